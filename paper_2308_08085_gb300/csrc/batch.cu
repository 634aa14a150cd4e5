// Batched instances: many independent block forests advanced together.  The
// recursive level step of Section 4.1 has the same shape for every instance
// (an instance without level L+1 contributes no work there).  Three forms:
//  * graph: each level operation is one launch over an instance-major list
//    of (instance, block) items, and the batched coarse step is captured as
//    a CUDA graph (one per parity of level 0);
//  * persistent: one launch per call advances every member by n coarse steps
//    through a work queue of (step, phase, member, tile) items with
//    per-member dependency counters (PersistArgs in lbm_ops.h);
//  * members: one CUDA graph per coarse step whose independent branches are
//    the members' own coarse steps (their per-instance kernels, with the
//    exchange fused into the parent level and the listed averaging), so that
//    the small levels of different members run side by side.
// The form and its tile shape are picked by timing the candidates on the
// batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "amr_internal.h"
#include "lattice.cuh"

namespace amr {

struct Batch {
  std::vector<Instance*> inst;
  int n = 0, dim = 0, q = 0, storage = 0, lmax = 0;
  cudaStream_t stream = nullptr, capture_stream = nullptr;
  const LbmOps* ops = nullptr;
  InstDesc* descs = nullptr;                  // device [n]
  uint32_t* act[BATCH_MAX_LEVELS] = {};       // device item lists
  uint32_t* par[BATCH_MAX_LEVELS] = {};
  int64_t n_act[BATCH_MAX_LEVELS] = {}, n_par[BATCH_MAX_LEVELS] = {},
          n_ids[BATCH_MAX_LEVELS] = {};
  int64_t list_cap = 0;
  unsigned cur = 0;
  int variant = 512;   // threads per CTA of the batched collide-stream
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graph_valid = false;
  int64_t launches = 0, graph_launches[2] = {0, 0};
  // persistent form
  int mode = AMR_BATCH_GRAPH;
  int p_threads = 128, p_tile = 2, p_ctas = 0;
  long long wait_limit = 1ll << 31;
  int n_phase_cap = 0, n_phase = 0, tiles_per_step = 0;
  bool plan_valid = false;
  PersistPhase* d_phases = nullptr;    // device [2][n_phase_cap]
  int32_t* d_tile_off = nullptr;       // device [n_phase_cap][n + 1]
  int32_t* d_item_off = nullptr;
  int32_t* d_dep = nullptr;            // device [n_phase_cap][n]
  uint32_t* d_done = nullptr;          // device [n_phase_cap][n], then the queue head
  unsigned long long* d_head = nullptr;
  int32_t* d_abort = nullptr;
  // member-graph form
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t mgraph[2] = {nullptr, nullptr};
  bool mgraph_valid = false;
  int64_t mgraph_launches[2] = {0, 0};
};

// phases of one coarse step: 2^(lmax+1) - 3 (interpolation, collide-stream
// and averaging of every level visit of the recursion)
static int phase_cap(int lmax) { return (1 << (lmax + 1)) - 3; }

static size_t align256b(size_t x) { return (x + 255) & ~size_t(255); }

static int64_t sum_caps(amr_t* const* in, int n) {
  int64_t s = 0;
  for (int i = 0; i < n; ++i) s += reinterpret_cast<Instance*>(in[i])->cap;
  return s;
}

static int max_levels(amr_t* const* in, int n) {
  int m = 0;
  for (int i = 0; i < n; ++i) m = std::max(m, reinterpret_cast<Instance*>(in[i])->lmax);
  return m;
}

__global__ void k_pack_items(const int32_t* __restrict__ list, int n, int inst,
                             uint32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = ((uint32_t)inst << BATCH_SHIFT) | (uint32_t)list[i];
}

static int refresh(Batch* b) {
  std::vector<InstDesc> h(b->n);
  for (int i = 0; i < b->n; ++i) {
    Instance* a = b->inst[i];
    InstDesc& d = h[i];
    std::memset(&d, 0, sizeof(d));
    d.f[0] = a->f[0];
    d.f[1] = a->f[1];
    d.nbr = a->nbr;
    d.child0 = a->child0;
    d.cellmask = a->cellmask;
    for (int L = 0; L < a->lmax; ++L) {
      d.omega[L] = 1.0 / a->tau[L];
      if (L + 1 < a->lmax) {
        d.r_cf[L] = a->tau[L + 1] / (2.0 * a->tau[L]);
        d.r_fc[L] = 2.0 * a->tau[L] / a->tau[L + 1];
      }
    }
    d.faces = a->prm.faces;
    d.wait_flag = a->prm.wait_flag;
  }
  AMR_CUDA(cudaMemcpyAsync(b->descs, h.data(), sizeof(InstDesc) * b->n, cudaMemcpyHostToDevice,
                           b->stream));
  for (int L = 0; L < b->lmax; ++L) {
    int64_t oa = 0, op = 0, ni = 0;
    for (int i = 0; i < b->n; ++i) {
      Instance* a = b->inst[i];
      if (L >= a->lmax) continue;
      const int64_t na = a->n_active[L], np = a->n_parents[L];
      if (na > 0)
        k_pack_items<<<(int)((na + 255) / 256), 256, 0, b->stream>>>(
            a->active + (size_t)L * a->cap, (int)na, i, b->act[L] + oa);
      if (np > 0)
        k_pack_items<<<(int)((np + 255) / 256), 256, 0, b->stream>>>(
            a->parents + (size_t)L * a->cap, (int)np, i, b->par[L] + op);
      oa += na;
      op += np;
      ni += a->n_ids[L];
    }
    b->n_act[L] = oa;
    b->n_par[L] = op;
    b->n_ids[L] = ni;
  }
  AMR_CUDA(cudaGetLastError());
  AMR_CUDA(cudaStreamSynchronize(b->stream));   // the host descriptor copy must finish
  for (auto& g : b->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  b->graph_valid = false;
  b->plan_valid = false;
  for (auto& g : b->mgraph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  b->mgraph_valid = false;
  return AMR_OK;
}

static void advance_batch(Batch* b, int L) {
  const bool fine = L + 1 < b->lmax && b->n_ids[L + 1] > 0;
  const int64_t np = b->n_par[L];
  const int wl = (int)((b->cur >> L) & 1u);
  if (fine && np > 0) {
    b->ops->interp_batch(b->stream, b->par[L], (int)np, b->descs, L, wl,
                         (int)((b->cur >> (L + 1)) & 1u));
    b->launches += 1;
  }
  if (b->n_act[L] > 0) {
    b->ops->collide_stream_batch(b->stream, b->act[L], (int)b->n_act[L], b->descs, L, wl,
                                 b->variant);
    b->launches += 1;
  }
  b->cur ^= 1u << L;
  if (fine) {
    advance_batch(b, L + 1);
    advance_batch(b, L + 1);
    if (np > 0) {
      b->ops->average_batch(b->stream, b->par[L], (int)np, b->descs, L,
                            (int)((b->cur >> L) & 1u), (int)((b->cur >> (L + 1)) & 1u));
      b->launches += 1;
    }
  }
}

static int build_batch_graphs(Batch* b) {
  const unsigned saved = b->cur;
  cudaStream_t user = b->stream;
  b->stream = b->capture_stream;
  for (int parity = 0; parity < 2; ++parity) {
    b->cur = (saved & ~1u) | (unsigned)parity;
    cudaGraph_t g = nullptr;
    const int64_t before = b->launches;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      advance_batch(b, 0);
      e = cudaStreamEndCapture(b->stream, &g);
    }
    b->graph_launches[parity] = b->launches - before;
    b->launches = before;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->stream = user;
      b->cur = saved;
      set_error(std::string("batch graph capture: ") + cudaGetErrorString(e));
      cudaGetLastError();
      return AMR_E_CUDA;
    }
  }
  b->stream = user;
  b->cur = saved;
  b->graph_valid = true;
  return AMR_OK;
}

// ------------------------------------------------------------ persistent form
struct PhaseRec {
  int op, level, which_in, which_ch;
};

// What the plan of the persistent form depends on: per member, its level
// count and per-level counts ([n][lmax], 0 beyond the member's levels), the
// batch's level count, the CTA and tile shape, the buffer parities.
struct PlanCounts {
  int dim = 3, n = 0, lmax = 0, threads = 128, tile = 2;
  unsigned cur = 0;
  std::vector<int> member_lmax;
  std::vector<int64_t> n_ids, n_active, n_parents;
  int64_t ids(int i, int L) const { return n_ids[(size_t)i * lmax + L]; }
  int64_t act(int i, int L) const { return n_active[(size_t)i * lmax + L]; }
  int64_t par(int i, int L) const { return n_parents[(size_t)i * lmax + L]; }
  int64_t sum(int64_t (PlanCounts::*f)(int, int) const, int L) const {
    int64_t t = 0;
    for (int i = 0; i < n; ++i) t += (this->*f)(i, L);
    return t;
  }
};

struct HostPlan {
  std::vector<PhaseRec> rec[2];           // steps starting with cur bit 0 clear / set
  std::vector<int32_t> toff, ioff, dep;   // [phase][n + 1], [phase][n + 1], [phase][n]
  int64_t tiles_per_step = 0;
};

// The phases of one coarse step in the order of advance_batch.
static void plan_rec(const PlanCounts& c, int L, unsigned& cur, std::vector<PhaseRec>& out) {
  const bool fine = L + 1 < c.lmax && c.sum(&PlanCounts::ids, L + 1) > 0;
  const int64_t np = c.sum(&PlanCounts::par, L);
  const int wl = (int)((cur >> L) & 1u);
  if (fine && np > 0) out.push_back({PH_INTERP, L, wl, (int)((cur >> (L + 1)) & 1u)});
  if (c.sum(&PlanCounts::act, L) > 0) out.push_back({PH_COLLIDE, L, wl, 0});
  cur ^= 1u << L;
  if (fine) {
    plan_rec(c, L + 1, cur, out);
    plan_rec(c, L + 1, cur, out);
    if (np > 0)
      out.push_back({PH_AVERAGE, L, (int)((cur >> L) & 1u), (int)((cur >> (L + 1)) & 1u)});
  }
}

// Items of member i in a phase, and the tiles they make: M_L blocks per
// collide-stream tile, threads / 4^D parents per interpolation tile and
// threads / 4^D children per averaging tile.
static int64_t member_items(const PlanCounts& c, int i, const PhaseRec& r) {
  if (r.level >= c.member_lmax[i]) return 0;
  return r.op == PH_COLLIDE ? c.act(i, r.level) : c.par(i, r.level);
}

static int64_t member_tiles(const PlanCounts& c, int i, const PhaseRec& r) {
  const int64_t ni = member_items(c, i, r);
  const int M = c.dim == 2 ? 16 : 64, NC = c.dim == 2 ? 4 : 8;
  const int U = c.threads / M;
  if (r.op == PH_COLLIDE) return (ni + c.tile - 1) / c.tile;
  if (r.op == PH_INTERP) return (ni + U - 1) / U;
  return (ni * NC + U - 1) / U;
}

static int make_plan(const PlanCounts& c, int max_phases, HostPlan* hp) {
  for (int parity = 0; parity < 2; ++parity) {
    unsigned cur = (c.cur & ~1u) | (unsigned)parity;
    plan_rec(c, 0, cur, hp->rec[parity]);
  }
  const int n = c.n;
  const int np = (int)hp->rec[0].size();
  if (np == 0 || np > max_phases || hp->rec[1].size() != hp->rec[0].size()) {
    set_error("persistent batch: unexpected phase list");
    return AMR_E_INVAL;
  }
  hp->toff.assign((size_t)np * (n + 1), 0);
  hp->ioff.assign((size_t)np * (n + 1), 0);
  hp->dep.assign((size_t)np * n, 0);
  int64_t tile0 = 0;
  for (int k = 0; k < np; ++k) {
    int64_t t = 0, it = 0;
    for (int i = 0; i < n; ++i) {
      hp->toff[(size_t)k * (n + 1) + i] = (int32_t)t;
      hp->ioff[(size_t)k * (n + 1) + i] = (int32_t)it;
      t += member_tiles(c, i, hp->rec[0][k]);
      it += member_items(c, i, hp->rec[0][k]);
    }
    hp->toff[(size_t)k * (n + 1) + n] = (int32_t)t;
    hp->ioff[(size_t)k * (n + 1) + n] = (int32_t)it;
    tile0 += t;
    if (tile0 >= (1ll << 30)) {
      set_error("persistent batch: more than 2^30 tiles per coarse step");
      return AMR_E_INVAL;
    }
  }
  // dependencies: the member's previous phase with tiles, cyclically
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < np; ++k) {
      int d = -1, wrap = 0;
      for (int back = 1; back <= np; ++back) {
        const int kk = k - back;
        const int kc = kk < 0 ? kk + np : kk;
        if (hp->toff[(size_t)kc * (n + 1) + i + 1] > hp->toff[(size_t)kc * (n + 1) + i]) {
          d = kc;
          wrap = kk < 0 ? 1 : 0;
          break;
        }
      }
      hp->dep[(size_t)k * n + i] = d < 0 ? 1 : 2 * d + wrap;   // no tiles at all: never waits
    }
  hp->tiles_per_step = tile0;
  return AMR_OK;
}

static int build_plan(Batch* b) {
  PlanCounts c;
  c.dim = b->dim;
  c.n = b->n;
  c.lmax = b->lmax;
  c.threads = b->p_threads;
  c.tile = b->p_tile;
  c.cur = b->cur;
  c.member_lmax.resize(b->n);
  c.n_ids.assign((size_t)b->n * b->lmax, 0);
  c.n_active.assign((size_t)b->n * b->lmax, 0);
  c.n_parents.assign((size_t)b->n * b->lmax, 0);
  for (int i = 0; i < b->n; ++i) {
    const Instance* a = b->inst[i];
    c.member_lmax[i] = a->lmax;
    for (int L = 0; L < a->lmax; ++L) {
      c.n_ids[(size_t)i * b->lmax + L] = a->n_ids[L];
      c.n_active[(size_t)i * b->lmax + L] = a->n_active[L];
      c.n_parents[(size_t)i * b->lmax + L] = a->n_parents[L];
    }
  }
  HostPlan hp;
  const int rc = make_plan(c, b->n_phase_cap, &hp);
  if (rc != AMR_OK) return rc;
  const int np = (int)hp.rec[0].size();
  std::vector<PersistPhase> ph(2 * (size_t)np);
  for (int k = 0; k < np; ++k)
    for (int parity = 0; parity < 2; ++parity) {
      const PhaseRec& r = hp.rec[parity][k];
      PersistPhase& p = ph[(size_t)parity * np + k];
      p.op = r.op;
      p.level = r.level;
      p.which_in = r.which_in;
      p.which_ch = r.which_ch;
      p.tile0 = k == 0 ? 0 : ph[(size_t)parity * np + k - 1].tile0 +
                                 ph[(size_t)parity * np + k - 1].n_tiles;
      p.n_tiles = hp.toff[(size_t)k * (b->n + 1) + b->n];
      p.items = r.op == PH_COLLIDE ? b->act[r.level] : b->par[r.level];
    }
  cudaStream_t s = b->stream;
  AMR_CUDA(cudaMemcpyAsync(b->d_phases, ph.data(), sizeof(PersistPhase) * ph.size(),
                           cudaMemcpyHostToDevice, s));
  AMR_CUDA(cudaMemcpyAsync(b->d_tile_off, hp.toff.data(), 4 * hp.toff.size(),
                           cudaMemcpyHostToDevice, s));
  AMR_CUDA(cudaMemcpyAsync(b->d_item_off, hp.ioff.data(), 4 * hp.ioff.size(),
                           cudaMemcpyHostToDevice, s));
  AMR_CUDA(cudaMemcpyAsync(b->d_dep, hp.dep.data(), 4 * hp.dep.size(), cudaMemcpyHostToDevice, s));
  AMR_CUDA(cudaStreamSynchronize(s));   // the host vectors go out of scope
  b->n_phase = np;
  b->tiles_per_step = (int)hp.tiles_per_step;
  b->plan_valid = true;
  return AMR_OK;
}

static int launch_persistent(Batch* b, int n, int stall, long long limit) {
  if (!b->plan_valid) {
    const int rc = build_plan(b);
    if (rc != AMR_OK) return rc;
  }
  // counters stay below 2^30 within a launch
  const int64_t per_launch = std::max<int64_t>(1, (1ll << 30) / std::max(1, b->tiles_per_step));
  for (int done = 0; done < n;) {
    const int chunk = (int)std::min<int64_t>(n - done, per_launch);
    AMR_CUDA(cudaMemsetAsync(b->d_done, 0, align256b((size_t)b->n_phase_cap * b->n * 4) + 8,
                             b->stream));
    PersistArgs a{};
    a.descs = b->descs;
    a.phases = b->d_phases;
    a.tile_off = b->d_tile_off;
    a.item_off = b->d_item_off;
    a.dep = b->d_dep;
    a.done = b->d_done;
    a.head = b->d_head;
    a.abort = b->d_abort;
    a.n_phase = b->n_phase;
    a.n_inst = b->n;
    a.tiles_per_step = b->tiles_per_step;
    a.parity0 = (int)(b->cur & 1u);
    a.n_steps = chunk;
    a.tile_blocks = b->p_tile;
    a.wait_limit = limit;
    a.stall = stall;
    const int64_t tiles = (int64_t)b->tiles_per_step * chunk;
    const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(b->p_ctas, tiles));
    b->ops->batch_persistent(b->stream, a, b->p_threads, ctas);
    AMR_CUDA(cudaGetLastError());
    b->launches += 1;
    if (stall) return AMR_OK;
    b->cur ^= (unsigned)(chunk & 1);
    done += chunk;
  }
  return AMR_OK;
}

// ------------------------------------------------------------ member graphs
static int build_member_graphs(Batch* b) {
  if (b->branch.empty()) {
    b->branch.assign(b->n, nullptr);
    b->joins.assign(b->n, nullptr);
    for (int i = 0; i < b->n; ++i) {
      AMR_CUDA(cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking));
      AMR_CUDA(cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming));
    }
    AMR_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  }
  cudaStream_t cs = b->capture_stream;
  for (int parity = 0; parity < 2; ++parity) {
    cudaGraph_t g = nullptr;
    int64_t launched = 0;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, cs);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
      e = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
      if (e != cudaSuccess) break;
      launched += coarse_step_into(b->inst[i], b->branch[i], parity);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(b->joins[i], b->branch[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, b->joins[i], 0);
    }
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->mgraph[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      set_error(std::string("member graph capture: ") + cudaGetErrorString(e));
      cudaGetLastError();
      return AMR_E_CUDA;
    }
    b->mgraph_launches[parity] = launched;
  }
  b->mgraph_valid = true;
  return AMR_OK;
}

static int step_batch(Batch* b, int n) {
  for (Instance* a : b->inst)
    if (a->cur != b->cur) {
      set_error("batch members were stepped outside the batch (buffer parities differ)");
      return AMR_E_INVAL;
    }
  if (b->mode == AMR_BATCH_PERSISTENT) {
    const int rc = launch_persistent(b, n, 0, b->wait_limit);
    if (rc != AMR_OK) return rc;
    for (Instance* a : b->inst) {
      a->cur = b->cur;
      a->coarse_steps += n;
    }
    return AMR_OK;
  }
  if (b->mode == AMR_BATCH_MEMBERS) {
    if (!b->mgraph_valid) {
      const int rc = build_member_graphs(b);
      if (rc != AMR_OK) return rc;
    }
    for (int s = 0; s < n; ++s) {
      const int parity = (int)(b->cur & 1u);
      AMR_CUDA(cudaGraphLaunch(b->mgraph[parity], b->stream));
      b->launches += b->mgraph_launches[parity];
      b->cur ^= 1u;
    }
    for (Instance* a : b->inst) {
      a->cur = b->cur;
      a->coarse_steps += n;
    }
    AMR_CUDA(cudaGetLastError());
    return AMR_OK;
  }
  if (!b->graph_valid) {
    const int rc = build_batch_graphs(b);
    if (rc != AMR_OK) return rc;
  }
  for (int s = 0; s < n; ++s) {
    const int parity = (int)(b->cur & 1u);
    AMR_CUDA(cudaGraphLaunch(b->graph[parity], b->stream));
    b->launches += b->graph_launches[parity];
    b->cur ^= 1u;
  }
  for (Instance* a : b->inst) {
    a->cur = b->cur;
    a->coarse_steps += n;
  }
  AMR_CUDA(cudaGetLastError());
  return AMR_OK;
}

}  // namespace amr

using namespace amr;

extern "C" {

size_t amr_batch_arena_bytes(amr_t* const* instances, int n) {
  if (!instances || n <= 0) return 0;
  const int64_t caps = sum_caps(instances, n);
  const int lmax = max_levels(instances, n);
  const size_t npc = (size_t)phase_cap(lmax);
  return align256b(sizeof(InstDesc) * n) + 2 * (size_t)lmax * align256b((size_t)caps * 4) +
         align256b(2 * npc * sizeof(PersistPhase)) + 2 * align256b(npc * (n + 1) * 4) +
         align256b(npc * n * 4) + align256b(npc * n * 4) + 256 + 256;
}

int amr_batch_create(amr_t* const* instances, int n, void* dev_arena, size_t arena_bytes,
                     void* stream, amr_batch_t** out) {
  if (!out || !instances || n <= 0) return AMR_E_INVAL;
  *out = nullptr;
  if (n > (1 << (32 - BATCH_SHIFT)) - 1) {
    set_error("too many instances for one batch");
    return AMR_E_INVAL;
  }
  Instance* a0 = reinterpret_cast<Instance*>(instances[0]);
  for (int i = 0; i < n; ++i) {
    Instance* a = reinterpret_cast<Instance*>(instances[i]);
    if (!a || a->dim != a0->dim || a->q != a0->q || a->storage != a0->storage) {
      set_error("batch members must share the velocity set and storage");
      return AMR_E_INVAL;
    }
    if (a->solid) {
      set_error("batch members may not have a solid prism");
      return AMR_E_INVAL;
    }
    if (a->cfg.interp != AMR_INTERP_LINEAR) {
      set_error("batch members use linear interpolation");
      return AMR_E_INVAL;
    }
    if (a->cap > (int64_t)BATCH_MASK) {
      set_error("batch member capacity exceeds 2^25 blocks");
      return AMR_E_INVAL;
    }
    if (a->lmax > BATCH_MAX_LEVELS || a->cur != a0->cur) {
      set_error("batch members must have equal buffer parities");
      return AMR_E_INVAL;
    }
  }
  const size_t need = amr_batch_arena_bytes(instances, n);
  if (!dev_arena || arena_bytes < need || ((uintptr_t)dev_arena & 255u)) {
    set_error("batch arena needs " + std::to_string(need) + " bytes, 256-byte aligned");
    return AMR_E_ARENA;
  }
  Batch* b = new Batch();
  for (int i = 0; i < n; ++i) b->inst.push_back(reinterpret_cast<Instance*>(instances[i]));
  b->n = n;
  b->dim = a0->dim;
  b->q = a0->q;
  b->storage = a0->storage;
  b->lmax = max_levels(instances, n);
  b->ops = a0->ops;
  b->stream = (cudaStream_t)stream;
  b->cur = a0->cur;
  b->list_cap = sum_caps(instances, n);
  char* base = (char*)dev_arena;
  b->descs = (InstDesc*)base;
  size_t off = align256b(sizeof(InstDesc) * n);
  for (int L = 0; L < b->lmax; ++L) {
    b->act[L] = (uint32_t*)(base + off);
    off += align256b((size_t)b->list_cap * 4);
    b->par[L] = (uint32_t*)(base + off);
    off += align256b((size_t)b->list_cap * 4);
  }
  b->n_phase_cap = phase_cap(b->lmax);
  const size_t npc = (size_t)b->n_phase_cap;
  b->d_phases = (PersistPhase*)(base + off);
  off += align256b(2 * npc * sizeof(PersistPhase));
  b->d_tile_off = (int32_t*)(base + off);
  off += align256b(npc * (n + 1) * 4);
  b->d_item_off = (int32_t*)(base + off);
  off += align256b(npc * (n + 1) * 4);
  b->d_dep = (int32_t*)(base + off);
  off += align256b(npc * n * 4);
  b->d_done = (uint32_t*)(base + off);                       // done, then the head
  off += align256b(npc * n * 4);
  b->d_head = (unsigned long long*)(base + off);
  off += 256;
  b->d_abort = (int32_t*)(base + off);
  if (cudaMemsetAsync(b->d_abort, 0, sizeof(int32_t), b->stream) != cudaSuccess) {
    delete b;
    set_error("cannot clear the batch abort word");
    return AMR_E_CUDA;
  }
  if (cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    set_error("cannot create capture stream");
    return AMR_E_CUDA;
  }
  const int rc = refresh(b);
  if (rc != AMR_OK) {
    cudaStreamDestroy(b->capture_stream);
    delete b;
    return rc;
  }
  *out = reinterpret_cast<amr_batch_t*>(b);
  return AMR_OK;
}

int amr_batch_refresh(amr_batch_t* h) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b) return AMR_E_INVAL;
  return refresh(b);
}

int amr_batch_step(amr_batch_t* h, int n_coarse_steps) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b || n_coarse_steps < 0) return AMR_E_INVAL;
  return step_batch(b, n_coarse_steps);
}

int amr_batch_configure(amr_batch_t* h, const amr_batch_config_t* cfg) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b || !cfg) return AMR_E_INVAL;
  if (cfg->mode == AMR_BATCH_GRAPH) {
    if (cfg->threads != 64 && cfg->threads != 128 && cfg->threads != 256 && cfg->threads != 512) {
      set_error("graph form: threads per CTA must be 64, 128, 256 or 512");
      return AMR_E_INVAL;
    }
    b->mode = AMR_BATCH_GRAPH;
    b->variant = cfg->threads;
    b->graph_valid = false;
    return AMR_OK;
  }
  if (cfg->mode == AMR_BATCH_MEMBERS) {
    b->mode = AMR_BATCH_MEMBERS;
    b->mgraph_valid = false;
    return AMR_OK;
  }
  if (cfg->mode != AMR_BATCH_PERSISTENT) {
    set_error("unknown batch mode");
    return AMR_E_INVAL;
  }
  if ((cfg->threads != 64 && cfg->threads != 128 && cfg->threads != 256) ||
      cfg->tile_blocks < 1 || cfg->tile_blocks > PERSIST_MAX_TILE || cfg->ctas < 0) {
    set_error("persistent form: threads 64, 128 or 256, tile_blocks 1..8, ctas >= 0");
    return AMR_E_INVAL;
  }
  const int resident = b->ops->persistent_ctas(cfg->threads);
  if (resident <= 0) {
    cudaGetLastError();
    set_error("persistent form: the kernel cannot be made resident with this CTA size");
    return AMR_E_CUDA;
  }
  b->mode = AMR_BATCH_PERSISTENT;
  b->p_threads = cfg->threads;
  b->p_tile = cfg->tile_blocks;
  b->p_ctas = cfg->ctas > 0 ? cfg->ctas : resident;
  b->plan_valid = false;
  return AMR_OK;
}

int amr_batch_get_config(amr_batch_t* h, amr_batch_config_t* out) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b || !out) return AMR_E_INVAL;
  out->mode = b->mode;
  out->threads = b->mode == AMR_BATCH_GRAPH ? b->variant
                                            : (b->mode == AMR_BATCH_PERSISTENT ? b->p_threads : 0);
  out->tile_blocks = b->mode == AMR_BATCH_GRAPH ? b->variant / (b->dim == 2 ? 16 : 64)
                                                : (b->mode == AMR_BATCH_PERSISTENT ? b->p_tile : 0);
  out->ctas = b->mode == AMR_BATCH_PERSISTENT ? b->p_ctas : 0;
  return AMR_OK;
}

int amr_batch_autotune(amr_batch_t* h, int trial_steps, int forms, amr_batch_config_t* chosen,
                       float* ms_out) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b || trial_steps < 1 || forms < 1 || forms > 7) return AMR_E_INVAL;
  // candidates in the order of ms_out: the graph form with 512 / 256 / 128 /
  // 64 threads per CTA (M_L = 8 / 4 / 2 / 1 blocks per CTA in 3D), then the
  // persistent form with M_L = 1, 2, 4, 8 blocks per tile x 64, 128, 256
  // threads per CTA, then the member-graph form
  std::vector<amr_batch_config_t> cand;
  for (int t : {512, 256, 128, 64}) cand.push_back({AMR_BATCH_GRAPH, t, 0, 0});
  for (int m : {1, 2, 4, 8})
    for (int t : {64, 128, 256}) cand.push_back({AMR_BATCH_PERSISTENT, t, m, 0});
  cand.push_back({AMR_BATCH_MEMBERS, 0, 0, 0});
  amr_batch_config_t keep{};
  amr_batch_get_config(h, &keep);
  cudaEvent_t e0, e1;
  AMR_CUDA(cudaEventCreate(&e0));
  AMR_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  amr_batch_config_t best_c = keep;
  int rc = AMR_OK;
  for (size_t c = 0; c < cand.size() && rc == AMR_OK; ++c) {
    if (ms_out) ms_out[c] = -1.f;
    const bool want = cand[c].mode == AMR_BATCH_GRAPH        ? (forms & 1)
                      : cand[c].mode == AMR_BATCH_PERSISTENT ? (forms & 2)
                                                             : (forms & 4);
    if (!want) continue;
    rc = amr_batch_configure(h, &cand[c]);
    if (rc != AMR_OK) break;
    rc = step_batch(b, 1);   // capture or plan, and warm
    if (rc != AMR_OK) break;
    if (cudaEventRecord(e0, b->stream) != cudaSuccess) rc = AMR_E_CUDA;
    if (rc == AMR_OK) rc = step_batch(b, trial_steps);
    if (rc == AMR_OK && cudaEventRecord(e1, b->stream) != cudaSuccess) rc = AMR_E_CUDA;
    if (rc == AMR_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = AMR_E_CUDA;
    float ms = 0.f;
    if (rc == AMR_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = AMR_E_CUDA;
    if (rc != AMR_OK) break;
    if (ms_out) ms_out[c] = ms / (float)trial_steps;
    if (ms < best) {
      best = ms;
      amr_batch_get_config(h, &best_c);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != AMR_OK) {
    if (rc == AMR_E_CUDA) set_error(std::string("batch autotune: ") + cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  best_c.ctas = 0;
  rc = amr_batch_configure(h, &best_c);
  if (rc != AMR_OK) return rc;
  if (chosen) amr_batch_get_config(h, chosen);
  return AMR_OK;
}

int amr_batch_sync(amr_batch_t* h) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b) return AMR_E_INVAL;
  int32_t ab = 0;
  AMR_CUDA(cudaMemcpyAsync(&ab, b->d_abort, sizeof(ab), cudaMemcpyDeviceToHost, b->stream));
  AMR_CUDA(cudaStreamSynchronize(b->stream));
  if (ab == 0) return AMR_OK;
  AMR_CUDA(cudaMemsetAsync(b->d_abort, 0, sizeof(int32_t), b->stream));
  for (Instance* a : b->inst)
    AMR_CUDA(cudaMemsetAsync(a->prm.wait_flag, 0, sizeof(int32_t), b->stream));
  AMR_CUDA(cudaStreamSynchronize(b->stream));
  set_error("a bounded wait of the persistent batched kernel timed out");
  return AMR_E_TIMEOUT;
}

int amr_batch_check_timeout(amr_batch_t* h, long long limit_cycles) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b) return AMR_E_INVAL;
  if (limit_cycles <= 0 || limit_cycles > (1ll << 32)) {
    set_error("limit_cycles must be in (0, 2^32]");
    return AMR_E_INVAL;
  }
  if (b->mode != AMR_BATCH_PERSISTENT) {
    set_error("amr_batch_check_timeout needs the persistent form");
    return AMR_E_INVAL;
  }
  int rc = amr_batch_sync(h);   // report (and clear) anything earlier first
  if (rc != AMR_OK) return rc;
  rc = launch_persistent(b, 1, 1, limit_cycles);
  if (rc != AMR_OK) return rc;
  return amr_batch_sync(h);
}

int amr_batch_plan(int dim, int n, int lmax, const int32_t* member_lmax, const int64_t* n_ids,
                   const int64_t* n_active, const int64_t* n_parents, int threads,
                   int tile_blocks, uint32_t cur, int max_phases, int32_t* n_phase,
                   int32_t* phases, int32_t* tile_off, int32_t* dep) {
  if ((dim != 2 && dim != 3) || n <= 0 || lmax < 1 || lmax > BATCH_MAX_LEVELS ||
      (threads != 64 && threads != 128 && threads != 256) || tile_blocks < 1 ||
      tile_blocks > PERSIST_MAX_TILE || max_phases < 1 || !member_lmax || !n_ids ||
      !n_active || !n_parents || !n_phase || !phases || !tile_off || !dep) {
    set_error("amr_batch_plan: bad arguments");
    return AMR_E_INVAL;
  }
  PlanCounts c;
  c.dim = dim;
  c.n = n;
  c.lmax = lmax;
  c.threads = threads;
  c.tile = tile_blocks;
  c.cur = cur;
  c.member_lmax.assign(member_lmax, member_lmax + n);
  for (int i = 0; i < n; ++i)
    if (c.member_lmax[i] < 1 || c.member_lmax[i] > lmax) {
      set_error("amr_batch_plan: a member's level count is out of range");
      return AMR_E_INVAL;
    }
  c.n_ids.assign(n_ids, n_ids + (size_t)n * lmax);
  c.n_active.assign(n_active, n_active + (size_t)n * lmax);
  c.n_parents.assign(n_parents, n_parents + (size_t)n * lmax);
  HostPlan hp;
  const int rc = make_plan(c, max_phases, &hp);
  if (rc != AMR_OK) return rc;
  const int np = (int)hp.rec[0].size();
  *n_phase = np;
  for (int k = 0; k < np; ++k) {
    const PhaseRec& r = hp.rec[c.cur & 1u][k];
    phases[4 * k] = r.op;
    phases[4 * k + 1] = r.level;
    phases[4 * k + 2] = r.which_in;
    phases[4 * k + 3] = r.which_ch;
  }
  std::copy(hp.toff.begin(), hp.toff.end(), tile_off);
  std::copy(hp.dep.begin(), hp.dep.end(), dep);
  return AMR_OK;
}

int64_t amr_batch_launches(amr_batch_t* h) {
  Batch* b = reinterpret_cast<Batch*>(h);
  return b ? b->launches : AMR_E_INVAL;
}

int amr_batch_free(amr_batch_t* h) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b) return AMR_E_INVAL;
  for (auto& g : b->graph)
    if (g) cudaGraphExecDestroy(g);
  for (auto& g : b->mgraph)
    if (g) cudaGraphExecDestroy(g);
  for (cudaStream_t st : b->branch)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->joins)
    if (ev) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  delete b;
  return AMR_OK;
}

}  // extern "C"
