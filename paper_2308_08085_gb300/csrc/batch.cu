// Batched instances: many independent block forests advanced together.  The
// recursive level step of Section 4.1 has the same shape for every instance
// (an instance without level L+1 contributes no work there).  Two forms:
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
  int p_threads = 128, p_tile = 2, p_ctas_req = 0, p_ctas = 0;
  long long wait_limit = 1ll << 31;
  int n_phase_cap = 0, n_phase = 0, tiles_per_step = 0, max_member_tiles = 0;
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

// The phases of one coarse step in the order of advance_batch.
static void plan_rec(const Batch* b, int L, unsigned& cur, std::vector<PhaseRec>& out) {
  const bool fine = L + 1 < b->lmax && b->n_ids[L + 1] > 0;
  const int64_t np = b->n_par[L];
  const int wl = (int)((cur >> L) & 1u);
  if (fine && np > 0) out.push_back({PH_INTERP, L, wl, (int)((cur >> (L + 1)) & 1u)});
  if (b->n_act[L] > 0) out.push_back({PH_COLLIDE, L, wl, 0});
  cur ^= 1u << L;
  if (fine) {
    plan_rec(b, L + 1, cur, out);
    plan_rec(b, L + 1, cur, out);
    if (np > 0)
      out.push_back({PH_AVERAGE, L, (int)((cur >> L) & 1u), (int)((cur >> (L + 1)) & 1u)});
  }
}

// Items of member a in a phase, and the tiles they make.
static int64_t member_items(const Instance* a, const PhaseRec& r) {
  if (r.level >= a->lmax) return 0;
  return r.op == PH_COLLIDE ? a->n_active[r.level] : a->n_parents[r.level];
}

static int64_t member_tiles(const Batch* b, const Instance* a, const PhaseRec& r) {
  const int64_t ni = member_items(a, r);
  const int M = b->dim == 2 ? 16 : 64, NC = b->dim == 2 ? 4 : 8;
  const int U = b->p_threads / M;
  if (r.op == PH_COLLIDE) return (ni + b->p_tile - 1) / b->p_tile;
  if (r.op == PH_INTERP) return (ni + U - 1) / U;
  return (ni * NC + U - 1) / U;
}

static int build_plan(Batch* b) {
  std::vector<PhaseRec> rec[2];
  for (int parity = 0; parity < 2; ++parity) {
    unsigned cur = (b->cur & ~1u) | (unsigned)parity;
    plan_rec(b, 0, cur, rec[parity]);
  }
  const int n = b->n;
  const int np = (int)rec[0].size();
  if (np == 0 || np > b->n_phase_cap || rec[1].size() != rec[0].size()) {
    set_error("persistent batch: unexpected phase list");
    return AMR_E_INVAL;
  }
  std::vector<int32_t> toff((size_t)np * (n + 1)), ioff((size_t)np * (n + 1)), dep((size_t)np * n);
  std::vector<PersistPhase> ph(2 * (size_t)np);
  int64_t tile0 = 0, max_tiles = 0;
  for (int k = 0; k < np; ++k) {
    int64_t t = 0, it = 0;
    for (int i = 0; i < n; ++i) {
      toff[(size_t)k * (n + 1) + i] = (int32_t)t;
      ioff[(size_t)k * (n + 1) + i] = (int32_t)it;
      const int64_t ti = member_tiles(b, b->inst[i], rec[0][k]);
      t += ti;
      it += member_items(b->inst[i], rec[0][k]);
      max_tiles = std::max(max_tiles, ti);
    }
    toff[(size_t)k * (n + 1) + n] = (int32_t)t;
    ioff[(size_t)k * (n + 1) + n] = (int32_t)it;
    for (int parity = 0; parity < 2; ++parity) {
      const PhaseRec& r = rec[parity][k];
      PersistPhase& p = ph[(size_t)parity * np + k];
      p.op = r.op;
      p.level = r.level;
      p.which_in = r.which_in;
      p.which_ch = r.which_ch;
      p.tile0 = (int32_t)tile0;
      p.n_tiles = (int32_t)t;
      p.items = r.op == PH_COLLIDE ? b->act[r.level] : b->par[r.level];
    }
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
        if (toff[(size_t)kc * (n + 1) + i + 1] > toff[(size_t)kc * (n + 1) + i]) {
          d = kc;
          wrap = kk < 0 ? 1 : 0;
          break;
        }
      }
      dep[(size_t)k * n + i] = d < 0 ? 1 : 2 * d + wrap;   // no tiles at all: never waits
    }
  cudaStream_t s = b->stream;
  AMR_CUDA(cudaMemcpyAsync(b->d_phases, ph.data(), sizeof(PersistPhase) * ph.size(),
                           cudaMemcpyHostToDevice, s));
  AMR_CUDA(cudaMemcpyAsync(b->d_tile_off, toff.data(), 4 * toff.size(), cudaMemcpyHostToDevice, s));
  AMR_CUDA(cudaMemcpyAsync(b->d_item_off, ioff.data(), 4 * ioff.size(), cudaMemcpyHostToDevice, s));
  AMR_CUDA(cudaMemcpyAsync(b->d_dep, dep.data(), 4 * dep.size(), cudaMemcpyHostToDevice, s));
  AMR_CUDA(cudaStreamSynchronize(s));   // the host vectors go out of scope
  b->n_phase = np;
  b->tiles_per_step = (int)tile0;
  b->max_member_tiles = (int)max_tiles;
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
  b->p_ctas_req = cfg->ctas;
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
