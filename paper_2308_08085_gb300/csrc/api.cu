// C ABI of the block-forest AMR-LBM library (include/amr.h): arena carving,
// the recursive level step of Section 4.1 (optionally replayed as a CUDA
// graph), the pre-adapt synchronisation and criterion of Section 4.4, field
// export/import, the FP64 mass audit, the momentum-exchange force, and
// per-kernel CUDA-event profiling.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "amr_internal.h"
#include "lattice.cuh"

static_assert(sizeof(amr_config) == 376, "amr_config layout is part of the ABI");
static_assert(sizeof(amr_adapt_stats) == 56, "amr_adapt_stats layout is part of the ABI");
static_assert(sizeof(amr_kernel_profile) == 64, "amr_kernel_profile layout is part of the ABI");

namespace amr {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

constexpr size_t STAGING_BYTES = size_t(32) << 20;

// host copies of the velocity vectors (same numbering as lattice.cuh)
static void host_velocities(int dim, int q, int (*c)[3], double* w) {
  if (dim == 2) {
    for (int p = 0; p < 9; ++p) {
      c[p][0] = VS<2, 9>::cx[p];
      c[p][1] = VS<2, 9>::cy[p];
      c[p][2] = 0;
      w[p] = VS<2, 9>::w[p];
    }
  } else if (q == 19) {
    for (int p = 0; p < 19; ++p) {
      c[p][0] = VS<3, 19>::cx[p];
      c[p][1] = VS<3, 19>::cy[p];
      c[p][2] = VS<3, 19>::cz[p];
      w[p] = VS<3, 19>::w[p];
    }
  } else {
    for (int p = 0; p < 27; ++p) {
      c[p][0] = VS<3, 27>::cx[p];
      c[p][1] = VS<3, 27>::cy[p];
      c[p][2] = VS<3, 27>::cz[p];
      w[p] = VS<3, 27>::w[p];
    }
  }
}

struct Layout {
  size_t off[32];
  size_t total;
};

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static size_t elem_bytes(int storage) {
  return storage == AMR_F64 ? 8 : (storage == AMR_F32 ? 4 : 2);
}

static int validate(const amr_config* c, std::string* why) {
  if (!c) { *why = "null config"; return AMR_E_INVAL; }
  const bool ok_set = (c->dim == 2 && c->q == 9) || (c->dim == 3 && (c->q == 19 || c->q == 27));
  if (!ok_set) { *why = "velocity set must be D2Q9, D3Q19 or D3Q27"; return AMR_E_INVAL; }
  if (c->storage < AMR_F64 || c->storage > AMR_F32_F16) { *why = "bad storage"; return AMR_E_INVAL; }
  if (c->dim == 2 && c->storage > AMR_F32) { *why = "16-bit storage is 3D only"; return AMR_E_INVAL; }
  const int n[3] = {c->nx, c->ny, c->dim == 3 ? c->nz : 4};
  for (int a = 0; a < 3; ++a)
    if (n[a] <= 0 || n[a] % 4) { *why = "root extents must be positive multiples of 4"; return AMR_E_INVAL; }
  if (c->max_levels < 1 || c->max_levels > AMR_MAX_LEVELS) { *why = "max_levels out of range"; return AMR_E_INVAL; }
  if (!(c->nu0 > 0) || !(c->length_x > 0)) { *why = "nu0 and length_x must be positive"; return AMR_E_INVAL; }
  for (int ax = 0; ax < c->dim; ++ax) {
    const bool p0 = c->faces[2 * ax].kind == AMR_FACE_PERIODIC;
    const bool p1 = c->faces[2 * ax + 1].kind == AMR_FACE_PERIODIC;
    if (p0 != p1) { *why = "periodic faces must come in pairs"; return AMR_E_INVAL; }
    for (int s = 0; s < 2; ++s) {
      const int k = c->faces[2 * ax + s].kind;
      if (k < AMR_FACE_NOSLIP || k > AMR_FACE_PERIODIC) { *why = "bad face kind"; return AMR_E_INVAL; }
    }
  }
  const int64_t n_root = (int64_t)(n[0] / 4) * (n[1] / 4) * (c->dim == 3 ? n[2] / 4 : 1);
  const int nc = c->dim == 2 ? 4 : 8;
  if (c->max_blocks < n_root || (c->max_blocks - n_root) % nc) {
    *why = "max_blocks must be >= root blocks and (max_blocks - root) a multiple of 2^dim";
    return AMR_E_INVAL;
  }
  if (c->max_blocks > (int64_t(1) << 31) / 64) { *why = "max_blocks too large"; return AMR_E_INVAL; }
  if (c->interp != AMR_INTERP_LINEAR && c->interp != AMR_INTERP_CUBIC) {
    *why = "interp must be AMR_INTERP_LINEAR or AMR_INTERP_CUBIC";
    return AMR_E_INVAL;
  }
  if (c->root_ids) {
    std::vector<char> seen((size_t)n_root, 0);
    for (int64_t i = 0; i < n_root; ++i) {
      const int32_t v = c->root_ids[i];
      if (v < 0 || v >= n_root || seen[(size_t)v]) {
        *why = "root_ids must be a permutation of 0 .. n_root-1";
        return AMR_E_INVAL;
      }
      seen[(size_t)v] = 1;
    }
  }
  return AMR_OK;
}

static Layout layout_for(const amr_config* c) {
  Layout L{};
  const int64_t cap = c->max_blocks;
  const int M = c->dim == 2 ? 16 : 64;
  const size_t fb = (size_t)cap * M * c->q * elem_bytes(c->storage);
  const int lmax = c->max_levels;
  const size_t sizes[] = {
      fb, fb,                                  // 0,1 populations A/B
      (size_t)cap * 4, (size_t)cap * 4,        // 2,3 level, status
      (size_t)cap * 4, (size_t)cap * 4,        // 4,5 child0, parent
      (size_t)cap * 12,                        // 6 X
      (size_t)cap * NBR_STRIDE * 4,            // 7 nbr
      (size_t)cap * 4,                         // 8 nonemask
      (size_t)cap * 8,                         // 9 solidmask
      (size_t)lmax * cap * 4,                  // 10 idset
      (size_t)lmax * cap * 4,                  // 11 active
      (size_t)lmax * cap * 4,                  // 12 parents
      (size_t)cap * 4,                         // 13 gap
      (size_t)cap,                             // 14 marks
      (size_t)cap * 8,                         // 15 w2
      (size_t)cap * 4, (size_t)cap * 4, (size_t)cap * 4,   // 16,17,18 tmp
      (size_t)cta_slots(cap) * 4,              // 19 cta
      64 * 4,                                  // 20 dcount
      8192 * 8,                                // 21 red
      64 * 4,                                  // 22 wall_code
      STAGING_BYTES,                           // 23 staging
      (size_t)cap * 16,                        // 24 cellmask
      (size_t)cap * 27 * 4,                    // 25 features
      (size_t)cap * 4,                         // 26 proposal probabilities
      (size_t)lmax * cap * 4,                  // 27 tree order of each level
      (size_t)lmax * cap * 4,                  // 28 blocks with a NONE neighbour, per level
      (size_t)cap * (c->dim == 2 ? 4 : 8) * 4, // 29 averaging groups, packed by level
  };
  size_t off = 0;
  int i = 0;
  for (size_t s : sizes) {
    L.off[i++] = off;
    off += align256(s);
  }
  L.total = off;
  return L;
}

struct Handle : Instance {
  void* staging = nullptr;
  cudaStream_t capture_stream = nullptr;
  char* arena = nullptr;       // the caller's arena (layout_for offsets)
  size_t arena_used = 0;       // bytes of it the layout occupies
};

// Header of a checkpoint image (amr_checkpoint): the configuration fields that
// fix the arena layout, then the host mirror of the mesh and time state.
struct CheckpointHeader {
  char tag[8];
  int32_t dim, q, storage, nx, ny, nz, max_levels, pad_;
  int64_t max_blocks;
  uint64_t arena_used;
  int64_t n_ids[AMR_MAX_LEVELS], n_active[AMR_MAX_LEVELS], n_parents[AMR_MAX_LEVELS],
      n_leaves[AMR_MAX_LEVELS], n_bnd[AMR_MAX_LEVELS], n_ghost_children[AMR_MAX_LEVELS],
      n_ghost_cells[AMR_MAX_LEVELS], n_iface_cells[AMR_MAX_LEVELS], n_agrp[AMR_MAX_LEVELS],
      agrp_off[AMR_MAX_LEVELS];
  int64_t n_gaps, coarse_steps;
  uint32_t cur, pad2_;
};
static const char kCheckpointTag[8] = {'A', 'M', 'R', 'C', 'K', 'P', 'T', '3'};

// ------------------------------------------------------------ profiling
static const char* kPkNames[PK_COUNT] = {
    "collide_stream", "interp",       "average",       "adapt_sync",
    "adapt_criterion", "adapt_marks", "adapt_alloc",   "adapt_idsets",
    "adapt_relink",   "adapt_children", "adapt_lists"};

static cudaEvent_t take_event(Instance* a) {
  if (!a->event_pool.empty()) {
    cudaEvent_t e = a->event_pool.back();
    a->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void adapt_phase(Instance* a, int kind) {
  if (a->profiling == 0) return;
  cudaEvent_t e = take_event(a);
  cudaEventRecord(e, a->stream);
  a->phase_marks.emplace_back(kind, e);
}

// Durations between consecutive phase marks of the finished adaptation.
static void harvest_phases(Instance* a) {
  if (a->phase_marks.empty()) return;
  cudaStreamSynchronize(a->stream);
  for (size_t i = 0; i + 1 < a->phase_marks.size(); ++i) {
    const int kind = a->phase_marks[i].first;
    float ms = 0.f;
    if (kind >= 0 && cudaEventElapsedTime(&ms, a->phase_marks[i].second,
                                          a->phase_marks[i + 1].second) == cudaSuccess) {
      a->acc[kind].launches += 1;
      a->acc[kind].ms += ms;
    }
  }
  for (auto& pm : a->phase_marks) a->event_pool.push_back(pm.second);
  a->phase_marks.clear();
}

struct ProfScope {
  Instance* a;
  ProfileSlot slot{};
  bool on;
  ProfScope(Instance* a_, int kind, double bytes, double cells)
      : a(a_), on(a_->profiling == 1 || (a_->profiling == 2 && a_->capturing)) {
    if (!on) return;
    slot.start = take_event(a);
    slot.stop = take_event(a);
    slot.kind = kind;
    slot.bytes = bytes;
    slot.cells = cells;
    record(slot.start);
  }
  // inside a stream capture the record must become an event node of the graph
  void record(cudaEvent_t e) {
    if (a->capturing) cudaEventRecordWithFlags(e, a->stream, cudaEventRecordExternal);
    else cudaEventRecord(e, a->stream);
  }
  ~ProfScope() {
    if (!on) return;
    record(slot.stop);
    if (a->capturing) a->gprof[a->capture_parity].push_back(slot);
    else a->prof.push_back(slot);
  }
};

static int drain_profile(Instance* a) {
  if (a->profiling == 2 && a->last_parity >= 0 && !a->gprof[a->last_parity].empty()) {
    // one sample: the launches of the most recently replayed coarse step
    AMR_CUDA(cudaStreamSynchronize(a->stream));
    for (auto& s : a->gprof[a->last_parity]) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, s.start, s.stop) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      auto& acc = a->acc[s.kind];
      acc.launches += 1;
      acc.ms += ms;
      acc.bytes += s.bytes;
      acc.cells += s.cells;
    }
    a->last_parity = -1;
  }
  if (a->prof.empty()) return AMR_OK;
  AMR_CUDA(cudaStreamSynchronize(a->stream));
  for (auto& s : a->prof) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s.start, s.stop);
    auto& acc = a->acc[s.kind];
    acc.launches += 1;
    acc.ms += ms;
    acc.bytes += s.bytes;
    acc.cells += s.cells;
    a->event_pool.push_back(s.start);
    a->event_pool.push_back(s.stop);
  }
  a->prof.clear();
  return AMR_OK;
}

// ------------------------------------------------------------ level step
static double ratio_cf(const Instance* a, int L) { return a->tau[L + 1] / (2.0 * a->tau[L]); }
static double ratio_fc(const Instance* a, int L) { return 2.0 * a->tau[L] / a->tau[L + 1]; }

// ghost_in: the first substep of level L > 0, whose ghost cells read the
// values the level step's interpolation left in their own output slots.
// xchg: level L's exchanging parents interpolate into their children's ghost
// cells (linear interpolation).
static void collide_stream_level(Instance* a, int L, bool ghost_in, const Exchange* xchg) {
  const int64_t n = a->n_active[L];
  // the parity flips even without active blocks: graph replay and batches
  // rely on level 0 flipping once and deeper levels an even number of times
  if (n == 0) {
    a->cur ^= 1u << L;
    return;
  }
  StepParams prm = a->prm;
  prm.omega = 1.0 / a->tau[L];
  double bytes = (double)n * a->M * 2.0 * a->q * a->elem;
  if (xchg) bytes += (double)a->n_ghost_cells[L] * a->q * a->elem;   // ghost cells written
  {
    ProfScope ps(a, PK_COLLIDE, bytes, (double)n * a->M);
    a->ops->collide_stream(a->stream, a->active + (size_t)L * a->cap, (int)n, a->fbuf(L, 0),
                           a->fbuf(L, 1), a->nbr, a->sm(), prm, a->solid,
                           ghost_in ? a->cellmask : nullptr, xchg);
    a->launches += 1;
  }
  a->cur ^= 1u << L;
}

// Recursive level step (Section 4.1): interpolate into level L+1, collide and
// stream level L, advance level L+1 twice, average level L+1 into level L.
// The interpolated ghost values go into their own slots of level L+1's output
// buffer, where the first of its two substeps (`first`) reads them.  With
// linear interpolation the interpolation is fused into level L's
// collide-stream (Exchange: its exchanging parents gather their cells anyway);
// cubic interpolation, which needs every cell of the parent, keeps its launch.
static void advance(Instance* a, int L, bool first) {
  const bool fine = L + 1 < a->lmax && a->n_ids[L + 1] > 0;
  const int64_t np = a->n_parents[L];
  const bool cubic = a->interp_bits() != 0;
  if (fine && np > 0 && cubic) {
    // algorithmic bytes: the 2^D parent cells under each child with ghost
    // cells (read) and the ghost cells (written)
    const double cells = (double)a->n_ghost_cells[L];
    ProfScope ps(a, PK_INTERP,
                 ((double)a->n_ghost_children[L] * a->nc + cells) * a->q * a->elem, cells);
    a->ops->interp(a->stream, a->parents + (size_t)L * a->cap, (int)np, a->fbuf(L, 0),
                   a->fbuf(L + 1, 1), a->child0, a->cellmask, a->nbr, a->sm(),
                   nullptr, nullptr, ratio_cf(a, L), 4 | a->interp_bits(), a->solid);
    a->launches += 1;
  }
  Exchange ex{};
  const bool xchg = fine && np > 0 && !cubic;
  if (xchg) {
    ex.fine_out = a->fbuf(L + 1, 1);
    ex.child0 = a->child0;
    ex.cellmask = a->cellmask;
    ex.r_cf = ratio_cf(a, L);
  }
  collide_stream_level(a, L, first && L > 0 && a->n_parents[L - 1] > 0, xchg ? &ex : nullptr);
  if (fine) {
    advance(a, L + 1, true);
    advance(a, L + 1, false);
    if (np > 0) {
      // algorithmic bytes: interface fine cells (read) and their parent
      // cells, one per 2^D children (written)
      const double cells = (double)a->n_iface_cells[L];
      ProfScope ps(a, PK_AVERAGE, cells * (1.0 + 1.0 / a->nc) * a->q * a->elem, cells);
      // cubic interpolation samples every cell of the parent, so with it the
      // parent cells over interior children are averaged as well (mode 1:
      // every cell whose children are not ghosts), else only those over
      // interface children: the groups of interface cells of the fine
      // level's boundary blocks, listed at adaptation
      if (cubic)
        a->ops->average(a->stream, a->parents + (size_t)L * a->cap, (int)np, true,
                        a->fbuf(L, 0), a->fbuf(L + 1, 0), a->child0, a->parent,
                        a->cellmask, a->status, a->nbr, a->sm(), ratio_fc(a, L), 1, a->solid);
      else
        a->ops->average_groups(a->stream, a->agrp + a->agrp_off[L + 1], (int)a->n_agrp[L + 1],
                               a->fbuf(L, 0), a->fbuf(L + 1, 0), a->child0,
                               a->parent, a->nbr, a->sm(), ratio_fc(a, L), a->solid);
      a->launches += 1;
    }
  }
}

// One coarse step of instance a, launched into stream s (a branch of a batch
// graph that holds every member's step; batch.cu) with the level buffers of
// coarse-step parity `parity`; the instance's stream, buffer parities and
// launch count are left as they were.  Returns the kernels launched.
int64_t coarse_step_into(Instance* a, cudaStream_t s, int parity) {
  const unsigned saved = a->cur;
  cudaStream_t user = a->stream;
  const int prof = a->profiling;
  a->stream = s;
  a->profiling = 0;
  a->cur = (saved & ~1u) | (unsigned)parity;
  const int64_t before = a->launches;
  advance(a, 0, false);
  const int64_t n = a->launches - before;
  a->launches = before;
  a->stream = user;
  a->cur = saved;
  a->profiling = prof;
  return n;
}

static int drain_profile(Instance* a);

static void destroy_graphs(Instance* a) {
  // keep the sample of the last replayed coarse step before its events go
  if (a->profiling == 2 && a->last_parity >= 0) drain_profile(a);
  for (auto& g : a->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  for (auto& v : a->gprof) {
    for (auto& s : v) {
      a->event_pool.push_back(s.start);
      a->event_pool.push_back(s.stop);
    }
    v.clear();
  }
  a->last_parity = -1;
  a->graph_valid = false;
}

static int build_graphs(Handle* h) {
  destroy_graphs(h);
  const unsigned saved = h->cur;
  cudaStream_t user = h->stream;
  h->stream = h->capture_stream;
  for (int parity = 0; parity < 2; ++parity) {
    h->cur = (saved & ~1u) | (unsigned)parity;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      h->capturing = true;
      h->capture_parity = parity;
      const int64_t before = h->launches;
      advance(h, 0, false);
      h->graph_launches[parity] = h->launches - before;
      h->launches = before;
      h->capturing = false;
      e = cudaStreamEndCapture(h->stream, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->stream = user;
      h->cur = saved;
      destroy_graphs(h);
      set_error(std::string("graph capture: ") + cudaGetErrorString(e));
      cudaGetLastError();
      return AMR_E_CUDA;
    }
  }
  h->stream = user;
  h->cur = saved;
  h->graph_valid = true;
  return AMR_OK;
}

// Pre-adapt synchronisation (Section 4.4): average every non-ghost child into
// its parent from the second-finest level up, then interpolate ghosts down.
static void level_sync(Instance* a) {
  for (int L = a->lmax - 2; L >= 0; --L) {
    if (a->n_ids[L + 1] == 0) continue;
    a->ops->average(a->stream, a->idset + (size_t)L * a->cap, (int)a->n_ids[L], true,
                    a->fbuf(L, 0), a->fbuf(L + 1, 0), a->child0, a->parent,
                    a->cellmask, a->status, a->nbr, a->sm(), ratio_fc(a, L), 1, a->solid);
    a->launches += 1;
  }
  for (int L = 0; L + 1 < a->lmax; ++L) {
    if (a->n_parents[L] == 0) continue;
    a->ops->interp(a->stream, a->parents + (size_t)L * a->cap, (int)a->n_parents[L],
                   a->fbuf(L, 0), a->fbuf(L + 1, 0), a->child0, a->cellmask,
                   a->nbr, a->sm(), nullptr, nullptr, ratio_cf(a, L), a->interp_bits(),
                   a->solid);
    a->launches += 1;
  }
}

// Vorticity criterion of every level and the distance rule into a->marks.
static int criterion_into_marks(Instance* a) {
  AMR_CUDA(cudaMemsetAsync(a->marks, 0, a->cap, a->stream));
  for (int L = 0; L < a->lmax; ++L) {
    if (a->n_ids[L] == 0) continue;
    const double inv_dx = a->cfg.nx * std::ldexp(1.0, L) / a->cfg.length_x;
    a->ops->criterion(a->stream, a->idset + (size_t)L * a->cap, (int)a->n_ids[L],
                      a->fbuf(L, 0), a->nbr, a->sm(), a->status, L, a->lmax, inv_dx,
                      a->cfg.crit_start, a->cfg.crit_inc, a->marks, a->w2);
    a->launches += 1;
  }
  AMR_CUDA(cudaGetLastError());
  return mesh_distance_marks(a);
}

// Block summaries of every block in the ID sets into a->features.
static int features_all(Instance* a) {
  if (a->dim != 3) {
    set_error("block summaries are defined for 3D forests");
    return AMR_E_INVAL;
  }
  AMR_CUDA(cudaMemsetAsync(a->features, 0, sizeof(float) * 27 * a->cap, a->stream));
  for (int L = 0; L < a->lmax; ++L) {
    if (a->n_ids[L] == 0) continue;
    const double inv_dx = a->cfg.nx * std::ldexp(1.0, L) / a->cfg.length_x;
    a->ops->features(a->stream, a->idset + (size_t)L * a->cap, (int)a->n_ids[L], a->fbuf(L, 0),
                     a->nbr, a->sm(), L, a->lmax, inv_dx, a->features);
    a->launches += 1;
  }
  AMR_CUDA(cudaGetLastError());
  return AMR_OK;
}

// leaves with probability above the threshold get a refine mark (+1) unless
// they already carry one
__global__ void k_propose(const int32_t* list, int n, const int32_t* status, const float* prob,
                          float threshold, int8_t* marks) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = list[i];
  if (status[b] == 1 && prob[b] > threshold && marks[b] <= 0) marks[b] = 1;
}

__global__ void k_sum_partials(int n, int nv, const double* partial, double* out) {
  __shared__ double s[256];
  for (int v = 0; v < nv; ++v) {
    double x = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x += partial[(size_t)i * nv + v];
    s[threadIdx.x] = x;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[v] = s[0];
    __syncthreads();
  }
}

}  // namespace amr

using namespace amr;

// ====================================================================== ABI
// A kernel whose bounded wait gave up sets this device counter; the next
// synchronising call (amr_adapt, amr_fields to host memory) reports it.
static int take_wait_flag(Instance* a) {
  int32_t v = 0;
  AMR_CUDA(cudaMemcpyAsync(&v, a->dcount + kWaitFlagSlot, sizeof(v), cudaMemcpyDeviceToHost,
                           a->stream));
  AMR_CUDA(cudaStreamSynchronize(a->stream));
  if (v == 0) return AMR_OK;
  AMR_CUDA(cudaMemsetAsync(a->dcount + kWaitFlagSlot, 0, sizeof(int32_t), a->stream));
  set_error("a bounded wait of the persistent batched kernel timed out");
  return AMR_E_TIMEOUT;
}

extern "C" {

const char* amr_strerror(int code) {
  switch (code) {
    case AMR_OK: return "ok";
    case AMR_E_INVAL: return "invalid argument";
    case AMR_E_CAPACITY: return "block capacity exhausted: refinement cancelled";
    case AMR_E_CUDA: return "CUDA error";
    case AMR_E_TIMEOUT: return "bounded device wait timed out";
    case AMR_E_UNSTABLE: return "non-finite mass or momentum";
    case AMR_E_ARENA: return "arena too small or misaligned";
    default: return "unknown error";
  }
}

const char* amr_last_error(void) { return g_last_error.c_str(); }

size_t amr_arena_bytes(const amr_config* cfg) {
  std::string why;
  if (validate(cfg, &why) != AMR_OK) {
    set_error(why);
    return 0;
  }
  return layout_for(cfg).total;
}

int amr_init(const amr_config* cfg, void* arena, size_t arena_bytes, void* stream,
             amr_t** out) {
  std::string why;
  if (!out) return AMR_E_INVAL;
  *out = nullptr;
  if (validate(cfg, &why) != AMR_OK) {
    set_error(why);
    return AMR_E_INVAL;
  }
  const Layout L = layout_for(cfg);
  if (!arena || arena_bytes < L.total || ((uintptr_t)arena & 255u)) {
    set_error("arena needs " + std::to_string(L.total) + " bytes, 256-byte aligned");
    return AMR_E_ARENA;
  }
  Handle* a = new Handle();
  a->arena = (char*)arena;
  a->arena_used = L.total;
  a->cfg = *cfg;
  a->dim = cfg->dim;
  a->q = cfg->q;
  a->M = cfg->dim == 2 ? 16 : 64;
  a->nc = cfg->dim == 2 ? 4 : 8;
  a->nk = cfg->dim == 2 ? 9 : 27;
  a->lmax = cfg->max_levels;
  a->storage = cfg->storage;
  a->cap = cfg->max_blocks;
  a->elem = elem_bytes(cfg->storage);
  a->stream = (cudaStream_t)stream;
  a->solid = cfg->has_solid != 0;
  a->use_graphs = cfg->use_graphs != 0;
  a->nroot[0] = cfg->nx / 4;
  a->nroot[1] = cfg->ny / 4;
  a->nroot[2] = cfg->dim == 3 ? cfg->nz / 4 : 1;
  a->n_root = (int64_t)a->nroot[0] * a->nroot[1] * a->nroot[2];
  a->ops = cfg->dim == 2 ? lbm_ops_d2q9(cfg->storage)
                         : (cfg->q == 19 ? lbm_ops_d3q19(cfg->storage) : lbm_ops_d3q27(cfg->storage));
  if (!a->ops) {
    delete a;
    set_error("no kernels for this velocity set / storage");
    return AMR_E_INVAL;
  }
  char* base = (char*)arena;
  int i = 0;
  a->f[0] = base + L.off[i++];
  a->f[1] = base + L.off[i++];
  a->level = (int32_t*)(base + L.off[i++]);
  a->status = (int32_t*)(base + L.off[i++]);
  a->child0 = (int32_t*)(base + L.off[i++]);
  a->parent = (int32_t*)(base + L.off[i++]);
  a->X = (float*)(base + L.off[i++]);
  a->nbr = (int32_t*)(base + L.off[i++]);
  a->nonemask = (uint32_t*)(base + L.off[i++]);
  a->solidmask = (uint64_t*)(base + L.off[i++]);
  a->idset = (int32_t*)(base + L.off[i++]);
  a->active = (int32_t*)(base + L.off[i++]);
  a->parents = (int32_t*)(base + L.off[i++]);
  a->gap = (int32_t*)(base + L.off[i++]);
  a->marks = (int8_t*)(base + L.off[i++]);
  a->w2 = (double*)(base + L.off[i++]);
  a->tmp0 = (int32_t*)(base + L.off[i++]);
  a->tmp1 = (int32_t*)(base + L.off[i++]);
  a->tmp2 = (int32_t*)(base + L.off[i++]);
  a->cta = (int32_t*)(base + L.off[i++]);
  a->dcount = (int32_t*)(base + L.off[i++]);
  a->red = (double*)(base + L.off[i++]);
  a->wall_code = (int32_t*)(base + L.off[i++]);
  a->staging = base + L.off[i++];
  a->cellmask = (uint64_t*)(base + L.off[i++]);
  a->features = (float*)(base + L.off[i++]);
  a->prob = (float*)(base + L.off[i++]);
  a->order = (int32_t*)(base + L.off[i++]);
  a->bnd = (int32_t*)(base + L.off[i++]);
  a->agrp = (int32_t*)(base + L.off[i++]);

  const double tau0 = 3.0 * cfg->nu0 + 0.5;
  for (int l = 0; l < a->lmax; ++l) a->tau[l] = 0.5 + std::ldexp(tau0 - 0.5, l);

  // boundary tables: wall code of every set of crossed faces, bounce-back terms
  static const int rank_of[4] = {1, 2, 3, 0};
  int32_t codes[64];
  for (int m = 0; m < 64; ++m) {
    int best = -1, br = 0;
    for (int f = 0; f < 6; ++f)
      if ((m >> f) & 1) {
        const int r = rank_of[cfg->faces[f].kind];
        if (r > br) { br = r; best = f; }
      }
    codes[m] = best >= 0 ? -2 - best : NONE;
  }
  int c[27][3];
  double w[27];
  host_velocities(a->dim, a->q, c, w);
  std::memset(&a->prm, 0, sizeof(a->prm));
  a->prm.variant = cfg->kernel_variant;
  a->prm.wait_flag = a->dcount + kWaitFlagSlot;
  if (a->ops->setup() != 0) {
    set_error(std::string("kernel setup: ") + cudaGetErrorString(cudaGetLastError()));
    delete a;
    return AMR_E_CUDA;
  }
  for (int f = 0; f < 6; ++f) {
    const amr_face& fc = cfg->faces[f];
    a->prm.faces.kind[f] = fc.kind;
    const double rho_w = fc.rho_w > 0 ? fc.rho_w : 1.0;
    a->prm.faces.rho_w[f] = rho_w;
    for (int p = 0; p < a->q; ++p) {
      const double cu = c[p][0] * fc.u[0] + c[p][1] * fc.u[1] + (a->dim == 3 ? c[p][2] * fc.u[2] : 0.0);
      a->prm.faces.bb[f][p] = fc.kind == AMR_FACE_MOVING ? -2.0 * w[p] * rho_w * cu * 3.0 : 0.0;
    }
  }
  int rc = AMR_OK;
  if (cudaStreamCreateWithFlags(&a->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("cannot create capture stream");
    delete a;
    return AMR_E_CUDA;
  }
  if (cudaMemcpyAsync(a->wall_code, codes, sizeof(codes), cudaMemcpyHostToDevice, a->stream) !=
      cudaSuccess) {
    set_error("wall code upload failed");
    rc = AMR_E_CUDA;
  }
  if (rc == AMR_OK && cudaMemsetAsync(a->dcount, 0, 64 * sizeof(int32_t), a->stream) != cudaSuccess) {
    set_error("counter reset failed");
    rc = AMR_E_CUDA;
  }
  if (rc == AMR_OK) {
    a->ops->init_rest(a->stream, a->cap, a->f[0]);
    a->ops->init_rest(a->stream, a->cap, a->f[1]);
    rc = mesh_init_root(a);
    a->cfg.root_ids = nullptr;   // read by amr_init only
  }
  if (rc == AMR_OK && cudaStreamSynchronize(a->stream) != cudaSuccess) {
    set_error(std::string("init: ") + cudaGetErrorString(cudaGetLastError()));
    rc = AMR_E_CUDA;
  }
  if (rc == AMR_OK && cfg->check_tables) {
    int64_t res[3];
    rc = check_instance_tables(a, res);
  }
  if (rc != AMR_OK) {
    cudaStreamDestroy(a->capture_stream);
    delete a;
    return rc;
  }
  *out = reinterpret_cast<amr_t*>(a);
  return AMR_OK;
}

int amr_check_tables(amr_t* h, int64_t* out3) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a || !out3) return AMR_E_INVAL;
  return check_instance_tables(a, out3);
}

int amr_step(amr_t* h, int n) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a || n < 0) return AMR_E_INVAL;
  const bool graphs = a->use_graphs && a->profiling != 1;
  if (graphs && !a->graph_valid) {
    int rc = build_graphs(a);
    if (rc != AMR_OK) return rc;
  }
  for (int s = 0; s < n; ++s) {
    if (graphs) {
      const int parity = (int)(a->cur & 1u);
      AMR_CUDA(cudaGraphLaunch(a->graph[parity], a->stream));
      a->launches += a->graph_launches[parity];
      a->last_parity = parity;
      a->cur ^= 1u;   // levels >= 1 flip an even number of times per coarse step
    } else {
      advance(a, 0, false);
    }
    a->coarse_steps += 1;
  }
  AMR_CUDA(cudaGetLastError());
  return AMR_OK;
}

int amr_adapt(amr_t* h, const int8_t* dev_marks, amr_adapt_stats* out) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a) return AMR_E_INVAL;
  const auto t0 = std::chrono::steady_clock::now();
  amr_adapt_stats st{};
  adapt_phase(a, PK_ADAPT_SYNC);
  level_sync(a);
  adapt_phase(a, PK_ADAPT_CRITERION);
  if (dev_marks) {
    AMR_CUDA(cudaMemcpyAsync(a->marks, dev_marks, a->cap, cudaMemcpyDeviceToDevice, a->stream));
  } else {
    const int crc = criterion_into_marks(a);
    if (crc != AMR_OK) return crc;
  }
  AMR_CUDA(cudaGetLastError());
  adapt_phase(a, PK_ADAPT_MARKS);
  int rc = mesh_adapt(a, dev_marks != nullptr, &st);
  adapt_phase(a, -1);
  if (rc != AMR_OK) return rc;
  destroy_graphs(a);
  AMR_CUDA(cudaStreamSynchronize(a->stream));
  harvest_phases(a);
  if (int wrc = take_wait_flag(a)) return wrc;
  if (a->cfg.check_tables) {
    int64_t res[3];
    if (int crc = check_instance_tables(a, res)) return crc;
  }
  int64_t nb = 0;
  for (int L = 0; L < a->lmax; ++L) nb += a->n_ids[L];
  st.n_blocks = nb;
  st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (out) *out = st;
  return st.capacity_error ? AMR_E_CAPACITY : AMR_OK;
}

int64_t amr_fields(amr_t* h, int what, void* dst, size_t dst_bytes, int dst_on_device) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a) return AMR_E_INVAL;
  const int64_t cap = a->cap;
  const int M = a->M, D = a->dim, Q = a->q;
  int64_t need = -1;
  switch (what) {
    case AMR_RHO_U: need = cap * M * (1 + D) * 8; break;
    case AMR_F: need = cap * M * Q * 8; break;
    case AMR_COUNTS: need = (4 + 4 * (int64_t)a->lmax) * 8; break;
    case AMR_MASS: need = (1 + D) * 8; break;
    case AMR_FORCE: need = 3 * 8; break;
    case AMR_FEATURES: need = cap * 27 * 4; break;
    default: need = mesh_export_bytes(a, what);
  }
  if (need < 0) {
    set_error("unknown field selector");
    return AMR_E_INVAL;
  }
  if (!dst) return need;
  if (!dst_on_device)
    if (int wrc = take_wait_flag(a)) return wrc;
  if ((int64_t)dst_bytes < need) {
    set_error("destination too small: need " + std::to_string(need) + " bytes");
    return AMR_E_INVAL;
  }
  cudaStream_t s = a->stream;
  if (what == AMR_COUNTS) {
    std::vector<int64_t> c(4 + 4 * a->lmax, 0);
    c[0] = a->lmax;
    c[1] = a->n_gaps;
    c[2] = a->coarse_steps;
    c[3] = a->launches;
    for (int L = 0; L < a->lmax; ++L) {
      c[4 + 4 * L] = a->n_ids[L];
      c[5 + 4 * L] = a->n_active[L];
      c[6 + 4 * L] = a->n_leaves[L];
      c[7 + 4 * L] = a->n_parents[L];
    }
    if (dst_on_device) {
      AMR_CUDA(cudaMemcpyAsync(dst, c.data(), need, cudaMemcpyHostToDevice, s));
      AMR_CUDA(cudaStreamSynchronize(s));
    } else {
      std::memcpy(dst, c.data(), need);
    }
    return need;
  }
  if (what == AMR_MASS || what == AMR_FORCE) {
    double* out_dev = a->red + 8000;
    if (what == AMR_MASS) {
      const int g = a->ops->mass_partial(s, cap, a->f[0], a->f[1], a->cur, a->level, a->status,
                                         a->nbr, a->sm(), a->red);
      k_sum_partials<<<1, 256, 0, s>>>(g, 4, a->red, out_dev);
    } else {
      AMR_CUDA(cudaMemsetAsync(out_dev + 4, 0, 3 * 8, s));
      double* acc = out_dev + 8;
      AMR_CUDA(cudaMemsetAsync(acc, 0, 3 * 8, s));
      std::vector<double> tot(3, 0.0), part(3);
      for (int L = 0; L < a->lmax; ++L) {
        if (a->n_active[L] == 0 || !a->solid) continue;
        const double dx = a->cfg.length_x / (a->cfg.nx * std::ldexp(1.0, L));
        const int g = a->ops->force_partial(s, a->active + (size_t)L * cap, (int)a->n_active[L],
                                            a->fbuf(L, 0), a->nbr, a->status,
                                            a->solidmask, 1.0 / a->tau[L], dx, a->red);
        k_sum_partials<<<1, 256, 0, s>>>(g, 3, a->red, out_dev + 4);
        AMR_CUDA(cudaMemcpyAsync(part.data(), out_dev + 4, 24, cudaMemcpyDeviceToHost, s));
        AMR_CUDA(cudaStreamSynchronize(s));
        for (int v = 0; v < 3; ++v) tot[v] += part[v];
      }
      AMR_CUDA(cudaMemcpyAsync(out_dev, tot.data(), 24, cudaMemcpyHostToDevice, s));
    }
    AMR_CUDA(cudaGetLastError());
    AMR_CUDA(cudaMemcpyAsync(dst, out_dev, need,
                             dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    AMR_CUDA(cudaStreamSynchronize(s));
    if (what == AMR_MASS) {
      double hv[4] = {0, 0, 0, 0};
      if (dst_on_device) {
        AMR_CUDA(cudaMemcpy(hv, out_dev, need, cudaMemcpyDeviceToHost));
      } else {
        std::memcpy(hv, dst, need);
      }
      for (int v = 0; v <= D; ++v)
        if (!std::isfinite(hv[v])) {
          set_error("mass audit found a non-finite value");
          return AMR_E_UNSTABLE;
        }
    }
    return need;
  }
  if (what == AMR_FEATURES) {
    level_sync(a);
    const int frc = features_all(a);
    if (frc != AMR_OK) return frc;
    if (dst_on_device) {
      AMR_CUDA(cudaMemcpyAsync(dst, a->features, need, cudaMemcpyDeviceToDevice, s));
    } else {
      AMR_CUDA(cudaMemcpyAsync(dst, a->features, need, cudaMemcpyDeviceToHost, s));
      AMR_CUDA(cudaStreamSynchronize(s));
    }
    return need;
  }
  if (what == AMR_RHO_U) level_sync(a);
  if (dst_on_device) {
    if (what == AMR_RHO_U) {
      a->ops->export_rho_u(s, cap, 0, cap, a->f[0], a->f[1], a->cur, a->level, a->nbr, a->sm(),
                           (double*)dst);
    } else if (what == AMR_F) {
      a->ops->export_f(s, cap, 0, cap, a->f[0], a->f[1], a->cur, a->level, a->nbr, a->sm(),
                       (double*)dst);
    } else {
      int rc = mesh_export(a, what, dst);
      if (rc != AMR_OK) return rc;
    }
    AMR_CUDA(cudaGetLastError());
    return need;
  }
  // host destination: through the staging area of the arena, in block chunks
  if (what == AMR_RHO_U || what == AMR_F) {
    const int64_t per_block = (int64_t)M * (what == AMR_F ? Q : 1 + D) * 8;
    const int64_t chunk = std::max<int64_t>(1, (int64_t)STAGING_BYTES / per_block);
    for (int64_t b0 = 0; b0 < cap; b0 += chunk) {
      const int64_t nb = std::min(chunk, cap - b0);
      double* st = (double*)a->staging;
      if (what == AMR_RHO_U) {
        a->ops->export_rho_u(s, cap, b0, nb, a->f[0], a->f[1], a->cur, a->level, a->nbr, a->sm(),
                             st);
        AMR_CUDA(cudaMemcpyAsync((char*)dst + b0 * per_block, st, nb * per_block,
                                 cudaMemcpyDeviceToHost, s));
      } else {
        a->ops->export_f(s, cap, b0, nb, a->f[0], a->f[1], a->cur, a->level, a->nbr, a->sm(), st);
        AMR_CUDA(cudaMemcpy2DAsync((char*)dst + b0 * M * 8, (size_t)cap * M * 8, st,
                                   (size_t)nb * M * 8, (size_t)nb * M * 8, Q,
                                   cudaMemcpyDeviceToHost, s));
      }
      AMR_CUDA(cudaGetLastError());
      AMR_CUDA(cudaStreamSynchronize(s));
    }
    return need;
  }
  if (what == AMR_NBR) {
    AMR_CUDA(cudaMemcpy2DAsync(dst, a->nk * 4, a->nbr, NBR_STRIDE * 4, a->nk * 4, cap,
                               cudaMemcpyDeviceToHost, s));
    AMR_CUDA(cudaStreamSynchronize(s));
    return need;
  }
  if (what == AMR_BLOCKS || what == AMR_IDSETS || what == AMR_GAPS) {
    const int32_t* srcs[4] = {a->level, a->status, a->child0, a->parent};
    if (what == AMR_BLOCKS) {
      for (int k = 0; k < 4; ++k)
        AMR_CUDA(cudaMemcpyAsync((int32_t*)dst + k * cap, srcs[k], cap * 4, cudaMemcpyDeviceToHost, s));
    } else {
      AMR_CUDA(cudaMemcpyAsync(dst, what == AMR_IDSETS ? a->idset : a->gap, need,
                               cudaMemcpyDeviceToHost, s));
    }
    AMR_CUDA(cudaStreamSynchronize(s));
    return need;
  }
  // remaining small tables: export into staging in one piece when it fits
  if (need > (int64_t)STAGING_BYTES) {
    set_error("table larger than the staging area: use a device destination");
    return AMR_E_INVAL;
  }
  int rc = mesh_export(a, what, a->staging);
  if (rc != AMR_OK) return rc;
  AMR_CUDA(cudaMemcpyAsync(dst, a->staging, need, cudaMemcpyDeviceToHost, s));
  AMR_CUDA(cudaStreamSynchronize(s));
  return need;
}

int amr_set_fields(amr_t* h, int what, const void* src, size_t src_bytes, int src_on_device) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a || what != AMR_F || !src) return AMR_E_INVAL;
  const int64_t cap = a->cap;
  const int M = a->M, Q = a->q;
  const int64_t need = cap * M * Q * 8;
  if ((int64_t)src_bytes < need) {
    set_error("source too small");
    return AMR_E_INVAL;
  }
  cudaStream_t s = a->stream;
  if (src_on_device) {
    a->ops->import_f(s, cap, 0, cap, a->f[0], a->f[1], a->cur, a->level, a->nbr, a->sm(),
                     (const double*)src);
  } else {
    const int64_t per_block = (int64_t)M * Q * 8;
    const int64_t chunk = std::max<int64_t>(1, (int64_t)STAGING_BYTES / per_block);
    for (int64_t b0 = 0; b0 < cap; b0 += chunk) {
      const int64_t nb = std::min(chunk, cap - b0);
      double* st = (double*)a->staging;
      AMR_CUDA(cudaMemcpy2DAsync(st, (size_t)nb * M * 8, (const char*)src + b0 * M * 8,
                                 (size_t)cap * M * 8, (size_t)nb * M * 8, Q,
                                 cudaMemcpyHostToDevice, s));
      a->ops->import_f(s, cap, b0, nb, a->f[0], a->f[1], a->cur, a->level, a->nbr, a->sm(), st);
      AMR_CUDA(cudaGetLastError());
      AMR_CUDA(cudaStreamSynchronize(s));
    }
  }
  AMR_CUDA(cudaGetLastError());
  return AMR_OK;
}

int amr_criterion_marks(amr_t* h, int8_t* dev_marks) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a || !dev_marks) return AMR_E_INVAL;
  level_sync(a);
  const int rc = criterion_into_marks(a);
  if (rc != AMR_OK) return rc;
  AMR_CUDA(cudaMemcpyAsync(dev_marks, a->marks, a->cap, cudaMemcpyDeviceToDevice, a->stream));
  AMR_CUDA(cudaStreamSynchronize(a->stream));
  return AMR_OK;
}

int amr_propose_marks(amr_t* h, const void* params_half, float threshold, int with_criterion,
                      int8_t* dev_marks) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a || !params_half || !dev_marks) return AMR_E_INVAL;
  level_sync(a);
  int rc = with_criterion ? criterion_into_marks(a) : AMR_OK;
  if (rc != AMR_OK) return rc;
  if (!with_criterion) AMR_CUDA(cudaMemsetAsync(a->marks, 0, a->cap, a->stream));
  rc = features_all(a);
  if (rc != AMR_OK) return rc;
  for (int L = 0; L < a->lmax; ++L) {
    const int64_t n = a->n_ids[L];
    if (n == 0) continue;
    const int32_t* ids = a->idset + (size_t)L * a->cap;
    mlp_infer_list(a->stream, params_half, a->features, ids, n, a->prob);
    k_propose<<<(int)((n + 255) / 256), 256, 0, a->stream>>>(ids, (int)n, a->status, a->prob,
                                                             threshold, a->marks);
    a->launches += 2;
  }
  AMR_CUDA(cudaGetLastError());
  AMR_CUDA(cudaMemcpyAsync(dev_marks, a->marks, a->cap, cudaMemcpyDeviceToDevice, a->stream));
  AMR_CUDA(cudaStreamSynchronize(a->stream));
  return AMR_OK;
}

int amr_profile(amr_t* h, int mode) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a || mode < 0 || mode > 2) return AMR_E_INVAL;
  int rc = drain_profile(a);
  if (rc != AMR_OK) return rc;
  if (mode != a->profiling) destroy_graphs(a);
  a->profiling = mode;
  return AMR_OK;
}

int amr_profile_read(amr_t* h, amr_kernel_profile* out, int max, int reset) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a) return AMR_E_INVAL;
  int rc = drain_profile(a);
  if (rc != AMR_OK) return rc;
  for (int k = 0; k < PK_COUNT && k < max; ++k) {
    std::memset(&out[k], 0, sizeof(out[k]));
    std::snprintf(out[k].name, sizeof(out[k].name), "%s", kPkNames[k]);
    out[k].launches = a->acc[k].launches;
    out[k].ms = a->acc[k].ms;
    out[k].bytes = a->acc[k].bytes;
    out[k].cells = a->acc[k].cells;
  }
  if (reset)
    for (auto& acc : a->acc) acc = Instance::Acc{};
  return PK_COUNT;
}

int64_t amr_checkpoint_bytes(amr_t* h) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a) return AMR_E_INVAL;
  return (int64_t)(sizeof(CheckpointHeader) + a->arena_used);
}

int amr_checkpoint(amr_t* h, void* dst, size_t dst_bytes) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a || !dst || dst_bytes < sizeof(CheckpointHeader) + a->arena_used) {
    set_error("checkpoint destination missing or smaller than amr_checkpoint_bytes");
    return AMR_E_INVAL;
  }
  drain_profile(a);
  CheckpointHeader hd{};
  std::memcpy(hd.tag, kCheckpointTag, sizeof(hd.tag));
  hd.dim = a->cfg.dim;
  hd.q = a->cfg.q;
  hd.storage = a->cfg.storage;
  hd.nx = a->cfg.nx;
  hd.ny = a->cfg.ny;
  hd.nz = a->cfg.nz;
  hd.max_levels = a->cfg.max_levels;
  hd.max_blocks = a->cfg.max_blocks;
  hd.arena_used = a->arena_used;
  for (int L = 0; L < AMR_MAX_LEVELS; ++L) {
    hd.n_ids[L] = a->n_ids[L];
    hd.n_active[L] = a->n_active[L];
    hd.n_parents[L] = a->n_parents[L];
    hd.n_leaves[L] = a->n_leaves[L];
    hd.n_bnd[L] = a->n_bnd[L];
    hd.n_agrp[L] = a->n_agrp[L];
    hd.agrp_off[L] = a->agrp_off[L];
    hd.n_ghost_children[L] = a->n_ghost_children[L];
    hd.n_ghost_cells[L] = a->n_ghost_cells[L];
    hd.n_iface_cells[L] = a->n_iface_cells[L];
  }
  hd.n_gaps = a->n_gaps;
  hd.coarse_steps = a->coarse_steps;
  hd.cur = a->cur;
  AMR_CUDA(cudaStreamSynchronize(a->stream));
  std::memcpy(dst, &hd, sizeof(hd));
  AMR_CUDA(cudaMemcpy((char*)dst + sizeof(hd), a->arena, a->arena_used, cudaMemcpyDeviceToHost));
  return AMR_OK;
}

int amr_restore(amr_t* h, const void* src, size_t src_bytes) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a || !src || src_bytes < sizeof(CheckpointHeader)) {
    set_error("checkpoint image missing or truncated");
    return AMR_E_INVAL;
  }
  CheckpointHeader hd;
  std::memcpy(&hd, src, sizeof(hd));
  const bool same = std::memcmp(hd.tag, kCheckpointTag, sizeof(hd.tag)) == 0 &&
                    hd.dim == a->cfg.dim && hd.q == a->cfg.q && hd.storage == a->cfg.storage &&
                    hd.nx == a->cfg.nx && hd.ny == a->cfg.ny && hd.nz == a->cfg.nz &&
                    hd.max_levels == a->cfg.max_levels && hd.max_blocks == a->cfg.max_blocks &&
                    hd.arena_used == a->arena_used &&
                    src_bytes >= sizeof(hd) + a->arena_used;
  if (!same) {
    set_error("checkpoint image does not match this instance's configuration");
    return AMR_E_INVAL;
  }
  drain_profile(a);
  destroy_graphs(a);
  AMR_CUDA(cudaStreamSynchronize(a->stream));
  AMR_CUDA(cudaMemcpy(a->arena, (const char*)src + sizeof(hd), a->arena_used,
                      cudaMemcpyHostToDevice));
  for (int L = 0; L < AMR_MAX_LEVELS; ++L) {
    a->n_ids[L] = hd.n_ids[L];
    a->n_active[L] = hd.n_active[L];
    a->n_parents[L] = hd.n_parents[L];
    a->n_leaves[L] = hd.n_leaves[L];
    a->n_bnd[L] = hd.n_bnd[L];
    a->n_agrp[L] = hd.n_agrp[L];
    a->agrp_off[L] = hd.agrp_off[L];
    a->n_ghost_children[L] = hd.n_ghost_children[L];
    a->n_ghost_cells[L] = hd.n_ghost_cells[L];
    a->n_iface_cells[L] = hd.n_iface_cells[L];
  }
  a->n_gaps = hd.n_gaps;
  a->coarse_steps = hd.coarse_steps;
  a->cur = hd.cur;
  return AMR_OK;
}

int amr_free(amr_t* h) {
  Handle* a = reinterpret_cast<Handle*>(h);
  if (!a) return AMR_E_INVAL;
  drain_profile(a);
  destroy_graphs(a);
  for (auto e : a->event_pool) cudaEventDestroy(e);
  if (a->capture_stream) cudaStreamDestroy(a->capture_stream);
  delete a;
  return AMR_OK;
}

}  // extern "C"
