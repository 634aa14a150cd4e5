// Internal state of one AMR-LBM instance and the mesh-adaptation entry points
// shared between the translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/amr.h"
#include "lbm_ops.h"

namespace amr {

void set_error(const std::string& msg);

struct ProfileSlot {
  cudaEvent_t start, stop;
  int kind;
  double bytes, cells;
};

struct Instance {
  amr_config cfg{};
  int dim = 0, q = 0, M = 0, nc = 0, nk = 0, lmax = 0, storage = 0;
  int64_t cap = 0, n_root = 0;
  int nroot[3] = {1, 1, 1};
  size_t elem = 0;                 // bytes per stored population
  cudaStream_t stream = nullptr;
  const LbmOps* ops = nullptr;
  bool solid = false;

  // device arrays carved from the caller's arena
  void* f[2] = {nullptr, nullptr};
  int32_t *level = nullptr, *status = nullptr, *child0 = nullptr, *parent = nullptr;
  float* X = nullptr;              // [cap][3] block corners, root-cell units
  int32_t* nbr = nullptr;          // [cap][NBR_STRIDE]
  uint32_t* nonemask = nullptr;    // bit k set when nbr[b][k] == NONE
  uint64_t* solidmask = nullptr;   // bit l set when cell l is solid
  uint64_t* cellmask = nullptr;    // [cap][2]: ghost cells, interface cells (bit l)
  float* features = nullptr;       // [cap][27] block summaries
  float* prob = nullptr;           // [cap] proposal probabilities
  int32_t *idset = nullptr, *active = nullptr, *parents = nullptr;   // [lmax][cap]
  // [lmax][cap]: the blocks of each level in tree order -- roots by position
  // (x fastest), then the children of each refined block in child order; the
  // active and parent lists are taken from it, so blocks that are neighbours
  // in space are advanced close together in time whatever their IDs
  int32_t* order = nullptr;
  int32_t* bnd = nullptr;          // [lmax][cap]: blocks with a NONE neighbour, tree order
  int32_t* agrp = nullptr;         // [cap * N_c]: averaging groups (block << 3 | group) of
                                   // the boundary blocks, level L at agrp_off[L]
  int32_t* gap = nullptr;          // [cap]
  int8_t* marks = nullptr;         // [cap]
  double* w2 = nullptr;            // [cap] criterion block maxima
  int32_t *tmp0 = nullptr, *tmp1 = nullptr, *tmp2 = nullptr;   // [cap]
  int32_t* cta = nullptr;          // [cta_slots(cap)]
  int32_t* dcount = nullptr;       // [64] device counters
  double* red = nullptr;           // [8192] reduction partials
  int32_t* wall_code = nullptr;    // [64] code of a set of crossed faces

  // host mirror of the mesh sizes and time-stepping state
  int64_t n_ids[AMR_MAX_LEVELS] = {}, n_active[AMR_MAX_LEVELS] = {},
          n_parents[AMR_MAX_LEVELS] = {}, n_leaves[AMR_MAX_LEVELS] = {},
          n_bnd[AMR_MAX_LEVELS] = {}, n_agrp[AMR_MAX_LEVELS] = {},
          agrp_off[AMR_MAX_LEVELS] = {};
  // per level L: over the children of level L's exchanging parents, the
  // children holding ghost cells, their ghost cells and their interface cells
  // (the algorithmic work of interpolation into and averaging from level L+1)
  int64_t n_ghost_children[AMR_MAX_LEVELS] = {}, n_ghost_cells[AMR_MAX_LEVELS] = {},
          n_iface_cells[AMR_MAX_LEVELS] = {};
  int64_t n_gaps = 0;
  int64_t coarse_steps = 0;
  int64_t launches = 0;            // kernels launched by this instance
  int64_t graph_launches[2] = {0, 0};   // kernels per captured coarse step
  unsigned cur = 0;                // bit L: current population buffer of level L
  double tau[AMR_MAX_LEVELS] = {};
  StepParams prm{};

  // CUDA graphs of one coarse step, one per parity of level 0
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graph_valid = false;
  bool use_graphs = true;

  // profiling: 1 = events around every launch (graphs off); 2 = events captured
  // inside the graphs, the last replayed coarse step sampled on each read
  int profiling = 0;
  bool capturing = false;
  int capture_parity = 0;
  int last_parity = -1;
  std::vector<ProfileSlot> prof;
  std::vector<ProfileSlot> gprof[2];
  std::vector<cudaEvent_t> event_pool;
  struct Acc { int64_t launches = 0; double ms = 0, bytes = 0, cells = 0; };
  Acc acc[16];
  // adaptation phase boundaries of the current amr_adapt call (profiling on)
  std::vector<std::pair<int, cudaEvent_t>> phase_marks;

  // solid-cell bits for the kernels (null: no solid cells in this instance)
  const uint64_t* sm() const { return solid ? solidmask : nullptr; }
  // interpolation mode bit of LbmOps::interp for this configuration
  int interp_bits() const { return cfg.interp == AMR_INTERP_CUBIC ? 2 : 0; }
  size_t f_bytes() const { return (size_t)cap * M * q * elem; }
  void* fbuf(int level, int which) const {   // which: 0 current, 1 other
    return f[((cur >> level) & 1u) ^ (unsigned)which];
  }
};

// dcount slot of the device wait-timeout flag (StepParams::wait_flag)
constexpr int kWaitFlagSlot = 16;
// entries of the compaction's per-CTA count array: one per 256 items of the
// longest compaction, the averaging groups of every block (8 per block)
inline int64_t cta_slots(int64_t cap) { return cap * 8 / 256 + 2; }

// api.cu: one coarse step of `a` (its own fused kernels) launched into `s`
// with the buffers of coarse-step parity `parity`; returns the launches
int64_t coarse_step_into(Instance* a, cudaStream_t s, int parity);

// check.cu: validate the instance's block tables, lists and averaging groups
// (amr_check_tables); out3 as there
int check_instance_tables(Instance* a, int64_t* out3);

enum ProfileKind {
  PK_COLLIDE = 0, PK_INTERP = 1, PK_AVERAGE = 2,
  // phases of an adaptation (the paper's Pre and S1-S8 grouped by what runs
  // here): synchronisation, criterion, marks with 2:1 enforcement, ID
  // allocation and gap pushes, ID sets, relinking, new children, level lists
  PK_ADAPT_SYNC = 3, PK_ADAPT_CRITERION = 4, PK_ADAPT_MARKS = 5, PK_ADAPT_ALLOC = 6,
  PK_ADAPT_IDSETS = 7, PK_ADAPT_RELINK = 8, PK_ADAPT_CHILDREN = 9, PK_ADAPT_LISTS = 10,
  PK_COUNT = 11
};

// Start adaptation phase `kind` (a PK_ADAPT_* value; -1 closes the last one):
// records an event on the stream when profiling is on, else does nothing.
void adapt_phase(Instance* a, int kind);

// mesh.cu
int mesh_init_root(Instance* a);
int mesh_adapt(Instance* a, bool external, amr_adapt_stats* st);
int mesh_export(Instance* a, int what, void* dst_dev);
int mesh_refresh_lists(Instance* a);
int mesh_distance_marks(Instance* a);
// mlp.cu
void mlp_infer_list(cudaStream_t s, const void* params_half, const float* x, const int32_t* list,
                    int64_t n, float* prob);
int64_t mesh_export_bytes(const Instance* a, int what);

#define AMR_CUDA(call)                                                             \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ::amr::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));       \
      return AMR_E_CUDA;                                                           \
    }                                                                              \
  } while (0)

}  // namespace amr
