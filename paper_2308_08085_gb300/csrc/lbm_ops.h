// Host-side interface to the per-velocity-set LBM kernels.  Each translation
// unit lbm_*.cu instantiates the kernels of one velocity set for its storage
// types and returns a table of launchers.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace amr {

struct FaceParams {
  int32_t kind[6];      // AMR_FACE_*
  double rho_w[6];
  double bb[6][27];     // bounce-back term -2 w_p rho_w (c_p . u_w) / cs^2
};

// Descriptor of one instance inside a batch (Section 4.1 level step applied to
// many forests in lock-step).  Work items pack inst << BATCH_SHIFT | block.
constexpr int BATCH_SHIFT = 25;
constexpr uint32_t BATCH_MASK = (1u << BATCH_SHIFT) - 1u;
constexpr int BATCH_MAX_LEVELS = 8;

struct InstDesc {
  void* f[2];                       // population buffers A / B
  const int32_t* nbr;
  const int32_t* child0;
  const uint64_t* cellmask;
  double omega[BATCH_MAX_LEVELS];   // 1 / tau_L
  double r_cf[BATCH_MAX_LEVELS];    // tau_{L+1} / (2 tau_L)
  double r_fc[BATCH_MAX_LEVELS];    // 2 tau_L / tau_{L+1}
  FaceParams faces;
  int32_t* wait_flag;               // the member's device wait-timeout flag
};

// The persistent form of the batched level step: one launch advances every
// member by n_steps coarse steps.  The recursive level step (Section 4.1) is
// unrolled on the host into a list of phases (interpolation into level L+1,
// collide-stream of level L, averaging of level L+1 into L), the same list
// for every member; the items of a phase are cut into tiles of one member
// each.  CTAs take tiles in queue order (step, phase, member, tile) from one
// counter, and a tile first waits until its member has completed the
// member's previous phase that has tiles: each member advances on its own,
// with no grid-wide barrier.  A tile only waits for tiles taken before it and
// a CTA holds one tile at a time, so the earliest unfinished tile can always
// run whatever the number of resident CTAs.
constexpr int PH_INTERP = 0;
constexpr int PH_COLLIDE = 1;
constexpr int PH_AVERAGE = 2;
constexpr int PERSIST_MAX_TILE = 8;    // blocks per collide-stream tile (M_L)

struct PersistPhase {
  int32_t op, level;
  int32_t which_in;       // buffer of level L (collide input; interpolation / averaging parent)
  int32_t which_ch;       // buffer of level L + 1 (interpolation / averaging children)
  int32_t tile0;          // first tile of the phase within a coarse step
  int32_t n_tiles;
  const uint32_t* items;  // the phase's instance-major item list (active blocks or parents)
};

struct PersistArgs {
  const InstDesc* descs;
  const PersistPhase* phases;   // [2][n_phase]: steps starting with cur bit 0 clear / set
  const int32_t* tile_off;      // [n_phase][n_inst + 1]: first tile of each member
  const int32_t* item_off;      // [n_phase][n_inst + 1]: first item of each member
  const int32_t* dep;           // [n_phase][n_inst]: 2 k + wrap, the member's previous phase
                                // with tiles (wrap: in the previous coarse step)
  uint32_t* done;               // [n_phase][n_inst]: tiles completed, summed over the launch
  unsigned long long* head;     // queue head
  int32_t* abort;               // raised when a wait gave up; sticky until read by the host
  int n_phase, n_inst, tiles_per_step, parity0, n_steps, tile_blocks;
  long long wait_limit;         // clock64 cycles a tile may wait
  int stall;                    // check of the timeout path: no wait can be satisfied
};

// The coarse-to-fine interpolation of the level step (Section 4.1) fused
// into the collide-stream of a level's exchanging parent blocks: every parent
// cell's pre-collision value, rescaled to the fine level, goes to shared
// memory, and the ghost cells of its children are interpolated (Section
// 3.4.1) into their own slots of the fine output buffer, where their first
// substep reads them.
struct Exchange {
  void* fine_out;              // the fine level's output buffer
  const int32_t* child0;
  const uint64_t* cellmask;    // [2 b]: ghost cells, [2 b + 1]: interface cells
  double r_cf;                 // coarse -> fine rescale, tau_F / (2 tau_C)
};

struct StepParams {
  double omega;         // 1 / tau_L
  int variant;          // collide-stream kernel variant (amr_config.kernel_variant)
  FaceParams faces;
  int32_t* wait_flag;   // device int set to 1 by a kernel whose bounded wait gave up
};

// Every kernel reads the populations of a cell through the gather and writes
// them through the scatter of collide_stream.cuh, so the neighbour table
// (`nbr`, NBR_STRIDE int32 per block) and the solid-cell bits (`solidmask`,
// one uint64 per block, null when the instance has no solid cells) go with
// every population buffer.
struct LbmOps {
  // one-time kernel attributes (SM count); call outside any stream capture
  int (*setup)();
  // fused BGK collision + pull streaming over `list` (active blocks of a level)
  // (ghostmask: the first substep of a level below the coarsest -- its ghost
  // cells read their interpolated pre-collision values from their own slots
  // of fout, see interp mode bit 2; null otherwise)
  // xchg: null, or the exchange with the next finer level fused into the
  // parent blocks of this level (linear interpolation only)
  void (*collide_stream)(cudaStream_t, const int32_t* list, int n, const void* fin, void* fout,
                         const int32_t* nbr, const uint64_t* solidmask, const StepParams& prm,
                         bool solid, const uint64_t* ghostmask, const Exchange* xchg);
  // coarse-to-fine interpolation: parents in `list`, into their children
  // (mode bit 0: every cell of new children, else their ghost cells; bit 1:
  // cubic instead of linear interpolation; bit 2, the level step: the ghost
  // values are written as they are into the ghost cells' own slots of `fch`,
  // the children's output buffer, for their next collide-stream to read,
  // instead of being scattered into the stored form).  With bit 0, `parent`
  // and `marks` (> 0: refined in this adaptation) tell new blocks from old.
  void (*interp)(cudaStream_t, const int32_t* list, int n, const void* fpar, void* fch,
                 const int32_t* child0, const uint64_t* cellmask,
                 const int32_t* nbr, const uint64_t* solidmask, const int32_t* parent,
                 const int8_t* marks, double ratio, int mode, bool solid);
  // fine-to-coarse averaging: by_parent -- `list` holds parents, all their
  // children are visited; else `list` holds children (boundary blocks of the
  // fine level) and parent[] leads to their parents.  mode 0: parent cells
  // over interface children, 1: over every non-ghost child (refined parents)
  void (*average)(cudaStream_t, const int32_t* list, int n, bool by_parent, void* fpar,
                  const void* fch, const int32_t* child0, const int32_t* parent,
                  const uint64_t* cellmask, const int32_t* status, const int32_t* nbr,
                  const uint64_t* solidmask, double ratio, int mode_sync, bool solid);
  // the averaging of the level step over (block << 3 | group) items: the
  // groups of 2^D interface cells of the fine level's boundary blocks, each
  // into its parent cell (the work of average mode 0, listed in advance)
  void (*average_groups)(cudaStream_t, const int32_t* items, int n, void* fpar, const void* fch,
                         const int32_t* child0, const int32_t* parent,
                         const int32_t* nbr, const uint64_t* solidmask, double ratio,
                         bool solid);
  // vorticity criterion marks (+1/-1/0) and block max |w|^2
  void (*criterion)(cudaStream_t, const int32_t* list, int n, const void* f, const int32_t* nbr, const uint64_t* solidmask, const int32_t* status,
                    int level, int lmax, double inv_dx, int n_start, int n_inc, int8_t* marks,
                    double* w2out);
  // exports / imports of the blocks b0 .. b0+nb-1; the buffer of block b is
  // bufs[(cur >> level[b]) & 1].  AMR_F layout [Q][nb][M], AMR_RHO_U [nb][M][1+D]
  void (*export_f)(cudaStream_t, int64_t cap, int64_t b0, int64_t nb, const void* fa,
                   const void* fb, unsigned cur, const int32_t* level, const int32_t* nbr,
                   const uint64_t* solidmask, double* out);
  void (*import_f)(cudaStream_t, int64_t cap, int64_t b0, int64_t nb, void* fa, void* fb,
                   unsigned cur, const int32_t* level, const int32_t* nbr,
                   const uint64_t* solidmask, const double* in);
  void (*export_rho_u)(cudaStream_t, int64_t cap, int64_t b0, int64_t nb, const void* fa,
                       const void* fb, unsigned cur, const int32_t* level, const int32_t* nbr,
                       const uint64_t* solidmask, double* out);
  void (*init_rest)(cudaStream_t, int64_t cap, void* f);
  // FP64 audit: per-CTA partial sums of rho V and rho u V over leaf cells into
  // `partial` [grid][4]; returns the grid size used
  int (*mass_partial)(cudaStream_t, int64_t cap, const void* fa, const void* fb, unsigned cur,
                      const int32_t* level, const int32_t* status, const int32_t* nbr,
                      const uint64_t* solidmask, double* partial);
  // momentum-exchange force (Section 5.3) partial sums [grid][3] over the
  // leaves in `list` (one level, buffer f); returns the grid size used
  int (*force_partial)(cudaStream_t, const int32_t* list, int n, const void* f, const int32_t* nbr, const int32_t* status, const uint64_t* solidmask,
                       double omega, double dx, double* partial);
  // batched instances: one launch over an instance-major list of work items;
  // buffer A / B choice per launch (every instance of a batch shares parities)
  void (*collide_stream_batch)(cudaStream_t, const uint32_t* items, int n, const InstDesc* descs,
                               int level, int which_in, int variant);
  void (*interp_batch)(cudaStream_t, const uint32_t* items, int n, const InstDesc* descs,
                       int level, int which_par, int which_ch);
  void (*average_batch)(cudaStream_t, const uint32_t* items, int n, const InstDesc* descs,
                        int level, int which_par, int which_ch);
  // persistent form (PersistArgs): the number of CTAs of `threads` threads
  // that stay resident together (0: unsupported CTA size), after setting the
  // kernel's shared-memory attribute; call outside any stream capture
  int (*persistent_ctas)(int threads);
  void (*batch_persistent)(cudaStream_t, const PersistArgs& a, int threads, int ctas);
  // 27 block summaries of the learned refinement proposal (3D only)
  void (*features)(cudaStream_t, const int32_t* list, int n, const void* f, const int32_t* nbr, const uint64_t* solidmask, int level, int lmax,
                   double inv_dx, float* out);
  // adaptation, before the children of the coarsen-marked blocks in `list`
  // are removed: a same-level neighbour that stays takes back, into its own
  // slots, the values that were stored in the removed blocks for it
  void (*coarsen_fixup)(cudaStream_t, const int32_t* list, int n, const int32_t* child0,
                        const int32_t* parent, const int8_t* marks, const int32_t* nbr,
                        const uint64_t* solidmask, const int32_t* level, void* fa, void* fb,
                        unsigned cur);
};

const LbmOps* lbm_ops_d2q9(int storage);
const LbmOps* lbm_ops_d3q19(int storage);
const LbmOps* lbm_ops_d3q27(int storage);

}  // namespace amr
