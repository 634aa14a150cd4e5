/*
 * amr.h -- C ABI of the GB300-native block-forest AMR lattice Boltzmann
 * library (method of arXiv 2308.08085, "GPU-Native Adaptive Mesh Refinement
 * with Application to Lattice Boltzmann Simulations").
 *
 * Every entry point takes plain pointers and sizes.  The caller owns device
 * memory (one arena, carved by the library) and the CUDA stream; the library
 * allocates no device memory of its own.  All calls are asynchronous on the
 * caller's stream except amr_adapt, amr_fields / amr_set_fields with host
 * buffers, and amr_profile_read, which synchronise that stream.
 *
 * Return values: AMR_OK (0) or a negative AMR_E_* code; amr_fields returns a
 * byte count (>= 0) or a negative code.  amr_last_error() gives a one-line
 * description of the most recent failure on the calling thread.
 *
 * Layouts (see also the per-call comments)
 *   block      4^dim cells; cell l = i + 4 j + 16 k (x fastest)
 *   block IDs  0 .. max_blocks-1; root blocks 0 .. n_root-1 numbered
 *              x-fastest over the root grid of blocks
 *   directions velocity-set numbering of the paper's velocity-set figure
 *              (Section 2): D2Q9 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+,+),
 *              6 (-,+), 7 (-,-), 8 (+,-); D3Q19/D3Q27 opposite pairs
 *              (2k-1, 2k): +-x, +-y, +-z, +-(x+y), +-(x+z), +-(y+z),
 *              +-(x-y), +-(x-z), +-(y-z), +-(1,1,1), +-(1,1,-1),
 *              +-(1,-1,1), +-(-1,1,1).  Block neighbours use the D2Q9 /
 *              D3Q27 numbering; neighbour 0 is the block itself.
 *   sentinels  AMR_NONE (-1): no same-level neighbour / no children;
 *              AMR_WALL(face) = -2 - face: the neighbour position leaves the
 *              domain through wall `face` (x-, x+, y-, y+, z-, z+ = 0..5).
 *
 * Stored populations.  The paper's state is the post-streaming
 * (pre-collision) populations f_p(x) of every cell (Section 4.1).  The arena
 * holds, for every cell y and direction p, the value that streams out of y
 * along c_p: the post-collision f*_p(y) of the last step (the step is pulled:
 * f_p(x) = f*_p(x - c_p)).  Where x - c_p is not a fluid cell of x's level (a
 * coarse-fine interface, a wall, a solid cell) f_p(x) is kept in x's own slot
 * of the opposite direction, with the link's boundary rule already applied.
 * amr_fields(AMR_F / AMR_RHO_U / AMR_MASS) and amr_set_fields(AMR_F) convert:
 * they read and write the paper's f_p(x); only the raw arena (checkpoints,
 * amr_mass_audit_noalloc's inputs) is in the stored form.  Its layout is
 * block-major: the stored value of direction p, block b, cell l is element
 * b Q M + p M + l of a buffer (M = 4^dim), so each block's Q M values are
 * one contiguous run.
 */
#ifndef AMR_H
#define AMR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define AMR_OK 0
#define AMR_E_INVAL (-1)     /* bad argument or configuration                 */
#define AMR_E_CAPACITY (-2)  /* gap set too small: refinement of the call was
                                cancelled, coarsening still applied            */
#define AMR_E_CUDA (-3)      /* a CUDA runtime call failed                     */
#define AMR_E_TIMEOUT (-4)   /* a bounded device wait gave up                  */
#define AMR_E_UNSTABLE (-5)  /* the FP64 mass audit found a non-finite value   */
#define AMR_E_ARENA (-6)     /* arena too small or misaligned                   */

/* ----------------------------------------------------------------- storage */
#define AMR_F64 0        /* populations stored and computed in FP64          */
#define AMR_F32 1        /* populations stored and computed in FP32          */
#define AMR_F32_BF16 2   /* stored as BF16 shifted values f - w_p, FP32 math */
#define AMR_F32_F16 3    /* stored as FP16 shifted values f - w_p, FP32 math */

/* ------------------------------------------------------------- face kinds */
#define AMR_FACE_NOSLIP 0    /* bounce-back, u_w = 0                          */
#define AMR_FACE_MOVING 1    /* bounce-back with known wall velocity u_w      */
#define AMR_FACE_OUTLET 2    /* anti-bounce-back with rho_w, u_w = cell u     */
#define AMR_FACE_PERIODIC 3  /* both faces of an axis must be periodic        */

/* --------------------------------------------------------- block statuses */
#define AMR_ST_INACTIVE 0
#define AMR_ST_UNREFINED 1          /* leaf                                   */
#define AMR_ST_REFINED 2            /* refined, every child a leaf            */
#define AMR_ST_REFINED_WITH_CHILD 3 /* refined, some child refined            */
#define AMR_ST_REFINED_PERMANENT 4  /* refined, never coarsened               */

/* ------------------------------------------------------------ cell classes */
#define AMR_CELL_INTERIOR 0
#define AMR_CELL_INTERFACE 1
#define AMR_CELL_GHOST 2

#define AMR_NONE (-1)
#define AMR_WALL(face) (-2 - (face))
#define AMR_MAX_LEVELS 8

typedef struct {
  int32_t kind;      /* AMR_FACE_*                                            */
  int32_t pad_;
  double u[3];       /* wall velocity (lattice units) for AMR_FACE_MOVING     */
  double rho_w;      /* wall density; the paper uses 1                        */
} amr_face;

typedef struct {
  int32_t dim, q;          /* (2,9) | (3,19) | (3,27)                          */
  int32_t storage;         /* AMR_F64 | AMR_F32 | AMR_F32_BF16 | AMR_F32_F16   */
  int32_t nx, ny, nz;      /* root grid in cells, multiples of 4 (nz ignored
                              in 2D)                                           */
  int32_t max_levels;      /* L_max, 1 .. AMR_MAX_LEVELS                       */
  int32_t crit_start;      /* N_start of the vorticity criterion (Alg. 3)      */
  int32_t crit_inc;        /* N_inc of the vorticity criterion (Alg. 3)        */
  int32_t has_solid;       /* 1: square prism (a square in 2D, spanning z in 3D;
                              see solid[])                                     */
  int64_t max_blocks;      /* block capacity; (max_blocks - n_root) must be a
                              multiple of 2^dim                                 */
  double nu0;              /* viscosity, root-lattice units                     */
  double length_x;         /* physical length of the x extent (dx_0 = len/nx)  */
  double solid[4];         /* x0, x1, y0, y1 (root-cell units): a cell whose
                              centre is strictly inside is solid               */
  amr_face faces[6];       /* x-, x+, y-, y+, z-, z+ (first 4 used in 2D)      */
  int32_t use_graphs;      /* 1: replay the coarse step as a CUDA graph         */
  int32_t kernel_variant;  /* collide-stream kernel (fused BGK + pull
                              streaming): 1 / 2 / 3 / 4: 512 / 256 / 128 /
                              64 threads per CTA (8 / 4 / 2 / 1 blocks in 3D);
                              5: 128 threads with 512 more resident threads
                              per SM (tighter register budget); 0 (default):
                              64 threads, with the tighter budget for D3Q27
                              with 16-bit storage                              */
  double refine_dist;      /* distance refinement (Section 4.4): a leaf on level
                              L within refine_dist / 2^L (physical units) of a
                              target is marked for refinement; 0 = off        */
  int32_t refine_dist_targets; /* bit 0: the solid prism, bit 1: outlet faces,
                                  bit 2: wall faces (no-slip and moving)      */
  int32_t refine_dist_freeze;  /* 1: blocks refined by distance become
                                  AMR_ST_REFINED_PERMANENT                    */
  const int32_t* root_ids; /* NULL: root block IDs in lexicographic order of
                              their position, b = bx + nbx (by + nby bz).
                              Else a host array of the n_root root blocks
                              (read by amr_init only): root_ids[i] is the ID
                              of the root at lexicographic position i; it must
                              be a permutation of 0 .. n_root-1 (AMR_E_INVAL
                              otherwise).  The ID set of level 0 stays in
                              ascending ID order, so the order of the IDs is
                              the order of the blocks in memory.             */
  int32_t interp;          /* coarse-to-fine interpolation (Section 3.4):
                              AMR_INTERP_LINEAR (0) or AMR_INTERP_CUBIC (3)  */
  int32_t check_tables;    /* 1: validate the block tables on the device at
                              amr_init and after every amr_adapt
                              (amr_check_tables); a bad entry fails the call
                              with AMR_E_INVAL                              */
} amr_config;

#define AMR_INTERP_LINEAR 0
#define AMR_INTERP_CUBIC 3

typedef struct {
  int64_t n_marked_refine;   /* eligible refine marks before capacity check  */
  int64_t n_marked_coarsen;  /* eligible coarsen marks before 2:1 reversion  */
  int64_t n_refined;         /* blocks refined by the call                    */
  int64_t n_coarsened;       /* blocks coarsened by the call                  */
  int64_t n_blocks;          /* active blocks after the call                  */
  int32_t capacity_error;    /* 1 when refinement was cancelled               */
  int32_t pad_;
  double ms_total;           /* host wall time of the call                    */
} amr_adapt_stats;

typedef struct {
  char name[32];         /* kernel class                                     */
  int64_t launches;
  double ms;             /* summed CUDA-event durations                      */
  double bytes;          /* summed algorithmic bytes (see amr_profile)       */
  double cells;          /* summed cells: updates (collide-stream), ghost
                            cells written (interp), interface fine cells read
                            (average)                                        */
} amr_kernel_profile;

typedef struct amr_t amr_t;

/* Bytes of device arena that amr_init needs for `cfg` (0 if cfg is invalid).
 * The arena must be 256-byte aligned. */
size_t amr_arena_bytes(const amr_config* cfg);

/* Build the root grid of blocks (Section 3.2: structured root grid, ID set of
 * level 0, gap set enumerated in reverse) and initialise every population to
 * the rest equilibrium (rho = 1, u = 0).  `dev_arena` (device memory of
 * `arena_bytes`, owned by the caller, kept alive until amr_free) holds every
 * array; `stream` is a cudaStream_t (NULL: legacy default stream).
 * Errors: AMR_E_INVAL (config), AMR_E_ARENA, AMR_E_CUDA. */
int amr_init(const amr_config* cfg, void* dev_arena, size_t arena_bytes,
             void* stream, amr_t** out);

/* Advance `n_coarse_steps` root time steps with the recursive level step of
 * Section 4.1: on level L, interpolate level L to the ghost cells of L+1
 * (Section 3.4.1), collide and stream L (Sections 4.2, 4.3, BGK with
 * tau_L = 1/2 + 2^L (tau_0 - 1/2)), advance L+1 twice, average the interface
 * cells of L+1 into L (Section 3.4.3).  Asynchronous.  Errors: AMR_E_INVAL,
 * AMR_E_CUDA. */
int amr_step(amr_t* a, int n_coarse_steps);

/* Adapt the mesh (Sections 3.3 and 4.4): synchronise all levels (average
 * bottom-up, interpolate ghosts top-down), mark blocks -- from the vorticity
 * criterion of Algorithm 3 and the distance rule (refine_dist) when
 * `dev_marks` is NULL, else from the caller's device array of int8 marks
 * indexed by block ID (+1 refine, +2 refine and freeze, -1 coarsen, 0 keep;
 * max_blocks entries) -- keep the eligible marks (refine: leaf below
 * L_max-1 with every same-level neighbour present; coarsen: status REFINED),
 * revert coarsening that would break 2:1 balance, allocate children from the
 * gap set, remove children, update ID sets, statuses, connectivity and cell
 * classes, and interpolate every cell of the new children.  Synchronous.
 * `out` may be NULL.  Errors: AMR_E_CAPACITY (refinement cancelled, mesh
 * otherwise updated), AMR_E_INVAL, AMR_E_CUDA. */
int amr_adapt(amr_t* a, const int8_t* dev_marks, amr_adapt_stats* out);

/* Field selectors for amr_fields / amr_set_fields.  B = max_blocks,
 * M = 4^dim, K = 3^dim. */
#define AMR_RHO_U 0     /* double [B][M][1+dim]: rho, u after a sync (the
                           call runs the level synchronisation first)          */
#define AMR_F 1         /* double [Q][B][M]: populations of every block at
                           its level's current time (unshifted values)         */
#define AMR_BLOCKS 2    /* int32 [4][B]: level, status, child0, parent         */
#define AMR_COORDS 3    /* double [B][dim]: block corner, root-cell units      */
#define AMR_NBR 4       /* int32 [B][K]: neighbour IDs / sentinels             */
#define AMR_NBR_CHILD 5 /* int32 [B][K]: first child of each neighbour,
                           AMR_NONE if absent/unrefined, wall code if wall     */
#define AMR_IDSETS 6    /* int32 [L_max][B]: ID set of each level; lengths
                           from AMR_COUNTS                                      */
#define AMR_GAPS 7      /* int32 [B]: gap stack, bottom first; length from
                           AMR_COUNTS                                          */
#define AMR_MASKS 8     /* uint8 [B][M]: AMR_CELL_* class of every cell        */
#define AMR_COUNTS 9    /* int64 [4 + 4 L_max]: L_max, n_gaps, coarse steps,
                           kernels launched so far, then per level: ID-set
                           size, active blocks, leaves, parent blocks
                           exchanging with children                            */
#define AMR_MASS 10     /* double [1 + dim]: FP64 sum over leaf cells of
                           rho V and rho u V, V = cell volume (root units)     */
#define AMR_FORCE 11    /* double [3]: momentum-exchange force on the solid
                           (Section 5.3), physical units of dx                 */
#define AMR_FEATURES 12 /* float [B][27]: block summaries of the learned
                           refinement proposal (3D only; after a sync; 0 for
                           blocks outside the mesh), see amr_propose_marks     */

/* Copy field `what` into `dst` (device pointer if dst_on_device, else host):
 * the populations and moments the recursive level step (Section 4.1) leaves,
 * after the level synchronisation of Section 4.4 for AMR_RHO_U; the block
 * tables, ID sets and gap stack of the forest (Sections 3.2-3.3); the cell
 * classes (Section 3.4); the momentum-exchange force (Section 5.3).
 * dst == NULL returns the required bytes.  Returns bytes written or a
 * negative code (AMR_E_INVAL if dst_bytes is too small; AMR_E_TIMEOUT, for
 * a host destination, when a bounded device wait gave up since the last
 * synchronising call). */
int64_t amr_fields(amr_t* a, int what, void* dst, size_t dst_bytes,
                   int dst_on_device);

/* Overwrite the populations (what == AMR_F, same layout as amr_fields) of
 * every active block from `src`.  Synchronous for host sources. */
int amr_set_fields(amr_t* a, int what, const void* src, size_t src_bytes,
                   int src_on_device);

/* Per-kernel CUDA-event timing.  mode 0: off.  mode 1: events around every
 * launch of amr_step (graph replay is off while on).  mode 2: events are
 * captured inside the coarse-step graphs; each amr_profile_read adds one
 * sample, the launches of the most recently replayed coarse step.
 * amr_profile_read synchronises, fills up to `max` entries (collide_stream,
 * interp, average, then the phases of amr_adapt: adapt_sync, adapt_criterion,
 * adapt_marks, adapt_alloc, adapt_idsets, adapt_relink, adapt_children,
 * adapt_lists, timed between events at their boundaries) and returns how many
 * classes exist; reset != 0
 * clears the sums.  Bytes are algorithmic, N_p bytes per stored population:
 * collide-stream 2 Q N_p per cell update (Section 4.2, read and write once);
 * interp Q N_p per ghost cell written plus 2^D Q N_p per child block with
 * ghost cells (its parent cells, Section 3.4.1); average Q N_p per interface
 * fine cell read plus Q N_p per parent cell written, one per 2^D fine cells
 * (Section 3.4.3). */
int amr_profile(amr_t* a, int mode);
int amr_profile_read(amr_t* a, amr_kernel_profile* out, int max, int reset);

/* FP64 mass and momentum audit that allocates nothing.  The paper has no
 * counterpart: this is a service of this library for callers that cannot
 * allocate device memory -- code running under a memory budget fixed by a
 * host framework, code that must not call the CUDA allocator inside a
 * latency-critical loop, or code that holds population buffers in this
 * library's layout but no amr_t instance and no arena.
 *
 * Inputs (device pointers, owned by the caller): the two population buffers
 * f_a, f_b of `n_blocks` blocks in this library's storage layout of
 * `storage` ([n_blocks][Q][4^dim] stored values -- the outgoing
 * post-collision populations, see "Stored populations" above; 16-bit
 * storages hold value - w_p), a per-level buffer choice `cur` (bit L set:
 * blocks of level L are read from f_b), int32 level[n_blocks] /
 * status[n_blocks] (AMR_BLOCKS rows 0 and 1), the neighbour table
 * nbr[n_blocks][32] (int32, 32 per block, the first 3^dim in the AMR_NBR
 * order, the layout of the arena's table) and the solid-cell bits
 * solidmask[n_blocks] (uint64, bit l = cell l; null when there are no solid
 * cells).  Output: out_dev[0 .. dim] (device, caller-owned) = the sum over
 * leaf blocks (status AMR_ST_UNREFINED) of rho V and rho u V,
 * V = 2^(-dim level), rho and u the moments of the cell's pre-collision
 * populations.  Asynchronous on `stream`.
 *
 * Scratch: a file-scope device array of AMR_NOALLOC_MAX_PARTIALS rows of 4
 * doubles (512 KiB), held by every GPU that loads the library until the
 * process exits.  One row per 64 blocks, so n_blocks may not exceed
 * 64 * AMR_NOALLOC_MAX_PARTIALS (1,048,576); larger inputs return
 * AMR_E_INVAL with a message and launch nothing.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * Every call on a device shares the array and leaves its partial sums there;
 * each call writes every row it reads, so nothing needs clearing, but calls
 * that overlap on the GPU (different streams, or different host threads)
 * race on it.  Calls no cudaMalloc, cudaFree or allocating library routine.
 * Errors: AMR_E_INVAL, AMR_E_CUDA (also when a CUDA error from earlier work
 * is already pending on the calling thread: it is left for its owner). */
#define AMR_NOALLOC_MAX_PARTIALS 16384
int amr_mass_audit_noalloc(int dim, int q, int storage, int64_t n_blocks,
                           const void* f_a, const void* f_b, uint32_t cur,
                           const int32_t* level, const int32_t* status,
                           const int32_t* nbr, const uint64_t* solidmask,
                           double* out_dev, void* stream);

/* Release host-side state (the arena stays owned by the caller). */
int amr_free(amr_t* a);

/* ------------------------------------------------- block-table validation
 * The stand-in for a device bounds checker (the paper has no counterpart).
 * Every block ID a kernel dereferences comes from the block tables (neighbour
 * rows, child0, parent), the per-level work lists or the averaging groups;
 * these checks verify each entry against its range and the forest's
 * invariants on the device, dereferencing an index only once it is known to
 * be in range, and count the bad entries in a device word instead of trapping.
 *
 * For every block b < cap: status in 0 .. 4; an inactive block (status 0)
 * has level -1, child0 = parent = AMR_NONE and an all-AMR_NONE neighbour
 * row; an active one has 0 <= level < max_levels, nbr[b][0] = b, entries
 * 1 .. 3^dim - 1 each AMR_NONE, a wall code (-2 .. -7) or an active block of
 * the same level, the remaining entries of the 32 AMR_NONE; child0 AMR_NONE
 * for a leaf, else 2^dim consecutive active children one level down whose
 * parent is b; parent AMR_NONE on level 0, else an active refined block one
 * level up whose children include b.  Gap stack entries: inactive IDs.
 *
 * amr_validate_tables: caller-owned device tables in the layout of the
 *   AMR_BLOCKS rows (level, status, child0, parent: int32[cap]) and of the
 *   arena's neighbour table (int32[cap][32], first 3^dim used), and the gap
 *   stack gap[n_gaps] (may be NULL when n_gaps is 0).  Synchronous on
 *   `stream`; the result words are a file-scope device array, so calls on
 *   different streams must not overlap.
 * amr_check_tables: the instance's own tables, gap stack, work lists (ID
 *   set, tree order, active, parent and boundary lists: IDs of their level)
 *   and averaging groups.  Synchronous.  AMR_E_INVAL when an entry is bad.
 * out3[0] = bad entries, out3[1] = the smallest block with a bad entry (-1
 * when none, or when the gap count itself is out of range), out3[2] = the
 * AMR_CHECK_* code of its first failed check. */
#define AMR_CHECK_STATUS 1
#define AMR_CHECK_INACTIVE 2
#define AMR_CHECK_LEVEL 3
#define AMR_CHECK_SELF 4
#define AMR_CHECK_NEIGHBOUR 5
#define AMR_CHECK_UNUSED 6
#define AMR_CHECK_CHILDREN 7
#define AMR_CHECK_PARENT 8
#define AMR_CHECK_GAP 9
#define AMR_CHECK_LIST 10
#define AMR_CHECK_GROUP 11
int amr_validate_tables(int dim, int max_levels, int64_t cap, const int32_t* level,
                        const int32_t* status, const int32_t* child0, const int32_t* parent,
                        const int32_t* nbr, const int32_t* gap, int64_t n_gaps, int64_t* out3,
                        void* stream);
int amr_check_tables(amr_t* a, int64_t* out3);

/* ---------------------------------------------------- checkpoint / resume
 * The paper keeps all state on the device and has no checkpoint; this is a
 * service of the library.  A checkpoint is a host byte image of the whole
 * instance: a header (format tag, the configuration fields that fix the
 * arena layout, the host mirror of the mesh sizes, the coarse-step count and
 * the level buffer parities) followed by the device arena.
 * amr_checkpoint_bytes: the image size.  amr_checkpoint: synchronises and
 * writes the image to host memory `dst` (caller-owned, >= the image size).
 * amr_restore: loads an image into an instance created by amr_init with the
 * same velocity set, storage, root grid, level count and capacity
 * (AMR_E_INVAL otherwise, leaving the instance unchanged); graph use and
 * stream may differ.  Stepping a restored instance with the same kernel
 * variant reproduces the original bit for bit (other variants are compiled
 * separately and may round differently).  Both calls are synchronous.
 * Errors: AMR_E_INVAL, AMR_E_CUDA. */
int64_t amr_checkpoint_bytes(amr_t* a);
int amr_checkpoint(amr_t* a, void* dst, size_t dst_bytes);
int amr_restore(amr_t* a, const void* src, size_t src_bytes);

/* ------------------------------------------------ learned refinement proposal
 * Not in the paper: a per-block MLP (27 -> 64 -> 64 -> 1, ReLU, sigmoid)
 * proposes refinement ahead of the vorticity criterion so that adaptation can
 * run less often; the plain criterion stays the fallback.  Inputs are the 27
 * block summaries of AMR_FEATURES: for the velocity-gradient components
 * du_a/dx_b their block mean and max |.|, mean and max-min of rho, mean
 * velocity and max |u|, mean and max |vorticity|, level / L_max (gradient and
 * vorticity entries compressed as sign(x) log(1 + |x|)).  Parameters are a flat
 * float array of amr_mlp_param_count() entries: W1[64][27], b1[64],
 * W2[64][64], b2[64], w3[64], b3 (FP32 master), plus an FP16 copy of the same
 * layout that inference reads.  All pointers are device pointers. */
#define AMR_MLP_INPUTS 27
#define AMR_MLP_HIDDEN 64

typedef struct {
  float* params;       /* FP32 master weights                                */
  float* adam_m;       /* Adam first moments (zero-initialised by the caller) */
  float* adam_v;       /* Adam second moments (zero-initialised)             */
  void* params_half;   /* FP16 copy, refreshed by every update               */
  float* grad;         /* scratch: summed gradient of a minibatch            */
  float* loss;         /* scratch: one float                                 */
  int64_t step;        /* Adam step counter (host side, updated)             */
} amr_mlp_state;

int amr_mlp_param_count(void);
/* Glorot-uniform weights and zero biases from a counter-based generator;
 * writes the FP16 copy too when params_half is not NULL. */
int amr_mlp_init(float* params, void* params_half, uint64_t seed, void* stream);
/* Summed gradient (into grad[param_count]) and summed loss (into *loss) of the
 * class-weighted binary cross-entropy  pw y softplus(-z) + (1-y) softplus(z)
 * over n samples x[n][27], labels y[n] in {0, 1}; nothing is updated. */
int amr_mlp_grad(const float* params, const float* x, const float* y, int64_t n, float pos_weight,
                 float* grad, float* loss, void* stream);
/* One epoch of minibatch Adam (beta 0.9 / 0.999, eps 1e-8) over n samples in
 * an order fixed by epoch_seed; *mean_loss (host, may be NULL; synchronises)
 * receives the mean loss of the epoch. */
int amr_mlp_train_epoch(const amr_mlp_state* st, const float* x, const float* y, int64_t n,
                        int batch, float lr, float pos_weight, uint64_t epoch_seed,
                        double* mean_loss, void* stream);
/* prob[i] = sigmoid(MLP(x[i])) with the FP16 weights, i < n. */
int amr_mlp_infer(const void* params_half, const float* x, int64_t n, float* prob, void* stream);

/* The plain criterion as a dry run: sync, vorticity criterion and distance
 * rule; writes the raw marks (+1 / +2 refine a leaf, -1 coarsen a REFINED
 * block, 0) of every block to dev_marks[max_blocks]; the mesh is unchanged.
 * Synchronous. */
int amr_criterion_marks(amr_t* a, int8_t* dev_marks);

/* Refinement proposal: sync, block summaries, the MLP (FP16 weights) on every
 * leaf; a leaf with probability > threshold is marked +1.  With
 * with_criterion != 0 the marks of the plain criterion are merged in (a
 * refine mark from either source refines; coarsening comes from the
 * criterion).  Writes dev_marks[max_blocks] for amr_adapt.  3D only.
 * Synchronous. */
int amr_propose_marks(amr_t* a, const void* params_half, float threshold, int with_criterion,
                      int8_t* dev_marks);

/* ---------------------------------------------------------- batched instances
 * Many independent instances (same velocity set and storage, no solid) are
 * advanced together.  The recursive level step (Section 4.1) has the same
 * shape for every member, so a batch runs it in one of two forms:
 *
 * AMR_BATCH_GRAPH       each level operation is one launch over an
 *                       instance-major list of (instance, block) items, and
 *                       the batched coarse step is replayed as a CUDA graph.
 * AMR_BATCH_PERSISTENT  one launch advances every member by n coarse steps.
 *                       The level step is unrolled into a list of phases
 *                       (interpolation into level L+1, collide-stream of
 *                       level L, averaging of level L+1 into L); a phase's
 *                       items are cut into tiles of one member each, and the
 *                       CTAs take tiles in (step, phase, member, tile) order
 *                       from one device queue.  Before it runs, a tile waits
 *                       until its member has finished the member's previous
 *                       phase; members advance independently, with no
 *                       grid-wide barrier.  Every wait is bounded (about one
 *                       second of clock64 cycles): when one gives up, the
 *                       launch stops, every member's wait flag is raised, and
 *                       amr_batch_sync returns AMR_E_TIMEOUT.
 * AMR_BATCH_MEMBERS     one CUDA graph per coarse step whose independent
 *                       branches are the members' own coarse steps (the
 *                       per-instance kernels of amr_step), so that the small
 *                       levels of different members run side by side.
 *
 * The paper runs one forest per GPU; batching is this library's extension.
 * Members keep their own arenas; the batch arena holds the instance
 * descriptors, the per-level item lists and the persistent form's phase
 * tables and counters.  Results of the two forms agree to rounding (the
 * kernels are compiled separately).
 *
 * amr_batch_arena_bytes: device bytes for a batch of these instances.
 * amr_batch_create: members must have equal buffer parities (equally many
 *   coarse steps since amr_init, modulo 2) and capacities below 2^25 blocks;
 *   at most 127 members.  `stream` as in amr_init.  Starts in the graph form
 *   with 512 threads per CTA.
 * amr_batch_refresh: rebuild the item lists after any member was adapted.
 * amr_batch_step: advance every member by n coarse steps (asynchronous);
 *   AMR_E_INVAL if a member was stepped outside the batch since.  After a
 *   timeout the persistent form does nothing until amr_batch_sync has
 *   reported it; the members' populations are then part-way through a step.
 * amr_batch_configure: select the form and its tile shape.  Graph form:
 *   threads per CTA of the batched collide-stream 64, 128, 256 or 512 (the
 *   CTA takes threads / 4^D blocks); tile_blocks and ctas are ignored.
 *   Persistent form: threads 64, 128 or 256 per CTA, tile_blocks M_L = 1..8
 *   blocks per collide-stream tile (an interpolation or averaging tile holds
 *   threads / 4^D parents or children), ctas = CTAs launched (0: as many as
 *   stay resident together; the queue needs no co-residency).
 *   Member-graph form: threads, tile_blocks and ctas are ignored.
 * amr_batch_get_config: the current form; in the graph form tile_blocks is
 *   threads / 4^D and ctas is 0; in the member-graph form all three are 0.
 * amr_batch_autotune: time `trial_steps` coarse steps of each candidate
 *   (forms: bit 0 the graph form with 512, 256, 128, 64 threads; bit 1 the
 *   persistent form with M_L = 1, 2, 4, 8 x threads 64, 128, 256, resident
 *   CTAs; bit 2 the member-graph form), keep the fastest and write it to
 *   *chosen (may be NULL).  ms_out (NULL, or 17 floats) receives
 *   milliseconds per coarse step in that candidate order, -1 for a
 *   candidate not timed.  The members advance.
 *   Synchronous.
 * amr_batch_sync: wait for the batch's stream; AMR_E_TIMEOUT (once) if a
 *   bounded wait of the persistent form gave up since the last call.
 * amr_batch_check_timeout: a check of the failure path of the persistent
 *   form that needs no GPU fault: one launch in which no tile's wait can be
 *   satisfied, with waits of `limit_cycles` clock64 cycles (0 < limit <=
 *   2^32).  Returns AMR_E_TIMEOUT when the waits gave up and the launch
 *   ended (the expected result).  The members are left part-way through a
 *   step: use it on a batch whose results are not needed.  Synchronous.
 * amr_batch_launches: kernels launched by the batch so far.
 * Errors: AMR_E_INVAL, AMR_E_ARENA, AMR_E_CUDA, AMR_E_TIMEOUT. */
#define AMR_BATCH_GRAPH 0
#define AMR_BATCH_PERSISTENT 1
#define AMR_BATCH_MEMBERS 2
typedef struct amr_batch_t amr_batch_t;
typedef struct {
  int32_t mode;         /* AMR_BATCH_GRAPH, _PERSISTENT or _MEMBERS */
  int32_t threads;      /* threads per CTA                          */
  int32_t tile_blocks;  /* M_L: blocks per collide-stream tile      */
  int32_t ctas;         /* persistent form: CTAs launched (0: all resident) */
} amr_batch_config_t;
size_t amr_batch_arena_bytes(amr_t* const* instances, int n);
int amr_batch_create(amr_t* const* instances, int n, void* dev_arena, size_t arena_bytes,
                     void* stream, amr_batch_t** out);
int amr_batch_refresh(amr_batch_t* b);
int amr_batch_step(amr_batch_t* b, int n_coarse_steps);
int amr_batch_configure(amr_batch_t* b, const amr_batch_config_t* cfg);
int amr_batch_get_config(amr_batch_t* b, amr_batch_config_t* out);
int amr_batch_autotune(amr_batch_t* b, int trial_steps, int forms, amr_batch_config_t* chosen,
                       float* ms_out);
int amr_batch_sync(amr_batch_t* b);
int amr_batch_check_timeout(amr_batch_t* b, long long limit_cycles);

/* The persistent form's plan for members with the given counts, computed on
 * the host (no device work; what amr_batch_step builds for the persistent
 * form, for inspection and tests).  n members; lmax = the batch's level
 * count (the largest member L_max); member_lmax[n]; n_ids, n_active,
 * n_parents [n][lmax] (AMR_COUNTS per level: ID-set size, active blocks,
 * exchanging parents; 0 beyond a member's levels); threads and tile_blocks
 * as in amr_batch_configure; cur: the level buffer parities at the start of
 * the coarse step.  Outputs, sized for max_phases phases: *n_phase;
 * phases[4 k .. 4 k + 3] = kind (0 interpolation into level + 1,
 * 1 collide-stream, 2 averaging of level + 1 into level), level, buffer of
 * the level read (interpolation, collide-stream) or written (averaging),
 * buffer of level + 1; tile_off[k (n + 1) + i] = first tile of member i in
 * phase k, tile_off[k (n + 1) + n] = the phase's tiles; dep[k n + i] = 2 k'
 * + wrap: the member's previous phase with tiles, wrap 1 when it lies in the
 * previous coarse step.  AMR_E_INVAL on bad arguments or when the phases do
 * not fit. */
int amr_batch_plan(int dim, int n, int lmax, const int32_t* member_lmax, const int64_t* n_ids,
                   const int64_t* n_active, const int64_t* n_parents, int threads,
                   int tile_blocks, uint32_t cur, int max_phases, int32_t* n_phase,
                   int32_t* phases, int32_t* tile_off, int32_t* dep);
int64_t amr_batch_launches(amr_batch_t* b);
int amr_batch_free(amr_batch_t* b);

/* ------------------------------------------------ cell-based uniform solver
 * The cell arrangement of the paper's comparison of cell- and block-based
 * grids on a single level (Section 5, "Cell vs. Block Arrangement"): a
 * uniform grid of nx x ny (x nz) cells, periodic in every axis, in which
 * every cell is its own element.  One kernel launch per time step: BGK
 * collision with tau = 3 nu0 + 1/2 (FP32 arithmetic) and push streaming of
 * each post-collision population f*_p to the element one link c_p
 * downstream.  Populations: two caller-owned device buffers f_a, f_b of
 * q * n FP32 values, [q][n] by element ID (n = nx ny, or nx ny nz in 3D).
 *
 * Element IDs are a permutation of the cell positions (x-fastest position
 * i = x + nx (y + ny z)): id_of_pos[i] is the ID of the cell at position i.
 * Connectivity:
 *   AMR_CELLS_CALCULATED  IDs are the positions themselves; a thread derives
 *                         the downstream IDs from its own ID (no table).
 *   AMR_CELLS_RETRIEVED   downstream IDs are read from table[p * n + id]
 *                         (device, int32, q * n entries, caller-owned), as
 *                         filled by amr_cells_table for the same grid.
 *
 * amr_cells_table (host only, no GPU): fills the caller's host array
 *   table[q * n] with table[p * n + id_of_pos[i]] = id_of_pos[j], j the
 *   position one link c_p downstream of position i (periodic).  id_of_pos
 *   (host, n entries) may be NULL for the x-fastest numbering.  AMR_E_INVAL,
 *   with nothing written, when id_of_pos is not a permutation of 0 .. n-1,
 *   for an unsupported velocity set, an empty grid, or n >= 2^31.
 * amr_cells_step: n_steps steps on `stream` (asynchronous); step k reads
 *   f_a and writes f_b when k is even, the reverse when k is odd, so the
 *   result of an odd count is in f_b.  AMR_E_INVAL for a null or aliased
 *   buffer, a missing table with AMR_CELLS_RETRIEVED, n_steps < 0 or
 *   nu0 <= 0; AMR_E_CUDA when a launch fails.  A table that amr_cells_table
 *   did not fill for this grid is undefined behaviour.
 * amr_cells_rest: writes the rest equilibrium (rho = 1, u = 0: f_p = w_p)
 *   into the device buffer f of q * n FP32 values (asynchronous on `stream`);
 *   AMR_E_INVAL for a null buffer or a grid amr_cells_table rejects. */
#define AMR_CELLS_CALCULATED 0
#define AMR_CELLS_RETRIEVED 1
int amr_cells_table(int dim, int q, int nx, int ny, int nz, const int32_t* id_of_pos,
                    int32_t* table);
int amr_cells_step(int dim, int q, int nx, int ny, int nz, int connectivity, double nu0,
                   const int32_t* table, float* f_a, float* f_b, int n_steps, void* stream);
int amr_cells_rest(int dim, int q, int nx, int ny, int nz, float* f, void* stream);

const char* amr_strerror(int code);
const char* amr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AMR_H */
