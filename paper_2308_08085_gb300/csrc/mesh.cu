// On-device mesh adaptation of the block forest (Sections 3.2-3.3, Alg. 1,
// Alg. 2): root grid, eligibility of marks, 2:1 coarsening reversion, ID
// allocation from the gap stack, removal, ID-set maintenance, statuses,
// connectivity of children from their parents, cell classes, per-level work
// lists.  Thrust calls of the paper are replaced by one stable compaction
// primitive (CTA counts with __syncthreads_count, a single-CTA scan, and a
// warp-ballot scatter).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>

#include "amr_internal.h"
#include "lattice.cuh"

namespace amr {

constexpr int ST_INACTIVE = 0, ST_UNREFINED = 1, ST_REFINED = 2, ST_RWC = 3, ST_PERM = 4;

// ====================================================== stable compaction
template <class Pred>
__global__ void __launch_bounds__(256) k_count(int n, Pred pred, int32_t* cta) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  const int flag = (i < n) && pred(i);
  const int c = __syncthreads_count(flag);
  if (threadIdx.x == 0) cta[blockIdx.x] = c;
}

// Exclusive scan of cta[0..nb) in place (one CTA of 1024 threads); writes the
// total to *total.
__global__ void __launch_bounds__(1024) k_scan(int nb, int32_t* cta, int32_t* total) {
  __shared__ int32_t wsum[32];
  __shared__ int32_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? cta[i] : 0;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = wsum[lane];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    const int excl = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - v;
    if (i < nb) cta[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

template <class Pred, class Val>
__global__ void __launch_bounds__(256)
    k_scatter(int n, Pred pred, Val val, const int32_t* cta, int32_t* out) {
  __shared__ int32_t wsum[8];
  const int i = blockIdx.x * 256 + threadIdx.x;
  const bool flag = (i < n) && pred(i);
  const unsigned bal = __ballot_sync(0xffffffffu, flag);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wsum[warp] = __popc(bal);
  __syncthreads();
  int off = cta[blockIdx.x];
  for (int w = 0; w < warp; ++w) off += wsum[w];
  if (flag) out[off + __popc(bal & ((1u << lane) - 1u))] = val(i);
}

struct VIdent {
  __device__ int operator()(int i) const { return i; }
};
struct VList {
  const int32_t* l;
  __device__ int operator()(int i) const { return l[i]; }
};
struct PMarkEq {
  const int8_t* m;
  int v;
  __device__ bool operator()(int i) const { return m[i] == v; }
};
struct PMarkPos {   // refine marks: +1, or +2 (refine and freeze)
  const int8_t* m;
  __device__ bool operator()(int i) const { return m[i] > 0; }
};
struct PLevelEq {
  const int32_t* list;
  const int32_t* level;
  int L;
  __device__ bool operator()(int i) const { return level[list[i]] == L; }
};
struct PAlive {
  const int32_t* list;
  const int32_t* status;
  __device__ bool operator()(int i) const { return status[list[i]] != ST_INACTIVE; }
};
struct PNoneNbr {   // blocks with a missing same-level neighbour (NONE)
  const int32_t* list;
  const uint32_t* nonemask;
  __device__ bool operator()(int i) const { return nonemask[list[i]] != 0u; }
};
struct PHasKids {
  const int32_t* list;
  const int32_t* child0;
  __device__ bool operator()(int i) const { return child0[list[i]] >= 0; }
};
struct PLeaf {
  const int32_t* list;
  const int32_t* status;
  __device__ bool operator()(int i) const { return status[list[i]] == ST_UNREFINED; }
};
// Averaging work of the level step (Section 3.4.3): group g of 2^D cells of
// boundary block list[i / N_c] (the cells under one parent cell) when they
// are interface cells and that parent cell is fluid
template <int D>
struct PAvgGroup {
  const int32_t* list;
  const uint64_t* cellmask;
  const int32_t* parent;
  const int32_t* child0;
  const uint64_t* solidmask;
  __device__ bool operator()(int i) const {
    constexpr int NC = Block<D>::NC;
    const int ch = list[i / NC], g = i % NC;
    const int f0 = Block<D>::cell(2 * (g & 1), 2 * ((g >> 1) & 1), 2 * ((g >> 2) & 1));
    if (!((cellmask[2 * (size_t)ch + 1] >> f0) & 1ull)) return false;
    if (!solidmask) return true;
    const int P = parent[ch], c = ch - child0[P];
    const int pc = Block<D>::cell(2 * (c & 1) + (g & 1), 2 * ((c >> 1) & 1) + ((g >> 1) & 1),
                                  2 * ((c >> 2) & 1) + ((g >> 2) & 1));
    return !((solidmask[P] >> pc) & 1ull);
  }
};
template <int D>
struct VAvgGroup {   // block << 3 | group
  const int32_t* list;
  __device__ int32_t operator()(int i) const {
    return (list[i / Block<D>::NC] << 3) | (i % Block<D>::NC);
  }
};

// leaves, and refined blocks with a child that has a NONE neighbour
struct PActive {
  const int32_t* list;
  const int32_t* status;
  const int32_t* child0;
  const uint32_t* nonemask;
  int nc;
  bool parents_only;
  __device__ bool operator()(int i) const {
    const int b = list[i];
    const int st = status[b];
    if (st == ST_UNREFINED) return !parents_only;
    if (st < ST_REFINED) return false;
    const int c0 = child0[b];
    for (int c = 0; c < nc; ++c)
      if (nonemask[c0 + c] != 0u) return true;
    return false;
  }
};

// Launch a stable compaction of the indices i < n with pred(i), writing
// val(i) to out in ascending i.  The count lands in dcount[slot]; when
// `count` is non-null the stream is synchronised and it is returned.
template <class Pred, class Val>
static int compact(Instance* a, int64_t n, Pred pred, Val val, int32_t* out, int64_t* count,
                   int slot = 0, bool scatter = true) {
  cudaStream_t s = a->stream;
  if (n <= 0) {
    AMR_CUDA(cudaMemsetAsync(a->dcount + slot, 0, sizeof(int32_t), s));
    if (count) *count = 0;
    return AMR_OK;
  }
  const int nb = (int)((n + 255) / 256);
  if (nb > cta_slots(a->cap)) {
    set_error("compaction of " + std::to_string(n) + " items exceeds its count array");
    return AMR_E_INVAL;
  }
  k_count<<<nb, 256, 0, s>>>((int)n, pred, a->cta);
  k_scan<<<1, 1024, 0, s>>>(nb, a->cta, a->dcount + slot);
  if (scatter) k_scatter<<<nb, 256, 0, s>>>((int)n, pred, val, a->cta, out);
  a->launches += scatter ? 3 : 2;
  AMR_CUDA(cudaGetLastError());
  if (count) {
    int32_t c = 0;
    AMR_CUDA(cudaMemcpyAsync(&c, a->dcount + slot, sizeof(c), cudaMemcpyDeviceToHost, s));
    AMR_CUDA(cudaStreamSynchronize(s));
    *count = c;
  }
  return AMR_OK;
}

static inline int blocks_for(int64_t n, int t = 256) {
  return (int)std::max<int64_t>(1, (n + t - 1) / t);
}

#define AMR_TRY(x)            \
  do {                        \
    int r_ = (x);             \
    if (r_ != AMR_OK) return r_; \
  } while (0)

// ============================================================== root grid
// Root blocks b = bx + nbx (by + nby bz) at 4 * (bx, by, bz); neighbours by
// position with periodic wrap, else the wall code of the crossed faces.
// id_of_pos / pos_of_id: the root numbering (root ID of a lexicographic
// position and its inverse), or null for the lexicographic numbering.
template <int D>
__global__ void k_init_root(int64_t cap, int n_root, int nbx, int nby, int nbz,
                            unsigned periodic, const int32_t* __restrict__ wall_code,
                            const int32_t* __restrict__ id_of_pos,
                            const int32_t* __restrict__ pos_of_id, int32_t* level,
                            int32_t* status, int32_t* child0, int32_t* parent, float* X,
                            int32_t* nbr, uint32_t* nonemask, uint64_t* cellmask, int32_t* gap,
                            int32_t* idset0, int32_t* order0) {
  using NV = typename Nbr<D>::V;
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= cap) return;
  if (b < cap - n_root) gap[b] = (int32_t)(cap - 1 - b);
  child0[b] = NONE;
  parent[b] = NONE;
  nonemask[b] = 0u;
  cellmask[2 * b] = cellmask[2 * b + 1] = 0ull;
  int32_t* row = nbr + (size_t)b * NBR_STRIDE;
  if (b >= n_root) {
    level[b] = -1;
    status[b] = ST_INACTIVE;
    X[3 * b] = X[3 * b + 1] = X[3 * b + 2] = 0.f;
    for (int k = 0; k < NBR_STRIDE; ++k) row[k] = NONE;
    return;
  }
  idset0[b] = (int32_t)b;
  level[b] = 0;
  status[b] = ST_UNREFINED;
  const int64_t pos = pos_of_id ? pos_of_id[b] : b;
  order0[pos] = (int32_t)b;
  const int bx = (int)(pos % nbx), by = (int)((pos / nbx) % nby),
            bz = (int)(pos / ((int64_t)nbx * nby));
  X[3 * b] = 4.f * bx;
  X[3 * b + 1] = 4.f * by;
  X[3 * b + 2] = D == 3 ? 4.f * bz : 0.f;
  for (int k = Nbr<D>::K; k < NBR_STRIDE; ++k) row[k] = NONE;
  static_for<0, Nbr<D>::K>([&](auto P) {
    constexpr int ex = NV::cx[P], ey = NV::cy[P], ez = NV::cz[P];
    int pos[3] = {bx + ex, by + ey, bz + ez};
    const int nbs[3] = {nbx, nby, nbz};
    unsigned crossed = 0;
    for (int ax = 0; ax < D; ++ax) {
      if (pos[ax] < 0 || pos[ax] >= nbs[ax]) {
        if ((periodic >> ax) & 1u) {
          pos[ax] = (pos[ax] + nbs[ax]) % nbs[ax];
        } else {
          crossed |= 1u << (2 * ax + (pos[ax] < 0 ? 0 : 1));
        }
      }
    }
    const int64_t npos = pos[0] + nbx * (pos[1] + (int64_t)nby * (D == 3 ? pos[2] : 0));
    row[P] = crossed ? wall_code[crossed] : (id_of_pos ? id_of_pos[npos] : (int32_t)npos);
  });
}

// solid bits of the cells of the blocks in `list` (cell centre strictly inside
// the prism [x0,x1] x [y0,y1] spanning z, root-cell units)
template <int D>
__global__ void k_solidmask(const int32_t* list, int n, const int32_t* level, const float* X,
                            double x0, double x1, double y0, double y1, uint64_t* sm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = list ? list[i] : i;
  const double h = 1.0 / (double)(1 << level[b]);
  uint64_t m = 0;
  for (int l = 0; l < Block<D>::M; ++l) {
    const double cx = X[3 * b] + (Block<D>::ci(l) + 0.5) * h;
    const double cy = X[3 * b + 1] + (Block<D>::cj(l) + 0.5) * h;
    if (cx > x0 && cx < x1 && cy > y0 && cy < y1) m |= 1ull << l;
  }
  sm[b] = m;
}

// ============================================================ adaptation
// keep a refine mark only for a leaf below L_max-1 without NONE neighbours,
// a coarsen mark only for a REFINED block
__global__ void k_eligible(int64_t cap, int8_t* marks, const int32_t* status,
                           const int32_t* level, const uint32_t* nonemask, int lmax) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= cap) return;
  const int m = marks[b];
  const int st = status[b];
  int8_t out = 0;
  if (m > 0 && st == ST_UNREFINED && level[b] < lmax - 1 && nonemask[b] == 0u) out = m > 1 ? 2 : 1;
  else if (m < 0 && st == ST_REFINED) out = -1;
  marks[b] = out;
}

__global__ void k_clear_refine(int64_t cap, int8_t* marks) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < cap && marks[b] > 0) marks[b] = 0;
}

// Step 3: a coarsen mark is reverted when a child has a same-level neighbour
// (any direction, including itself) that has children or is marked refine.
__global__ void k_revert(int64_t cap, int8_t* marks, const int32_t* child0, const int32_t* nbr,
                         int nk, int nc) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= cap || marks[b] != -1) return;
  const int c0 = child0[b];
  bool violating = false;
  for (int c = 0; c < nc && !violating; ++c) {
    const int32_t* row = nbr + (size_t)(c0 + c) * NBR_STRIDE;
    for (int k = 0; k < nk; ++k) {
      const int nb = row[k];
      if (nb >= 0 && (child0[nb] >= 0 || marks[nb] > 0)) {
        violating = true;
        break;
      }
    }
  }
  if (violating) marks[b] = 0;
}

// Steps 2 + 4 (Alg. 1): group i of N_c IDs popped from the gap stack top goes
// to the i-th refine-marked block; child c = head + c at X_P + offset * w.
template <int D>
__global__ void k_alloc(const int32_t* R, int nR, const int32_t* gap, int64_t n_gaps,
                        int32_t* child0, int32_t* level, float* X, int32_t* status,
                        int32_t* parent, int32_t* err) {
  constexpr int NC = Block<D>::NC;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nR * NC) return;
  const int i = t / NC, c = t - i * NC;
  const int P = R[i];
  const int64_t top = n_gaps - 1 - (int64_t)i * NC;
  const int head = gap[top];
  const int ch = head + c;
  if (gap[top - c] != ch) atomicExch(err, 1);   // groups must stay contiguous
  if (c == 0) child0[P] = head;
  const int lq = level[P] + 1;
  const float w = 4.f / (float)(1 << lq);
  level[ch] = lq;
  X[3 * ch] = X[3 * P] + (float)(c & 1) * w;
  X[3 * ch + 1] = X[3 * P + 1] + (float)((c >> 1) & 1) * w;
  X[3 * ch + 2] = X[3 * P + 2] + (D == 3 ? (float)((c >> 2) & 1) * w : 0.f);
  status[ch] = ST_UNREFINED;
  child0[ch] = NONE;
  parent[ch] = P;
}

// Step 5: freed child IDs, listed by (level, parent, child), are appended to
// the gap stack in reverse so that later pops return them in that order.
template <int D>
__global__ void k_push_gaps(const int32_t* CL, int n, const int32_t* child0, int32_t* gap,
                            int64_t base, int64_t total, int64_t off) {
  constexpr int NC = Block<D>::NC;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * NC) return;
  const int i = t / NC, c = t - i * NC;
  const int64_t idx = off + (int64_t)i * NC + c;
  gap[base + total - 1 - idx] = child0[CL[i]] + c;
}

template <int D>
__global__ void k_remove_children(const int32_t* C, int n, const int32_t* child0,
                                  int32_t* status, int32_t* level, int32_t* parent,
                                  int32_t* nbr, uint32_t* nonemask, uint64_t* cellmask) {
  constexpr int NC = Block<D>::NC;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * NC) return;
  const int i = t / NC, c = t - i * NC;
  const int ch = child0[C[i]] + c;
  status[ch] = ST_INACTIVE;
  level[ch] = -1;
  parent[ch] = NONE;
  nonemask[ch] = 0u;
  cellmask[2 * ch] = cellmask[2 * ch + 1] = 0ull;
  for (int k = 0; k < NBR_STRIDE; ++k) nbr[(size_t)ch * NBR_STRIDE + k] = NONE;
}

__global__ void k_finish_coarsened(const int32_t* C, int n, int32_t* child0, int32_t* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  child0[C[i]] = NONE;
  status[C[i]] = ST_UNREFINED;
}

// refined blocks: REFINED, or REFINED_PERMANENT when the mark froze them
__global__ void k_set_refined(const int32_t* list, int n, const int8_t* marks, int32_t* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) status[list[i]] = marks[list[i]] == 2 ? ST_PERM : ST_REFINED;
}

template <int D>
__global__ void k_append_children(const int32_t* R, int n, const int32_t* child0, int32_t* out) {
  constexpr int NC = Block<D>::NC;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * NC) return;
  const int i = t / NC, c = t - i * NC;
  out[t] = child0[R[i]] + c;
}

// Step 7: a refined block with a refined child is REFINED_WITH_CHILD.
__global__ void k_branch_leaf(int64_t cap, int32_t* status, const int32_t* child0, int nc) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= cap) return;
  const int st = status[b];
  if (st != ST_REFINED && st != ST_RWC) return;
  const int c0 = child0[b];
  bool any = false;
  for (int c = 0; c < nc; ++c) any |= status[c0 + c] >= ST_REFINED;
  status[b] = any ? ST_RWC : ST_REFINED;
}

// Step 8 (Alg. 2): neighbours of a child from its parent's neighbours.  Child c
// at (cx,cy,cz) in {0,1}^D looks in direction e at position c + e in
// {-1..2}^D of its parent's 2x2(x2) neighbourhood: the parent-level direction
// is floor((c+e)/2) and the child index there is (c+e) mod 2.  A parent-level
// neighbour without children gives NONE; wall codes pass through.
template <int D>
__global__ void k_relink(const int32_t* list, int n, const int32_t* parent,
                         const int32_t* child0, int32_t* nbr, uint32_t* nonemask,
                         uint64_t* cellmask) {
  using NV = typename Nbr<D>::V;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int X = list[i];
  const int P = parent[X];
  const int c = X - child0[P];
  const int cxyz[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
  const int32_t* prow = nbr + (size_t)P * NBR_STRIDE;
  int32_t* row = nbr + (size_t)X * NBR_STRIDE;
  uint32_t nm = 0u;
  static_for<0, Nbr<D>::K>([&](auto K) {
    constexpr int ex = NV::cx[K], ey = NV::cy[K], ez = NV::cz[K];
    const int e[3] = {ex, ey, ez};
    int code = 0, sub = 0, mul = 1, sub_mul = 1;
    for (int ax = 0; ax < D; ++ax) {
      const int t = cxyz[ax] + e[ax];
      const int s = t < 0 ? -1 : (t > 1 ? 1 : 0);
      code += (s + 1) * mul;
      sub += (t - 2 * s) * sub_mul;
      mul *= 3;
      sub_mul *= 2;
    }
    int kp = 0;
    static_for<0, Nbr<D>::K>([&](auto J) {
      constexpr int jcode = (NV::cx[J] + 1) + 3 * (NV::cy[J] + 1) + (D == 3 ? 9 * (NV::cz[J] + 1) : 0);
      if (jcode == code) kp = J;
    });
    const int pn = prow[kp];
    int v;
    if (pn >= 0) {
      const int pc = child0[pn];
      v = pc >= 0 ? pc + sub : NONE;
    } else {
      v = pn;
    }
    row[K] = v;
    if (v == NONE) nm |= 1u << K;
  });
  nonemask[X] = nm;
  // ghost and interface cells of the block (Section 3.4 cell classes)
  uint64_t gm = 0ull, im = 0ull;
  if (nm != 0u) {
    for (int l = 0; l < Block<D>::M; ++l) {
      const int cls = cell_class<D>(nm, Block<D>::ci(l), Block<D>::cj(l), Block<D>::ck(l));
      if (cls == 2) gm |= 1ull << l;
      else if (cls == 1) im |= 1ull << l;
    }
  }
  cellmask[2 * (size_t)X] = gm;
  cellmask[2 * (size_t)X + 1] = im;
}

// Distance rule (Section 4.4): a leaf on level L within thr (root-cell units,
// compared squared) of the solid prism or an outlet face is marked +1 (+2 when
// frozen); a refined block within thr loses its coarsening mark.  Products and
// sums are rounded separately so the decision is that of plain FP64.
__global__ void k_distance_marks(const int32_t* list, int n, int level, const int32_t* status,
                                 const float* X, int8_t* marks, double thr2, int targets,
                                 int has_solid, double sx0, double sx1, double sy0, double sy1,
                                 unsigned face_mask, double ex, double ey, double ez,
                                 int freeze) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = list[i];
  const double w = 4.0 / (double)(1 << level);
  const double x = (double)X[3 * b], y = (double)X[3 * b + 1], z = (double)X[3 * b + 2];
  bool within = false;
  if ((targets & 1) && has_solid) {
    const double dx = fmax(fmax(__dsub_rn(sx0, __dadd_rn(x, w)), __dsub_rn(x, sx1)), 0.0);
    const double dy = fmax(fmax(__dsub_rn(sy0, __dadd_rn(y, w)), __dsub_rn(y, sy1)), 0.0);
    within = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < thr2;
  }
  if (targets & 6) {   // outlet faces (bit 1), wall faces (bit 2): face_mask
    const double lo[3] = {x, y, z};
    const double ext[3] = {ex, ey, ez};
    for (int f = 0; f < 6; ++f) {
      if (!((face_mask >> f) & 1u)) continue;
      const int ax = f >> 1;
      const double d = (f & 1) ? __dsub_rn(ext[ax], __dadd_rn(lo[ax], w)) : lo[ax];
      if (__dmul_rn(d, d) < thr2) within = true;
    }
  }
  if (!within) return;
  const int st = status[b];
  if (st == ST_UNREFINED) marks[b] = freeze ? 2 : 1;
  else if (marks[b] < 0) marks[b] = 0;
}

int mesh_distance_marks(Instance* a) {
  const amr_config& c = a->cfg;
  if (!(c.refine_dist > 0.0) || c.refine_dist_targets == 0) return AMR_OK;
  unsigned faces = 0;   // the faces whose distance counts
  for (int f = 0; f < 2 * a->dim; ++f) {
    const int k = c.faces[f].kind;
    if ((c.refine_dist_targets & 2) && k == AMR_FACE_OUTLET) faces |= 1u << f;
    if ((c.refine_dist_targets & 4) && (k == AMR_FACE_NOSLIP || k == AMR_FACE_MOVING))
      faces |= 1u << f;
  }
  for (int L = 0; L < a->lmax; ++L) {
    if (a->n_ids[L] == 0) continue;
    const double thr = (c.refine_dist * c.nx / c.length_x) / std::ldexp(1.0, L);
    k_distance_marks<<<blocks_for(a->n_ids[L]), 256, 0, a->stream>>>(
        a->idset + (size_t)L * a->cap, (int)a->n_ids[L], L, a->status, a->X, a->marks, thr * thr,
        c.refine_dist_targets, c.has_solid, c.solid[0], c.solid[1], c.solid[2], c.solid[3],
        faces, (double)c.nx, (double)c.ny, (double)(a->dim == 3 ? c.nz : 0), c.refine_dist_freeze);
    a->launches += 1;
    AMR_CUDA(cudaGetLastError());
  }
  return AMR_OK;
}

// ================================================================ exports
template <int D>
__global__ void k_export_nbr(int64_t cap, const int32_t* nbr, const int32_t* child0, int mode,
                             int32_t* out) {
  constexpr int K = Nbr<D>::K;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cap * K) return;
  const int64_t b = t / K;
  const int k = (int)(t - b * K);
  const int v = nbr[(size_t)b * NBR_STRIDE + k];
  if (mode == 0) out[t] = v;
  else out[t] = v <= -2 ? v : (v >= 0 ? child0[v] : NONE);
}

template <int D>
__global__ void k_export_masks(int64_t cap, const int32_t* status, const uint64_t* cellmask,
                               uint8_t* out) {
  constexpr int M = Block<D>::M;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cap * M) return;
  const int64_t b = t / M;
  const int l = (int)(t - b * M);
  const bool ghost = (cellmask[2 * b] >> l) & 1ull;
  const bool iface = (cellmask[2 * b + 1] >> l) & 1ull;
  out[t] = status[b] == ST_INACTIVE ? 0 : (ghost ? 2 : (iface ? 1 : 0));
}

__global__ void k_export_coords(int64_t cap, int dim, const float* X, double* out) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= cap) return;
  for (int a = 0; a < dim; ++a) out[b * dim + a] = (double)X[3 * b + a];
}

// ============================================================ host side

template <int D>
static int init_root_t(Instance* a) {
  cudaStream_t s = a->stream;
  unsigned periodic = 0;
  for (int ax = 0; ax < D; ++ax)
    if (a->cfg.faces[2 * ax].kind == AMR_FACE_PERIODIC) periodic |= 1u << ax;
  const int32_t *id_of_pos = nullptr, *pos_of_id = nullptr;
  if (a->cfg.root_ids) {
    // both directions of the numbering, staged in the adaptation scratch lists
    std::vector<int32_t> inv((size_t)a->n_root);
    for (int64_t i = 0; i < a->n_root; ++i) inv[(size_t)a->cfg.root_ids[i]] = (int32_t)i;
    AMR_CUDA(cudaMemcpyAsync(a->tmp0, a->cfg.root_ids, sizeof(int32_t) * a->n_root,
                             cudaMemcpyHostToDevice, s));
    AMR_CUDA(cudaMemcpyAsync(a->tmp1, inv.data(), sizeof(int32_t) * a->n_root,
                             cudaMemcpyHostToDevice, s));
    AMR_CUDA(cudaStreamSynchronize(s));   // inv is a host temporary
    id_of_pos = a->tmp0;
    pos_of_id = a->tmp1;
  }
  k_init_root<D><<<blocks_for(a->cap), 256, 0, s>>>(
      a->cap, (int)a->n_root, a->nroot[0], a->nroot[1], a->nroot[2], periodic, a->wall_code,
      id_of_pos, pos_of_id, a->level, a->status, a->child0, a->parent, a->X, a->nbr, a->nonemask,
      a->cellmask, a->gap, a->idset, a->order);
  AMR_CUDA(cudaGetLastError());
  AMR_CUDA(cudaMemsetAsync(a->solidmask, 0, sizeof(uint64_t) * a->cap, s));
  if (a->solid) {
    k_solidmask<D><<<blocks_for(a->n_root), 256, 0, s>>>(nullptr, (int)a->n_root, a->level, a->X,
                                                         a->cfg.solid[0], a->cfg.solid[1],
                                                         a->cfg.solid[2], a->cfg.solid[3],
                                                         a->solidmask);
    AMR_CUDA(cudaGetLastError());
  }
  a->n_gaps = a->cap - a->n_root;
  for (int L = 0; L < a->lmax; ++L) a->n_ids[L] = 0;
  a->n_ids[0] = a->n_root;
  return mesh_refresh_lists(a);
}

int mesh_init_root(Instance* a) { return a->dim == 2 ? init_root_t<2>(a) : init_root_t<3>(a); }

// Per parent of a level's exchange list: how many of its children hold ghost
// cells, and the ghost and interface cells of its children (popcounts of the
// children's cell masks), summed into out[0..2].
__global__ void __launch_bounds__(256)
    k_exchange_cells(const int32_t* __restrict__ parents, int n,
                     const int32_t* __restrict__ child0, const uint64_t* __restrict__ cellmask,
                     int nc, unsigned long long* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long kids = 0, ghost = 0, iface = 0;
  if (i < n) {
    const int c0 = child0[parents[i]];
    for (int c = 0; c < nc; ++c) {
      const uint64_t g = cellmask[2 * (size_t)(c0 + c)];
      kids += g != 0ull;
      ghost += __popcll(g);
      iface += __popcll(cellmask[2 * (size_t)(c0 + c) + 1]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    kids += __shfl_down_sync(0xffffffffu, kids, o);
    ghost += __shfl_down_sync(0xffffffffu, ghost, o);
    iface += __shfl_down_sync(0xffffffffu, iface, o);
  }
  if ((threadIdx.x & 31) == 0 && (kids | ghost | iface)) {
    atomicAdd(out, kids);
    atomicAdd(out + 1, ghost);
    atomicAdd(out + 2, iface);
  }
}

int mesh_refresh_lists(Instance* a) {
  for (int L = 0; L < a->lmax; ++L) {
    int32_t* ord = a->order + (size_t)L * a->cap;
    const int64_t n = a->n_ids[L];
    if (L > 0) {
      // tree order of level L: the children of the refined blocks of level
      // L-1, taken in that level's tree order (roots were placed at init)
      const int32_t* up = a->order + (size_t)(L - 1) * a->cap;
      int64_t n_ref = 0;
      AMR_TRY(compact(a, a->n_ids[L - 1], PHasKids{up, a->child0}, VList{up}, a->tmp2, &n_ref));
      if (n_ref * a->nc != n) {
        set_error("tree order: the children of level " + std::to_string(L - 1) +
                  " do not match the ID set of level " + std::to_string(L));
        return AMR_E_CUDA;
      }
      if (n_ref > 0) {
        if (a->dim == 2)
          k_append_children<2><<<blocks_for(n), 256, 0, a->stream>>>(a->tmp2, (int)n_ref,
                                                                       a->child0, ord);
        else
          k_append_children<3><<<blocks_for(n), 256, 0, a->stream>>>(a->tmp2, (int)n_ref,
                                                                       a->child0, ord);
        a->launches += 1;
        AMR_CUDA(cudaGetLastError());
      }
    }
    PActive act{ord, a->status, a->child0, a->nonemask, a->nc, false};
    PActive par{ord, a->status, a->child0, a->nonemask, a->nc, true};
    AMR_TRY(compact(a, n, act, VList{ord}, a->active + (size_t)L * a->cap, &a->n_active[L]));
    AMR_TRY(compact(a, n, par, VList{ord}, a->parents + (size_t)L * a->cap, &a->n_parents[L]));
    AMR_TRY(compact(a, n, PLeaf{ord, a->status}, VIdent{}, nullptr, &a->n_leaves[L], 0, false));
    AMR_TRY(compact(a, n, PNoneNbr{ord, a->nonemask}, VList{ord}, a->bnd + (size_t)L * a->cap,
                    &a->n_bnd[L]));
  }
  // averaging groups of every level's boundary blocks, packed by level
  int64_t off = 0;
  for (int L = 0; L < a->lmax; ++L) {
    a->agrp_off[L] = off;
    a->n_agrp[L] = 0;
    if (L == 0 || a->n_bnd[L] == 0) continue;
    const int32_t* bl = a->bnd + (size_t)L * a->cap;
    if (a->dim == 2)
      AMR_TRY(compact(a, a->n_bnd[L] * 4,
                      PAvgGroup<2>{bl, a->cellmask, a->parent, a->child0, a->sm()},
                      VAvgGroup<2>{bl}, a->agrp + off, &a->n_agrp[L]));
    else
      AMR_TRY(compact(a, a->n_bnd[L] * 8,
                      PAvgGroup<3>{bl, a->cellmask, a->parent, a->child0, a->sm()},
                      VAvgGroup<3>{bl}, a->agrp + off, &a->n_agrp[L]));
    off += a->n_agrp[L];
  }
  // exchange work per level, for the profile's algorithmic bytes
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(a->red);
  AMR_CUDA(cudaMemsetAsync(cnt, 0, 3 * sizeof(unsigned long long) * a->lmax, a->stream));
  for (int L = 0; L + 1 < a->lmax; ++L) {
    if (a->n_parents[L] == 0) continue;
    k_exchange_cells<<<blocks_for(a->n_parents[L]), 256, 0, a->stream>>>(
        a->parents + (size_t)L * a->cap, (int)a->n_parents[L], a->child0, a->cellmask, a->nc,
        cnt + 3 * L);
    a->launches += 1;
  }
  AMR_CUDA(cudaGetLastError());
  unsigned long long h[3 * AMR_MAX_LEVELS] = {};
  AMR_CUDA(cudaMemcpyAsync(h, cnt, 3 * sizeof(unsigned long long) * a->lmax,
                           cudaMemcpyDeviceToHost, a->stream));
  AMR_CUDA(cudaStreamSynchronize(a->stream));
  for (int L = 0; L < a->lmax; ++L) {
    a->n_ghost_children[L] = (int64_t)h[3 * L];
    a->n_ghost_cells[L] = (int64_t)h[3 * L + 1];
    a->n_iface_cells[L] = (int64_t)h[3 * L + 2];
  }
  return AMR_OK;
}

template <int D>
static int adapt_t(Instance* a, amr_adapt_stats* st) {
  constexpr int NC = Block<D>::NC;
  cudaStream_t s = a->stream;
  const int64_t cap = a->cap;
  int32_t* R = a->tmp0;        // refine-marked blocks, ascending
  int32_t* C = a->tmp1;        // coarsen-marked blocks, ascending
  int32_t* W = a->tmp2;        // work list

  k_eligible<<<blocks_for(cap), 256, 0, s>>>(cap, a->marks, a->status, a->level, a->nonemask,
                                              a->lmax);
  a->launches += 1;
  AMR_CUDA(cudaGetLastError());
  int64_t nR = 0, nC = 0, nC0 = 0;
  AMR_TRY(compact(a, cap, PMarkPos{a->marks}, VIdent{}, R, &nR));
  AMR_TRY(compact(a, cap, PMarkEq{a->marks, -1}, VIdent{}, nullptr, &nC0, 0, false));
  st->n_marked_refine = nR;
  st->n_marked_coarsen = nC0;
  if (nR * NC > a->n_gaps) {
    st->capacity_error = 1;
    k_clear_refine<<<blocks_for(cap), 256, 0, s>>>(cap, a->marks);
    a->launches += 1;
    nR = 0;
  }
  k_revert<<<blocks_for(cap), 256, 0, s>>>(cap, a->marks, a->child0, a->nbr, a->nk, NC);
  a->launches += 1;
  AMR_CUDA(cudaGetLastError());
  AMR_TRY(compact(a, cap, PMarkEq{a->marks, -1}, VIdent{}, C, &nC));
  st->n_refined = nR;
  st->n_coarsened = nC;
  if (nR == 0 && nC == 0) return AMR_OK;

  // refine-marked blocks grouped by level (stable): R_L = C + offR[L] below
  std::vector<int64_t> nRL(a->lmax, 0), offR(a->lmax + 1, 0);
  std::vector<int64_t> nCL(a->lmax, 0);

  adapt_phase(a, PK_ADAPT_ALLOC);
  // allocation (reads the gap stack top before any push)
  AMR_CUDA(cudaMemsetAsync(a->dcount + 8, 0, sizeof(int32_t), s));
  if (nR > 0) {
    k_alloc<D><<<blocks_for(nR * NC), 256, 0, s>>>(R, (int)nR, a->gap, a->n_gaps, a->child0,
                                                    a->level, a->X, a->status, a->parent,
                                                    a->dcount + 8);
    a->launches += 1;
    AMR_CUDA(cudaGetLastError());
  }
  a->n_gaps -= nR * NC;
  // gap pushes, level by level
  int64_t off = 0;
  for (int L = 0; L < a->lmax; ++L) {
    AMR_TRY(compact(a, nC, PLevelEq{C, a->level, L}, VList{C}, W, &nCL[L]));
    if (nCL[L] > 0) {
      k_push_gaps<D><<<blocks_for(nCL[L] * NC), 256, 0, s>>>(W, (int)nCL[L], a->child0, a->gap,
                                                              a->n_gaps, nC * NC, off);
      a->launches += 1;
      AMR_CUDA(cudaGetLastError());
    }
    off += nCL[L] * NC;
  }
  if (nC > 0) {
    // values stored in the removed children for their staying neighbours go
    // back to those neighbours (the neighbour rows still hold the old links)
    a->ops->coarsen_fixup(s, C, (int)nC, a->child0, a->parent, a->marks, a->nbr, a->sm(),
                          a->level, a->f[0], a->f[1], a->cur);
    a->launches += 1;
    k_remove_children<D><<<blocks_for(nC * NC), 256, 0, s>>>(C, (int)nC, a->child0, a->status,
                                                              a->level, a->parent, a->nbr,
                                                              a->nonemask, a->cellmask);
    a->launches += 1;
    k_finish_coarsened<<<blocks_for(nC), 256, 0, s>>>(C, (int)nC, a->child0, a->status);
    a->launches += 1;
    AMR_CUDA(cudaGetLastError());
  }
  a->n_gaps += nC * NC;
  if (nR > 0) {
    k_set_refined<<<blocks_for(nR), 256, 0, s>>>(R, (int)nR, a->marks, a->status);
    a->launches += 1;
    AMR_CUDA(cudaGetLastError());
  }
  adapt_phase(a, PK_ADAPT_IDSETS);
  // R grouped by level into C's storage (C is no longer needed)
  for (int L = 0; L < a->lmax; ++L) {
    AMR_TRY(compact(a, nR, PLevelEq{R, a->level, L}, VList{R}, C + offR[L], &nRL[L]));
    offR[L + 1] = offR[L] + nRL[L];
  }
  // ID sets
  for (int L = 1; L < a->lmax; ++L) {
    int32_t* ids = a->idset + (size_t)L * cap;
    int64_t kept = 0;
    AMR_TRY(compact(a, a->n_ids[L], PAlive{ids, a->status}, VList{ids}, W, &kept));
    const int64_t nadd = nRL[L - 1] * NC;
    if (nadd > 0) {
      k_append_children<D><<<blocks_for(nadd), 256, 0, s>>>(C + offR[L - 1], (int)nRL[L - 1],
                                                            a->child0, W + kept);
      a->launches += 1;
      AMR_CUDA(cudaGetLastError());
    }
    if (kept + nadd > 0)
      AMR_CUDA(cudaMemcpyAsync(ids, W, sizeof(int32_t) * (kept + nadd), cudaMemcpyDeviceToDevice, s));
    a->n_ids[L] = kept + nadd;
  }
  adapt_phase(a, PK_ADAPT_RELINK);
  k_branch_leaf<<<blocks_for(cap), 256, 0, s>>>(cap, a->status, a->child0, NC);
  a->launches += 1;
  AMR_CUDA(cudaGetLastError());
  for (int L = 1; L < a->lmax; ++L) {
    if (a->n_ids[L] == 0) continue;
    k_relink<D><<<blocks_for(a->n_ids[L], 128), 128, 0, s>>>(a->idset + (size_t)L * cap,
                                                        (int)a->n_ids[L], a->parent, a->child0,
                                                        a->nbr, a->nonemask, a->cellmask);
    a->launches += 1;
    AMR_CUDA(cudaGetLastError());
  }
  adapt_phase(a, PK_ADAPT_CHILDREN);
  // solid bits of the new children, then every cell of them from the parents
  for (int L = 0; L + 1 < a->lmax; ++L) {
    if (nRL[L] == 0) continue;
    const int64_t nnew = nRL[L] * NC;
    k_append_children<D><<<blocks_for(nnew), 256, 0, s>>>(C + offR[L], (int)nRL[L], a->child0, W);
    a->launches += 1;
    if (a->solid)
      k_solidmask<D><<<blocks_for(nnew), 256, 0, s>>>(W, (int)nnew, a->level, a->X,
                                                      a->cfg.solid[0], a->cfg.solid[1],
                                                      a->cfg.solid[2], a->cfg.solid[3],
                                                      a->solidmask);
      a->launches += 1;
    AMR_CUDA(cudaGetLastError());
    const double ratio = a->tau[L + 1] / (2.0 * a->tau[L]);
    a->ops->interp(s, C + offR[L], (int)nRL[L], a->fbuf(L, 0), a->fbuf(L + 1, 0), a->child0, a->cellmask, a->nbr, a->sm(), a->parent, a->marks, ratio,
                   1 | a->interp_bits(), a->solid);
    a->launches += 1;
    AMR_CUDA(cudaGetLastError());
  }
  int32_t err = 0;
  AMR_CUDA(cudaMemcpyAsync(&err, a->dcount + 8, sizeof(err), cudaMemcpyDeviceToHost, s));
  AMR_CUDA(cudaStreamSynchronize(s));
  if (err) {
    set_error("gap stack lost its group structure");
    return AMR_E_INVAL;
  }
  adapt_phase(a, PK_ADAPT_LISTS);
  return mesh_refresh_lists(a);
}

int mesh_adapt(Instance* a, bool /*external*/, amr_adapt_stats* st) {
  return a->dim == 2 ? adapt_t<2>(a, st) : adapt_t<3>(a, st);
}

int64_t mesh_export_bytes(const Instance* a, int what) {
  const int64_t cap = a->cap;
  switch (what) {
    case AMR_BLOCKS: return 4 * cap * 4;
    case AMR_COORDS: return cap * a->dim * 8;
    case AMR_NBR:
    case AMR_NBR_CHILD: return cap * a->nk * 4;
    case AMR_IDSETS: return (int64_t)a->lmax * cap * 4;
    case AMR_GAPS: return cap * 4;
    case AMR_MASKS: return cap * a->M;
    default: return -1;
  }
}

int mesh_export(Instance* a, int what, void* dst) {
  cudaStream_t s = a->stream;
  const int64_t cap = a->cap;
  const bool d3 = a->dim == 3;
  switch (what) {
    case AMR_BLOCKS: {
      int32_t* o = (int32_t*)dst;
      AMR_CUDA(cudaMemcpyAsync(o, a->level, cap * 4, cudaMemcpyDeviceToDevice, s));
      AMR_CUDA(cudaMemcpyAsync(o + cap, a->status, cap * 4, cudaMemcpyDeviceToDevice, s));
      AMR_CUDA(cudaMemcpyAsync(o + 2 * cap, a->child0, cap * 4, cudaMemcpyDeviceToDevice, s));
      AMR_CUDA(cudaMemcpyAsync(o + 3 * cap, a->parent, cap * 4, cudaMemcpyDeviceToDevice, s));
      return AMR_OK;
    }
    case AMR_COORDS:
      k_export_coords<<<blocks_for(cap), 256, 0, s>>>(cap, a->dim, a->X, (double*)dst);
      break;
    case AMR_NBR:
    case AMR_NBR_CHILD: {
      const int mode = what == AMR_NBR ? 0 : 1;
      if (d3)
        k_export_nbr<3><<<blocks_for(cap * 27), 256, 0, s>>>(cap, a->nbr, a->child0, mode, (int32_t*)dst);
      else
        k_export_nbr<2><<<blocks_for(cap * 9), 256, 0, s>>>(cap, a->nbr, a->child0, mode, (int32_t*)dst);
      break;
    }
    case AMR_IDSETS:
      AMR_CUDA(cudaMemcpyAsync(dst, a->idset, (size_t)a->lmax * cap * 4, cudaMemcpyDeviceToDevice, s));
      return AMR_OK;
    case AMR_GAPS:
      AMR_CUDA(cudaMemcpyAsync(dst, a->gap, cap * 4, cudaMemcpyDeviceToDevice, s));
      return AMR_OK;
    case AMR_MASKS:
      if (d3)
        k_export_masks<3><<<blocks_for(cap * 64), 256, 0, s>>>(cap, a->status, a->cellmask, (uint8_t*)dst);
      else
        k_export_masks<2><<<blocks_for(cap * 16), 256, 0, s>>>(cap, a->status, a->cellmask, (uint8_t*)dst);
      break;
    default:
      return AMR_E_INVAL;
  }
  AMR_CUDA(cudaGetLastError());
  return AMR_OK;
}

}  // namespace amr
