// Templated LBM kernels of the block forest.  Included once per velocity-set
// translation unit, which instantiates them through AMR_LBM_OPS.
//
// Population layout (every storage type): block-major, g[b * Q M + p * M + l],
// M = 4^D cells per block, l = i + 4 j + 16 k (collide_stream.cuh).  Two buffers A/B
// are used per level in ping-pong; a level's current buffer is bit L of `cur`.
// The stored values are the outgoing post-collision populations; every kernel
// reads a cell's pre-collision populations with gather_cell and writes them
// with scatter_cell (collide_stream.cuh).
#pragma once
#include "collide_stream.cuh"

#include <algorithm>

namespace amr {

// =========================================== coarse-to-fine linear interpolation
// Per parent block: every parent cell rescales its populations to the fine
// level (f_eq + (f - f_eq) r, Section 3.4.1) into shared memory; then, for
// each child c, fine cell (I,J,K) takes the multilinear interpolant of the
// 2^D parent cells of quadrant c at local coordinates -1/4 + I/2.  Writes the
// ghost cells of every child (mode_all = 0) or every cell (mode_all = 1).
// Neighbour rows of the blocks a CTA works on, copied to shared memory
// (the gathers and scatters read one entry per link).
template <int D>
__device__ __forceinline__ void stage_row(int32_t* dst, const int32_t* __restrict__ nbr, int b,
                                          int t, int nt) {
  constexpr int NK = Nbr<D>::K;
  for (int k = t; k < NK; k += nt) dst[k] = b >= 0 ? __ldg(nbr + (size_t)b * NBR_STRIDE + k) : NONE;
}

template <int D, int Q, class T, bool SOLID, bool COH = false>
__device__ __forceinline__ void interp_stage(typename Store<T>::R (*sF)[Block<D>::M],
                                             const T* __restrict__ fpar, int P,
                                             int l, double ratio, const int32_t* prow,
                                             const uint64_t* __restrict__ solidmask) {
  using S = Store<T>;
  using R = typename S::R;
  R f[Q];
  gather_cell<D, Q, T, SOLID, COH>(f, fpar, P, l, prow, solidmask);
  R rho, ux, uy, uz;
  moments<D, Q>(f, rho, ux, uy, uz);
  const R usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
  const R r = R(ratio);
  static_for<0, Q>([&](auto Pp) {
    const R e = feq<D, Q, Pp>(rho, ux, uy, uz, usq15);
    sF[Pp][l] = e + (f[Pp] - e) * r;
  });
}

// Store the interpolated populations v of cell l of child ch.  mode_all (new
// children of an adaptation): values that old neighbours stored in the new
// block's place are moved first (scatter_cell MOVE); a solid cell takes the
// rest state.
template <int D, int Q, class T, bool SOLID>
__device__ __forceinline__ void store_child_cell(typename Store<T>::R (&v)[Q], T* __restrict__ fch,
                                                 int ch, int l, const int32_t* row,
                                                 const uint64_t* __restrict__ solidmask,
                                                 const int32_t* __restrict__ parent,
                                                 const int8_t* __restrict__ marks, int mode_all) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  if (mode_all & 4) {   // the level step: as they are, into the child's own slots
    const size_t own = (size_t)ch * (Q * M) + l;
    static_for<0, Q>([&](auto Pp) { fch[own + (size_t)Pp * M] = S::template save<D, Q, Pp>(v[Pp]); });
    return;
  }
  if (mode_all & 1) {
    auto is_new = [&](int blk) {
      const int pp = __ldg(parent + blk);
      return pp >= 0 && __ldg(marks + pp) > 0;
    };
    scatter_cell<D, Q, T, SOLID, true>(v, fch, ch, l, row, solidmask, is_new);
  } else {
    scatter_cell<D, Q, T, SOLID>(v, fch, ch, l, row, solidmask);
  }
}

template <int D, int Q, class T, bool SOLID>
__device__ __forceinline__ void interp_children(const typename Store<T>::R (*sF)[Block<D>::M],
                                                int l, T* __restrict__ fch, int c0, const uint64_t* __restrict__ cellmask,
                                                const int32_t (*crow)[Nbr<D>::K],
                                                const uint64_t* __restrict__ solidmask,
                                                const int32_t* __restrict__ parent,
                                                const int8_t* __restrict__ marks, int mode_all) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int NC = Block<D>::NC;
  const int i = Block<D>::ci(l), j = Block<D>::cj(l), k = Block<D>::ck(l);
  const R x = R(-0.25) + R(0.5) * R(i);
  const R y = R(-0.25) + R(0.5) * R(j);
  const R z = R(-0.25) + R(0.5) * R(k);
  R wgt[NC];
#pragma unroll
  for (int a = 0; a < NC; ++a) {
    R wv = ((a & 1) ? x : R(1) - x) * ((a & 2) ? y : R(1) - y);
    if (D == 3) wv *= (a & 4) ? z : R(1) - z;
    wgt[a] = wv;
  }
#pragma unroll 1
  for (int c = 0; c < NC; ++c) {
    const int ch = c0 + c;
    if (!(mode_all & 1)) {
      const uint64_t gm = __ldg(cellmask + 2 * (size_t)ch);   // ghost cells of the child
      if (gm == 0ull) continue;
      if (!((gm >> l) & 1ull)) continue;
    }
    R v[Q];
    if (SOLID && solidmask && ((__ldg(solidmask + ch) >> l) & 1ull)) {
      if (!(mode_all & 1)) continue;                 // solid cells keep the rest state
      static_for<0, Q>([&](auto Pp) { v[Pp] = R(VS<D, Q>::w[Pp]); });
    } else {
      const int qx = c & 1, qy = (c >> 1) & 1, qz = (c >> 2) & 1;
      int corner[NC];
#pragma unroll
      for (int a = 0; a < NC; ++a)
        corner[a] = Block<D>::cell(2 * qx + (a & 1), 2 * qy + ((a >> 1) & 1),
                                   2 * qz + ((a >> 2) & 1));
      static_for<0, Q>([&](auto Pp) {
        R acc = R(0);
#pragma unroll
        for (int a = 0; a < NC; ++a) acc += wgt[a] * sF[Pp][corner[a]];
        v[Pp] = acc;
      });
    }
    store_child_cell<D, Q, T, SOLID>(v, fch, ch, l, crow[c], solidmask, parent, marks,
                                     mode_all);
  }
}

template <int D, int Q, class T, bool SOLID>
__global__ void __launch_bounds__(128, 8)
    k_interp(const int32_t* __restrict__ list, int n, const T* __restrict__ fpar,
             T* __restrict__ fch, const int32_t* __restrict__ child0,
             const uint64_t* __restrict__ cellmask, const int32_t* __restrict__ nbr,
             const uint64_t* __restrict__ solidmask, const int32_t* __restrict__ parent,
             const int8_t* __restrict__ marks, double ratio, int mode_all) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  constexpr int NK = Nbr<D>::K;
  constexpr int BPC = 128 / M;
  __shared__ R sF[BPC][Q][M];
  __shared__ int32_t s_row[BPC][1 + NC][NK];   // the parent's row, then its children's
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int bi = blockIdx.x * BPC + slot;
  const bool valid = bi < n;
  const int P = valid ? list[bi] : 0;
  const int c0 = valid ? child0[P] : 0;
  for (int r = 0; r <= NC; ++r)
    stage_row<D>(s_row[slot][r], nbr, valid ? (r == 0 ? P : c0 + r - 1) : NONE, l, M);
  __syncthreads();
  if (valid) interp_stage<D, Q, T, SOLID>(sF[slot], fpar, P, l, ratio, s_row[slot][0],
                                          solidmask);
  __syncthreads();
  if (!valid) return;
  interp_children<D, Q, T, SOLID>(sF[slot], l, fch, c0, cellmask, s_row[slot] + 1,
                                  solidmask, parent, marks, mode_all);
}

// ========================================== coarse-to-fine cubic interpolation
// Section 3.4.2: the interpolant is the polynomial with exponents 0..3 in
// each direction through all 4^D rescaled cells of the parent block, on the
// unit square / cube spanned by the corner cell centres (parent cell m at
// m/3).  That polynomial is the tensor product of 1D cubic Lagrange bases on
// the nodes 0, 1/3, 2/3, 1, so it is evaluated one direction at a time: child
// c's cell I sits at x = -1/12 + I/6 + c_x 2/3, i.e. at position q = I + 4 c_x
// of eight, and F(x, y, z) = sum_l w_K(l) sum_n w_J(n) sum_m w_I(m) F_mnl.
// A CTA of 64 threads handles 64/M parents: every thread rescales one parent
// cell into shared memory; then, child by child, the x, y (and z) sums run in
// three passes through shared memory, each thread producing one of the 4^D
// partial sums per pass (4 multiply-adds per population).
struct CubicW {
  double w[8][4];   // w[q][m]: weight of node m at position q = I + 4 c_d
};
constexpr CubicW make_cubic_w() {
  CubicW t{};
  for (int q = 0; q < 8; ++q)
    for (int m = 0; m < 4; ++m) {
      // in units of 1/12: position 2q - 1, nodes 0, 4, 8, 12
      double v = 1.0;
      for (int j = 0; j < 4; ++j)
        if (j != m) v *= double(2 * q - 1 - 4 * j) / double(4 * m - 4 * j);
      t.w[q][m] = v;
    }
  return t;
}
static __constant__ CubicW c_cubic_w = make_cubic_w();

template <int D, int Q, class T, bool SOLID>
__global__ void __launch_bounds__(64)
    k_interp_cubic(const int32_t* __restrict__ list, int n, const T* __restrict__ fpar,
                   T* __restrict__ fch, const int32_t* __restrict__ child0,
                   const uint64_t* __restrict__ cellmask, const int32_t* __restrict__ nbr,
                   const uint64_t* __restrict__ solidmask, const int32_t* __restrict__ parent,
                   const int8_t* __restrict__ marks, double ratio, int mode_all) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  constexpr int PPC = 64 / M;   // parents per CTA
  __shared__ R sF[PPC][Q][M];   // rescaled parent cells
  __shared__ R sA[PPC][Q][M];   // x sums
  __shared__ R sB[D == 3 ? PPC : 1][D == 3 ? Q : 1][M];   // x-y sums (3D)
  __shared__ R sw[8][4];
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int i = Block<D>::ci(l), j = Block<D>::cj(l), k = Block<D>::ck(l);
  if (threadIdx.x < 32) sw[threadIdx.x >> 2][threadIdx.x & 3] = R(c_cubic_w.w[threadIdx.x >> 2][threadIdx.x & 3]);
  constexpr int NK = Nbr<D>::K;
  __shared__ int32_t s_row[PPC][1 + NC][NK];   // the parent's row, then its children's
  const int bi = blockIdx.x * PPC + slot;
  const bool valid = bi < n;
  const int P = valid ? list[bi] : 0;
  const int c0 = valid ? child0[P] : 0;
  for (int r = 0; r <= NC; ++r)
    stage_row<D>(s_row[slot][r], nbr, valid ? (r == 0 ? P : c0 + r - 1) : NONE, l, M);
  __syncthreads();
  if (valid) interp_stage<D, Q, T, SOLID>(sF[slot], fpar, P, l, ratio, s_row[slot][0],
                                          solidmask);
  __syncthreads();
  for (int c = 0; c < NC; ++c) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    const int ch = c0 + c;
    uint64_t gm = 0ull;
    if (valid) gm = (mode_all & 1) ? ~0ull : __ldg(cellmask + 2 * (size_t)ch);
    const bool need = gm != 0ull;   // uniform over the parent's threads
    // pass 1: thread (i, j, k) -> sum_m w_i(m) F(m, j, k)
    if (need) {
      const R w0 = sw[i + 4 * cx][0], w1 = sw[i + 4 * cx][1], w2 = sw[i + 4 * cx][2],
              w3 = sw[i + 4 * cx][3];
      const int r = 4 * j + 16 * k;
      static_for<0, Q>([&](auto Pp) {
        const R* f = sF[slot][Pp];
        sA[slot][Pp][l] = w0 * f[r] + w1 * f[r + 1] + w2 * f[r + 2] + w3 * f[r + 3];
      });
    }
    __syncthreads();
    // pass 2: thread (i, j, k) -> sum_n w_j(n) A(i, n, k)
    R out2[D == 2 ? Q : 1];
    if (need) {
      const R w0 = sw[j + 4 * cy][0], w1 = sw[j + 4 * cy][1], w2 = sw[j + 4 * cy][2],
              w3 = sw[j + 4 * cy][3];
      const int r = i + 16 * k;
      static_for<0, Q>([&](auto Pp) {
        const R* a = sA[slot][Pp];
        const R v = w0 * a[r] + w1 * a[r + 4] + w2 * a[r + 8] + w3 * a[r + 12];
        if constexpr (D == 3) sB[slot][Pp][l] = v;
        else out2[Pp] = v;
      });
    }
    if constexpr (D == 3) {
      __syncthreads();
    }
    // pass 3 (3D): thread (i, j, k) -> sum_l w_k(l) B(i, j, l); then the write
    if (need && ((gm >> l) & 1ull)) {
      R v[Q];
      const bool solid_cell = SOLID && solidmask && ((__ldg(solidmask + ch) >> l) & 1ull);
      if (solid_cell) {
        static_for<0, Q>([&](auto Pp) { v[Pp] = R(VS<D, Q>::w[Pp]); });
      } else if constexpr (D == 3) {
        const R w0 = sw[k + 4 * cz][0], w1 = sw[k + 4 * cz][1], w2 = sw[k + 4 * cz][2],
                w3 = sw[k + 4 * cz][3];
        const int r = i + 4 * j;
        static_for<0, Q>([&](auto Pp) {
          const R* b = sB[slot][Pp];
          v[Pp] = w0 * b[r] + w1 * b[r + 16] + w2 * b[r + 32] + w3 * b[r + 48];
        });
      } else {
        static_for<0, Q>([&](auto Pp) { v[Pp] = out2[Pp]; });
      }
      // solid cells: the rest state for new children, untouched otherwise
      if (!solid_cell || (mode_all & 1))
        store_child_cell<D, Q, T, SOLID>(v, fch, ch, l, s_row[slot][1 + c], solidmask,
                                         parent, marks, mode_all);
    }
    (void)cz;
    // 2D: pass 1 of the next child rewrites the x sums that pass 2 just read
    if constexpr (D == 2) __syncthreads();
  }
}

// ===================================================== fine-to-coarse averaging
// Section 3.4.3.  A child covers 2^D parent cells (g = gx + 2 gy [+ 4 gz]),
// each the mean of a 2^D group of the child's fine cells, which share one
// class.  A group is taken when its cells are interface cells (mode_sync = 0)
// or not ghosts (mode_sync = 1), and its parent cell is not solid.  One thread
// per fine cell gathers it and rescales it to the coarse level
// (f_eq + (f - f_eq) r) into shared memory; then one thread per taken group
// sums its 2^D cells and scatters the mean into the parent cell.
template <int D>
__device__ __forceinline__ bool average_group_taken(const uint64_t* __restrict__ cellmask, int ch,
                                                    int g, int mode_sync) {
  const int f0 = Block<D>::cell(2 * (g & 1), 2 * ((g >> 1) & 1), 2 * ((g >> 2) & 1));
  if (mode_sync) return !((__ldg(cellmask + 2 * (size_t)ch) >> f0) & 1ull);
  return (__ldg(cellmask + 2 * (size_t)ch + 1) >> f0) & 1ull;
}

template <int D, int Q, class T, bool SOLID, bool COH = false>
__device__ __forceinline__ void average_child(typename Store<T>::R (*sR)[Block<D>::M],
                                              bool valid, int P, int c, int ch,
                                              int l, T* __restrict__ fpar,
                                              const T* __restrict__ fch, const uint64_t* __restrict__ cellmask,
                                              const int32_t* crow, const int32_t* prow,
                                              const uint64_t* __restrict__ solidmask,
                                              double ratio, int mode_sync) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  const int i = Block<D>::ci(l), j = Block<D>::cj(l), k = Block<D>::ck(l);
  const int g = (i >> 1) + 2 * (j >> 1) + (D == 3 ? 4 * (k >> 1) : 0);
  auto parent_cell = [&](int gg) {
    return Block<D>::cell(2 * (c & 1) + (gg & 1), 2 * ((c >> 1) & 1) + ((gg >> 1) & 1),
                          2 * ((c >> 2) & 1) + ((gg >> 2) & 1));
  };
  // group gg is taken: its class matches and its parent cell is not solid
  auto taken = [&](int gg) {
    return average_group_taken<D>(cellmask, ch, gg, mode_sync) &&
           !(SOLID && solidmask && ((__ldg(solidmask + P) >> parent_cell(gg)) & 1ull));
  };
  if (valid && taken(g)) {
    R f[Q];
    gather_cell<D, Q, T, SOLID, COH>(f, fch, ch, l, crow, solidmask);
    R rho, ux, uy, uz;
    moments<D, Q>(f, rho, ux, uy, uz);
    const R usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
    const R r = R(ratio);
    static_for<0, Q>([&](auto Pp) {
      const R e = feq<D, Q, Pp>(rho, ux, uy, uz, usq15);
      sR[Pp][l] = e + (f[Pp] - e) * r;
    });
  }
  __syncthreads();
  // one thread per taken group: the mean of its 2^D rescaled cells,
  // scattered into the parent cell
  if (valid && l < NC && taken(l)) {
    const int f0 = Block<D>::cell(2 * (l & 1), 2 * ((l >> 1) & 1), 2 * ((l >> 2) & 1));
    R acc[Q];
    const R inv = R(1) / R(NC);
    static_for<0, Q>([&](auto Pp) {
      R a = R(0);
#pragma unroll
      for (int s = 0; s < NC; ++s) a += sR[Pp][f0 + Block<D>::cell(s & 1, (s >> 1) & 1, (s >> 2) & 1)];
      acc[Pp] = a * inv;
    });
    scatter_cell<D, Q, T, SOLID>(acc, fpar, P, parent_cell(l), prow, solidmask);
  }
}

// 128 threads = 128 / 4^D children.  by_parent: child item i is child i % N_c
// of list[i / N_c] (skipped when the parent has no children, or, in
// mode_sync, is not refined); else child item i is the block list[i] (a
// block with a NONE neighbour: the only blocks with interface cells).
template <int D, int Q, class T, bool SOLID>
__global__ void __launch_bounds__(128)
    k_average(const int32_t* __restrict__ list, int64_t n_items, bool by_parent,
              T* __restrict__ fpar, const T* __restrict__ fch, const int32_t* __restrict__ child0, const int32_t* __restrict__ parent,
              const uint64_t* __restrict__ cellmask, const int32_t* __restrict__ status,
              const int32_t* __restrict__ nbr, const uint64_t* __restrict__ solidmask,
              double ratio, int mode_sync) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  constexpr int NK = Nbr<D>::K;
  constexpr int CPC = 128 / M;
  __shared__ R sR[CPC][Q][M];
  __shared__ int32_t s_row[CPC][2][NK];   // the child's row and its parent's
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int64_t item = (int64_t)blockIdx.x * CPC + slot;
  bool valid = item < n_items;
  int P = 0, c = 0, ch = 0;
  if (valid) {
    if (by_parent) {
      P = list[item / NC];
      c = (int)(item % NC);
      const int c0 = child0[P];
      valid = c0 >= 0 && !(mode_sync && status[P] < ST_REFINED);
      ch = c0 + c;
    } else {
      ch = list[item];
      P = parent[ch];
      c = ch - child0[P];
    }
  }
  stage_row<D>(s_row[slot][0], nbr, valid ? ch : NONE, l, M);
  stage_row<D>(s_row[slot][1], nbr, valid ? P : NONE, l, M);
  __syncthreads();
  average_child<D, Q, T, SOLID>(sR[slot], valid, P, c, ch, l, fpar, fch, cellmask, s_row[slot][0], s_row[slot][1], solidmask, ratio,
                                mode_sync);
}

// The level step's averaging (mode 0) over a list of (child block, group)
// items, the groups of 2^D interface cells of the fine level's boundary
// blocks whose parent cell is fluid.  One lane per fine cell gathers and
// rescales it (f_eq + (f - f_eq) r, Section 3.4.3); the 2^D lanes of a group
// sum their values with a butterfly that halves the directions each lane
// carries at every exchange (a reduce-scatter: afterwards each lane holds the
// sums of ceil(Q / 2^D) directions), and each lane stores the means of its
// directions into the parent cell's slots.  No shared memory, no barrier,
// every lane busy.
template <int D, int Q, class T, bool SOLID>
__global__ void __launch_bounds__(128, 8)
    k_average_groups(const int32_t* __restrict__ items, int n, T* __restrict__ fpar,
                     const T* __restrict__ fch, const int32_t* __restrict__ child0,
                     const int32_t* __restrict__ parent, const int32_t* __restrict__ nbr,
                     const uint64_t* __restrict__ solidmask, double ratio) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int NC = Block<D>::NC;            // lanes of a group
  constexpr int PER = (Q + NC - 1) / NC;      // directions a lane keeps
  constexpr int QP = PER * NC;
  const int s = threadIdx.x & (NC - 1);
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / NC;
  const bool valid = item < n;                // the same for the lanes of a group
  int ch = 0, g = 0, P = 0, c = 0;
  if (valid) {
    const int it = __ldg(items + item);
    ch = it >> 3;
    g = it & 7;
    P = __ldg(parent + ch);
    c = ch - __ldg(child0 + P);
  }
  const int l = Block<D>::cell(2 * (g & 1) + (s & 1), 2 * ((g >> 1) & 1) + ((s >> 1) & 1),
                               2 * ((g >> 2) & 1) + ((s >> 2) & 1));
  R v[QP];
#pragma unroll
  for (int p = 0; p < QP; ++p) v[p] = R(0);
  if (valid) {
    R f[Q];
    gather_cell<D, Q, T, SOLID>(f, fch, ch, l, nbr + (size_t)ch * NBR_STRIDE, solidmask);
    R rho, ux, uy, uz;
    moments<D, Q>(f, rho, ux, uy, uz);
    const R usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
    const R r = R(ratio);
    static_for<0, Q>([&](auto Pp) {
      const R e = feq<D, Q, Pp>(rho, ux, uy, uz, usq15);
      v[Pp] = e + (f[Pp] - e) * r;
    });
  }
  // reduce-scatter over the group: at the exchange with lane s ^ m, the lane
  // with bit m set keeps the upper half of its K directions, the other the
  // lower half, each adding the partner's copy of the half it keeps
  int base = 0;
#pragma unroll
  for (int m = NC / 2, K = QP; m >= 1; m >>= 1, K >>= 1) {
    const bool hi = (s & m) != 0;
    if (hi) base += K / 2;
#pragma unroll
    for (int i = 0; i < K / 2; ++i) {
      const R send = hi ? v[i] : v[i + K / 2];
      const R recv = __shfl_xor_sync(0xffffffffu, send, m);
      v[i] = (hi ? v[i + K / 2] : v[i]) + recv;
    }
  }
  if (!valid) return;
  const int pc = Block<D>::cell(2 * (c & 1) + (g & 1), 2 * ((c >> 1) & 1) + ((g >> 1) & 1),
                                2 * ((c >> 2) & 1) + ((g >> 2) & 1));
  const int32_t* prow = nbr + (size_t)P * NBR_STRIDE;
  const R inv = R(1) / R(NC);
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int p = base + j;
    if (p < Q)
      fpar[src_slot<D, Q>(p, P, pc, prow, SOLID ? solidmask : nullptr)] =
          save_rt<D, Q, T>(v[j] * inv, p);
  }
}

// ================================================ batched instances (lock-step)
// Work items pack (instance, block) as inst << BATCH_SHIFT | block; each
// instance's buffers, tables and per-level factors come from its descriptor.
// The same pull step as k_collide_stream (no solid cells in a batch).
template <int D, int Q, class T, int THREADS>
__global__ void __launch_bounds__(THREADS, (one_pass_min_blocks<T, Q, THREADS>()))
    k_collide_stream_batch(const uint32_t* __restrict__ items, int n,
                           const InstDesc* __restrict__ descs, int level, int which_in) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  constexpr int NCODE = D == 2 ? 9 : 27;
  constexpr int CENTER = D == 2 ? 4 : 13;
  constexpr int BPC = THREADS / M;
  __shared__ int32_t s_nb[BPC][NCODE];
  __shared__ int32_t s_inst[BPC];
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int first = blockIdx.x * BPC;
  for (int t = threadIdx.x; t < BPC * NCODE; t += THREADS) {
    const int s = t / NCODE, code = t - s * NCODE;
    const int bi = first + s;
    int v = NONE;
    if (bi < n) {
      const uint32_t it = __ldg(items + bi);
      const int inst = (int)(it >> BATCH_SHIFT);
      const int b = (int)(it & BATCH_MASK);
      v = __ldg(descs[inst].nbr + (size_t)b * NBR_STRIDE + geo_to_k<D>(code));
      if (code == 0) s_inst[s] = inst;
    }
    s_nb[s][code] = v;
  }
  __syncthreads();
  int flags;
  {
    const int v = s_nb[slot][l % NCODE];
    const unsigned lanes = M >= 32 ? 0xffffffffu : (((1u << M) - 1u) << ((threadIdx.x & 31) & ~(M - 1)));
    const unsigned outside = __ballot_sync(0xffffffffu, v < 0) & lanes;
    // (a slot past the end of the list has only NONE entries: no descriptor read)
    const unsigned wall = __ballot_sync(
        0xffffffffu, v <= -2 && descs[s_inst[slot]].faces.kind[-2 - v] != FACE_NOSLIP) & lanes;
    const unsigned outlet = __ballot_sync(
        0xffffffffu, v <= -2 && descs[s_inst[slot]].faces.kind[-2 - v] == FACE_OUTLET) & lanes;
    flags = (outside ? BF_OUTSIDE : 0) | (wall ? BF_WALL : 0) | (outlet ? BF_OUTLET : 0);
  }
  if (first + slot >= n) return;
  const InstDesc& d = descs[s_inst[slot]];
  const int b = s_nb[slot][CENTER];
  const T* __restrict__ gin = (const T*)d.f[which_in];
  T* __restrict__ gout = (T*)d.f[which_in ^ 1];
  const size_t own = (size_t)b * (Q * M) + l;
  const int32_t* nb = s_nb[slot];
  if (flags == 0) {
    R f[Q];
    static_for<0, Q>([&](auto P) {
      constexpr int p = P;
      if constexpr (p == 0) {
        f[0] = S::template load<D, Q, 0>(gin[own]);
      } else {
        const int e = link_entry<D, Q, p>(g_src_geo<D, Q>, l);
        f[p] = S::template load<D, Q, p>(
            gin[(size_t)nb[e & 31] * (Q * M) + (size_t)p * M + (e >> 5)]);
      }
    });
    R ux, uy, uz, usq15;
    bgk<D, Q>(f, R(d.omega[level]), ux, uy, uz, usq15);
    static_for<0, Q>([&](auto P) {
      gout[own + (size_t)P * M] = S::template save<D, Q, P>(f[P]);
    });
  } else {
    if (flags & BF_OUTLET)
      step_cell_checked<D, Q, T, false, true>(gin, gout, own, l, nb, nullptr, flags,
                                              d.omega[level], d.faces, false);
    else
      step_cell_checked<D, Q, T, false, false>(gin, gout, own, l, nb, nullptr, flags,
                                               d.omega[level], d.faces, false);
  }
}

template <int D, int Q, class T>
__global__ void __launch_bounds__(128, 5)
    k_interp_batch(const uint32_t* __restrict__ items, int n, const InstDesc* __restrict__ descs,
                   int level, int which_par, int which_ch) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  constexpr int NK = Nbr<D>::K;
  constexpr int BPC = 128 / M;
  __shared__ R sF[BPC][Q][M];
  __shared__ int32_t s_row[BPC][1 + NC][NK];
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int bi = blockIdx.x * BPC + slot;
  const bool valid = bi < n;
  int inst = 0, P = 0, c0 = 0;
  if (valid) {
    const uint32_t it = __ldg(items + bi);
    inst = (int)(it >> BATCH_SHIFT);
    P = (int)(it & BATCH_MASK);
    c0 = descs[inst].child0[P];
  }
  const InstDesc& d = descs[inst];
  for (int r = 0; r <= NC; ++r)
    stage_row<D>(s_row[slot][r], d.nbr, valid ? (r == 0 ? P : c0 + r - 1) : NONE, l, M);
  __syncthreads();
  if (valid)
    interp_stage<D, Q, T, false>(sF[slot], (const T*)d.f[which_par], P, l,
                                 d.r_cf[level], s_row[slot][0], nullptr);
  __syncthreads();
  if (!valid) return;
  interp_children<D, Q, T, false>(sF[slot], l, (T*)d.f[which_ch], c0, d.cellmask,
                                  s_row[slot] + 1, nullptr, nullptr, nullptr, 0);
}

// items are parents; child item i is child i % N_c of items[i / N_c]; one
// child per 4^D threads as in k_average
template <int D, int Q, class T>
__global__ void __launch_bounds__(128)
    k_average_batch(const uint32_t* __restrict__ items, int64_t n_items,
                    const InstDesc* __restrict__ descs, int level, int which_par, int which_ch) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  constexpr int NK = Nbr<D>::K;
  constexpr int CPC = 128 / M;
  __shared__ R sR[CPC][Q][M];
  __shared__ int32_t s_row[CPC][2][NK];
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int64_t item = (int64_t)blockIdx.x * CPC + slot;
  const bool valid = item < n_items;
  int inst = 0, P = 0, c = 0, ch = 0;
  if (valid) {
    const uint32_t it = __ldg(items + item / NC);
    inst = (int)(it >> BATCH_SHIFT);
    P = (int)(it & BATCH_MASK);
    c = (int)(item % NC);
    ch = descs[inst].child0[P] + c;
  }
  const InstDesc& d = descs[inst];
  stage_row<D>(s_row[slot][0], d.nbr, valid ? ch : NONE, l, M);
  stage_row<D>(s_row[slot][1], d.nbr, valid ? P : NONE, l, M);
  __syncthreads();
  average_child<D, Q, T, false>(sR[slot], valid, P, c, ch, l, (T*)d.f[which_par],
                                (const T*)d.f[which_ch], d.cellmask, s_row[slot][0],
                                s_row[slot][1], nullptr, d.r_fc[level], 0);
}

// ============================ batched instances: persistent form (PersistArgs)
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait until *cnt >= target.  False when *abort is raised, or when `limit`
// clock64 cycles have passed (then this wait raises *abort itself).
__device__ __forceinline__ bool persist_wait(const uint32_t* cnt, uint32_t target, int32_t* abort,
                                             long long limit) {
  const long long t0 = clock64();
  for (;;) {
    if (ld_acquire_u32(cnt) >= target) return true;
    if (*(volatile int32_t*)abort) return false;
    if (clock64() - t0 > limit) {
      atomicExch(abort, 1);
      return false;
    }
    __nanosleep(64);
  }
}

// Collide-stream tile: `nblk` (<= PERSIST_MAX_TILE) active blocks of one
// member, the cells spread over the CTA's threads.  The same pull step as
// k_collide_stream_batch, with every population read from L2.
template <int D, int Q, class T, int THREADS>
__device__ __forceinline__ void persist_collide(const InstDesc& d, const uint32_t* items, int nblk,
                                                int level, int which_in,
                                                int32_t (*s_nb)[D == 2 ? 9 : 27],
                                                int32_t* s_flags) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  constexpr int NCODE = D == 2 ? 9 : 27;
  constexpr int CENTER = D == 2 ? 4 : 13;
  for (int e = threadIdx.x; e < nblk * NCODE; e += THREADS) {
    const int s = e / NCODE, code = e - s * NCODE;
    const int b = (int)(__ldg(items + s) & BATCH_MASK);
    s_nb[s][code] = __ldg(d.nbr + (size_t)b * NBR_STRIDE + geo_to_k<D>(code));
  }
  __syncthreads();
  if (threadIdx.x < nblk) {
    int flags = 0;
    for (int code = 0; code < NCODE; ++code) {
      const int v = s_nb[threadIdx.x][code];
      if (v < 0) flags |= BF_OUTSIDE;
      if (v <= -2 && d.faces.kind[-2 - v] != FACE_NOSLIP) flags |= BF_WALL;
      if (v <= -2 && d.faces.kind[-2 - v] == FACE_OUTLET) flags |= BF_OUTLET;
    }
    s_flags[threadIdx.x] = flags;
  }
  __syncthreads();
  const T* gin = (const T*)d.f[which_in];
  T* gout = (T*)d.f[which_in ^ 1];
  const double omega = d.omega[level];
  for (int c = threadIdx.x; c < nblk * M; c += THREADS) {
    const int s = c / M, l = c - s * M;
    const int32_t* nb = s_nb[s];
    const size_t own = (size_t)nb[CENTER] * (Q * M) + l;
    const int flags = s_flags[s];
    if (flags == 0) {
      R f[Q];
      static_for<0, Q>([&](auto P) {
        constexpr int p = P;
        if constexpr (p == 0) {
          f[0] = S::template load<D, Q, 0>(__ldcg(gin + own));
        } else {
          const int e = link_entry<D, Q, p>(g_src_geo<D, Q>, l);
          f[p] = S::template load<D, Q, p>(
              __ldcg(gin + (size_t)nb[e & 31] * (Q * M) + (size_t)p * M + (e >> 5)));
        }
      });
      R ux, uy, uz, usq15;
      bgk<D, Q>(f, R(omega), ux, uy, uz, usq15);
      static_for<0, Q>([&](auto P) {
        gout[own + (size_t)P * M] = S::template save<D, Q, P>(f[P]);
      });
    } else if (flags & BF_OUTLET) {
      step_cell_checked<D, Q, T, false, true, false, true>(gin, gout, own, l, nb, nullptr,
                                                           flags, omega, d.faces, false);
    } else {
      step_cell_checked<D, Q, T, false, false, false, true>(gin, gout, own, l, nb,
                                                            nullptr, flags, omega, d.faces, false);
    }
  }
}

// Interpolation tile: THREADS / M parents of one member (as k_interp_batch).
// Out of line, like the averaging tile, so that their register needs do not
// weigh on the collide-stream tiles.
template <int D, int Q, class T, int THREADS>
__device__ __noinline__ void persist_interp(const InstDesc& d, const uint32_t* items, int ni,
                                            int tile, int level, int win, int wch,
                                            typename Store<T>::R (*sF)[Q][Block<D>::M],
                                            int32_t (*s_rows)[1 + Block<D>::NC][Nbr<D>::K]) {
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int j = tile * (THREADS / M) + slot;
  const bool valid = j < ni;
  int P = 0, c0 = 0;
  if (valid) {
    P = (int)(__ldg(items + j) & BATCH_MASK);
    c0 = __ldg(d.child0 + P);
  }
  for (int rr = 0; rr <= NC; ++rr)
    stage_row<D>(s_rows[slot][rr], d.nbr, valid ? (rr == 0 ? P : c0 + rr - 1) : NONE, l, M);
  __syncthreads();
  if (valid)
    interp_stage<D, Q, T, false, true>(sF[slot], (const T*)d.f[win], P, l,
                                       d.r_cf[level], s_rows[slot][0], nullptr);
  __syncthreads();
  if (valid)
    interp_children<D, Q, T, false>(sF[slot], l, (T*)d.f[wch], c0, d.cellmask,
                                    s_rows[slot] + 1, nullptr, nullptr, nullptr, 0);
}

// Averaging tile: THREADS / M children of one member; child item j is child
// j % N_c of parent item j / N_c (as k_average_batch).
template <int D, int Q, class T, int THREADS>
__device__ __noinline__ void persist_average(const InstDesc& d, const uint32_t* items, int ni,
                                             int tile, int level, int win, int wch,
                                             typename Store<T>::R (*sF)[Q][Block<D>::M],
                                             int32_t (*s_rows)[1 + Block<D>::NC][Nbr<D>::K]) {
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int j = tile * (THREADS / M) + slot;
  const bool valid = j < ni * NC;
  int P = 0, c = 0, ch = 0;
  if (valid) {
    P = (int)(__ldg(items + j / NC) & BATCH_MASK);
    c = j % NC;
    ch = __ldg(d.child0 + P) + c;
  }
  stage_row<D>(s_rows[slot][0], d.nbr, valid ? ch : NONE, l, M);
  stage_row<D>(s_rows[slot][1], d.nbr, valid ? P : NONE, l, M);
  __syncthreads();
  average_child<D, Q, T, false, true>(sF[slot], valid, P, c, ch, l, (T*)d.f[win],
                                      (const T*)d.f[wch], d.cellmask, s_rows[slot][0],
                                      s_rows[slot][1], nullptr, d.r_fc[level], 0);
}

// The persistent kernel.  Dynamic shared memory: the rescaled populations of
// the THREADS / M parents (interpolation) or children (averaging) of a tile,
// then their neighbour rows.
template <int D, int Q, class T, int THREADS>
__global__ void __launch_bounds__(THREADS, (one_pass_min_blocks<T, Q, THREADS>()))
    k_batch_persistent(PersistArgs a) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  constexpr int NK = Nbr<D>::K;
  constexpr int U = THREADS / M;     // parents or children per interface tile
  extern __shared__ __align__(16) unsigned char s_dyn[];
  R (*sF)[Q][M] = reinterpret_cast<R (*)[Q][M]>(s_dyn);
  int32_t (*s_rows)[1 + NC][NK] =
      reinterpret_cast<int32_t (*)[1 + NC][NK]>(s_dyn + sizeof(R) * U * Q * M);
  __shared__ int32_t s_nb[PERSIST_MAX_TILE][D == 2 ? 9 : 27];
  __shared__ int32_t s_flags[PERSIST_MAX_TILE];
  __shared__ long long s_take;
  __shared__ int32_t s_go;
  const long long total = (long long)a.tiles_per_step * a.n_steps;
  for (;;) {
    if (threadIdx.x == 0) {
      long long t = -1;
      if (!*(volatile int32_t*)a.abort) {
        const unsigned long long q = atomicAdd(a.head, 1ull);
        if ((long long)q < total) t = (long long)q;
      }
      s_take = t;
    }
    __syncthreads();
    const long long t = s_take;
    if (t < 0) return;
    const int step = (int)(t / a.tiles_per_step);
    const int r = (int)(t - (long long)step * a.tiles_per_step);
    const PersistPhase* list = a.phases + (size_t)((a.parity0 + step) & 1) * a.n_phase;
    // the phase: the last one starting at or before tile r (every listed
    // phase has tiles); the member: the last one whose tiles start at or
    // before the phase-local tile
    int lo = 0, hi = a.n_phase - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&list[mid].tile0) <= r) lo = mid;
      else hi = mid - 1;
    }
    const int k = lo;
    const int tt = r - __ldg(&list[k].tile0);
    const int32_t* toff = a.tile_off + (size_t)k * (a.n_inst + 1);
    int ilo = 0, ihi = a.n_inst - 1;
    while (ilo < ihi) {
      const int mid = (ilo + ihi + 1) >> 1;
      if (__ldg(toff + mid) <= tt) ilo = mid;
      else ihi = mid - 1;
    }
    const int inst = ilo;
    const int tile = tt - __ldg(toff + inst);
    if (threadIdx.x == 0) {
      int go = 1;
      const int dep = __ldg(a.dep + (size_t)k * a.n_inst + inst);
      const int dk = dep >> 1;
      const long long need = (long long)step + 1 - (dep & 1);   // coarse steps of phase dk
      if (need > 0) {
        const int32_t* doff = a.tile_off + (size_t)dk * (a.n_inst + 1);
        uint32_t target = (uint32_t)need * (uint32_t)(__ldg(doff + inst + 1) - __ldg(doff + inst));
        if (a.stall) target += 1u << 30;
        go = persist_wait(a.done + (size_t)dk * a.n_inst + inst, target, a.abort, a.wait_limit);
        if (!go)
          for (int i = 0; i < a.n_inst; ++i) atomicExch(a.descs[i].wait_flag, 1);
      }
      __threadfence();
      s_go = go;
    }
    __syncthreads();
    if (!s_go) return;
    const InstDesc& d = a.descs[inst];
    const int op = __ldg(&list[k].op), level = __ldg(&list[k].level);
    const int win = __ldg(&list[k].which_in), wch = __ldg(&list[k].which_ch);
    const int32_t i0 = __ldg(a.item_off + (size_t)k * (a.n_inst + 1) + inst);
    const int32_t ni = __ldg(a.item_off + (size_t)k * (a.n_inst + 1) + inst + 1) - i0;
    const uint32_t* items = list[k].items + i0;
    if (op == PH_COLLIDE) {
      const int first = tile * a.tile_blocks;
      const int nblk = min(a.tile_blocks, ni - first);
      persist_collide<D, Q, T, THREADS>(d, items + first, nblk, level, win, s_nb, s_flags);
    } else if (op == PH_INTERP) {
      persist_interp<D, Q, T, THREADS>(d, items, ni, tile, level, win, wch, sF, s_rows);
    } else {
      persist_average<D, Q, T, THREADS>(d, items, ni, tile, level, win, wch, sF, s_rows);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(a.done + (size_t)k * a.n_inst + inst, 1u);
    }
  }
}

template <int D, int Q, class T, int THREADS>
constexpr size_t persist_smem_bytes() {
  return sizeof(typename Store<T>::R) * THREADS * Q +
         sizeof(int32_t) * (THREADS / Block<D>::M) * (1 + Block<D>::NC) * Nbr<D>::K;
}

// ================================================================ criterion
// Vorticity magnitude from block-local first-order differences (forward, and
// backward at the last cell), block maximum of |w|^2, desired level of
// Algorithm 3 (eps < T evaluated as |w|^2 < 4^T), mark: +1 for a leaf with
// L_des > L, -1 for a REFINED block with L_des <= L.
template <int D, int Q, class T>
__global__ void __launch_bounds__(128)
    k_criterion(const int32_t* __restrict__ list, int n, const T* __restrict__ f, const int32_t* __restrict__ nbr, const uint64_t* __restrict__ solidmask,
                const int32_t* __restrict__ status, int level, int lmax, double inv_dx,
                int n_start, int n_inc, int8_t* __restrict__ marks, double* __restrict__ w2out) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  constexpr int BPC = 128 / M;
  __shared__ R su[BPC][3][M];
  __shared__ R sw[4];
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int bi = blockIdx.x * BPC + slot;
  const bool valid = bi < n;
  int b = 0;
  if (valid) {
    b = list[bi];
    R fl[Q];
    gather_cell<D, Q, T, true>(fl, f, b, l, nbr + (size_t)b * NBR_STRIDE, solidmask);
    R rho, ux, uy, uz;
    moments<D, Q>(fl, rho, ux, uy, uz);
    su[slot][0][l] = ux;
    su[slot][1][l] = uy;
    su[slot][2][l] = uz;
  }
  __syncthreads();
  R w2 = R(0);
  if (valid) {
    const int i = Block<D>::ci(l), j = Block<D>::cj(l), k = Block<D>::ck(l);
    // d(u_c)/d(axis) in lattice differences
    auto diff = [&](int comp, int axis) -> R {
      const int pos = axis == 0 ? i : (axis == 1 ? j : k);
      const int st = axis == 0 ? 1 : (axis == 1 ? 4 : 16);
      return pos < 3 ? su[slot][comp][l + st] - su[slot][comp][l]
                     : su[slot][comp][l] - su[slot][comp][l - st];
    };
    const R s = R(inv_dx);
    if constexpr (D == 2) {
      const R wz = (diff(1, 0) - diff(0, 1)) * s;
      w2 = wz * wz;
    } else {
      const R wx = (diff(2, 1) - diff(1, 2)) * s;
      const R wy = (diff(0, 2) - diff(2, 0)) * s;
      const R wz = (diff(1, 0) - diff(0, 1)) * s;
      w2 = wx * wx + wy * wy + wz * wz;
    }
  }
  // block maximum
  constexpr int START = M < 32 ? M / 2 : 16;
#pragma unroll
  for (int off = START; off > 0; off >>= 1) w2 = max(w2, __shfl_xor_sync(0xffffffffu, w2, off));
  if constexpr (M > 32) {
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) sw[warp] = w2;
    __syncthreads();
    w2 = max(sw[2 * slot], sw[2 * slot + 1]);
  }
  if (!valid || l != 0) return;
  const double w2d = (double)w2;
  int ldes = lmax - 1;
  for (int p = 1; p < lmax; ++p) {
    const int T_ = n_start - p * n_inc;
    if (T_ > 1 || w2d < ldexp(1.0, 2 * T_)) ldes = (lmax - 1) - p;
  }
  const int st = status[b];
  int8_t m = 0;
  if (st == ST_UNREFINED && ldes > level) m = 1;
  else if (st == ST_REFINED && ldes <= level) m = -1;
  marks[b] = m;
  if (w2out) w2out[b] = w2d;
}


// ============================================ block summaries (27 features)
// Inputs of the learned refinement proposal, per 4^3 block after the level
// synchronisation: for the 9 velocity-gradient components G_ab = du_a/dx_b
// (block-local first-order differences as in the criterion, physical units)
// their mean and max |.|; mean and max-min of rho; mean u_x, u_y, u_z and
// max |u|; mean and max |w|; level / L_max.  Gradient and vorticity entries
// are compressed as sign(x) log(1 + |x|); density entries are (rho - 1) * 100
// and (max - min) * 100; velocities are scaled by 20.
constexpr int N_FEATURES = 27;

__device__ __forceinline__ float squash(float x) { return copysignf(log1pf(fabsf(x)), x); }

template <int Q, class T>
__global__ void __launch_bounds__(128)
    k_features(const int32_t* __restrict__ list, int n, const T* __restrict__ f, const int32_t* __restrict__ nbr, const uint64_t* __restrict__ solidmask,
               int level, int lmax, double inv_dx, float* __restrict__ out) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int D = 3, M = 64, BPC = 2, NV = 15;
  __shared__ float su[BPC][4][M];            // ux, uy, uz, rho
  __shared__ float sv[BPC][NV][M];           // per-cell values to reduce
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int bi = blockIdx.x * BPC + slot;
  const bool valid = bi < n;
  int b = 0;
  if (valid) {
    b = list[bi];
    R fl[Q];
    gather_cell<D, Q, T, true>(fl, f, b, l, nbr + (size_t)b * NBR_STRIDE, solidmask);
    R rho, ux, uy, uz;
    moments<D, Q>(fl, rho, ux, uy, uz);
    su[slot][0][l] = (float)ux;
    su[slot][1][l] = (float)uy;
    su[slot][2][l] = (float)uz;
    su[slot][3][l] = (float)rho;
  }
  __syncthreads();
  if (valid) {
    const int i = l & 3, j = (l >> 2) & 3, k = l >> 4;
    const float s = (float)inv_dx;
    float G[9];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const int pos = ax == 0 ? i : (ax == 1 ? j : k);
        const int st = ax == 0 ? 1 : (ax == 1 ? 4 : 16);
        const float d = pos < 3 ? su[slot][c][l + st] - su[slot][c][l]
                                : su[slot][c][l] - su[slot][c][l - st];
        G[3 * c + ax] = d * s;
      }
    const float wx = G[7] - G[5], wy = G[2] - G[6], wz = G[3] - G[1];
    const float ux = su[slot][0][l], uy = su[slot][1][l], uz = su[slot][2][l];
#pragma unroll
    for (int q = 0; q < 9; ++q) sv[slot][q][l] = G[q];
    sv[slot][9][l] = su[slot][3][l];
    sv[slot][10][l] = ux;
    sv[slot][11][l] = uy;
    sv[slot][12][l] = uz;
    sv[slot][13][l] = sqrtf(ux * ux + uy * uy + uz * uz);
    sv[slot][14][l] = sqrtf(wx * wx + wy * wy + wz * wz);
  }
  __syncthreads();
  if (!valid || l >= N_FEATURES) return;
  // thread l reduces feature l over the block's 64 cells
  const int q = l;
  float acc;
  if (q < 9) {                                   // mean of G_q
    acc = 0.f;
    for (int c = 0; c < M; ++c) acc += sv[slot][q][c];
    acc = squash(acc / M);
  } else if (q < 18) {                           // max |G_q|
    acc = 0.f;
    for (int c = 0; c < M; ++c) acc = fmaxf(acc, fabsf(sv[slot][q - 9][c]));
    acc = squash(acc);
  } else if (q == 18) {                          // mean rho
    acc = 0.f;
    for (int c = 0; c < M; ++c) acc += sv[slot][9][c];
    acc = (acc / M - 1.f) * 100.f;
  } else if (q == 19) {                          // max - min rho
    float lo = sv[slot][9][0], hi = lo;
    for (int c = 1; c < M; ++c) {
      lo = fminf(lo, sv[slot][9][c]);
      hi = fmaxf(hi, sv[slot][9][c]);
    }
    acc = (hi - lo) * 100.f;
  } else if (q < 23) {                           // mean u_x, u_y, u_z
    acc = 0.f;
    for (int c = 0; c < M; ++c) acc += sv[slot][10 + (q - 20)][c];
    acc = acc / M * 20.f;
  } else if (q == 23) {                          // max |u|
    acc = 0.f;
    for (int c = 0; c < M; ++c) acc = fmaxf(acc, sv[slot][13][c]);
    acc *= 20.f;
  } else if (q == 24) {                          // mean |w|
    acc = 0.f;
    for (int c = 0; c < M; ++c) acc += sv[slot][14][c];
    acc = squash(acc / M);
  } else if (q == 25) {                          // max |w|
    acc = 0.f;
    for (int c = 0; c < M; ++c) acc = fmaxf(acc, sv[slot][14][c]);
    acc = squash(acc);
  } else {                                       // level / L_max
    acc = (float)level / (float)lmax;
  }
  out[(size_t)b * N_FEATURES + q] = acc;
}

// ============================================================ exports/imports
template <int D, int Q, class T>
__global__ void k_export_f(int64_t cap, int64_t b0, int64_t nb, const T* __restrict__ fa,
                           const T* __restrict__ fb, unsigned cur,
                           const int32_t* __restrict__ level, const int32_t* __restrict__ nbr,
                           const uint64_t* __restrict__ solidmask, double* __restrict__ out) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nb * M) return;
  const int64_t b = b0 + g / M;
  const int l = (int)(g % M);
  const int L = level[b];
  if (L < 0) {
    for (int p = 0; p < Q; ++p) out[(size_t)p * nb * M + g] = 0.0;
    return;
  }
  const T* f = ((cur >> L) & 1u) ? fb : fa;
  R fl[Q];
  gather_cell<D, Q, T, true>(fl, f, (int)b, l, nbr + (size_t)b * NBR_STRIDE, solidmask);
  static_for<0, Q>([&](auto P) { out[(size_t)P * nb * M + g] = (double)fl[P]; });
}

template <int D, int Q, class T>
__global__ void k_import_f(int64_t cap, int64_t b0, int64_t nb, T* __restrict__ fa,
                           T* __restrict__ fb, unsigned cur, const int32_t* __restrict__ level,
                           const int32_t* __restrict__ nbr, const uint64_t* __restrict__ solidmask,
                           const double* __restrict__ in) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nb * M) return;
  const int64_t b = b0 + g / M;
  const int l = (int)(g % M);
  const int L = level[b];
  if (L < 0) return;
  T* f = ((cur >> L) & 1u) ? fb : fa;
  R v[Q];
  static_for<0, Q>([&](auto P) { v[P] = (R)in[(size_t)P * nb * M + g]; });
  scatter_cell<D, Q, T, true>(v, f, (int)b, l, nbr + (size_t)b * NBR_STRIDE, solidmask);
}

template <int D, int Q, class T>
__global__ void k_export_rho_u(int64_t cap, int64_t b0, int64_t nb, const T* __restrict__ fa,
                               const T* __restrict__ fb, unsigned cur,
                               const int32_t* __restrict__ level,
                               const int32_t* __restrict__ nbr,
                               const uint64_t* __restrict__ solidmask, double* __restrict__ out) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nb * M) return;
  const int64_t b = b0 + g / M;
  const int l = (int)(g % M);
  const int L = level[b];
  double* o = out + (size_t)g * (1 + D);
  if (L < 0) {
    for (int a = 0; a <= D; ++a) o[a] = 0.0;
    return;
  }
  const T* f = ((cur >> L) & 1u) ? fb : fa;
  R fl[Q];
  gather_cell<D, Q, T, true>(fl, f, (int)b, l, nbr + (size_t)b * NBR_STRIDE, solidmask);
  R rho, ux, uy, uz;
  moments<D, Q>(fl, rho, ux, uy, uz);
  o[0] = rho;
  o[1] = ux;
  o[2] = uy;
  if (D == 3) o[3] = uz;
}

// The rest state (f = w_p in every slot; the gather of it is w_p everywhere).
template <int D, int Q, class T>
__global__ void k_init_rest(int64_t cap, T* __restrict__ f) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= cap * M) return;
  const size_t own = (size_t)(g / M) * (Q * M) + (size_t)(g % M);
  static_for<0, Q>([&](auto P) {
    constexpr double wp = VS<D, Q>::w[P];
    f[own + (size_t)P * M] = Store<T>::template save<D, Q, P>(R(wp));
  });
}

// Adaptation: for every cell x of a child about to be removed and every link
// p whose target y = x + c_p lies in a same-level block that stays, the value
// stored in x's slot p is y's pre-collision f_p; once the block is gone y
// reads it from its own opposite slot, so it is moved there.  One thread per
// (removed child, cell).
template <int D, int Q, class T>
__global__ void k_coarsen_fixup(const int32_t* __restrict__ list, int n,
                                const int32_t* __restrict__ child0,
                                const int32_t* __restrict__ parent,
                                const int8_t* __restrict__ marks,
                                const int32_t* __restrict__ nbr,
                                const uint64_t* __restrict__ solidmask,
                                const int32_t* __restrict__ level, T* __restrict__ fa,
                                T* __restrict__ fb, unsigned cur) {
  constexpr int M = Block<D>::M, NC = Block<D>::NC;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * NC * M) return;
  const int l = (int)(t % M);
  const int64_t it = t / M;
  const int x = child0[list[it / NC]] + (int)(it % NC);
  if (solidmask && ((solidmask[x] >> l) & 1ull)) return;
  T* g = ((cur >> level[x]) & 1u) ? fb : fa;
  const int32_t* row = nbr + (size_t)x * NBR_STRIDE;
  static_for<1, Q>([&](auto P) {
    constexpr int p = P;
    constexpr int pb = VS<D, Q>::opp[p];
    const int e = link_entry<D, Q, p>(g_tgt_k<D, Q>, l);
    const int k = e & 31, tl = e >> 5;
    if (k == 0) return;
    const int y = row[k];
    if (y < 0) return;
    const int py = parent[y];
    if (py >= 0 && marks[py] == -1) return;       // removed as well
    if (solidmask && ((solidmask[y] >> tl) & 1ull)) return;
    g[(size_t)y * (Q * M) + (size_t)pb * M + tl] = g[(size_t)x * (Q * M) + (size_t)p * M + l];
  });
}

// ------------------------------------------------------- block reductions
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* out) {
  __shared__ double sred[NV][32];
#pragma unroll
  for (int a = 0; a < NV; ++a)
    for (int off = 16; off > 0; off >>= 1) v[a] += __shfl_xor_sync(0xffffffffu, v[a], off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int a = 0; a < NV; ++a) sred[a][warp] = v[a];
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    for (int a = 0; a < NV; ++a) {
      double x = lane < nw ? sred[a][lane] : 0.0;
      for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      if (lane == 0) out[(size_t)blockIdx.x * NV + a] = x;
    }
  }
}

// FP64 audit of mass and momentum over leaf cells (grid-fixed grid).
template <int D, int Q, class T>
__global__ void __launch_bounds__(256)
    k_mass_partial(int64_t cap, const T* __restrict__ fa, const T* __restrict__ fb, unsigned cur,
                   const int32_t* __restrict__ level, const int32_t* __restrict__ status,
                   const int32_t* __restrict__ nbr, const uint64_t* __restrict__ solidmask,
                   double* __restrict__ partial) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < cap * M;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = g / M;
    if (status[b] != ST_UNREFINED) continue;
    const int L = level[b];
    const T* f = ((cur >> L) & 1u) ? fb : fa;
    R fl[Q];
    gather_cell<D, Q, T, true>(fl, f, (int)b, (int)(g % M),
                               nbr + (size_t)b * NBR_STRIDE, solidmask);
    double r = 0, jx = 0, jy = 0, jz = 0;
    static_for<0, Q>([&](auto P) {
      const double v = (double)fl[P];
      constexpr int cx = VS<D, Q>::cx[P], cy = VS<D, Q>::cy[P], cz = VS<D, Q>::cz[P];
      r += v;
      jx += cx * v;
      jy += cy * v;
      jz += cz * v;
    });
    const double vol = ldexp(1.0, -D * L);
    acc[0] += r * vol;
    acc[1] += jx * vol;
    acc[2] += jy * vol;
    acc[3] += jz * vol;
  }
  block_sum_store<4>(acc, partial);
}

// Momentum-exchange force: F = 2 dx^(D-1) sum over fluid cells and links p
// whose target x + c_p is solid of f*_p c_p (Section 5.3, with dt = dx per
// link), f* recomputed by BGK from the stored state.
template <int D, int Q, class T>
__global__ void __launch_bounds__(256)
    k_force_partial(const int32_t* __restrict__ list, int n, const T* __restrict__ f,
                    const int32_t* __restrict__ nbr,
                    const int32_t* __restrict__ status, const uint64_t* __restrict__ solidmask,
                    double omega, double dx, double* __restrict__ partial) {
  using V = VS<D, Q>;
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  constexpr int BPC = 256 / M;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int bi0 = blockIdx.x * BPC; bi0 < n; bi0 += gridDim.x * BPC) {
    const int slot = threadIdx.x / M, l = threadIdx.x - slot * M;
    const int bi = bi0 + slot;
    if (bi >= n) continue;
    const int b = list[bi];
    if (status[b] != ST_UNREFINED) continue;
    if ((solidmask[b] >> l) & 1ull) continue;
    R fl[Q];
    gather_cell<D, Q, T, true>(fl, f, b, l, nbr + (size_t)b * NBR_STRIDE, solidmask);
    R rho, ux, uy, uz;
    moments<D, Q>(fl, rho, ux, uy, uz);
    const R usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
    const int i = Block<D>::ci(l), j = Block<D>::cj(l), k = Block<D>::ck(l);
    static_for<1, Q>([&](auto P) {
      constexpr int p = P;
      constexpr int cx = V::cx[p], cy = V::cy[p], cz = V::cz[p];
      const int ti = i + cx, tj = j + cy, tk = k + cz;
      const int sx = ti < 0 ? -1 : (ti > 3 ? 1 : 0);
      const int sy = tj < 0 ? -1 : (tj > 3 ? 1 : 0);
      const int sz = tk < 0 ? -1 : (tk > 3 ? 1 : 0);
      const int code = (sx + 1) + 3 * (sy + 1) + (D == 3 ? 9 * (sz + 1) : 0);
      const int tb = nbr[(size_t)b * NBR_STRIDE + geo_to_k<D>(code)];
      if (tb < 0) return;
      const int tl = (ti & 3) + 4 * (tj & 3) + (D == 3 ? 16 * (tk & 3) : 0);
      if (!((solidmask[tb] >> tl) & 1ull)) return;
      const R fs = fl[p] + R(omega) * (feq<D, Q, p>(rho, ux, uy, uz, usq15) - fl[p]);
      acc[0] += (double)fs * cx;
      acc[1] += (double)fs * cy;
      acc[2] += (double)fs * cz;
    });
  }
  const double scale = 2.0 * pow(dx, (double)(D - 1));
  for (int a = 0; a < 3; ++a) acc[a] *= scale;
  block_sum_store<3>(acc, partial);
}

// =============================================================== launchers
inline int grid_for(int64_t n, int per) { return (int)((n + per - 1) / per); }

template <int D, int Q, class T>
struct Launch {
  static constexpr int M = Block<D>::M;
  static inline int sm_count = 152;

  static int setup() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    sm_count = sms;
    return 0;
  }

  template <bool SOLID, int THREADS, bool DENSE = false>
  static void one_pass(cudaStream_t s, const int32_t* list, int n, const void* fin, void* fout,
                       const int32_t* nbr, const uint64_t* sm, const StepParams& prm,
                       const uint64_t* gm, const Exchange* xchg) {
    const int grid = grid_for(n, THREADS / M);
    const T* in = (const T*)fin;
    T* out = (T*)fout;
    Exchange ex{};
    if (xchg) ex = *xchg;
    if (gm && xchg)
      k_collide_stream<D, Q, T, SOLID, THREADS, DENSE, true, true>
          <<<grid, THREADS, 0, s>>>(list, n, in, out, nbr, sm, prm, gm, ex);
    else if (gm)
      k_collide_stream<D, Q, T, SOLID, THREADS, DENSE, true, false>
          <<<grid, THREADS, 0, s>>>(list, n, in, out, nbr, sm, prm, gm, ex);
    else if (xchg)
      k_collide_stream<D, Q, T, SOLID, THREADS, DENSE, false, true>
          <<<grid, THREADS, 0, s>>>(list, n, in, out, nbr, sm, prm, nullptr, ex);
    else
      k_collide_stream<D, Q, T, SOLID, THREADS, DENSE, false, false>
          <<<grid, THREADS, 0, s>>>(list, n, in, out, nbr, sm, prm, nullptr, ex);
  }

  template <bool SOLID>
  static void collide_stream_t(cudaStream_t s, const int32_t* list, int n, const void* fin,
                               void* fout, const int32_t* nbr, const uint64_t* sm,
                               const StepParams& prm, const uint64_t* gm, const Exchange* x) {
    // kernel_variant: 1 / 2 / 3 / 4: 512 / 256 / 128 / 64 threads per CTA
    // (8 / 4 / 2 / 1 blocks of 4^3 cells); 5: 128 threads with 512 more
    // resident threads per SM (tighter register budget); 0 (auto): 64
    // threads (the fastest in the 3D cavity's AMR step, where the blocks of
    // a CTA take different paths), with the tighter budget for D3Q27 with
    // 16-bit storage.  Launches with exchanging parents always run 64
    // threads per CTA, so that a parent's barrier holds no other block.
    constexpr bool kDenseAuto = Q == 27 && sizeof(T) == 2;
    if (x) {
      one_pass<SOLID, 64, kDenseAuto>(s, list, n, fin, fout, nbr, sm, prm, gm, x);
      return;
    }
    switch (prm.variant) {
      case 1: one_pass<SOLID, 512>(s, list, n, fin, fout, nbr, sm, prm, gm, nullptr); break;
      case 2: one_pass<SOLID, 256>(s, list, n, fin, fout, nbr, sm, prm, gm, nullptr); break;
      case 3: one_pass<SOLID, 128>(s, list, n, fin, fout, nbr, sm, prm, gm, nullptr); break;
      case 4: one_pass<SOLID, 64>(s, list, n, fin, fout, nbr, sm, prm, gm, nullptr); break;
      case 5: one_pass<SOLID, 128, true>(s, list, n, fin, fout, nbr, sm, prm, gm, nullptr); break;
      default: one_pass<SOLID, 64, kDenseAuto>(s, list, n, fin, fout, nbr, sm, prm, gm, nullptr);
    }
  }

  static void collide_stream(cudaStream_t s, const int32_t* list, int n, const void* fin,
                             void* fout, const int32_t* nbr, const uint64_t* sm,
                             const StepParams& prm, bool solid, const uint64_t* gm,
                             const Exchange* x) {
    if (n <= 0) return;
    if (solid) collide_stream_t<true>(s, list, n, fin, fout, nbr, sm, prm, gm, x);
    else collide_stream_t<false>(s, list, n, fin, fout, nbr, nullptr, prm, gm, x);
  }

  static void interp(cudaStream_t s, const int32_t* list, int n, const void* fpar, void* fch,
                     const int32_t* child0, const uint64_t* nm,
                     const int32_t* nbr, const uint64_t* sm, const int32_t* parent,
                     const int8_t* marks, double ratio, int mode_all, bool solid) {
    if (n <= 0) return;
    // mode bit 0: every cell (new children), else ghost cells; bit 1: cubic;
    // bit 2: direct writes into the children's own slots
    const int all = mode_all & 5;
    if (mode_all & 2) {
      const int grid = grid_for(n, 64 / M);
      if (solid)
        k_interp_cubic<D, Q, T, true><<<grid, 64, 0, s>>>(list, n, (const T*)fpar, (T*)fch,
                                                         child0, nm, nbr, sm, parent,
                                                         marks, ratio, all);
      else
        k_interp_cubic<D, Q, T, false><<<grid, 64, 0, s>>>(list, n, (const T*)fpar, (T*)fch,
                                                          child0, nm, nbr, nullptr,
                                                          parent, marks, ratio, all);
      return;
    }
    const int grid = grid_for(n, 128 / M);
    if (solid)
      k_interp<D, Q, T, true><<<grid, 128, 0, s>>>(list, n, (const T*)fpar, (T*)fch, child0, nm, nbr, sm, parent, marks, ratio, all);
    else
      k_interp<D, Q, T, false><<<grid, 128, 0, s>>>(list, n, (const T*)fpar, (T*)fch, child0, nm, nbr, nullptr, parent, marks, ratio,
                                                   all);
  }
  static void average(cudaStream_t s, const int32_t* list, int n, bool by_parent, void* fpar,
                      const void* fch, const int32_t* child0,
                      const int32_t* parent, const uint64_t* nm, const int32_t* status,
                      const int32_t* nbr, const uint64_t* sm, double ratio, int mode_sync,
                      bool solid) {
    if (n <= 0) return;
    const int64_t items = by_parent ? (int64_t)n * Block<D>::NC : (int64_t)n;
    const int grid = (int)((items + 128 / M - 1) / (128 / M));
    if (solid)
      k_average<D, Q, T, true><<<grid, 128, 0, s>>>(list, items, by_parent, (T*)fpar,
                                                   (const T*)fch, child0, parent, nm,
                                                   status, nbr, sm, ratio, mode_sync);
    else
      k_average<D, Q, T, false><<<grid, 128, 0, s>>>(list, items, by_parent, (T*)fpar,
                                                    (const T*)fch, child0, parent, nm,
                                                    status, nbr, nullptr, ratio, mode_sync);
  }
  static void criterion(cudaStream_t s, const int32_t* list, int n, const void* f, const int32_t* nbr, const uint64_t* sm, const int32_t* status, int level,
                        int lmax, double inv_dx, int ns, int ni, int8_t* marks, double* w2out) {
    if (n <= 0) return;
    k_criterion<D, Q, T><<<grid_for(n, 128 / M), 128, 0, s>>>(
        list, n, (const T*)f, nbr, sm, status, level, lmax, inv_dx, ns, ni, marks, w2out);
  }
  static void export_f(cudaStream_t s, int64_t cap, int64_t b0, int64_t nb, const void* fa,
                       const void* fb, unsigned cur, const int32_t* level, const int32_t* nbr,
                       const uint64_t* sm, double* out) {
    k_export_f<D, Q, T><<<grid_for(nb * M, 256), 256, 0, s>>>(
        cap, b0, nb, (const T*)fa, (const T*)fb, cur, level, nbr, sm, out);
  }
  static void import_f(cudaStream_t s, int64_t cap, int64_t b0, int64_t nb, void* fa, void* fb,
                       unsigned cur, const int32_t* level, const int32_t* nbr,
                       const uint64_t* sm, const double* in) {
    k_import_f<D, Q, T><<<grid_for(nb * M, 256), 256, 0, s>>>(cap, b0, nb, (T*)fa, (T*)fb, cur,
                                                               level, nbr, sm, in);
  }
  static void export_rho_u(cudaStream_t s, int64_t cap, int64_t b0, int64_t nb, const void* fa,
                           const void* fb, unsigned cur, const int32_t* level,
                           const int32_t* nbr, const uint64_t* sm, double* out) {
    k_export_rho_u<D, Q, T><<<grid_for(nb * M, 256), 256, 0, s>>>(
        cap, b0, nb, (const T*)fa, (const T*)fb, cur, level, nbr, sm, out);
  }
  static void init_rest(cudaStream_t s, int64_t cap, void* f) {
    k_init_rest<D, Q, T><<<grid_for(cap * M, 256), 256, 0, s>>>(cap, (T*)f);
  }
  static int mass_partial(cudaStream_t s, int64_t cap, const void* fa, const void* fb,
                          unsigned cur, const int32_t* level, const int32_t* status,
                          const int32_t* nbr, const uint64_t* sm, double* partial) {
    const int grid = 152 * 4;
    k_mass_partial<D, Q, T><<<grid, 256, 0, s>>>(cap, (const T*)fa, (const T*)fb, cur, level,
                                                 status, nbr, sm, partial);
    return grid;
  }
  static int force_partial(cudaStream_t s, const int32_t* list, int n, const void* f,
                           const int32_t* nbr, const int32_t* status,
                           const uint64_t* sm, double omega, double dx, double* partial) {
    const int grid = 152 * 2;
    k_force_partial<D, Q, T><<<grid, 256, 0, s>>>(list, n, (const T*)f, nbr, status, sm,
                                                  omega, dx, partial);
    return grid;
  }
  static void features(cudaStream_t s, const int32_t* list, int n, const void* f, const int32_t* nbr, const uint64_t* sm, int level, int lmax,
                       double inv_dx, float* out) {
    if constexpr (D == 3) {
      if (n > 0)
        k_features<Q, T><<<grid_for(n, 2), 128, 0, s>>>(list, n, (const T*)f, nbr, sm,
                                                        level, lmax, inv_dx, out);
    }
  }
  static void coarsen_fixup(cudaStream_t s, const int32_t* list, int n, const int32_t* child0,
                            const int32_t* parent, const int8_t* marks, const int32_t* nbr,
                            const uint64_t* sm, const int32_t* level, void* fa, void* fb,
                            unsigned cur) {
    if (n <= 0) return;
    const int64_t threads = (int64_t)n * Block<D>::NC * M;
    k_coarsen_fixup<D, Q, T><<<(int)((threads + 255) / 256), 256, 0, s>>>(
        list, n, child0, parent, marks, nbr, sm, level, (T*)fa, (T*)fb, cur);
  }

  static void collide_stream_batch(cudaStream_t s, const uint32_t* items, int n,
                                   const InstDesc* descs, int level, int which_in, int variant) {
    if (n <= 0) return;
    // variant = threads per CTA: 64 / 128 / 256 / 512, i.e. M_L = 64/M .. 512/M
    // blocks per CTA (anything else: 512)
    switch (variant) {
      case 64:
        k_collide_stream_batch<D, Q, T, 64><<<grid_for(n, 64 / M), 64, 0, s>>>(items, n, descs,
                                                                              level, which_in);
        break;
      case 128:
        k_collide_stream_batch<D, Q, T, 128><<<grid_for(n, 128 / M), 128, 0, s>>>(
            items, n, descs, level, which_in);
        break;
      case 256:
        k_collide_stream_batch<D, Q, T, 256><<<grid_for(n, 256 / M), 256, 0, s>>>(
            items, n, descs, level, which_in);
        break;
      default:
        k_collide_stream_batch<D, Q, T, 512><<<grid_for(n, 512 / M), 512, 0, s>>>(
            items, n, descs, level, which_in);
    }
  }
  static void interp_batch(cudaStream_t s, const uint32_t* items, int n, const InstDesc* descs,
                           int level, int which_par, int which_ch) {
    if (n <= 0) return;
    k_interp_batch<D, Q, T><<<grid_for(n, 128 / M), 128, 0, s>>>(items, n, descs, level,
                                                                   which_par, which_ch);
  }
  static void average_batch(cudaStream_t s, const uint32_t* items, int n, const InstDesc* descs,
                            int level, int which_par, int which_ch) {
    if (n <= 0) return;
    const int64_t kids = (int64_t)n * Block<D>::NC;
    k_average_batch<D, Q, T><<<(int)((kids + 128 / M - 1) / (128 / M)), 128, 0, s>>>(
        items, kids, descs, level, which_par, which_ch);
  }

  static void average_groups(cudaStream_t s, const int32_t* items, int n, void* fpar,
                             const void* fch, const int32_t* child0,
                             const int32_t* parent, const int32_t* nbr, const uint64_t* sm,
                             double ratio, bool solid) {
    if (n <= 0) return;
    const int grid = (int)(((int64_t)n * Block<D>::NC + 127) / 128);
    if (solid)
      k_average_groups<D, Q, T, true><<<grid, 128, 0, s>>>(items, n, (T*)fpar, (const T*)fch,
                                                           child0, parent, nbr, sm,
                                                           ratio);
    else
      k_average_groups<D, Q, T, false><<<grid, 128, 0, s>>>(items, n, (T*)fpar, (const T*)fch,
                                                            child0, parent, nbr,
                                                            nullptr, ratio);
  }

  template <int THREADS>
  static int persistent_ctas_t() {
    constexpr size_t smem = persist_smem_bytes<D, Q, T, THREADS>();
    auto k = k_batch_persistent<D, Q, T, THREADS>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, THREADS, smem) != cudaSuccess)
      return 0;
    return per_sm * sm_count;
  }
  static int persistent_ctas(int threads) {
    switch (threads) {
      case 64: return persistent_ctas_t<64>();
      case 128: return persistent_ctas_t<128>();
      case 256: return persistent_ctas_t<256>();
      default: return 0;
    }
  }
  static void batch_persistent(cudaStream_t s, const PersistArgs& a, int threads, int ctas) {
    switch (threads) {
      case 64:
        k_batch_persistent<D, Q, T, 64><<<ctas, 64, persist_smem_bytes<D, Q, T, 64>(), s>>>(a);
        break;
      case 128:
        k_batch_persistent<D, Q, T, 128><<<ctas, 128, persist_smem_bytes<D, Q, T, 128>(), s>>>(a);
        break;
      default:
        k_batch_persistent<D, Q, T, 256><<<ctas, 256, persist_smem_bytes<D, Q, T, 256>(), s>>>(a);
    }
  }

  static const LbmOps* ops() {
    static const LbmOps o = {setup,         collide_stream, interp,   average,
                             average_groups, criterion,     export_f,       import_f, export_rho_u,
                             init_rest,     mass_partial,   force_partial,
                             collide_stream_batch, interp_batch, average_batch,
                             persistent_ctas, batch_persistent, features,
                             coarsen_fixup};
    return &o;
  }
};

}  // namespace amr
