// Fused collide + stream of one level (Sections 4.2, 4.3) in pull form, and
// the link tables and the gather / scatter of a cell's populations that every
// other kernel uses to read or write the state.  Included by lbm_kernels.cuh.
//
// Population layout (every storage type): block-major, g[b * Q M + p * M + l],
// M = 4^D cells per block, l = i + 4 j + 16 k: the Q planes of a block are one
// contiguous run, so blocks with unrelated IDs still move whole DRAM pages.
//
// What is stored.  The paper stores the post-streaming (pre-collision)
// populations f(x, t) of every cell.  This library stores, for every cell y
// and direction p, the value that will stream out of y along c_p: the
// post-collision f*_p(y) of the last step.  The pre-collision state is
// therefore spread over the neighbours and is read by a gather:
//
//   f_p(x) = g_p(x - c_p)        when x - c_p is a fluid cell of the same level
//          = g_pbar(x)           otherwise (no same-level block there -- the
//                                coarse-fine interface --, a wall, or a solid
//                                cell), pbar the opposite of p.
//
// In the second case the slot g_pbar(x) holds the value that bounced back
// into x: the step that wrote it applied the boundary rule of the link (the
// moving-wall term or the anti-bounce-back outlet value, Section 2), so the
// gather needs no boundary arithmetic.  Writing a pre-collision value f_p(x)
// (interpolation, averaging, imports) is the scatter into the same slot.
// Each slot is the source of exactly one (cell, direction) pair, so gathers
// and scatters of different cells never collide, and the whole method
// (interpolation, averaging, criterion, exports) sees exactly the state of
// the paper's formulation.  The fused step reads its Q values through the
// gather (loads shifted across block edges, served by L1/L2) and writes all
// Q post-collision values of a cell to its own slots: every store is a whole
// row of the block, and no store crosses a block edge.
#pragma once
#include "lattice.cuh"
#include "lbm_ops.h"

#include <algorithm>

namespace amr {

constexpr int ST_UNREFINED = 1;
constexpr int ST_REFINED = 2;
constexpr int CLS_INTERIOR = 0, CLS_INTERFACE = 1, CLS_GHOST = 2;
constexpr int FACE_NOSLIP = 0, FACE_OUTLET = 2;

// geometric neighbour code (sx+1) + 3 (sy+1) [+ 9 (sz+1)] -> neighbour index k
struct GeoTable {
  int8_t k_of_code[27];
};
template <int D>
constexpr GeoTable make_geo() {
  GeoTable t{};
  for (int c = 0; c < 27; ++c) {
    int sx = c % 3 - 1, sy = (c / 3) % 3 - 1, sz = c / 9 - 1;
    if (D == 2) t.k_of_code[c] = (c < 9) ? (int8_t)Nbr<2>::dir_of(sx, sy, 0) : (int8_t)-1;
    else t.k_of_code[c] = (int8_t)Nbr<3>::dir_of(sx, sy, sz);
  }
  return t;
}
static __constant__ GeoTable c_geo2 = make_geo<2>();
static __constant__ GeoTable c_geo3 = make_geo<3>();

template <int D>
__device__ __forceinline__ int geo_to_k(int code) {
  return D == 2 ? c_geo2.k_of_code[code] : c_geo3.k_of_code[code];
}

// Link tables: for direction p and cell l, the block that holds the cell
// x + s c_p (s = +1: the target of the link leaving x, s = -1: the source of
// the link arriving at x) and the cell index inside it, packed as
// e = blk | (cell << 5).  blk is the geometric code of the neighbour block
// (0 .. 3^D - 1, centre = the block itself) or, in the _K tables, its index
// k in the block's neighbour row (0 = the block itself).
template <int D, int Q>
struct LinkTable {
  uint16_t e[Q * Block<D>::M];
};
template <int D, int Q, int SIGN, bool BY_K>
constexpr LinkTable<D, Q> make_link_table() {
  LinkTable<D, Q> t{};
  constexpr int M = Block<D>::M;
  for (int p = 0; p < Q; ++p)
    for (int l = 0; l < M; ++l) {
      const int ti = Block<D>::ci(l) + SIGN * VS<D, Q>::cx[p];
      const int tj = Block<D>::cj(l) + SIGN * VS<D, Q>::cy[p];
      const int tk = Block<D>::ck(l) + SIGN * VS<D, Q>::cz[p];
      const int sx = ti < 0 ? -1 : (ti > 3 ? 1 : 0);
      const int sy = tj < 0 ? -1 : (tj > 3 ? 1 : 0);
      const int sz = tk < 0 ? -1 : (tk > 3 ? 1 : 0);
      const int blk = BY_K ? Nbr<D>::dir_of(sx, sy, sz)
                           : (sx + 1) + 3 * (sy + 1) + (D == 3 ? 9 * (sz + 1) : 0);
      const int cell = (ti & 3) + 4 * (tj & 3) + (D == 3 ? 16 * (tk & 3) : 0);
      t.e[p * M + l] = (uint16_t)(blk | (cell << 5));
    }
  return t;
}
template <int D, int Q>
__device__ const LinkTable<D, Q> g_src_geo = make_link_table<D, Q, -1, false>();
template <int D, int Q>
__device__ const LinkTable<D, Q> g_tgt_geo = make_link_table<D, Q, +1, false>();
template <int D, int Q>
__device__ const LinkTable<D, Q> g_src_k = make_link_table<D, Q, -1, true>();
template <int D, int Q>
__device__ const LinkTable<D, Q> g_tgt_k = make_link_table<D, Q, +1, true>();

template <int D, int Q, int P>
__device__ __forceinline__ int link_entry(const LinkTable<D, Q>& t, int l) {
  return __ldg(&t.e[P * Block<D>::M + l]);
}

// A population load.  COH: the value may have been stored by another CTA of
// the same launch (the persistent batched kernel), so it is read from L2
// (ld.global.cg), never through a path that may hold an older copy.
template <bool COH, class T>
__device__ __forceinline__ T ld_pop(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// --------------------------------------------------------- gather / scatter
// Pre-collision populations of cell l of block b (see the file comment).
// `row` is the block's neighbour row (neighbour-index order), in global or
// shared memory.  A solid cell holds its own (rest) values.  With
// SOLID, `solidmask` (one bit per cell) may still be null: no solid cells.
template <int D, int Q, class T, bool SOLID, bool COH = false>
__device__ __forceinline__ void gather_cell(typename Store<T>::R (&f)[Q],
                                            const T* __restrict__ g, int b, int l,
                                            const int32_t* __restrict__ row,
                                            const uint64_t* __restrict__ solidmask) {
  using S = Store<T>;
  constexpr int M = Block<D>::M;
  const size_t own = (size_t)b * (Q * M) + l;
  const bool has_sm = SOLID && solidmask != nullptr;
  const bool solid_cell = has_sm && ((__ldg(solidmask + b) >> l) & 1ull);
  static_for<0, Q>([&](auto P) {
    constexpr int p = P;
    constexpr int pb = VS<D, Q>::opp[p];
    if constexpr (p == 0) {
      f[0] = S::template load<D, Q, 0>(ld_pop<COH>(g + own));
    } else {
      const int e = link_entry<D, Q, p>(g_src_k<D, Q>, l);
      const int k = e & 31, sl = e >> 5;
      const int src = k == 0 ? b : row[k];
      bool back = src < 0;
      if (has_sm && !back) back = (__ldg(solidmask + src) >> sl) & 1ull;
      const size_t at = solid_cell ? own + (size_t)p * M
                                   : (back ? own + (size_t)pb * M
                                           : (size_t)src * (Q * M) + (size_t)p * M + sl);
      f[p] = S::template load<D, Q, p>(ld_pop<COH>(g + at));
    }
  });
}

// Opposite directions as a device table (for loops over runtime p).
template <int D, int Q>
struct OppTable {
  int8_t o[Q];
};
template <int D, int Q>
constexpr OppTable<D, Q> make_opp() {
  OppTable<D, Q> t{};
  for (int p = 0; p < Q; ++p) t.o[p] = (int8_t)VS<D, Q>::opp[p];
  return t;
}
template <int D, int Q>
__device__ const OppTable<D, Q> g_opp = make_opp<D, Q>();

// The element of g that holds the pre-collision f_p of cell l of block b
// (the scatter rule of scatter_cell for one runtime direction p).
template <int D, int Q>
__device__ __forceinline__ size_t src_slot(int p, int b, int l, const int32_t* row,
                                           const uint64_t* __restrict__ solidmask) {
  constexpr int M = Block<D>::M;
  const size_t own = (size_t)b * (Q * M) + l;
  if (p == 0) return own;
  const int e = __ldg(&g_src_k<D, Q>.e[p * M + l]);
  const int k = e & 31, sl = e >> 5;
  const int src = k == 0 ? b : row[k];
  bool back = src < 0;
  if (solidmask && !back) back = (__ldg(solidmask + src) >> sl) & 1ull;
  if (solidmask && ((__ldg(solidmask + b) >> l) & 1ull)) return own + (size_t)p * M;
  return back ? own + (size_t)g_opp<D, Q>.o[p] * M : (size_t)src * (Q * M) + (size_t)p * M + sl;
}

// Store pre-collision populations f of cell l of block b so that gather_cell
// returns them.  MOVE (new blocks of an adaptation): where the source cell
// x - c_p lies in a block that existed before (is_new(block) false), its slot
// still holds the value that bounced back into that old cell, which now has
// to come from this cell: it is moved to this cell's opposite slot first.
template <int D, int Q, class T, bool SOLID, bool MOVE = false, class IsNew = int>
__device__ __forceinline__ void scatter_cell(const typename Store<T>::R (&f)[Q],
                                             T* __restrict__ g, int b, int l,
                                             const int32_t* __restrict__ row,
                                             const uint64_t* __restrict__ solidmask,
                                             IsNew is_new = 0) {
  using S = Store<T>;
  constexpr int M = Block<D>::M;
  const size_t own = (size_t)b * (Q * M) + l;
  const bool has_sm = SOLID && solidmask != nullptr;
  const bool solid_cell = has_sm && ((__ldg(solidmask + b) >> l) & 1ull);
  static_for<0, Q>([&](auto P) {
    constexpr int p = P;
    constexpr int pb = VS<D, Q>::opp[p];
    if constexpr (p == 0) {
      g[own] = S::template save<D, Q, 0>(f[0]);
    } else {
      const int e = link_entry<D, Q, p>(g_src_k<D, Q>, l);
      const int k = e & 31, sl = e >> 5;
      const int src = k == 0 ? b : row[k];
      bool back = src < 0;
      if (has_sm && !back) back = (__ldg(solidmask + src) >> sl) & 1ull;
      if (solid_cell) {
        g[own + (size_t)p * M] = S::template save<D, Q, p>(f[p]);
      } else if (back) {
        g[own + (size_t)pb * M] = S::template save<D, Q, p>(f[p]);
      } else {
        T* slot = g + (size_t)src * (Q * M) + (size_t)p * M + sl;
        if constexpr (MOVE) {
          if (k != 0 && !is_new(src)) g[own + (size_t)pb * M] = *slot;
        }
        *slot = S::template save<D, Q, p>(f[p]);
      }
    }
  });
}

// ------------------------------------------------------------ BGK collision
template <int D, int Q, class R>
__device__ __forceinline__ void bgk(R (&f)[Q], R om, R& ux, R& uy, R& uz, R& usq15) {
  R rho;
  moments<D, Q>(f, rho, ux, uy, uz);
  usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
  static_for<0, Q>([&](auto P) {
    f[P] = f[P] + om * (feq<D, Q, P>(rho, ux, uy, uz, usq15) - f[P]);
  });
}

// The BGK step (Section 2) on shifted populations g_p = f_p - w_p, as the
// 16-bit storages hold them: rho = 1 + sum_p g_p and j = sum_p c_p g_p (the
// weights have no first moment), and f_eq,p - w_p = w_p (rho - 1) + w_p rho
// (3 c.u + 4.5 (c.u)^2 - 1.5 u^2), so the shift is neither added on load nor
// removed on store.
template <int D, int Q, class R>
__device__ __forceinline__ void bgk_shifted(R (&g)[Q], R om) {
  using V = VS<D, Q>;
  R dr = 0, jx = 0, jy = 0, jz = 0;
  static_for<0, Q>([&](auto P) {
    constexpr int p = P;
    constexpr int cx = V::cx[p], cy = V::cy[p], cz = V::cz[p];
    dr += g[p];
    if constexpr (cx != 0) jx += cx > 0 ? g[p] : -g[p];
    if constexpr (cy != 0) jy += cy > 0 ? g[p] : -g[p];
    if constexpr (cz != 0) jz += cz > 0 ? g[p] : -g[p];
  });
  const R rho = R(1) + dr;
  const R inv = R(1) / rho;
  const R ux = jx * inv, uy = jy * inv, uz = D == 3 ? jz * inv : R(0);
  const R usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
  static_for<0, Q>([&](auto P) {
    constexpr int p = P;
    constexpr int cx = V::cx[p], cy = V::cy[p], cz = V::cz[p];
    R cu = R(0);
    if constexpr (cx != 0) cu += cx > 0 ? ux : -ux;
    if constexpr (cy != 0) cu += cy > 0 ? uy : -uy;
    if constexpr (cz != 0) cu += cz > 0 ? uz : -uz;
    constexpr double wp = V::w[p];
    const R geq = R(wp) * (dr + rho * (R(3) * cu + R(4.5) * cu * cu - usq15));
    g[p] = g[p] + om * (geq - g[p]);
  });
}

// Value stored in the own slot p of a cell whose link p leaves through wall
// face `face` (Section 2 boundary equations): the moving-wall bounce-back
// f* + bb, or the anti-bounce-back outlet value with the cell's velocity.
template <int D, int Q, int P, class R>
__device__ __forceinline__ R wall_value(R fs, int face, R ux, R uy, R uz, R usq15,
                                        const FaceParams& faces) {
  using V = VS<D, Q>;
  constexpr int cx = V::cx[P], cy = V::cy[P], cz = V::cz[P];
  if (faces.kind[face] == FACE_OUTLET) {
    R cu = R(0);
    if constexpr (cx != 0) cu += cx > 0 ? ux : -ux;
    if constexpr (cy != 0) cu += cy > 0 ? uy : -uy;
    if constexpr (cz != 0) cu += cz > 0 ? uz : -uz;
    constexpr double wp = V::w[P];
    return -fs + R(2.0 * wp * faces.rho_w[face]) * (R(1) + R(4.5) * cu * cu - usq15);
  }
  return fs + R(faces.bb[face][P]);
}

// ================================================= fused collide + stream
// One thread per cell, THREADS / M blocks per CTA (tree order).  The
// neighbour rows of the CTA's blocks are staged in shared memory in
// geometric order.  Blocks whose 3^D neighbourhood is complete and free of
// solid cells take a branch-free path (every source is a same-level cell);
// the others test each link: a source across a missing block, a wall or a
// solid cell reads the cell's own opposite slot, and the links that leave
// through a wall store the wall value.  Solid cells are not advanced.
// resident threads per SM targeted: 1536 for FP32 math with Q <= 19 (40
// registers), fewer for the larger register footprints (+512 with DENSE: a
// tighter register budget)
template <class T, int Q, int THREADS, bool DENSE = false>
constexpr int one_pass_min_blocks() {
  const int threads_per_sm = (sizeof(typename Store<T>::R) == 4 ? (Q <= 19 ? 1536 : 1024)
                                                                 : (Q <= 19 ? 1024 : 512)) +
                             (DENSE ? 512 : 0);
  return threads_per_sm / THREADS > 0 ? threads_per_sm / THREADS : 1;
}

constexpr int BF_OUTSIDE = 1;   // a neighbour block is missing or a wall
constexpr int BF_WALL = 2;      // a neighbour is a moving wall or an outlet (a no-slip wall
                                // bounces back with no added term, like a missing block)
constexpr int BF_SOLID = 4;     // the block or a neighbour has solid cells
constexpr int BF_OUTLET = 8;    // a neighbour is an outlet face

// The step of one cell of a block whose neighbourhood has a missing block, a
// wall or solid cells: every source is tested, and the links whose source
// lies outside (bit p of `back`) are the links p-bar that leave the cell
// through a wall, which store the wall value.  Kept out of line so that the
// branch-free path of the other blocks keeps its registers.  OUTLET: a
// neighbour is an outlet face (anti-bounce-back needs the cell's velocity).
template <int D, int Q, class T, bool SOLID, bool OUTLET, bool GHOST = false, bool COH = false>
__device__ __noinline__ void step_cell_checked(const T* __restrict__ gin, T* __restrict__ gout,
                                               size_t own, int l,
                                               const int32_t* nb, const uint64_t* sm, int flags,
                                               double omega, const FaceParams& faces,
                                               bool ghost_in) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  R f[Q];
  uint32_t back = 0u;
  // ghost_in: a ghost cell at the first substep of its level reads the values
  // the interpolation left in its own slots of the output buffer (the same
  // loads with another address, so that the cells of a warp do not diverge)
  if constexpr (!GHOST) ghost_in = false;
  const T* gsrc = ghost_in ? (const T*)gout : gin;
  static_for<0, Q>([&](auto P) {
    constexpr int p = P;
    constexpr int pb = VS<D, Q>::opp[p];
    if constexpr (p == 0) {
      f[0] = S::template load<D, Q, 0>(ld_pop<COH>(gsrc + own));
    } else {
      const int e = link_entry<D, Q, p>(g_src_geo<D, Q>, l);
      const int code = e & 31, sl = e >> 5;
      const int src = nb[code];
      bool out = src < 0;
      if constexpr (SOLID) out = out || ((sm[code] >> sl) & 1ull);
      back |= (uint32_t)out << p;
      const size_t at = ghost_in ? own + (size_t)p * M
                                 : (out ? own + (size_t)pb * M
                                        : (size_t)src * (Q * M) + (size_t)p * M + sl);
      f[p] = S::template load<D, Q, p>(ld_pop<COH>(gsrc + at));
    }
  });
  R ux, uy, uz, usq15;
  bgk<D, Q>(f, R(omega), ux, uy, uz, usq15);
  if (!(flags & BF_WALL)) back = 0u;
  static_for<0, Q>([&](auto P) {
    constexpr int p = P;
    constexpr int pb = VS<D, Q>::opp[p];
    R v = f[p];
    if constexpr (p != 0) {
      if ((back >> pb) & 1u) {   // the target of link p is outside
        const int tgt = nb[link_entry<D, Q, p>(g_tgt_geo<D, Q>, l) & 31];
        if (tgt <= -2) {
          if constexpr (OUTLET) v = wall_value<D, Q, p>(v, -2 - tgt, ux, uy, uz, usq15, faces);
          else v += R(faces.bb[-2 - tgt][p]);
        }
      }
    }
    gout[own + (size_t)p * M] = S::template save<D, Q, p>(v);
  });
}

// An exchanging parent cell (see Exchange): the checked step of
// step_cell_checked, with the cell's pre-collision values rescaled to the
// fine level (f_eq + (f - f_eq) r_cf, Section 3.4.1) stored to rc[p * M + l]
// for the interpolation into the children.
template <int D, int Q, class T, bool SOLID, bool OUTLET>
__device__ __noinline__ void step_cell_parent(const T* __restrict__ gin, T* __restrict__ gout,
                                              size_t own, int l,
                                              const int32_t* nb, const uint64_t* sm, int flags,
                                              double omega, const FaceParams& faces, double r_cf,
                                              typename Store<T>::R* rc) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  R f[Q];
  uint32_t back = 0u;
  static_for<0, Q>([&](auto P) {
    constexpr int p = P;
    constexpr int pb = VS<D, Q>::opp[p];
    if constexpr (p == 0) {
      f[0] = S::template load<D, Q, 0>(gin[own]);
    } else {
      const int e = link_entry<D, Q, p>(g_src_geo<D, Q>, l);
      const int code = e & 31, sl = e >> 5;
      const int src = nb[code];
      bool out = src < 0;
      if constexpr (SOLID) out = out || ((sm[code] >> sl) & 1ull);
      back |= (uint32_t)out << p;
      f[p] = out ? S::template load<D, Q, p>(gin[own + (size_t)pb * M])
                 : S::template load<D, Q, p>(gin[(size_t)src * (Q * M) + (size_t)p * M + sl]);
    }
  });
  R rho, ux, uy, uz;
  moments<D, Q>(f, rho, ux, uy, uz);
  const R usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
  const R om = R(omega), rcf = R(r_cf);
  static_for<0, Q>([&](auto P) {
    const R e = feq<D, Q, P>(rho, ux, uy, uz, usq15);
    rc[P * M + l] = e + (f[P] - e) * rcf;
    f[P] = f[P] + om * (e - f[P]);
  });
  if (!(flags & BF_WALL)) back = 0u;
  static_for<0, Q>([&](auto P) {
    constexpr int p = P;
    constexpr int pb = VS<D, Q>::opp[p];
    R v = f[p];
    if constexpr (p != 0) {
      if ((back >> pb) & 1u) {
        const int tgt = nb[link_entry<D, Q, p>(g_tgt_geo<D, Q>, l) & 31];
        if (tgt <= -2) {
          if constexpr (OUTLET) v = wall_value<D, Q, p>(v, -2 - tgt, ux, uy, uz, usq15, faces);
          else v += R(faces.bb[-2 - tgt][p]);
        }
      }
    }
    gout[own + (size_t)p * M] = S::template save<D, Q, p>(v);
  });
}

// The ghost cells of the children of an exchanging parent: cell l of every
// child c with ghost cells takes the multilinear interpolant of the 2^D
// rescaled parent cells of quadrant c (child cell I at -1/4 + I/2 between the
// parent cell centres; Section 3.4.1), written as it is into its own slots of
// the fine output buffer.  Solid cells are skipped.
template <int D, int Q, class T>
__device__ __noinline__ void interp_out(const typename Store<T>::R* rc, int l, int c0,
                                        const uint64_t* cgm, T* __restrict__ fout,
                                        const uint64_t* __restrict__ solidmask) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  const R x = R(-0.25) + R(0.5) * R(Block<D>::ci(l));
  const R y = R(-0.25) + R(0.5) * R(Block<D>::cj(l));
  const R z = R(-0.25) + R(0.5) * R(Block<D>::ck(l));
  R wgt[NC];
#pragma unroll
  for (int a = 0; a < NC; ++a) {
    R wv = ((a & 1) ? x : R(1) - x) * ((a & 2) ? y : R(1) - y);
    if (D == 3) wv *= (a & 4) ? z : R(1) - z;
    wgt[a] = wv;
  }
#pragma unroll 1
  for (int c = 0; c < NC; ++c) {
    if (!((cgm[2 * c] >> l) & 1ull)) continue;   // cgm[2 c]: ghost cells of child c
    const int ch = c0 + c;
    if (solidmask && ((__ldg(solidmask + ch) >> l) & 1ull)) continue;
    const int qx = c & 1, qy = (c >> 1) & 1, qz = (c >> 2) & 1;
    int corner[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a)
      corner[a] = Block<D>::cell(2 * qx + (a & 1), 2 * qy + ((a >> 1) & 1), 2 * qz + ((a >> 2) & 1));
    const size_t own = (size_t)ch * (Q * M) + l;
    static_for<0, Q>([&](auto P) {
      R acc = R(0);
#pragma unroll
      for (int a = 0; a < NC; ++a) acc += wgt[a] * rc[P * M + corner[a]];
      fout[own + (size_t)P * M] = S::template save<D, Q, P>(acc);
    });
  }
}

// GHOST_IN (the first of the two substeps of a level below the coarsest):
// the coarse-to-fine interpolation of the level step (Section 4.1) wrote the
// pre-collision values of this level's ghost cells into their own slots of
// the output buffer (a direct write, see LbmOps::interp); the ghost cells read
// them there instead of gathering, and overwrite them with their
// post-collision values.  `ghostmask` (= the cell-class table's ghost bits,
// cellmask[2 b]) tells the ghost cells.
// XCHG: the level has exchanging parents; they run step_cell_parent and then,
// after a barrier, interp_out (see Exchange): the coarse-to-fine interpolation
// of the level step fused into the parent level's collide-stream.
template <int D, int Q, class T, bool SOLID, int THREADS, bool DENSE = false, bool GHOST_IN = false,
          bool XCHG = false>
__global__ void __launch_bounds__(THREADS, (one_pass_min_blocks<T, Q, THREADS, DENSE>()))
    k_collide_stream(const int32_t* __restrict__ list, int n, const T* __restrict__ gin,
                     T* __restrict__ gout, const int32_t* __restrict__ nbr,
                     const uint64_t* __restrict__ solidmask, StepParams prm,
                     const uint64_t* __restrict__ ghostmask, Exchange ex) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  constexpr int NCODE = D == 2 ? 9 : 27;
  constexpr int CENTER = D == 2 ? 4 : 13;
  constexpr int BPC = THREADS / M;
  static_assert(THREADS % M == 0 && THREADS >= 32, "whole blocks per CTA");
  __shared__ int32_t s_nb[BPC][NCODE];
  __shared__ uint64_t s_sm[SOLID ? BPC : 1][SOLID ? NCODE : 1];
  __shared__ uint64_t s_gm[GHOST_IN ? BPC : 1];                 // ghost cells of the block
  __shared__ int32_t s_c0[XCHG ? BPC : 1];                       // first child, or NONE
  __shared__ uint64_t s_cm[XCHG ? BPC : 1][XCHG ? 2 * NC : 1];   // children's ghost, interface
  __shared__ R s_rc[XCHG ? BPC : 1][XCHG ? Q * M : 1];           // rescaled parent cells

  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int first = blockIdx.x * BPC;
  for (int t = threadIdx.x; t < BPC * NCODE; t += THREADS) {
    const int s = t / NCODE, code = t - s * NCODE;
    const int bi = first + s;
    int v = NONE;
    if (bi < n) {
      const int b = __ldg(list + bi);
      v = __ldg(nbr + (size_t)b * NBR_STRIDE + geo_to_k<D>(code));
      if (GHOST_IN && code == 0) s_gm[s] = __ldg(ghostmask + 2 * (size_t)b);
      if (XCHG && code == 0) s_c0[s] = __ldg(ex.child0 + b);
    } else if (XCHG && code == 0) {
      s_c0[s] = NONE;
    }
    s_nb[s][code] = v;
    if constexpr (SOLID) s_sm[s][code] = (v >= 0) ? __ldg(solidmask + v) : 0ull;
  }
  __syncthreads();
  int c0 = NONE;
  if constexpr (XCHG) {
    c0 = s_c0[slot];
    if (c0 >= 0 && l < 2 * NC) s_cm[slot][l] = __ldg(ex.cellmask + 2 * (size_t)c0 + l);
    __syncthreads();
  }
  // block flags from the neighbour codes: every warp reads all codes of its
  // block (32 consecutive cells cover every residue mod 3^D) and votes
  int flags;
  {
    const int code = l % NCODE;
    const int v = s_nb[slot][code];
    const unsigned lanes = M >= 32 ? 0xffffffffu : (((1u << M) - 1u) << ((threadIdx.x & 31) & ~(M - 1)));
    const unsigned outside = __ballot_sync(0xffffffffu, v < 0) & lanes;
    const unsigned wall =
        __ballot_sync(0xffffffffu, v <= -2 && prm.faces.kind[-2 - v] != FACE_NOSLIP) & lanes;
    const unsigned outlet =
        __ballot_sync(0xffffffffu, v <= -2 && prm.faces.kind[-2 - v] == FACE_OUTLET) & lanes;
    unsigned solid = 0u;
    if constexpr (SOLID) solid = __ballot_sync(0xffffffffu, s_sm[slot][code] != 0ull) & lanes;
    flags = (outside ? BF_OUTSIDE : 0) | (wall ? BF_WALL : 0) | (solid ? BF_SOLID : 0) |
            (outlet ? BF_OUTLET : 0);
  }
  const bool active = first + slot < n;
  bool solid_cell = false;
  if constexpr (SOLID) solid_cell = (s_sm[slot][CENTER] >> l) & 1ull;   // not advanced
  const int b = s_nb[slot][CENTER];
  const size_t own = (size_t)b * (Q * M) + l;
  const int32_t* nb = s_nb[slot];
  if (XCHG && active && c0 >= 0) {
    // an exchanging parent (a refined block has every same-level neighbour,
    // so it never holds ghost cells)
    if (solid_cell) {
      static_for<0, Q>([&](auto P) { s_rc[slot][P * M + l] = R(VS<D, Q>::w[P]); });
    } else if (flags & BF_OUTLET) {
      step_cell_parent<D, Q, T, SOLID, true>(gin, gout, own, l, nb,
                                             SOLID ? s_sm[slot] : nullptr, flags, prm.omega,
                                             prm.faces, ex.r_cf, s_rc[slot]);
    } else {
      step_cell_parent<D, Q, T, SOLID, false>(gin, gout, own, l, nb,
                                              SOLID ? s_sm[slot] : nullptr, flags, prm.omega,
                                              prm.faces, ex.r_cf, s_rc[slot]);
    }
  } else if (active && !solid_cell) {
    bool ghost_in = false;
    if constexpr (GHOST_IN) ghost_in = (s_gm[slot] >> l) & 1ull;
    if (flags == 0) {   // (a block with ghost cells has a missing neighbour: flags != 0)
      R f[Q];
      static_for<0, Q>([&](auto P) {
        constexpr int p = P;
        size_t at = own;
        if constexpr (p != 0) {
          const int e = link_entry<D, Q, p>(g_src_geo<D, Q>, l);
          at = (size_t)nb[e & 31] * (Q * M) + (size_t)p * M + (e >> 5);
        }
        if constexpr (S::kShifted) f[p] = S::raw(gin[at]);
        else f[p] = S::template load<D, Q, p>(gin[at]);
      });
      if constexpr (S::kShifted) {
        bgk_shifted<D, Q>(f, R(prm.omega));
        static_for<0, Q>([&](auto P) { gout[own + (size_t)P * M] = S::from_raw(f[P]); });
      } else {
        R ux, uy, uz, usq15;
        bgk<D, Q>(f, R(prm.omega), ux, uy, uz, usq15);
        static_for<0, Q>([&](auto P) {
          gout[own + (size_t)P * M] = S::template save<D, Q, P>(f[P]);
        });
      }
    } else {
      if (flags & BF_OUTLET)
        step_cell_checked<D, Q, T, SOLID, true, GHOST_IN>(gin, gout, own, l, nb,
                                                          SOLID ? s_sm[slot] : nullptr, flags,
                                                          prm.omega, prm.faces, ghost_in);
      else
        step_cell_checked<D, Q, T, SOLID, false, GHOST_IN>(gin, gout, own, l, nb,
                                                           SOLID ? s_sm[slot] : nullptr, flags,
                                                           prm.omega, prm.faces, ghost_in);
    }
  }
  if constexpr (XCHG) {
    __syncthreads();
    if (active && c0 >= 0)
      interp_out<D, Q, T>(s_rc[slot], l, c0, s_cm[slot], (T*)ex.fine_out, solidmask);
  }
}

}  // namespace amr
