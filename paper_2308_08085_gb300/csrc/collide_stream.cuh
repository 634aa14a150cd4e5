// Fused collide + stream of one level (Sections 4.2, 4.3): the push-target
// tables, the per-cell BGK collision and push, and the kernel variants that
// drive it (one-pass, cp.async pipelined, bulk-copy staged).  Included by
// lbm_kernels.cuh.
//
// Population layout (every storage type): f[p * stride + b * M + l], stride =
// capacity * M, M = 4^D cells per block, l = i + 4 j + 16 k.
#pragma once
#include "lattice.cuh"
#include "lbm_ops.h"

#include <algorithm>

namespace amr {

constexpr int ST_UNREFINED = 1;
constexpr int ST_REFINED = 2;
constexpr int CLS_INTERIOR = 0, CLS_INTERFACE = 1, CLS_GHOST = 2;
constexpr int FACE_OUTLET = 2;

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


// Push targets of the fused collide-stream: for direction p and cell l the
// entry packs the geometric code of the block that holds x + c_p (5 bits)
// and the cell index inside it (6 bits): e = code | (cell << 5).
template <int D, int Q>
struct StreamTable {
  uint16_t e[Q * Block<D>::M];
};
template <int D, int Q, bool BY_K = false>
constexpr StreamTable<D, Q> make_stream_table() {
  StreamTable<D, Q> t{};
  constexpr int M = Block<D>::M;
  for (int p = 0; p < Q; ++p)
    for (int l = 0; l < M; ++l) {
      const int ti = Block<D>::ci(l) + VS<D, Q>::cx[p];
      const int tj = Block<D>::cj(l) + VS<D, Q>::cy[p];
      const int tk = Block<D>::ck(l) + VS<D, Q>::cz[p];
      const int sx = ti < 0 ? -1 : (ti > 3 ? 1 : 0);
      const int sy = tj < 0 ? -1 : (tj > 3 ? 1 : 0);
      const int sz = tk < 0 ? -1 : (tk > 3 ? 1 : 0);
      const int code = BY_K ? Nbr<D>::dir_of(sx, sy, sz)
                            : (sx + 1) + 3 * (sy + 1) + (D == 3 ? 9 * (sz + 1) : 0);
      const int cell = (ti & 3) + 4 * (tj & 3) + (D == 3 ? 16 * (tk & 3) : 0);
      t.e[p * M + l] = (uint16_t)(code | (cell << 5));
    }
  return t;
}
template <int D, int Q>
__device__ const StreamTable<D, Q> g_stream_table = make_stream_table<D, Q>();
// the same targets with the neighbour index k of the block's nbr row in place
// of the geometric code (for kernels that use the raw row)
template <int D, int Q>
__device__ const StreamTable<D, Q> g_stream_table_k = make_stream_table<D, Q, true>();

// One BGK collision + push of a cell whose populations are f[]: the common
// body of both collide-stream kernels.  `tab` is the stream table, in shared
// memory when TAB_SMEM, else the global copy read through the read-only
// path; `nb` the neighbour block IDs of the cell's block in geometric order.
template <int D, int Q, class T, bool SOLID, bool TAB_SMEM>
__device__ __forceinline__ void collide_push(typename Store<T>::R (&f)[Q], int l, int b,
                                             const uint16_t* __restrict__ tab,
                                             const int32_t* __restrict__ nb,
                                             const uint64_t* __restrict__ sm_nb,
                                             T* __restrict__ fout, size_t stride, double omega,
                                             const FaceParams& faces) {
  using V = VS<D, Q>;
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  R rho, ux, uy, uz;
  moments<D, Q>(f, rho, ux, uy, uz);
  const R usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
  const R om = R(omega);
  const int own = b * M + l;
  static_for<0, Q>([&](auto P) {
    constexpr int p = P;
    constexpr int cx = V::cx[p], cy = V::cy[p], cz = V::cz[p];
    constexpr int pb = V::opp[p];
    const R fs = f[p] + om * (feq<D, Q, p>(rho, ux, uy, uz, usq15) - f[p]);
    T* __restrict__ outp = fout + (size_t)p * stride;
    if constexpr (p == 0) {
      outp[own] = S::template save<D, Q, 0>(fs);
    } else {
      int e;
      if constexpr (TAB_SMEM) e = tab[p * M + l];
      else e = __ldg(tab + p * M + l);
      const int code = e & 31, tl = e >> 5;
      const int tgt = nb[code];
      bool bounce = tgt < 0;
      if constexpr (SOLID) bounce = bounce || ((sm_nb[code] >> tl) & 1ull);
      if (!bounce) {
        outp[tgt * M + tl] = S::template save<D, Q, p>(fs);
      } else {
        R v = fs;   // NONE (interface) or solid: halfway bounce-back
        if (tgt <= -2) {
          const int face = -2 - tgt;
          if (faces.kind[face] == FACE_OUTLET) {
            R cu = R(0);
            if constexpr (cx != 0) cu += cx > 0 ? ux : -ux;
            if constexpr (cy != 0) cu += cy > 0 ? uy : -uy;
            if constexpr (cz != 0) cu += cz > 0 ? uz : -uz;
            constexpr double wp = V::w[p];
            v = -fs + R(2.0 * wp * faces.rho_w[face]) * (R(1) + R(4.5) * cu * cu - usq15);
          } else {
            v = fs + R(faces.bb[face][p]);
          }
        }
        fout[(size_t)pb * stride + own] = S::template save<D, Q, pb>(v);
      }
    }
  });
}

// ===================================================== fused collide + stream
// One thread per cell, 256 threads = 256/M blocks per CTA.  Each cell loads its
// Q populations (coalesced planes), relaxes them with BGK (Section 4.3) and
// pushes f*_p to x + c_p in the other buffer (Section 4.2).  Neighbour block
// IDs are staged in shared memory in geometric order.  A push that leaves the
// level (NONE), hits a wall, or hits a solid cell lands in the cell's own
// opposite slot: halfway bounce-back, the moving-wall term, or the
// anti-bounce-back outlet value (Section 2 boundary equations).
// resident warps per SM targeted by the one-pass kernel: 48 for FP32 math
// with Q <= 19 (40 registers), fewer for the larger register footprints
// (+ 512 threads per SM with DENSE: a tighter register budget that may spill)
template <class T, int Q, int THREADS, bool DENSE = false>
constexpr int one_pass_min_blocks() {
  const int threads_per_sm = (sizeof(typename Store<T>::R) == 4 ? (Q <= 19 ? 1536 : 1024)
                                                                 : (Q <= 19 ? 1024 : 512)) +
                             (DENSE ? 512 : 0);
  return threads_per_sm / THREADS > 0 ? threads_per_sm / THREADS : 1;
}

template <int D, int Q, class T, bool SOLID, int THREADS, bool TAB_SMEM, bool DENSE = false>
__global__ void __launch_bounds__(THREADS, (one_pass_min_blocks<T, Q, THREADS, DENSE>()))
    k_collide_stream(const int32_t* __restrict__ list, int n, const T* __restrict__ fin,
                     T* __restrict__ fout, const int32_t* __restrict__ nbr,
                     const uint64_t* __restrict__ solidmask, StepParams prm) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  constexpr int NCODE = D == 2 ? 9 : 27;
  constexpr int CENTER = D == 2 ? 4 : 13;
  constexpr int BPC = THREADS / M;
  __shared__ int32_t s_nb[BPC][NCODE];
  __shared__ uint64_t s_sm[SOLID ? BPC : 1][SOLID ? NCODE : 1];
  __shared__ int s_near[SOLID ? BPC : 1];   // a neighbour (or the block) has solid cells
  __shared__ uint16_t s_tab[TAB_SMEM ? Q * M : 1];

  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int first = blockIdx.x * BPC;
  if constexpr (TAB_SMEM)
    for (int t = threadIdx.x; t < Q * M; t += THREADS) s_tab[t] = g_stream_table<D, Q>.e[t];
  if constexpr (SOLID) {
    if (threadIdx.x < BPC) s_near[threadIdx.x] = 0;
    __syncthreads();
  }
  for (int t = threadIdx.x; t < BPC * NCODE; t += THREADS) {
    const int s = t / NCODE, code = t - s * NCODE;
    const int k = geo_to_k<D>(code);
    const int bi = first + s;
    int v = NONE;
    if (bi < n) v = __ldg(nbr + (size_t)__ldg(list + bi) * NBR_STRIDE + k);
    s_nb[s][code] = v;
    if constexpr (SOLID) {
      const uint64_t sm = (v >= 0) ? __ldg(solidmask + v) : 0ull;
      s_sm[s][code] = sm;
      if (sm) s_near[s] = 1;
    }
  }
  __syncthreads();
  if (first + slot >= n) return;
  const int b = s_nb[slot][CENTER];
  if constexpr (SOLID) {
    if ((s_sm[slot][CENTER] >> l) & 1ull) return;   // solid cells are not advanced
  }
  const size_t stride = prm.stride;
  const int own = b * M + l;
  R f[Q];
  static_for<0, Q>([&](auto P) {
    f[P] = S::template load<D, Q, P>(fin[(size_t)P * stride + own]);
  });
  const uint16_t* tab = TAB_SMEM ? s_tab : g_stream_table<D, Q>.e;
  // blocks with no solid cell around them take the push without solid tests
  // (a branch uniform over the block's two warps)
  if (SOLID && s_near[SOLID ? slot : 0])
    collide_push<D, Q, T, SOLID, TAB_SMEM>(f, l, b, tab, s_nb[slot], SOLID ? s_sm[slot] : nullptr,
                                           fout, prm.stride, prm.omega, prm.faces);
  else
    collide_push<D, Q, T, false, TAB_SMEM>(f, l, b, tab, s_nb[slot], nullptr, fout, prm.stride,
                                           prm.omega, prm.faces);
}

// ================================== pipelined persistent collide + stream
// Same arithmetic as k_collide_stream.  Each CTA walks tiles of 256/M blocks
// (stride gridDim.x) and double-buffers them in shared memory: while tile t
// is collided and pushed from shared memory, the populations and neighbour
// rows of its next tile stream in with 16-byte cp.async copies, so the
// memory system always has loads in flight.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int D, int Q, class T, int STAGES>
struct PipeShape {
  static constexpr int M = Block<D>::M;
  static constexpr int TILE = 256 / M;
  static constexpr int STAGE_ELEMS = TILE * Q * M;
  static constexpr int PLANE_CHUNKS = M * (int)sizeof(T) / 16;
  static constexpr size_t SMEM =
      STAGES * ((size_t)STAGE_ELEMS * sizeof(T) + (size_t)TILE * NBR_STRIDE * 4);
};

template <int D, int Q, class T, bool SOLID, int STAGES>
__global__ void __launch_bounds__(256, (sizeof(T) == 8 && Q == 27) ? 1 : 2)
    k_collide_stream_pipe(const int32_t* __restrict__ list, int n, const T* __restrict__ fin,
                          T* __restrict__ fout, const int32_t* __restrict__ nbr,
                          const uint64_t* __restrict__ solidmask, StepParams prm) {
  using V = VS<D, Q>;
  using S = Store<T>;
  using R = typename S::R;
  using PS = PipeShape<D, Q, T, STAGES>;
  constexpr int M = PS::M, TILE = PS::TILE;
  constexpr int NCODE = D == 2 ? 9 : 27;
  constexpr int CENTER = D == 2 ? 4 : 13;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sf = reinterpret_cast<T*>(smem_raw);                           // [STAGES][TILE][Q][M]
  int32_t* srow = reinterpret_cast<int32_t*>(smem_raw + STAGES * (size_t)PS::STAGE_ELEMS * sizeof(T));
  __shared__ int32_t s_nb[TILE][NCODE];
  __shared__ uint64_t s_sm[SOLID ? TILE : 1][SOLID ? NCODE : 1];
  __shared__ uint16_t s_tab[Q * M];
  const size_t stride = prm.stride;
  const int n_tiles = (n + TILE - 1) / TILE;
  for (int t = threadIdx.x; t < Q * M; t += blockDim.x) s_tab[t] = g_stream_table<D, Q>.e[t];

  auto issue = [&](int tile, int stage) {
    constexpr int NCH = TILE * Q * PS::PLANE_CHUNKS;
#pragma unroll 1
    for (int c = threadIdx.x; c < NCH; c += blockDim.x) {
      const int s = c / (Q * PS::PLANE_CHUNKS);
      const int rem = c - s * Q * PS::PLANE_CHUNKS;
      const int p = rem / PS::PLANE_CHUNKS;
      const int ch = rem - p * PS::PLANE_CHUNKS;
      const int bi = tile * TILE + s;
      if (bi < n) {
        const int b = __ldg(list + bi);
        cp_async16(reinterpret_cast<char*>(sf + (size_t)stage * PS::STAGE_ELEMS + (s * Q + p) * M) + 16 * ch,
                   reinterpret_cast<const char*>(fin + (size_t)p * stride + (size_t)b * M) + 16 * ch);
      }
    }
#pragma unroll 1
    for (int c = threadIdx.x; c < TILE * (NBR_STRIDE / 4); c += blockDim.x) {
      const int s = c / (NBR_STRIDE / 4), ch = c - s * (NBR_STRIDE / 4);
      const int bi = tile * TILE + s;
      if (bi < n)
        cp_async16(srow + (stage * TILE + s) * NBR_STRIDE + 4 * ch,
                   nbr + (size_t)__ldg(list + bi) * NBR_STRIDE + 4 * ch);
    }
  };

  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  // prologue: the first STAGES-1 tiles of this CTA are requested up front
#pragma unroll
  for (int k = 0; k < STAGES - 1; ++k) {
    const int t = blockIdx.x + k * gridDim.x;
    if (t < n_tiles) issue(t, k);
    cp_async_commit();
  }
  int stage = 0;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int ahead = tile + (STAGES - 1) * gridDim.x;
    if (ahead < n_tiles) issue(ahead, (stage + STAGES - 1) % STAGES);
    cp_async_commit();
    cp_async_wait<STAGES - 1>();   // this tile's group has landed
    __syncthreads();
#pragma unroll 1
    for (int t = threadIdx.x; t < TILE * NCODE; t += blockDim.x) {
      const int s = t / NCODE, code = t - s * NCODE;
      const int v = (tile * TILE + s < n) ? srow[(stage * TILE + s) * NBR_STRIDE + geo_to_k<D>(code)]
                                          : NONE;
      s_nb[s][code] = v;
      if constexpr (SOLID) s_sm[s][code] = (v >= 0) ? __ldg(solidmask + v) : 0ull;
    }
    __syncthreads();
    const bool active = tile * TILE + slot < n;
    bool solid_cell = false;
    if constexpr (SOLID) solid_cell = active && ((s_sm[slot][CENTER] >> l) & 1ull);
    if (active && !solid_cell) {
      const int b = s_nb[slot][CENTER];
      const T* sblk = sf + (size_t)stage * PS::STAGE_ELEMS + slot * Q * M;
      R f[Q];
      static_for<0, Q>([&](auto P) { f[P] = S::template load<D, Q, P>(sblk[P * M + l]); });
      collide_push<D, Q, T, SOLID, true>(f, l, b, s_tab, s_nb[slot],
                                         SOLID ? s_sm[slot] : nullptr, fout, prm.stride,
                                         prm.omega, prm.faces);
    }
    __syncthreads();
    stage = (stage + 1) % STAGES;
  }
  cp_async_wait<0>();
}

// ============================ bulk-copy staged persistent collide + stream
// Same arithmetic as k_collide_stream.  Each CTA walks tiles of THREADS/M
// blocks (tile = blockIdx.x + k gridDim.x, one cell per thread).  Warp 0
// stages a tile into shared memory with bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on the stage's mbarrier): the Q
// population planes of each block (M N_p contiguous bytes each) and its
// 128-byte neighbour row.  STAGES tiles are in flight while the CTA collides
// the current one out of shared memory and pushes it to global memory.  The
// loads occupy no registers and no load instructions of the computing
// threads.  Every wait on an mbarrier is bounded (about a second); a CTA
// that gives up sets *wait_flag, waits (bounded) for its copies in flight
// and returns.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of `parity` to complete: false once `limit`
// cycles (default 2^31, about a second) have passed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long limit = 1ll << 31) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

template <int D, int Q, class T, int THREADS>
struct BulkTile {
  static constexpr int M = Block<D>::M;
  static constexpr int TB = THREADS / M;                       // blocks per tile
  static constexpr int PLANE = M * (int)sizeof(T);             // bytes, multiple of 16
  static constexpr int POPS = TB * Q * PLANE;                  // [TB][Q][M] values
  static constexpr int ROW = NBR_STRIDE * 4;                   // one neighbour row
  static constexpr int STAGE = POPS + TB * ROW;
  static constexpr size_t smem(int stages) { return (size_t)stages * STAGE + 8 * (size_t)stages; }
  static_assert(PLANE % 16 == 0 && ROW % 16 == 0, "bulk copies move multiples of 16 bytes");
  static_assert(TB <= 32, "one lane of warp 0 per block of a tile");
};

template <int D, int Q, class T, int THREADS, int STAGES>
__global__ void __launch_bounds__(THREADS, (THREADS >= 512 ? 2 : 4))
    k_collide_stream_bulk(const int32_t* __restrict__ list, int n, const T* __restrict__ fin,
                          T* __restrict__ fout, const int32_t* __restrict__ nbr,
                          StepParams prm) {
  using BT = BulkTile<D, Q, T, THREADS>;
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = BT::M, TB = BT::TB;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + STAGES * (size_t)BT::STAGE);
  __shared__ int s_contig[STAGES];   // 1: the stage was filled by one copy per plane
  const int n_tiles = (n + TB - 1) / TB;
  const int lane = threadIdx.x & 31;
  const bool producer = threadIdx.x < 32;
  if (threadIdx.x == 0) {
    for (int st = 0; st < STAGES; ++st) mbar_init(smem_addr(bars + st), 1);
    fence_mbar_init();
  }
  __syncthreads();

  // warp 0: request tile `tile` into stage `st`
  auto issue = [&](int tile, int st) {
    const int first = tile * TB;
    const int nb = min(TB, n - first);
    const uint32_t bar = smem_addr(bars + st);
    unsigned char* base = smem_raw + (size_t)st * BT::STAGE;
    const int my_b = lane < nb ? __ldg(list + first + lane) : 0;
    const int b0 = __shfl_sync(0xffffffffu, my_b, 0);
    // consecutive IDs (sibling groups, uniform forests): one copy per plane
    const bool contig = __all_sync(0xffffffffu, lane >= nb || my_b == b0 + lane);
    if (lane == 0) s_contig[st] = contig ? 1 : 0;   // published by the arrive below
    fence_proxy_async_smem();   // earlier generic reads of this stage before the async writes
    __syncwarp();
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)nb * (Q * BT::PLANE + BT::ROW));
    __syncwarp();
    if (contig) {
      for (int p = lane; p <= Q; p += 32) {
        if (p < Q)
          bulk_load(smem_addr(base + (size_t)p * BT::PLANE * TB),
                    fin + (size_t)p * prm.stride + (size_t)b0 * M, nb * BT::PLANE, bar);
        else
          bulk_load(smem_addr(base + BT::POPS), nbr + (size_t)b0 * NBR_STRIDE, nb * BT::ROW, bar);
      }
      return;
    }
#pragma unroll 1
    for (int s = 0; s < nb; ++s) {
      const int b = __shfl_sync(0xffffffffu, my_b, s);
      for (int p = lane; p <= Q; p += 32) {
        if (p < Q)
          bulk_load(smem_addr(base + (size_t)(s * Q + p) * BT::PLANE),
                    fin + (size_t)p * prm.stride + (size_t)b * M, BT::PLANE, bar);
        else
          bulk_load(smem_addr(base + BT::POPS + s * BT::ROW), nbr + (size_t)b * NBR_STRIDE,
                    BT::ROW, bar);
      }
    }
  };

  int k_issued = 0;   // tiles of this CTA requested so far
  if (producer)
    for (; k_issued < STAGES && blockIdx.x + k_issued * (int)gridDim.x < n_tiles; ++k_issued)
      issue(blockIdx.x + k_issued * gridDim.x, k_issued);
  if (producer) k_issued = __shfl_sync(0xffffffffu, k_issued, 0);

  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  int k = 0;
  bool failed = false;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
    const int st = k % STAGES;
    const uint32_t parity = (uint32_t)(k / STAGES) & 1u;
    const bool ok = mbar_wait(smem_addr(bars + st), parity);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    const unsigned char* base = smem_raw + (size_t)st * BT::STAGE;
    if (tile * TB + slot < n) {
      const int32_t* row = reinterpret_cast<const int32_t*>(base + BT::POPS + slot * BT::ROW);
      // plane-major [Q][TB][M] after a contiguous copy, else block-major [TB][Q][M]
      const bool contig = s_contig[st] != 0;
      const T* sf = reinterpret_cast<const T*>(base) + (contig ? (size_t)slot * M : (size_t)slot * Q * M);
      const int pstride = contig ? TB * M : M;
      R f[Q];
      static_for<0, Q>([&](auto P) { f[P] = S::template load<D, Q, P>(sf[P * pstride + l]); });
      collide_push<D, Q, T, false, false>(f, l, row[0], g_stream_table_k<D, Q>.e, row, nullptr,
                                          fout, prm.stride, prm.omega, prm.faces);
    }
    __syncthreads();   // stage st is free again
    const int next = tile + STAGES * (int)gridDim.x;
    if (producer && next < n_tiles) {
      issue(next, st);
      ++k_issued;
    }
  }
  if (failed) {
    // give up: report, then let the copies already requested land (bounded)
    if (threadIdx.x == 0) {
      atomicExch(prm.wait_flag, 1);
      for (int j = k; j < k_issued; ++j)
        (void)mbar_wait(smem_addr(bars + (j % STAGES)), (uint32_t)(j / STAGES) & 1u);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int st = 0; st < STAGES; ++st) mbar_inval(smem_addr(bars + st));
}

}  // namespace amr
