// Templated LBM kernels of the block forest.  Included once per velocity-set
// translation unit, which instantiates them through AMR_LBM_OPS.
//
// Population layout (every storage type): f[p * stride + b * M + l], stride =
// capacity * M, M = 4^D cells per block, l = i + 4 j + 16 k.  Two buffers A/B
// are used per level in ping-pong; a level's current buffer is bit L of `cur`.
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
  __shared__ uint16_t s_tab[TAB_SMEM ? Q * M : 1];

  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int first = blockIdx.x * BPC;
  if constexpr (TAB_SMEM)
    for (int t = threadIdx.x; t < Q * M; t += THREADS) s_tab[t] = g_stream_table<D, Q>.e[t];
  for (int t = threadIdx.x; t < BPC * NCODE; t += THREADS) {
    const int s = t / NCODE, code = t - s * NCODE;
    const int k = geo_to_k<D>(code);
    const int bi = first + s;
    int v = NONE;
    if (bi < n) v = __ldg(nbr + (size_t)__ldg(list + bi) * NBR_STRIDE + k);
    s_nb[s][code] = v;
    if constexpr (SOLID) s_sm[s][code] = (v >= 0) ? __ldg(solidmask + v) : 0ull;
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
  if constexpr (TAB_SMEM)
    collide_push<D, Q, T, SOLID, true>(f, l, b, s_tab, s_nb[slot], SOLID ? s_sm[slot] : nullptr,
                                       fout, prm.stride, prm.omega, prm.faces);
  else
    collide_push<D, Q, T, SOLID, false>(f, l, b, g_stream_table<D, Q>.e, s_nb[slot],
                                        SOLID ? s_sm[slot] : nullptr, fout, prm.stride,
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
// bounded wait for the phase of `parity` to complete: false after ~2^31 cycles
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
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
}

// =========================================== coarse-to-fine linear interpolation
// Per parent block: every parent cell rescales its populations to the fine
// level (f_eq + (f - f_eq) r, Section 3.4.1) into shared memory; then, for
// each child c, fine cell (I,J,K) takes the multilinear interpolant of the
// 2^D parent cells of quadrant c at local coordinates -1/4 + I/2.  Writes the
// ghost cells of every child (mode_all = 0) or every cell (mode_all = 1).
template <int D, int Q, class T>
__device__ __forceinline__ void interp_stage(typename Store<T>::R (*sF)[Block<D>::M],
                                             const T* __restrict__ fpar, size_t stride, int P,
                                             int l, double ratio) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  const size_t base = (size_t)P * M + l;
  R f[Q];
  static_for<0, Q>([&](auto Pp) {
    f[Pp] = S::template load<D, Q, Pp>(fpar[(size_t)Pp * stride + base]);
  });
  R rho, ux, uy, uz;
  moments<D, Q>(f, rho, ux, uy, uz);
  const R usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
  const R r = R(ratio);
  static_for<0, Q>([&](auto Pp) {
    const R e = feq<D, Q, Pp>(rho, ux, uy, uz, usq15);
    sF[Pp][l] = e + (f[Pp] - e) * r;
  });
}

template <int D, int Q, class T, bool SOLID>
__device__ __forceinline__ void interp_children(const typename Store<T>::R (*sF)[Block<D>::M],
                                                int l, T* __restrict__ fch, size_t stride,
                                                int c0, const uint64_t* __restrict__ cellmask,
                                                const uint64_t* __restrict__ solidmask,
                                                int mode_all) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
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
  for (int c = 0; c < NC; ++c) {
    const int ch = c0 + c;
    if (!mode_all) {
      const uint64_t gm = __ldg(cellmask + 2 * (size_t)ch);   // ghost cells of the child
      if (gm == 0ull) continue;
      if (!((gm >> l) & 1ull)) continue;
    }
    if constexpr (SOLID) {
      if ((__ldg(solidmask + ch) >> l) & 1ull) continue;
    }
    const int qx = c & 1, qy = (c >> 1) & 1, qz = (c >> 2) & 1;
    int corner[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a)
      corner[a] = Block<D>::cell(2 * qx + (a & 1), 2 * qy + ((a >> 1) & 1),
                                 2 * qz + ((a >> 2) & 1));
    const size_t base = (size_t)ch * M + l;
    static_for<0, Q>([&](auto Pp) {
      R v = R(0);
#pragma unroll
      for (int a = 0; a < NC; ++a) v += wgt[a] * sF[Pp][corner[a]];
      fch[(size_t)Pp * stride + base] = S::template save<D, Q, Pp>(v);
    });
  }
}

template <int D, int Q, class T, bool SOLID>
__global__ void __launch_bounds__(128)
    k_interp(const int32_t* __restrict__ list, int n, const T* __restrict__ fpar,
             T* __restrict__ fch, size_t stride, const int32_t* __restrict__ child0,
             const uint64_t* __restrict__ cellmask, const uint64_t* __restrict__ solidmask,
             double ratio, int mode_all) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  constexpr int BPC = 128 / M;
  __shared__ R sF[BPC][Q][M];
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int bi = blockIdx.x * BPC + slot;
  const bool valid = bi < n;
  const int P = valid ? list[bi] : 0;
  if (valid) interp_stage<D, Q, T>(sF[slot], fpar, stride, P, l, ratio);
  __syncthreads();
  if (!valid) return;
  interp_children<D, Q, T, SOLID>(sF[slot], l, fch, stride, child0[P], cellmask, solidmask,
                                  mode_all);
}

// ===================================================== fine-to-coarse averaging
// One thread per parent cell: the 2^D fine children (all of one child block)
// are rescaled to the coarse level (f_eq + (f - f_eq) r, Section 3.4.3) and
// averaged.  mode_sync = 0 writes parent cells over interface children;
// mode_sync = 1 writes every parent cell whose children are not ghosts.
template <int D, int Q, class T, bool SOLID>
__device__ __forceinline__ void average_cell(int P, int l, T* __restrict__ fpar,
                                             const T* __restrict__ fch, size_t stride, int c0,
                                             const uint64_t* __restrict__ cellmask,
                                             const uint64_t* __restrict__ solidmask,
                                             double ratio, int mode_sync) {
  using S = Store<T>;
  using R = typename S::R;
  constexpr int M = Block<D>::M;
  constexpr int NC = Block<D>::NC;
  const int i = Block<D>::ci(l), j = Block<D>::cj(l), k = Block<D>::ck(l);
  const int c = (i >> 1) + 2 * (j >> 1) + (D == 3 ? 4 * (k >> 1) : 0);
  const int ch = c0 + c;
  const int fi = 2 * (i & 1), fj = 2 * (j & 1), fk = 2 * (k & 1);
  // all 2^D children of a parent cell share one class; test the first
  const int f0 = Block<D>::cell(fi, fj, fk);
  if (!mode_sync && !((__ldg(cellmask + 2 * (size_t)ch + 1) >> f0) & 1ull)) return;
  if (mode_sync && ((__ldg(cellmask + 2 * (size_t)ch) >> f0) & 1ull)) return;
  if constexpr (SOLID) {
    if ((__ldg(solidmask + P) >> l) & 1ull) return;
  }
  const R r = R(ratio);
  R acc[Q];
  static_for<0, Q>([&](auto Pp) { acc[Pp] = R(0); });
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    const int fl = Block<D>::cell(fi + (s & 1), fj + ((s >> 1) & 1), fk + ((s >> 2) & 1));
    const size_t base = (size_t)ch * M + fl;
    R f[Q];
    static_for<0, Q>([&](auto Pp) {
      f[Pp] = S::template load<D, Q, Pp>(fch[(size_t)Pp * stride + base]);
    });
    R rho, ux, uy, uz;
    moments<D, Q>(f, rho, ux, uy, uz);
    const R usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
    static_for<0, Q>([&](auto Pp) {
      const R e = feq<D, Q, Pp>(rho, ux, uy, uz, usq15);
      acc[Pp] += e + (f[Pp] - e) * r;
    });
  }
  const size_t base = (size_t)P * M + l;
  const R inv = R(1) / R(NC);
  static_for<0, Q>([&](auto Pp) {
    fpar[(size_t)Pp * stride + base] = S::template save<D, Q, Pp>(acc[Pp] * inv);
  });
}

template <int D, int Q, class T, bool SOLID>
__global__ void __launch_bounds__(128)
    k_average(const int32_t* __restrict__ list, int n, T* __restrict__ fpar,
              const T* __restrict__ fch, size_t stride, const int32_t* __restrict__ child0,
              const uint64_t* __restrict__ cellmask, const int32_t* __restrict__ status,
              const uint64_t* __restrict__ solidmask, double ratio, int mode_sync) {
  constexpr int M = Block<D>::M;
  constexpr int BPC = 128 / M;
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int bi = blockIdx.x * BPC + slot;
  if (bi >= n) return;
  const int P = list[bi];
  if (mode_sync && status[P] < ST_REFINED) return;
  average_cell<D, Q, T, SOLID>(P, l, fpar, fch, stride, child0[P], cellmask, solidmask, ratio,
                               mode_sync);
}

// ================================================ batched instances (lock-step)
// Work items pack (instance, block) as inst << BATCH_SHIFT | block; each
// instance's buffers, tables and per-level factors come from its descriptor.
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
  if (first + slot >= n) return;
  const InstDesc& d = descs[s_inst[slot]];
  const int b = s_nb[slot][CENTER];
  const T* __restrict__ fin = (const T*)d.f[which_in];
  T* __restrict__ fout = (T*)d.f[which_in ^ 1];
  const size_t stride = d.stride;
  const int own = b * M + l;
  R f[Q];
  static_for<0, Q>([&](auto P) {
    f[P] = S::template load<D, Q, P>(fin[(size_t)P * stride + own]);
  });
  collide_push<D, Q, T, false, false>(f, l, b, g_stream_table<D, Q>.e, s_nb[slot], nullptr, fout,
                                      stride, d.omega[level], d.faces);
}

template <int D, int Q, class T>
__global__ void __launch_bounds__(128)
    k_interp_batch(const uint32_t* __restrict__ items, int n, const InstDesc* __restrict__ descs,
                   int level, int which_par, int which_ch) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  constexpr int BPC = 128 / M;
  __shared__ R sF[BPC][Q][M];
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int bi = blockIdx.x * BPC + slot;
  const bool valid = bi < n;
  int inst = 0, P = 0;
  if (valid) {
    const uint32_t it = __ldg(items + bi);
    inst = (int)(it >> BATCH_SHIFT);
    P = (int)(it & BATCH_MASK);
    const InstDesc& d = descs[inst];
    interp_stage<D, Q, T>(sF[slot], (const T*)d.f[which_par], d.stride, P, l, d.r_cf[level]);
  }
  __syncthreads();
  if (!valid) return;
  const InstDesc& d = descs[inst];
  interp_children<D, Q, T, false>(sF[slot], l, (T*)d.f[which_ch], d.stride, d.child0[P],
                                  d.cellmask, nullptr, 0);
}

template <int D, int Q, class T>
__global__ void __launch_bounds__(128)
    k_average_batch(const uint32_t* __restrict__ items, int n, const InstDesc* __restrict__ descs,
                    int level, int which_par, int which_ch) {
  constexpr int M = Block<D>::M;
  constexpr int BPC = 128 / M;
  const int slot = threadIdx.x / M;
  const int l = threadIdx.x - slot * M;
  const int bi = blockIdx.x * BPC + slot;
  if (bi >= n) return;
  const uint32_t it = __ldg(items + bi);
  const InstDesc& d = descs[it >> BATCH_SHIFT];
  const int P = (int)(it & BATCH_MASK);
  average_cell<D, Q, T, false>(P, l, (T*)d.f[which_par], (const T*)d.f[which_ch], d.stride,
                               d.child0[P], d.cellmask, nullptr, d.r_fc[level], 0);
}

// ================================================================ criterion
// Vorticity magnitude from block-local first-order differences (forward, and
// backward at the last cell), block maximum of |w|^2, desired level of
// Algorithm 3 (eps < T evaluated as |w|^2 < 4^T), mark: +1 for a leaf with
// L_des > L, -1 for a REFINED block with L_des <= L.
template <int D, int Q, class T>
__global__ void __launch_bounds__(128)
    k_criterion(const int32_t* __restrict__ list, int n, const T* __restrict__ f, size_t stride,
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
    static_for<0, Q>([&](auto P) {
      fl[P] = S::template load<D, Q, P>(f[(size_t)P * stride + (size_t)b * M + l]);
    });
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
    k_features(const int32_t* __restrict__ list, int n, const T* __restrict__ f, size_t stride,
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
    static_for<0, Q>([&](auto P) {
      fl[P] = S::template load<D, Q, P>(f[(size_t)P * stride + (size_t)b * M + l]);
    });
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
                           const int32_t* __restrict__ level, double* __restrict__ out) {
  constexpr int M = Block<D>::M;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nb * M) return;
  const int64_t b = b0 + g / M;
  const int L = level[b];
  const size_t stride = (size_t)cap * M;
  const size_t src = (size_t)b0 * M + g;
  const T* f = (L >= 0 && ((cur >> L) & 1u)) ? fb : fa;
  static_for<0, Q>([&](auto P) {
    out[(size_t)P * nb * M + g] =
        L >= 0 ? (double)Store<T>::template load<D, Q, P>(f[(size_t)P * stride + src]) : 0.0;
  });
}

template <int D, int Q, class T>
__global__ void k_import_f(int64_t cap, int64_t b0, int64_t nb, T* __restrict__ fa,
                           T* __restrict__ fb, unsigned cur, const int32_t* __restrict__ level,
                           const double* __restrict__ in) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nb * M) return;
  const int64_t b = b0 + g / M;
  const int L = level[b];
  if (L < 0) return;
  const size_t stride = (size_t)cap * M;
  const size_t dst = (size_t)b0 * M + g;
  T* f = ((cur >> L) & 1u) ? fb : fa;
  static_for<0, Q>([&](auto P) {
    f[(size_t)P * stride + dst] =
        Store<T>::template save<D, Q, P>((R)in[(size_t)P * nb * M + g]);
  });
}

template <int D, int Q, class T>
__global__ void k_export_rho_u(int64_t cap, int64_t b0, int64_t nb, const T* __restrict__ fa,
                               const T* __restrict__ fb, unsigned cur,
                               const int32_t* __restrict__ level, double* __restrict__ out) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nb * M) return;
  const int64_t b = b0 + g / M;
  const int L = level[b];
  double* o = out + (size_t)g * (1 + D);
  if (L < 0) {
    for (int a = 0; a <= D; ++a) o[a] = 0.0;
    return;
  }
  const size_t stride = (size_t)cap * M;
  const size_t src = (size_t)b0 * M + g;
  const T* f = ((cur >> L) & 1u) ? fb : fa;
  R fl[Q];
  static_for<0, Q>([&](auto P) {
    fl[P] = Store<T>::template load<D, Q, P>(f[(size_t)P * stride + src]);
  });
  R rho, ux, uy, uz;
  moments<D, Q>(fl, rho, ux, uy, uz);
  o[0] = rho;
  o[1] = ux;
  o[2] = uy;
  if (D == 3) o[3] = uz;
}

template <int D, int Q, class T>
__global__ void k_init_rest(int64_t cap, T* __restrict__ f) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= cap * M) return;
  const size_t stride = (size_t)cap * M;
  static_for<0, Q>([&](auto P) {
    constexpr double wp = VS<D, Q>::w[P];
    f[(size_t)P * stride + g] = Store<T>::template save<D, Q, P>(R(wp));
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

// FP64 audit of mass and momentum over leaf cells (grid-stride, fixed grid).
template <int D, int Q, class T>
__global__ void __launch_bounds__(256)
    k_mass_partial(int64_t cap, const T* __restrict__ fa, const T* __restrict__ fb, unsigned cur,
                   const int32_t* __restrict__ level, const int32_t* __restrict__ status,
                   double* __restrict__ partial) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  const size_t stride = (size_t)cap * M;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < cap * M;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = g / M;
    if (status[b] != ST_UNREFINED) continue;
    const int L = level[b];
    const T* f = ((cur >> L) & 1u) ? fb : fa;
    double r = 0, jx = 0, jy = 0, jz = 0;
    static_for<0, Q>([&](auto P) {
      const double v = (double)Store<T>::template load<D, Q, P>(f[(size_t)P * stride + g]);
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
                    size_t stride, const int32_t* __restrict__ nbr,
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
    static_for<0, Q>([&](auto P) {
      fl[P] = S::template load<D, Q, P>(f[(size_t)P * stride + (size_t)b * M + l]);
    });
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
  // persistent grid of the pipelined kernel: [solid][stages - 2]
  static inline int pipe_grid[2][2] = {{0, 0}, {0, 0}};

  template <bool SOLID, int STAGES>
  static int setup_one(int sms) {
    using PS = PipeShape<D, Q, T, STAGES>;
    const void* fn = (const void*)k_collide_stream_pipe<D, Q, T, SOLID, STAGES>;
    if (PS::SMEM > 227 * 1024) return 0;   // not launchable: leave grid 0
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PS::SMEM) !=
        cudaSuccess)
      return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, PS::SMEM) != cudaSuccess)
      return -1;
    pipe_grid[SOLID ? 1 : 0][STAGES - 2] = per_sm > 0 ? per_sm * sms : 0;
    return 0;
  }

  // persistent grids of the bulk-copy kernel: [threads 256/512][stages 2..4]
  static inline int bulk_grid[2][3] = {{0, 0, 0}, {0, 0, 0}};

  template <int THREADS, int STAGES>
  static int setup_bulk(int sms) {
    using BT = BulkTile<D, Q, T, THREADS>;
    const size_t bytes = BT::smem(STAGES);
    const void* fn = (const void*)k_collide_stream_bulk<D, Q, T, THREADS, STAGES>;
    if (bytes > 227 * 1024) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
      return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, THREADS, bytes) != cudaSuccess)
      return -1;
    bulk_grid[THREADS == 512 ? 1 : 0][STAGES - 2] = per_sm > 0 ? per_sm * sms : 0;
    return 0;
  }

  static int setup() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    if (setup_one<false, 2>(sms) || setup_one<true, 2>(sms) || setup_one<false, 3>(sms) ||
        setup_one<true, 3>(sms))
      return -1;
    if (setup_bulk<512, 2>(sms) || setup_bulk<512, 3>(sms) || setup_bulk<512, 4>(sms) ||
        setup_bulk<256, 2>(sms) || setup_bulk<256, 3>(sms) || setup_bulk<256, 4>(sms))
      return -1;
    return 0;
  }

  template <int THREADS, int STAGES>
  static bool launch_bulk(cudaStream_t s, const int32_t* list, int n, const void* fin, void* fout,
                          const int32_t* nbr, const StepParams& prm) {
    using BT = BulkTile<D, Q, T, THREADS>;
    const int g = bulk_grid[THREADS == 512 ? 1 : 0][STAGES - 2];
    if (g <= 0) return false;
    const int n_tiles = (n + BT::TB - 1) / BT::TB;
    k_collide_stream_bulk<D, Q, T, THREADS, STAGES>
        <<<std::min(n_tiles, g), THREADS, BT::smem(STAGES), s>>>(list, n, (const T*)fin,
                                                                (T*)fout, nbr, prm);
    return true;
  }

  template <bool SOLID, int STAGES>
  static void launch_pipe(cudaStream_t s, int grid, const int32_t* list, int n, const void* fin,
                          void* fout, const int32_t* nbr, const uint64_t* sm,
                          const StepParams& prm) {
    k_collide_stream_pipe<D, Q, T, SOLID, STAGES>
        <<<grid, 256, PipeShape<D, Q, T, STAGES>::SMEM, s>>>(list, n, (const T*)fin, (T*)fout,
                                                            nbr, sm, prm);
  }

  static void collide_stream(cudaStream_t s, const int32_t* list, int n, const void* fin,
                             void* fout, const int32_t* nbr, const uint64_t* sm,
                             const StepParams& prm, bool solid) {
    if (n <= 0) return;
    const int tile = 256 / M;
    const int n_tiles = (n + tile - 1) / tile;
    const bool sol = solid && D == 3;
    // variant 0 (auto): 2-stage pipeline for launches of at least two waves
    const int stages = prm.variant == 3 ? 3 : 2;
    const int pg = pipe_grid[sol ? 1 : 0][stages - 2];
    const bool pipe = pg > 0 && (prm.variant == 2 || prm.variant == 3);
    (void)n_tiles;
    if (pipe) {
      const int grid = std::min(n_tiles, pg);
      if (sol) {
        if (stages == 3) launch_pipe<true, 3>(s, grid, list, n, fin, fout, nbr, sm, prm);
        else launch_pipe<true, 2>(s, grid, list, n, fin, fout, nbr, sm, prm);
      } else {
        if (stages == 3) launch_pipe<false, 3>(s, grid, list, n, fin, fout, nbr, sm, prm);
        else launch_pipe<false, 2>(s, grid, list, n, fin, fout, nbr, sm, prm);
      }
      return;
    }
    // bulk-copy staged persistent kernel (no solid cells): 8 / 9 / 10: 512
    // threads, 2 / 3 / 4 stages; 11 / 12 / 13: 256 threads, 2 / 3 / 4 stages
    if (!sol && prm.variant >= 8 && prm.variant <= 13) {
      bool done = false;
      switch (prm.variant) {
        case 8: done = launch_bulk<512, 2>(s, list, n, fin, fout, nbr, prm); break;
        case 9: done = launch_bulk<512, 3>(s, list, n, fin, fout, nbr, prm); break;
        case 10: done = launch_bulk<512, 4>(s, list, n, fin, fout, nbr, prm); break;
        case 11: done = launch_bulk<256, 2>(s, list, n, fin, fout, nbr, prm); break;
        case 12: done = launch_bulk<256, 3>(s, list, n, fin, fout, nbr, prm); break;
        default: done = launch_bulk<256, 4>(s, list, n, fin, fout, nbr, prm); break;
      }
      if (done) return;
    }
    // one-pass kernel: 1: 512 threads, table in shared memory; 4: 256 threads,
    // shared; 5: 256 threads, table read through L1; 6 and 0 (auto, the fastest
    // on the 256^3 forest): 512 threads, table through L1; 7: as 6 with 512
    // more resident threads per SM (tighter register budget)
    const int v = prm.variant;
    if (sol) {
      if (v == 1) one_pass<true, 512, true>(s, list, n, fin, fout, nbr, sm, prm);
      else if (v == 4) one_pass<true, 256, true>(s, list, n, fin, fout, nbr, sm, prm);
      else if (v == 5) one_pass<true, 256, false>(s, list, n, fin, fout, nbr, sm, prm);
      else if (v == 7) one_pass<true, 512, false, true>(s, list, n, fin, fout, nbr, sm, prm);
      else one_pass<true, 512, false>(s, list, n, fin, fout, nbr, sm, prm);
    } else {
      if (v == 1) one_pass<false, 512, true>(s, list, n, fin, fout, nbr, sm, prm);
      else if (v == 4) one_pass<false, 256, true>(s, list, n, fin, fout, nbr, sm, prm);
      else if (v == 5) one_pass<false, 256, false>(s, list, n, fin, fout, nbr, sm, prm);
      else if (v == 7) one_pass<false, 512, false, true>(s, list, n, fin, fout, nbr, sm, prm);
      else one_pass<false, 512, false>(s, list, n, fin, fout, nbr, sm, prm);
    }
  }

  template <bool SOLID, int THREADS, bool TAB_SMEM, bool DENSE = false>
  static void one_pass(cudaStream_t s, const int32_t* list, int n, const void* fin, void* fout,
                       const int32_t* nbr, const uint64_t* sm, const StepParams& prm) {
    k_collide_stream<D, Q, T, SOLID, THREADS, TAB_SMEM, DENSE>
        <<<grid_for(n, THREADS / M), THREADS, 0, s>>>(list, n, (const T*)fin, (T*)fout, nbr, sm,
                                                      prm);
  }
  static void interp(cudaStream_t s, const int32_t* list, int n, const void* fpar, void* fch,
                     size_t stride, const int32_t* child0, const uint64_t* nm, const uint64_t* sm,
                     double ratio, int mode_all, bool solid) {
    if (n <= 0) return;
    const int grid = grid_for(n, 128 / M);
    if (solid && D == 3)
      k_interp<D, Q, T, true><<<grid, 128, 0, s>>>(list, n, (const T*)fpar, (T*)fch, stride,
                                                  child0, nm, sm, ratio, mode_all);
    else
      k_interp<D, Q, T, false><<<grid, 128, 0, s>>>(list, n, (const T*)fpar, (T*)fch, stride,
                                                   child0, nm, sm, ratio, mode_all);
  }
  static void average(cudaStream_t s, const int32_t* list, int n, void* fpar, const void* fch,
                      size_t stride, const int32_t* child0, const uint64_t* nm,
                      const int32_t* status, const uint64_t* sm, double ratio, int mode_sync,
                      bool solid) {
    if (n <= 0) return;
    const int grid = grid_for(n, 128 / M);
    if (solid && D == 3)
      k_average<D, Q, T, true><<<grid, 128, 0, s>>>(list, n, (T*)fpar, (const T*)fch, stride,
                                                   child0, nm, status, sm, ratio, mode_sync);
    else
      k_average<D, Q, T, false><<<grid, 128, 0, s>>>(list, n, (T*)fpar, (const T*)fch, stride,
                                                    child0, nm, status, sm, ratio, mode_sync);
  }
  static void criterion(cudaStream_t s, const int32_t* list, int n, const void* f, size_t stride,
                        const int32_t* status, int level, int lmax, double inv_dx, int ns, int ni,
                        int8_t* marks, double* w2out) {
    if (n <= 0) return;
    k_criterion<D, Q, T><<<grid_for(n, 128 / M), 128, 0, s>>>(
        list, n, (const T*)f, stride, status, level, lmax, inv_dx, ns, ni, marks, w2out);
  }
  static void export_f(cudaStream_t s, int64_t cap, int64_t b0, int64_t nb, const void* fa,
                       const void* fb, unsigned cur, const int32_t* level, double* out) {
    k_export_f<D, Q, T><<<grid_for(nb * M, 256), 256, 0, s>>>(cap, b0, nb, (const T*)fa,
                                                               (const T*)fb, cur, level, out);
  }
  static void import_f(cudaStream_t s, int64_t cap, int64_t b0, int64_t nb, void* fa, void* fb,
                       unsigned cur, const int32_t* level, const double* in) {
    k_import_f<D, Q, T><<<grid_for(nb * M, 256), 256, 0, s>>>(cap, b0, nb, (T*)fa, (T*)fb, cur,
                                                               level, in);
  }
  static void export_rho_u(cudaStream_t s, int64_t cap, int64_t b0, int64_t nb, const void* fa,
                           const void* fb, unsigned cur, const int32_t* level, double* out) {
    k_export_rho_u<D, Q, T><<<grid_for(nb * M, 256), 256, 0, s>>>(
        cap, b0, nb, (const T*)fa, (const T*)fb, cur, level, out);
  }
  static void init_rest(cudaStream_t s, int64_t cap, void* f) {
    k_init_rest<D, Q, T><<<grid_for(cap * M, 256), 256, 0, s>>>(cap, (T*)f);
  }
  static int mass_partial(cudaStream_t s, int64_t cap, const void* fa, const void* fb,
                          unsigned cur, const int32_t* level, const int32_t* status,
                          double* partial) {
    const int grid = 152 * 4;
    k_mass_partial<D, Q, T><<<grid, 256, 0, s>>>(cap, (const T*)fa, (const T*)fb, cur, level,
                                                 status, partial);
    return grid;
  }
  static int force_partial(cudaStream_t s, const int32_t* list, int n, const void* f,
                           size_t stride, const int32_t* nbr, const int32_t* status,
                           const uint64_t* sm, double omega, double dx, double* partial) {
    const int grid = 152 * 2;
    k_force_partial<D, Q, T><<<grid, 256, 0, s>>>(list, n, (const T*)f, stride, nbr, status, sm,
                                                  omega, dx, partial);
    return grid;
  }
  static void features(cudaStream_t s, const int32_t* list, int n, const void* f, size_t stride,
                       int level, int lmax, double inv_dx, float* out) {
    if constexpr (D == 3) {
      if (n > 0)
        k_features<Q, T><<<grid_for(n, 2), 128, 0, s>>>(list, n, (const T*)f, stride, level, lmax,
                                                        inv_dx, out);
    }
  }

  static void collide_stream_batch(cudaStream_t s, const uint32_t* items, int n,
                                   const InstDesc* descs, int level, int which_in, int variant) {
    if (n <= 0) return;
    if (variant == 4 || variant == 5)
      k_collide_stream_batch<D, Q, T, 256><<<grid_for(n, 256 / M), 256, 0, s>>>(
          items, n, descs, level, which_in);
    else
      k_collide_stream_batch<D, Q, T, 512><<<grid_for(n, 512 / M), 512, 0, s>>>(
          items, n, descs, level, which_in);
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
    k_average_batch<D, Q, T><<<grid_for(n, 128 / M), 128, 0, s>>>(items, n, descs, level,
                                                                    which_par, which_ch);
  }

  static const LbmOps* ops() {
    static const LbmOps o = {setup,         collide_stream, interp,   average,
                             criterion,     export_f,       import_f, export_rho_u,
                             init_rest,     mass_partial,   force_partial,
                             collide_stream_batch, interp_batch, average_batch, features};
    return &o;
  }
};

}  // namespace amr
