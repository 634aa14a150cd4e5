// Compile-time velocity sets, storage traits and block/cell geometry shared
// by the LBM kernels.  Numbering follows the paper's velocity-set figure
// (Section 2); weights are the standard Gauss-Hermite weights by speed shell.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace amr {

constexpr int NONE = -1;
constexpr int NBR_STRIDE = 32;   // int32 slots per block row of the nbr table

// ----------------------------------------------------------- static loops
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// ----------------------------------------------------------- velocity sets
template <int D, int Q> struct VS;

template <> struct VS<2, 9> {
  static constexpr int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  static constexpr int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  static constexpr int cz[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  static constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  static constexpr double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                  1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
};

#define AMR_D3_CX 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0
#define AMR_D3_CY 0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 1, -1
#define AMR_D3_CZ 0, 0, 0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 1, -1, 1
#define AMR_D3_OPP 0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17

template <> struct VS<3, 19> {
  static constexpr int cx[19] = {AMR_D3_CX};
  static constexpr int cy[19] = {AMR_D3_CY};
  static constexpr int cz[19] = {AMR_D3_CZ};
  static constexpr int opp[19] = {AMR_D3_OPP};
  static constexpr double w[19] = {1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                                   1.0 / 18, 1.0 / 18, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                                   1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                                   1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
};

template <> struct VS<3, 27> {
  static constexpr int cx[27] = {AMR_D3_CX, 1, -1, 1, -1, 1, -1, -1, 1};
  static constexpr int cy[27] = {AMR_D3_CY, 1, -1, 1, -1, -1, 1, 1, -1};
  static constexpr int cz[27] = {AMR_D3_CZ, 1, -1, -1, 1, 1, -1, 1, -1};
  static constexpr int opp[27] = {AMR_D3_OPP, 20, 19, 22, 21, 24, 23, 26, 25};
  static constexpr double w[27] = {
      8.0 / 27,  2.0 / 27,  2.0 / 27,  2.0 / 27,  2.0 / 27,  2.0 / 27,  2.0 / 27,
      1.0 / 54,  1.0 / 54,  1.0 / 54,  1.0 / 54,  1.0 / 54,  1.0 / 54,  1.0 / 54,
      1.0 / 54,  1.0 / 54,  1.0 / 54,  1.0 / 54,  1.0 / 54,  1.0 / 216, 1.0 / 216,
      1.0 / 216, 1.0 / 216, 1.0 / 216, 1.0 / 216, 1.0 / 216, 1.0 / 216};
};

// Block-neighbour numbering: D2Q9 in 2D, D3Q27 in 3D.  dir_of(sx,sy,sz)
// returns the index of the direction (sx,sy,sz) in {-1,0,1}^D.
template <int D> struct Nbr {
  static constexpr int K = D == 2 ? 9 : 27;
  using V = std::conditional_t<D == 2, VS<2, 9>, VS<3, 27>>;
  static constexpr int dir_of(int sx, int sy, int sz) {
    for (int k = 0; k < K; ++k)
      if (V::cx[k] == sx && V::cy[k] == sy && V::cz[k] == sz) return k;
    return -1;
  }
};

// ------------------------------------------------------------ block geometry
template <int D> struct Block {
  static constexpr int M = D == 2 ? 16 : 64;
  static constexpr int NC = D == 2 ? 4 : 8;
  __host__ __device__ static constexpr int ci(int l) { return l & 3; }
  __host__ __device__ static constexpr int cj(int l) { return (l >> 2) & 3; }
  __host__ __device__ static constexpr int ck(int l) { return D == 2 ? 0 : (l >> 4); }
  __host__ __device__ static constexpr int cell(int i, int j, int k) {
    return i + 4 * j + (D == 2 ? 0 : 16 * k);
  }
};

// Chebyshev distance (cells) from cell (i,j,k) to the nearest block region in
// a direction flagged in `none_mask` (bit k set when nbr[k] == NONE); 0 when
// no bit is set.  Class: d in {1,2} ghost, {3,4} interface, else interior
// (Section 3.4).
template <int D>
__device__ __forceinline__ int cell_class(uint32_t none_mask, int i, int j, int k) {
  using NV = typename Nbr<D>::V;
  int best = 99;
  uint32_t m = none_mask & ~1u;
  while (m) {
    int d = __ffs(m) - 1;
    m &= m - 1;
    int sx = 0, sy = 0, sz = 0;
    // direction vectors of the neighbour numbering
    static_for<1, Nbr<D>::K>([&](auto P) {
      constexpr int vx = NV::cx[P], vy = NV::cy[P], vz = NV::cz[P];
      if (P == d) { sx = vx; sy = vy; sz = vz; }
    });
    int dist = 0;
    dist = max(dist, sx < 0 ? i + 1 : (sx > 0 ? 4 - i : 0));
    dist = max(dist, sy < 0 ? j + 1 : (sy > 0 ? 4 - j : 0));
    if (D == 3) dist = max(dist, sz < 0 ? k + 1 : (sz > 0 ? 4 - k : 0));
    best = min(best, dist);
  }
  return best <= 2 ? 2 : (best <= 4 ? 1 : 0);   // GHOST, INTERFACE, INTERIOR
}

// ---------------------------------------------------------- storage traits
// Values are stored either as the population itself (FP64, FP32) or as the
// shifted value f - w_p in BF16 / FP16, rounded to nearest even.
template <class T> struct Store;
template <> struct Store<double> {
  using R = double;
  static constexpr bool kShifted = false;
  template <int D, int Q, int P> __device__ static R load(double v) { return v; }
  template <int D, int Q, int P> __device__ static double save(R v) { return v; }
};
template <> struct Store<float> {
  using R = float;
  static constexpr bool kShifted = false;
  template <int D, int Q, int P> __device__ static R load(float v) { return v; }
  template <int D, int Q, int P> __device__ static float save(R v) { return v; }
};
template <> struct Store<__nv_bfloat16> {
  using R = float;
  static constexpr bool kShifted = true;   // holds f - w_p
  __device__ static R raw(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __nv_bfloat16 from_raw(R v) { return __float2bfloat16_rn(v); }
  template <int D, int Q, int P> __device__ static R load(__nv_bfloat16 v) {
    constexpr float wp = float(VS<D, Q>::w[P]);
    return __bfloat162float(v) + wp;
  }
  template <int D, int Q, int P> __device__ static __nv_bfloat16 save(R v) {
    constexpr float wp = float(VS<D, Q>::w[P]);
    return __float2bfloat16_rn(v - wp);
  }
};
template <> struct Store<__half> {
  using R = float;
  static constexpr bool kShifted = true;   // holds f - w_p
  __device__ static R raw(__half v) { return __half2float(v); }
  __device__ static __half from_raw(R v) { return __float2half_rn(v); }
  template <int D, int Q, int P> __device__ static R load(__half v) {
    constexpr float wp = float(VS<D, Q>::w[P]);
    return __half2float(v) + wp;
  }
  template <int D, int Q, int P> __device__ static __half save(R v) {
    constexpr float wp = float(VS<D, Q>::w[P]);
    return __float2half_rn(v - wp);
  }
};

// Runtime-p variants (used off the hot path).
template <int D, int Q, class T>
__device__ __forceinline__ typename Store<T>::R load_rt(T v, int p) {
  typename Store<T>::R r = 0;
  static_for<0, Q>([&](auto P) {
    if (P == p) r = Store<T>::template load<D, Q, P>(v);
  });
  return r;
}
template <int D, int Q, class T>
__device__ __forceinline__ T save_rt(typename Store<T>::R v, int p) {
  T r{};
  static_for<0, Q>([&](auto P) {
    if (P == p) r = Store<T>::template save<D, Q, P>(v);
  });
  return r;
}

// ------------------------------------------------------- BGK building blocks
template <int D, int Q, class R>
__device__ __forceinline__ void moments(const R* f, R& rho, R& ux, R& uy, R& uz) {
  using V = VS<D, Q>;
  R r = 0, jx = 0, jy = 0, jz = 0;
  static_for<0, Q>([&](auto P) {
    constexpr int p = P;
    constexpr int cx = V::cx[p], cy = V::cy[p], cz = V::cz[p];
    r += f[p];
    if constexpr (cx != 0) jx += cx > 0 ? f[p] : -f[p];
    if constexpr (cy != 0) jy += cy > 0 ? f[p] : -f[p];
    if constexpr (cz != 0) jz += cz > 0 ? f[p] : -f[p];
  });
  rho = r;
  R inv = R(1) / r;
  ux = jx * inv;
  uy = jy * inv;
  uz = D == 3 ? jz * inv : R(0);
}

template <int D, int Q, int P, class R>
__device__ __forceinline__ R feq(R rho, R ux, R uy, R uz, R usq15) {
  using V = VS<D, Q>;
  constexpr int cx = V::cx[P], cy = V::cy[P], cz = V::cz[P];
  R cu = R(0);
  if constexpr (cx != 0) cu += cx > 0 ? ux : -ux;
  if constexpr (cy != 0) cu += cy > 0 ? uy : -uy;
  if constexpr (cz != 0) cu += cz > 0 ? uz : -uz;
  constexpr double wp = V::w[P];
  return R(wp) * rho * (R(1) + R(3) * cu + R(4.5) * cu * cu - usq15);
}

}  // namespace amr
