// FP64 mass / momentum audit that allocates nothing.
//
// Callers that cannot allocate device memory -- code running under a memory
// budget fixed by a host framework, code that must not touch the CUDA
// allocator inside a latency-critical loop, or code that holds population
// buffers but no AMR instance and no arena -- can still audit a population
// buffer pair laid out the way this library stores it.  The per-CTA partial
// sums live in a file-scope device array instead of caller- or
// library-allocated scratch.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/amr.h"
#include "collide_stream.cuh"

namespace amr {

void set_error(const std::string& msg);

namespace {

constexpr int kBlocksPerCta = 64;    // blocks summed by one CTA (one partial row)
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: one row of 4 doubles per CTA.
static __device__ __align__(256) double g_partials[AMR_NOALLOC_MAX_PARTIALS * 4];

std::mutex g_mu;
double* g_scratch[kMaxDevices] = {};

// Device address of g_partials for the current device, looked up once per
// device.  Host code must not use the symbol name as a device pointer.
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error("amr_mass_audit_noalloc: no usable current device");
    return AMR_E_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess || !p) {
      set_error(std::string("amr_mass_audit_noalloc: cudaGetSymbolAddress: ") +
                cudaGetErrorString(e));
      return AMR_E_CUDA;
    }
    g_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_scratch[dev];
  return AMR_OK;
}

// The pre-collision populations of a cell are read with the library's gather
// (its stored values are the outgoing post-collision populations), which needs
// the neighbour rows and the solid-cell bits.
template <int D, int Q, class T>
__global__ void __launch_bounds__(kThreads)
    k_mass_static(int64_t n_blocks, const T* __restrict__ fa, const T* __restrict__ fb,
                  unsigned cur, const int32_t* __restrict__ level,
                  const int32_t* __restrict__ status, const int32_t* __restrict__ nbr,
                  const uint64_t* __restrict__ solidmask, double* __restrict__ partials) {
  using R = typename Store<T>::R;
  constexpr int M = Block<D>::M;
  const int64_t first = (int64_t)blockIdx.x * kBlocksPerCta * M;
  const int64_t last = min((int64_t)(blockIdx.x + 1) * kBlocksPerCta, n_blocks) * M;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t g = first + threadIdx.x; g < last; g += kThreads) {
    const int64_t b = g / M;
    if (status[b] != 1) continue;   // leaves only
    const int L = level[b];
    const T* f = ((cur >> L) & 1u) ? fb : fa;
    R fl[Q];
    gather_cell<D, Q, T, true>(fl, f, (int)b, (int)(g % M), nbr + (size_t)b * NBR_STRIDE,
                               solidmask);
    double r = 0, jx = 0, jy = 0, jz = 0;
    static_for<0, Q>([&](auto P) {
      constexpr int cx = VS<D, Q>::cx[P], cy = VS<D, Q>::cy[P], cz = VS<D, Q>::cz[P];
      const double v = (double)fl[P];
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
  __shared__ double s[4][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    for (int off = 16; off > 0; off >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], off);
    if (lane == 0) s[a][warp] = acc[a];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += s[threadIdx.x][w];
    partials[(size_t)blockIdx.x * 4 + threadIdx.x] = t;
  }
}

// Sums rows 0 .. n-1 of the partials (written by the same call) into out.
__global__ void k_mass_static_sum(int n, int nv, const double* __restrict__ partials,
                                  double* __restrict__ out) {
  __shared__ double s[kThreads];
  for (int v = 0; v < nv; ++v) {
    double x = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) x += partials[(size_t)i * 4 + v];
    s[threadIdx.x] = x;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[v] = s[0];
    __syncthreads();
  }
}

struct Args {
  int64_t n_blocks;
  const void *fa, *fb;
  unsigned cur;
  const int32_t *level, *status, *nbr;
  const uint64_t* solidmask;
};

template <int D, int Q, class T>
void launch(int grid, cudaStream_t s, const Args& a, double* scratch) {
  k_mass_static<D, Q, T><<<grid, kThreads, 0, s>>>(a.n_blocks, (const T*)a.fa, (const T*)a.fb,
                                                   a.cur, a.level, a.status, a.nbr, a.solidmask,
                                                   scratch);
}

}  // namespace
}  // namespace amr

extern "C" int amr_mass_audit_noalloc(int dim, int q, int storage, int64_t n_blocks,
                                      const void* f_a, const void* f_b, uint32_t cur,
                                      const int32_t* level, const int32_t* status,
                                      const int32_t* nbr, const uint64_t* solidmask,
                                      double* out_dev, void* stream) {
  using namespace amr;
  // an error left pending by earlier work on this thread is not this call's
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) {
    set_error(std::string("amr_mass_audit_noalloc: CUDA error pending before the audit: ") +
              cudaGetErrorString(pending));
    return AMR_E_CUDA;
  }
  const bool ok_set = (dim == 2 && q == 9) || (dim == 3 && (q == 19 || q == 27));
  if (!ok_set || storage < AMR_F64 || storage > AMR_F32_F16 || (dim == 2 && storage > AMR_F32)) {
    set_error("amr_mass_audit_noalloc: unsupported velocity set / storage");
    return AMR_E_INVAL;
  }
  if (n_blocks <= 0 || !f_a || !f_b || !level || !status || !nbr || !out_dev) {
    set_error("amr_mass_audit_noalloc: null pointer or empty input");
    return AMR_E_INVAL;
  }
  const int64_t grid64 = (n_blocks + kBlocksPerCta - 1) / kBlocksPerCta;
  if (grid64 > AMR_NOALLOC_MAX_PARTIALS) {
    set_error("amr_mass_audit_noalloc: n_blocks " + std::to_string(n_blocks) +
              " exceeds the static scratch limit of " +
              std::to_string((int64_t)AMR_NOALLOC_MAX_PARTIALS * kBlocksPerCta) + " blocks");
    return AMR_E_INVAL;
  }
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != AMR_OK) return rc;
  const int grid = (int)grid64;
  cudaStream_t s = (cudaStream_t)stream;
  const Args args{n_blocks, f_a, f_b, cur, level, status, nbr, solidmask};
  if (dim == 2) {
    if (storage == AMR_F64) launch<2, 9, double>(grid, s, args, scratch);
    else launch<2, 9, float>(grid, s, args, scratch);
  } else if (q == 19) {
    if (storage == AMR_F64) launch<3, 19, double>(grid, s, args, scratch);
    else if (storage == AMR_F32) launch<3, 19, float>(grid, s, args, scratch);
    else if (storage == AMR_F32_BF16) launch<3, 19, __nv_bfloat16>(grid, s, args, scratch);
    else launch<3, 19, __half>(grid, s, args, scratch);
  } else {
    if (storage == AMR_F64) launch<3, 27, double>(grid, s, args, scratch);
    else if (storage == AMR_F32) launch<3, 27, float>(grid, s, args, scratch);
    else if (storage == AMR_F32_BF16) launch<3, 27, __nv_bfloat16>(grid, s, args, scratch);
    else launch<3, 27, __half>(grid, s, args, scratch);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("amr_mass_audit_noalloc: partial-sum launch: ") + cudaGetErrorString(e));
    return AMR_E_CUDA;
  }
  k_mass_static_sum<<<1, kThreads, 0, s>>>(grid, 1 + dim, scratch, out_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("amr_mass_audit_noalloc: final-sum launch: ") + cudaGetErrorString(e));
    return AMR_E_CUDA;
  }
  return AMR_OK;
}
