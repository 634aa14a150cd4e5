// Cell-based uniform solver: the cell arrangement of the paper's comparison of
// cell- and block-based grids on one level (Section 5, "Cell vs. Block
// Arrangement").  Every cell is its own element; elements are numbered by a
// caller-given permutation of the cell positions (x-fastest, Morton order,
// shuffled, ...).  One kernel per time step: BGK collision (Section 4.3) and
// push streaming (Section 4.2) of each element to the elements one link away,
// periodic in every axis.  Neighbour IDs are either computed from the element
// ID (x-fastest numbering only) or read from a table [Q][n] built on the host.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/amr.h"
#include "lattice.cuh"

namespace amr {

void set_error(const std::string& msg);

namespace {

constexpr int kCellThreads = 256;

// Position (x-fastest index) of the cell one link c_P downstream of (x, y, z),
// wrapped periodically.
template <int D, int Q, int P>
__host__ __device__ __forceinline__ int64_t downstream(int x, int y, int z, int nx, int ny,
                                                       int nz) {
  constexpr int cx = VS<D, Q>::cx[P], cy = VS<D, Q>::cy[P], cz = VS<D, Q>::cz[P];
  int tx = x + cx, ty = y + cy, tz = z + cz;
  tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
  ty = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
  if (D == 3) tz = tz < 0 ? tz + nz : (tz >= nz ? tz - nz : tz);
  else tz = 0;
  return (int64_t)tx + (int64_t)nx * ((int64_t)ty + (int64_t)ny * tz);
}

// One collide-push step.  f_in / f_out: [Q][n] FP32 by element ID.  TABLE:
// target IDs from table[P * n + id]; otherwise IDs are x-fastest positions and
// targets are computed.
template <int D, int Q, bool TABLE>
__global__ void __launch_bounds__(kCellThreads)
    k_cells_step(const float* __restrict__ fin, float* __restrict__ fout,
                 const int32_t* __restrict__ table, int64_t n, int nx, int ny, int nz,
                 float omega) {
  const int64_t id = (int64_t)blockIdx.x * kCellThreads + threadIdx.x;
  if (id >= n) return;
  float f[Q];
  static_for<0, Q>([&](auto P) { f[P] = __ldg(fin + (int64_t)P * n + id); });
  float rho, ux, uy, uz;
  moments<D, Q>(f, rho, ux, uy, uz);
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  int x = 0, y = 0, z = 0;
  if constexpr (!TABLE) {
    x = (int)(id % nx);
    y = (int)((id / nx) % ny);
    z = D == 3 ? (int)(id / ((int64_t)nx * ny)) : 0;
  }
  static_for<0, Q>([&](auto P) {
    constexpr int p = P;
    const float fs = f[p] + omega * (feq<D, Q, p>(rho, ux, uy, uz, usq15) - f[p]);
    int64_t t;
    if constexpr (TABLE) t = __ldg(table + (int64_t)p * n + id);
    else t = downstream<D, Q, p>(x, y, z, nx, ny, nz);
    fout[(int64_t)p * n + t] = fs;
  });
}

// Rest equilibrium (rho = 1, u = 0): f[P * n + i] = w_P.
template <int D, int Q>
__global__ void __launch_bounds__(kCellThreads) k_cells_rest(float* __restrict__ f, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * kCellThreads + threadIdx.x;
  if (i >= n) return;
  static_for<0, Q>([&](auto P) { f[(int64_t)P * n + i] = (float)VS<D, Q>::w[P]; });
}

template <int D, int Q>
void fill_table(int nx, int ny, int nz, const int32_t* id_of_pos, int32_t* table) {
  const int64_t nxy = (int64_t)nx * ny, n = nxy * (D == 3 ? nz : 1);
  for (int64_t pos = 0; pos < n; ++pos) {
    const int x = (int)(pos % nx), y = (int)((pos / nx) % ny), z = (int)(pos / nxy);
    const int64_t id = id_of_pos ? id_of_pos[pos] : pos;
    static_for<0, Q>([&](auto P) {
      const int64_t t = downstream<D, Q, P>(x, y, z, nx, ny, nz);
      table[(int64_t)P * n + id] = id_of_pos ? id_of_pos[t] : (int32_t)t;
    });
  }
}

template <int D, int Q>
void launch_cells(bool use_table, const float* fin, float* fout, const int32_t* table, int64_t n,
                  int nx, int ny, int nz, float omega, cudaStream_t s) {
  const unsigned grid = (unsigned)((n + kCellThreads - 1) / kCellThreads);
  if (use_table)
    k_cells_step<D, Q, true><<<grid, kCellThreads, 0, s>>>(fin, fout, table, n, nx, ny, nz, omega);
  else
    k_cells_step<D, Q, false><<<grid, kCellThreads, 0, s>>>(fin, fout, nullptr, n, nx, ny, nz,
                                                            omega);
}

// Number of cells, or a negative code with the error set.
int64_t cells_count(const char* who, int dim, int q, int nx, int ny, int nz) {
  const bool ok_set = (dim == 2 && q == 9) || (dim == 3 && (q == 19 || q == 27));
  if (!ok_set) {
    set_error(std::string(who) + ": unsupported velocity set");
    return AMR_E_INVAL;
  }
  if (nx < 1 || ny < 1 || (dim == 3 && nz < 1)) {
    set_error(std::string(who) + ": empty grid");
    return AMR_E_INVAL;
  }
  const int64_t n = (int64_t)nx * ny * (dim == 3 ? nz : 1);
  if (n * q > ((int64_t)1 << 40) || n > ((int64_t)1 << 31) - 1) {
    set_error(std::string(who) + ": grid too large for int32 element IDs");
    return AMR_E_INVAL;
  }
  return n;
}

}  // namespace
}  // namespace amr

extern "C" int amr_cells_table(int dim, int q, int nx, int ny, int nz, const int32_t* id_of_pos,
                               int32_t* table) {
  using namespace amr;
  const int64_t n = cells_count("amr_cells_table", dim, q, nx, ny, nz);
  if (n < 0) return (int)n;
  if (!table) {
    set_error("amr_cells_table: null table");
    return AMR_E_INVAL;
  }
  if (id_of_pos) {
    // the IDs must be a permutation of 0 .. n-1: every table entry is then an
    // in-range element ID
    std::vector<unsigned char> seen((size_t)n, 0);
    for (int64_t i = 0; i < n; ++i) {
      const int32_t v = id_of_pos[i];
      if (v < 0 || v >= n || seen[(size_t)v]) {
        set_error("amr_cells_table: id_of_pos is not a permutation of 0 .. n-1 (entry " +
                  std::to_string(i) + ")");
        return AMR_E_INVAL;
      }
      seen[(size_t)v] = 1;
    }
  }
  if (dim == 2) fill_table<2, 9>(nx, ny, 1, id_of_pos, table);
  else if (q == 19) fill_table<3, 19>(nx, ny, nz, id_of_pos, table);
  else fill_table<3, 27>(nx, ny, nz, id_of_pos, table);
  return AMR_OK;
}

extern "C" int amr_cells_step(int dim, int q, int nx, int ny, int nz, int connectivity,
                              double nu0, const int32_t* table, float* f_a, float* f_b,
                              int n_steps, void* stream) {
  using namespace amr;
  const int64_t n = cells_count("amr_cells_step", dim, q, nx, ny, nz);
  if (n < 0) return (int)n;
  if (connectivity != AMR_CELLS_CALCULATED && connectivity != AMR_CELLS_RETRIEVED) {
    set_error("amr_cells_step: unknown connectivity");
    return AMR_E_INVAL;
  }
  const bool use_table = connectivity == AMR_CELLS_RETRIEVED;
  if (!f_a || !f_b || f_a == f_b || (use_table && !table) || n_steps < 0 || !(nu0 > 0.0)) {
    set_error("amr_cells_step: null or aliased buffer, missing table, negative step count "
              "or non-positive viscosity");
    return AMR_E_INVAL;
  }
  const float omega = (float)(1.0 / (3.0 * nu0 + 0.5));
  cudaStream_t s = (cudaStream_t)stream;
  for (int k = 0; k < n_steps; ++k) {
    const float* fin = (k & 1) ? f_b : f_a;
    float* fout = (k & 1) ? f_a : f_b;
    if (dim == 2) launch_cells<2, 9>(use_table, fin, fout, table, n, nx, ny, 1, omega, s);
    else if (q == 19) launch_cells<3, 19>(use_table, fin, fout, table, n, nx, ny, nz, omega, s);
    else launch_cells<3, 27>(use_table, fin, fout, table, n, nx, ny, nz, omega, s);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("amr_cells_step: launch: ") + cudaGetErrorString(e));
    return AMR_E_CUDA;
  }
  return AMR_OK;
}

extern "C" int amr_cells_rest(int dim, int q, int nx, int ny, int nz, float* f, void* stream) {
  using namespace amr;
  const int64_t n = cells_count("amr_cells_rest", dim, q, nx, ny, nz);
  if (n < 0) return (int)n;
  if (!f) {
    set_error("amr_cells_rest: null buffer");
    return AMR_E_INVAL;
  }
  const unsigned grid = (unsigned)((n + kCellThreads - 1) / kCellThreads);
  cudaStream_t s = (cudaStream_t)stream;
  if (dim == 2) k_cells_rest<2, 9><<<grid, kCellThreads, 0, s>>>(f, n);
  else if (q == 19) k_cells_rest<3, 19><<<grid, kCellThreads, 0, s>>>(f, n);
  else k_cells_rest<3, 27><<<grid, kCellThreads, 0, s>>>(f, n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("amr_cells_rest: launch: ") + cudaGetErrorString(e));
    return AMR_E_CUDA;
  }
  return AMR_OK;
}
