// Validation of the block tables: the stand-in for a device bounds checker.
// Every block ID that a kernel dereferences comes from these tables (the
// neighbour rows, child0 / parent, the per-level work lists, the averaging
// groups) or from compile-time link tables.  The checks below verify each
// entry against its range and against the forest's invariants (Sections
// 3.2-3.3: same-level neighbours, 2^D consecutive children one level down
// whose parent is the block, free IDs on the gap stack), dereferencing an
// index only after it has been found in range.  A bad entry is counted in a
// device word, and the smallest failing block with the code of its check is
// kept; nothing traps.
#include <cuda_runtime.h>

#include <string>

#include "amr_internal.h"
#include "lattice.cuh"

namespace amr {

namespace {

constexpr int kInactive = 0, kUnrefined = 1;

// out[0]: bad entries; out[1]: min over bad entries of (block << 8 | code)
__device__ __forceinline__ void bad(unsigned long long* out, long long b, int code) {
  atomicAdd(out, 1ull);
  atomicMin(out + 1, ((unsigned long long)(b < 0 ? 0 : b) << 8) | (unsigned)code);
}

__global__ void k_validate_blocks(int nc, int nk, int lmax, int64_t cap,
                                  const int32_t* __restrict__ level,
                                  const int32_t* __restrict__ status,
                                  const int32_t* __restrict__ child0,
                                  const int32_t* __restrict__ parent,
                                  const int32_t* __restrict__ nbr, unsigned long long* out) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= cap) return;
  const int st = status[b], L = level[b], c0 = child0[b], pa = parent[b];
  const int32_t* row = nbr + (size_t)b * NBR_STRIDE;
  if (st < 0 || st > 4) {
    bad(out, b, AMR_CHECK_STATUS);
    return;
  }
  if (st == kInactive) {
    bool clean = L == -1 && c0 == NONE && pa == NONE;
    for (int k = 0; k < NBR_STRIDE; ++k) clean = clean && row[k] == NONE;
    if (!clean) bad(out, b, AMR_CHECK_INACTIVE);
    return;
  }
  if (L < 0 || L >= lmax) {
    bad(out, b, AMR_CHECK_LEVEL);
    return;
  }
  if (row[0] != (int32_t)b) bad(out, b, AMR_CHECK_SELF);
  for (int k = 1; k < NBR_STRIDE; ++k) {
    const int v = row[k];
    if (k >= nk) {
      if (v != NONE) bad(out, b, AMR_CHECK_UNUSED);
      continue;
    }
    if (v == NONE || (v <= -2 && v >= -7)) continue;   // missing, or a wall code
    if (v < 0 || v >= cap || status[v] == kInactive || level[v] != L) bad(out, b, AMR_CHECK_NEIGHBOUR);
  }
  if (st == kUnrefined) {
    if (c0 != NONE) bad(out, b, AMR_CHECK_CHILDREN);
  } else if (c0 < 0 || (int64_t)c0 + nc > cap) {
    bad(out, b, AMR_CHECK_CHILDREN);
  } else {
    for (int c = 0; c < nc; ++c) {
      const int ch = c0 + c;
      if (status[ch] == kInactive || level[ch] != L + 1 || parent[ch] != (int32_t)b) {
        bad(out, b, AMR_CHECK_CHILDREN);
        break;
      }
    }
  }
  if (L == 0) {
    if (pa != NONE) bad(out, b, AMR_CHECK_PARENT);
  } else if (pa < 0 || pa >= cap || status[pa] <= kUnrefined || level[pa] != L - 1 ||
             child0[pa] < 0 || b < child0[pa] || b >= (int64_t)child0[pa] + nc) {
    bad(out, b, AMR_CHECK_PARENT);
  }
}

__global__ void k_validate_gaps(int64_t cap, const int32_t* __restrict__ gap, int64_t n_gaps,
                                const int32_t* __restrict__ status, unsigned long long* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_gaps) return;
  const int g = gap[i];
  if (g < 0 || g >= cap || status[g] != kInactive) bad(out, g < 0 || g >= cap ? 0 : g, AMR_CHECK_GAP);
}

// entries of a per-level list: IDs in range, of level L (groups: block << 3 | group)
__global__ void k_validate_list(const int32_t* __restrict__ list, int64_t n, int L, int nc,
                                bool groups, int64_t cap, const int32_t* __restrict__ level,
                                unsigned long long* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int e = list[i];
  const int b = groups ? (e >> 3) : e;
  if (e < 0 || b >= cap || (groups && (e & 7) >= nc) || level[b] != L)
    bad(out, (e < 0 || b >= cap) ? 0 : b, groups ? AMR_CHECK_GROUP : AMR_CHECK_LIST);
}

// file-scope result words: calls on different streams must not overlap
__device__ unsigned long long g_check[2];

int blocks_of(int64_t n) { return (int)((n + 255) / 256); }

int begin(cudaStream_t s, unsigned long long** out) {
  AMR_CUDA(cudaGetSymbolAddress((void**)out, g_check));
  const unsigned long long init[2] = {0ull, ~0ull};
  AMR_CUDA(cudaMemcpyAsync(*out, init, sizeof(init), cudaMemcpyHostToDevice, s));
  AMR_CUDA(cudaStreamSynchronize(s));   // `init` is a host stack array
  return AMR_OK;
}

int finish(cudaStream_t s, unsigned long long* dev, int64_t* out3) {
  AMR_CUDA(cudaGetLastError());
  unsigned long long h[2] = {0ull, 0ull};
  AMR_CUDA(cudaMemcpyAsync(h, dev, sizeof(h), cudaMemcpyDeviceToHost, s));
  AMR_CUDA(cudaStreamSynchronize(s));
  out3[0] = (int64_t)h[0];
  out3[1] = h[0] ? (int64_t)(h[1] >> 8) : -1;
  out3[2] = h[0] ? (int64_t)(h[1] & 0xffu) : 0;
  return AMR_OK;
}

int validate_blocks(cudaStream_t s, int dim, int lmax, int64_t cap, const int32_t* level,
                    const int32_t* status, const int32_t* child0, const int32_t* parent,
                    const int32_t* nbr, const int32_t* gap, int64_t n_gaps,
                    unsigned long long* dev) {
  const int nc = dim == 2 ? 4 : 8, nk = dim == 2 ? 9 : 27;
  k_validate_blocks<<<blocks_of(cap), 256, 0, s>>>(nc, nk, lmax, cap, level, status, child0,
                                                   parent, nbr, dev);
  if (n_gaps > 0)
    k_validate_gaps<<<blocks_of(n_gaps), 256, 0, s>>>(cap, gap, n_gaps, status, dev);
  return AMR_OK;
}

}  // namespace

// The instance's own tables, lists and averaging groups; a bad entry fails
// with AMR_E_INVAL (see amr_check_tables).
int check_instance_tables(Instance* a, int64_t* out3) {
  cudaStream_t s = a->stream;
  unsigned long long* dev = nullptr;
  int rc = begin(s, &dev);
  if (rc != AMR_OK) return rc;
  if (a->n_gaps < 0 || a->n_gaps > a->cap) {
    out3[0] = 1;
    out3[1] = -1;
    out3[2] = AMR_CHECK_GAP;
  } else {
    validate_blocks(s, a->dim, a->lmax, a->cap, a->level, a->status, a->child0, a->parent,
                    a->nbr, a->gap, a->n_gaps, dev);
    for (int L = 0; L < a->lmax; ++L) {
      const size_t off = (size_t)L * a->cap;
      const int64_t lists[5] = {a->n_ids[L], a->n_active[L], a->n_parents[L], a->n_bnd[L],
                                a->n_ids[L]};
      const int32_t* ptr[5] = {a->idset + off, a->active + off, a->parents + off, a->bnd + off,
                               a->order + off};
      for (int j = 0; j < 5; ++j)
        if (lists[j] > 0)
          k_validate_list<<<blocks_of(lists[j]), 256, 0, s>>>(ptr[j], lists[j], L, a->nc, false,
                                                              a->cap, a->level, dev);
      if (a->n_agrp[L] > 0)
        k_validate_list<<<blocks_of(a->n_agrp[L]), 256, 0, s>>>(
            a->agrp + a->agrp_off[L], a->n_agrp[L], L, a->nc, true, a->cap, a->level, dev);
    }
    rc = finish(s, dev, out3);
    if (rc != AMR_OK) return rc;
  }
  if (out3[0] != 0) {
    set_error("block tables: " + std::to_string(out3[0]) + " bad entries, first at block " +
              std::to_string(out3[1]) + " (check " + std::to_string(out3[2]) + ")");
    return AMR_E_INVAL;
  }
  return AMR_OK;
}

}  // namespace amr

using namespace amr;

extern "C" {

int amr_validate_tables(int dim, int max_levels, int64_t cap, const int32_t* level,
                        const int32_t* status, const int32_t* child0, const int32_t* parent,
                        const int32_t* nbr, const int32_t* gap, int64_t n_gaps, int64_t* out3,
                        void* stream) {
  if ((dim != 2 && dim != 3) || max_levels < 1 || max_levels > AMR_MAX_LEVELS || cap <= 0 ||
      cap > (int64_t(1) << 31) / 64 || !level || !status || !child0 || !parent || !nbr ||
      !out3 || n_gaps < 0 || (n_gaps > 0 && !gap)) {
    set_error("amr_validate_tables: bad arguments");
    return AMR_E_INVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_gaps > cap) {
    out3[0] = 1;
    out3[1] = -1;
    out3[2] = AMR_CHECK_GAP;
    return AMR_OK;
  }
  unsigned long long* dev = nullptr;
  int rc = begin(s, &dev);
  if (rc != AMR_OK) return rc;
  validate_blocks(s, dim, max_levels, cap, level, status, child0, parent, nbr, gap, n_gaps, dev);
  return finish(s, dev, out3);
}

}  // extern "C"
