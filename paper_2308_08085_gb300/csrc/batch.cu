// Batched instances: many independent block forests advanced in lock-step by
// one sequence of launches.  The recursive level step of Section 4.1 has the
// same shape for every instance (an instance without level L+1 contributes no
// work there), so each level operation becomes one launch over an
// instance-major list of (instance, block) items.  The batched coarse step is
// captured as a CUDA graph (one per parity of level 0); the collide-stream
// variant is picked by timing the candidates on the batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "amr_internal.h"
#include "lattice.cuh"

namespace amr {

struct Batch {
  std::vector<Instance*> inst;
  int n = 0, dim = 0, q = 0, storage = 0, lmax = 0;
  cudaStream_t stream = nullptr, capture_stream = nullptr;
  const LbmOps* ops = nullptr;
  InstDesc* descs = nullptr;                  // device [n]
  uint32_t* act[BATCH_MAX_LEVELS] = {};       // device item lists
  uint32_t* par[BATCH_MAX_LEVELS] = {};
  int64_t n_act[BATCH_MAX_LEVELS] = {}, n_par[BATCH_MAX_LEVELS] = {},
          n_ids[BATCH_MAX_LEVELS] = {};
  int64_t list_cap = 0;
  unsigned cur = 0;
  int variant = 512;   // threads per CTA of the batched collide-stream
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graph_valid = false;
  int64_t launches = 0, graph_launches[2] = {0, 0};
};

static size_t align256b(size_t x) { return (x + 255) & ~size_t(255); }

static int64_t sum_caps(amr_t* const* in, int n) {
  int64_t s = 0;
  for (int i = 0; i < n; ++i) s += reinterpret_cast<Instance*>(in[i])->cap;
  return s;
}

static int max_levels(amr_t* const* in, int n) {
  int m = 0;
  for (int i = 0; i < n; ++i) m = std::max(m, reinterpret_cast<Instance*>(in[i])->lmax);
  return m;
}

__global__ void k_pack_items(const int32_t* __restrict__ list, int n, int inst,
                             uint32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = ((uint32_t)inst << BATCH_SHIFT) | (uint32_t)list[i];
}

static int refresh(Batch* b) {
  std::vector<InstDesc> h(b->n);
  for (int i = 0; i < b->n; ++i) {
    Instance* a = b->inst[i];
    InstDesc& d = h[i];
    std::memset(&d, 0, sizeof(d));
    d.f[0] = a->f[0];
    d.f[1] = a->f[1];
    d.nbr = a->nbr;
    d.child0 = a->child0;
    d.cellmask = a->cellmask;
    d.stride = a->stride();
    for (int L = 0; L < a->lmax; ++L) {
      d.omega[L] = 1.0 / a->tau[L];
      if (L + 1 < a->lmax) {
        d.r_cf[L] = a->tau[L + 1] / (2.0 * a->tau[L]);
        d.r_fc[L] = 2.0 * a->tau[L] / a->tau[L + 1];
      }
    }
    d.faces = a->prm.faces;
  }
  AMR_CUDA(cudaMemcpyAsync(b->descs, h.data(), sizeof(InstDesc) * b->n, cudaMemcpyHostToDevice,
                           b->stream));
  for (int L = 0; L < b->lmax; ++L) {
    int64_t oa = 0, op = 0, ni = 0;
    for (int i = 0; i < b->n; ++i) {
      Instance* a = b->inst[i];
      if (L >= a->lmax) continue;
      const int64_t na = a->n_active[L], np = a->n_parents[L];
      if (na > 0)
        k_pack_items<<<(int)((na + 255) / 256), 256, 0, b->stream>>>(
            a->active + (size_t)L * a->cap, (int)na, i, b->act[L] + oa);
      if (np > 0)
        k_pack_items<<<(int)((np + 255) / 256), 256, 0, b->stream>>>(
            a->parents + (size_t)L * a->cap, (int)np, i, b->par[L] + op);
      oa += na;
      op += np;
      ni += a->n_ids[L];
    }
    b->n_act[L] = oa;
    b->n_par[L] = op;
    b->n_ids[L] = ni;
  }
  AMR_CUDA(cudaGetLastError());
  AMR_CUDA(cudaStreamSynchronize(b->stream));   // the host descriptor copy must finish
  for (auto& g : b->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  b->graph_valid = false;
  return AMR_OK;
}

static void advance_batch(Batch* b, int L) {
  const bool fine = L + 1 < b->lmax && b->n_ids[L + 1] > 0;
  const int64_t np = b->n_par[L];
  const int wl = (int)((b->cur >> L) & 1u);
  if (fine && np > 0) {
    b->ops->interp_batch(b->stream, b->par[L], (int)np, b->descs, L, wl,
                         (int)((b->cur >> (L + 1)) & 1u));
    b->launches += 1;
  }
  if (b->n_act[L] > 0) {
    b->ops->collide_stream_batch(b->stream, b->act[L], (int)b->n_act[L], b->descs, L, wl,
                                 b->variant);
    b->launches += 1;
  }
  b->cur ^= 1u << L;
  if (fine) {
    advance_batch(b, L + 1);
    advance_batch(b, L + 1);
    if (np > 0) {
      b->ops->average_batch(b->stream, b->par[L], (int)np, b->descs, L,
                            (int)((b->cur >> L) & 1u), (int)((b->cur >> (L + 1)) & 1u));
      b->launches += 1;
    }
  }
}

static int build_batch_graphs(Batch* b) {
  const unsigned saved = b->cur;
  cudaStream_t user = b->stream;
  b->stream = b->capture_stream;
  for (int parity = 0; parity < 2; ++parity) {
    b->cur = (saved & ~1u) | (unsigned)parity;
    cudaGraph_t g = nullptr;
    const int64_t before = b->launches;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      advance_batch(b, 0);
      e = cudaStreamEndCapture(b->stream, &g);
    }
    b->graph_launches[parity] = b->launches - before;
    b->launches = before;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[parity], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->stream = user;
      b->cur = saved;
      set_error(std::string("batch graph capture: ") + cudaGetErrorString(e));
      cudaGetLastError();
      return AMR_E_CUDA;
    }
  }
  b->stream = user;
  b->cur = saved;
  b->graph_valid = true;
  return AMR_OK;
}

static int step_batch(Batch* b, int n) {
  for (Instance* a : b->inst)
    if (a->cur != b->cur) {
      set_error("batch members were stepped outside the batch (buffer parities differ)");
      return AMR_E_INVAL;
    }
  if (!b->graph_valid) {
    const int rc = build_batch_graphs(b);
    if (rc != AMR_OK) return rc;
  }
  for (int s = 0; s < n; ++s) {
    const int parity = (int)(b->cur & 1u);
    AMR_CUDA(cudaGraphLaunch(b->graph[parity], b->stream));
    b->launches += b->graph_launches[parity];
    b->cur ^= 1u;
  }
  for (Instance* a : b->inst) {
    a->cur = b->cur;
    a->coarse_steps += n;
  }
  AMR_CUDA(cudaGetLastError());
  return AMR_OK;
}

}  // namespace amr

using namespace amr;

extern "C" {

size_t amr_batch_arena_bytes(amr_t* const* instances, int n) {
  if (!instances || n <= 0) return 0;
  const int64_t caps = sum_caps(instances, n);
  const int lmax = max_levels(instances, n);
  return align256b(sizeof(InstDesc) * n) + 2 * (size_t)lmax * align256b((size_t)caps * 4);
}

int amr_batch_create(amr_t* const* instances, int n, void* dev_arena, size_t arena_bytes,
                     void* stream, amr_batch_t** out) {
  if (!out || !instances || n <= 0) return AMR_E_INVAL;
  *out = nullptr;
  if (n > (1 << (32 - BATCH_SHIFT)) - 1) {
    set_error("too many instances for one batch");
    return AMR_E_INVAL;
  }
  Instance* a0 = reinterpret_cast<Instance*>(instances[0]);
  for (int i = 0; i < n; ++i) {
    Instance* a = reinterpret_cast<Instance*>(instances[i]);
    if (!a || a->dim != a0->dim || a->q != a0->q || a->storage != a0->storage) {
      set_error("batch members must share the velocity set and storage");
      return AMR_E_INVAL;
    }
    if (a->solid) {
      set_error("batch members may not have a solid prism");
      return AMR_E_INVAL;
    }
    if (a->cfg.interp != AMR_INTERP_LINEAR) {
      set_error("batch members use linear interpolation");
      return AMR_E_INVAL;
    }
    if (a->cap > (int64_t)BATCH_MASK) {
      set_error("batch member capacity exceeds 2^25 blocks");
      return AMR_E_INVAL;
    }
    if (a->lmax > BATCH_MAX_LEVELS || a->cur != a0->cur) {
      set_error("batch members must have equal buffer parities");
      return AMR_E_INVAL;
    }
  }
  const size_t need = amr_batch_arena_bytes(instances, n);
  if (!dev_arena || arena_bytes < need || ((uintptr_t)dev_arena & 255u)) {
    set_error("batch arena needs " + std::to_string(need) + " bytes, 256-byte aligned");
    return AMR_E_ARENA;
  }
  Batch* b = new Batch();
  for (int i = 0; i < n; ++i) b->inst.push_back(reinterpret_cast<Instance*>(instances[i]));
  b->n = n;
  b->dim = a0->dim;
  b->q = a0->q;
  b->storage = a0->storage;
  b->lmax = max_levels(instances, n);
  b->ops = a0->ops;
  b->stream = (cudaStream_t)stream;
  b->cur = a0->cur;
  b->list_cap = sum_caps(instances, n);
  char* base = (char*)dev_arena;
  b->descs = (InstDesc*)base;
  size_t off = align256b(sizeof(InstDesc) * n);
  for (int L = 0; L < b->lmax; ++L) {
    b->act[L] = (uint32_t*)(base + off);
    off += align256b((size_t)b->list_cap * 4);
    b->par[L] = (uint32_t*)(base + off);
    off += align256b((size_t)b->list_cap * 4);
  }
  if (cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    set_error("cannot create capture stream");
    return AMR_E_CUDA;
  }
  const int rc = refresh(b);
  if (rc != AMR_OK) {
    cudaStreamDestroy(b->capture_stream);
    delete b;
    return rc;
  }
  *out = reinterpret_cast<amr_batch_t*>(b);
  return AMR_OK;
}

int amr_batch_refresh(amr_batch_t* h) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b) return AMR_E_INVAL;
  return refresh(b);
}

int amr_batch_step(amr_batch_t* h, int n_coarse_steps) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b || n_coarse_steps < 0) return AMR_E_INVAL;
  return step_batch(b, n_coarse_steps);
}

int amr_batch_autotune(amr_batch_t* h, int trial_steps, int* chosen) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b || trial_steps < 1) return AMR_E_INVAL;
  // CTA sizes of the batched collide-stream: 512 / 256 / 128 / 64 threads,
  // i.e. M_L = 8 / 4 / 2 / 1 blocks of 64 cells per CTA in 3D
  static const int candidates[] = {512, 256, 128, 64};
  cudaEvent_t e0, e1;
  AMR_CUDA(cudaEventCreate(&e0));
  AMR_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_v = b->variant;
  for (int v : candidates) {
    b->variant = v;
    b->graph_valid = false;
    int rc = step_batch(b, 1);   // capture and warm
    if (rc != AMR_OK) return rc;
    AMR_CUDA(cudaEventRecord(e0, b->stream));
    rc = step_batch(b, trial_steps);
    if (rc != AMR_OK) return rc;
    AMR_CUDA(cudaEventRecord(e1, b->stream));
    AMR_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->variant = best_v;
  b->graph_valid = false;
  if (chosen) *chosen = best_v;
  return AMR_OK;
}

int64_t amr_batch_launches(amr_batch_t* h) {
  Batch* b = reinterpret_cast<Batch*>(h);
  return b ? b->launches : AMR_E_INVAL;
}

int amr_batch_free(amr_batch_t* h) {
  Batch* b = reinterpret_cast<Batch*>(h);
  if (!b) return AMR_E_INVAL;
  for (auto& g : b->graph)
    if (g) cudaGraphExecDestroy(g);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  delete b;
  return AMR_OK;
}

}  // extern "C"
