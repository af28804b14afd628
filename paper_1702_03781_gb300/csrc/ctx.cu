// ctx.cu -- context creation, workspace ownership, status strings.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "ozaki.cuh"

namespace harp {
int g_last_cuda_error = 0;
std::atomic<unsigned long long> g_kernel_launches{0};
}

using namespace harp;

extern "C" const char* harp_status_string(int s) {
  if (s == HARP_OK) return "ok";
  if (s < 0) return "invalid argument";
  switch (s) {
    case HARP_E_COINCIDENT: return "coincident antennas (r == 0)";
    case HARP_E_NOCONV: return "iterative refinement did not reach tol";
    case HARP_E_TIMEOUT: return "bounded device wait gave up";
    case HARP_E_CUDA: return "CUDA runtime error";
    case HARP_E_NOMEM: return "device allocation failed";
    case HARP_E_UNSUPPORTED: return "size not supported by this build";
    case HARP_E_STATE: return "call order violated (no cached factorisation)";
    case HARP_E_NONFINITE: return "non-finite value in inputs or factors";
    default: return "exactly zero pivot (singular matrix)";
  }
}

extern "C" int harp_last_cuda_error(void) { return g_last_cuda_error; }

extern "C" unsigned long long harp_kernel_launches(void) { return g_kernel_launches.load(); }

static void free_all(harp_ctx* c) {
  void* ptrs[] = {c->z64, c->lu_re, c->lu_im, c->ipiv, c->w_re, c->w_im, c->x_re, c->x_im,
                  c->r_re, c->r_im, c->v_re, c->v_im, c->t_re, c->t_im, c->perm, c->zff, c->xff, c->rowsum, c->tc_a, c->tc_b, c->dinv_re, c->dinv_im, c->rpart, c->finv, c->finv_tmp, c->finv_split, c->pmap, c->gpair, c->red, c->dstatus,
                  c->oz_a, c->oz_y, c->oz_slots, c->oz_acc, c->oz_rexp, c->oz_cexp, c->oz_part,
                  c->oz_znorm};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int g = 0; g < 2; ++g)
    if (c->solve_graph[g]) cudaGraphExecDestroy(c->solve_graph[g]);
  for (int g = 0; g < 18; ++g)
    if (c->ref_graph[g]) cudaGraphExecDestroy(c->ref_graph[g]);
  if (c->zbuf) cudaFree(c->zbuf);
  if (c->fin) cudaFree(c->fin);
  if (c->gbuf) cudaFree(c->gbuf);
  if (c->blk_uinv) cudaFree(c->blk_uinv);
  if (c->eep_ws) cudaFree(c->eep_ws);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->lu_stream) cudaStreamDestroy(c->lu_stream);
  if (c->ev_lu_fork) cudaEventDestroy(c->ev_lu_fork);
  if (c->ev_lu_join) cudaEventDestroy(c->ev_lu_join);
  if (c->fill_stream) cudaStreamDestroy(c->fill_stream);
  for (int q = 0; q < 2; ++q) {
    if (c->inv_stream[q]) cudaStreamDestroy(c->inv_stream[q]);
    if (c->ev_inv[q]) cudaEventDestroy(c->ev_inv[q]);
  }
  if (c->ev_fill_fork) cudaEventDestroy(c->ev_fill_fork);
  if (c->ev_z64) cudaEventDestroy(c->ev_z64);
  for (int e = 0; e < c->n_events; ++e) {
    if (c->ev_fac && c->ev_fac[e]) cudaEventDestroy(c->ev_fac[e]);
    if (c->ev_big && c->ev_big[e]) cudaEventDestroy(c->ev_big[e]);
  }
  free(c->ev_fac);
  free(c->ev_big);
  if (c->stream) cudaStreamDestroy(c->stream);
  if (c->red_host) cudaFreeHost(c->red_host);
  if (c->hstatus) cudaFreeHost(c->hstatus);
}

extern "C" int harp_ctx_create(harp_ctx** out, int device, int max_N, int max_nrhs) {
  if (!out) return -1;
  *out = nullptr;
  int ndev = 0;
  HARP_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return -2;
  if (max_N < 1 || max_N > (1 << 17)) return -3;
  if (max_nrhs < 1 || max_nrhs > (1 << 20)) return -4;
  DeviceGuard g(device);
  if (!g.ok) return cuda_status(cudaGetLastError());

  harp_ctx* c = (harp_ctx*)calloc(1, sizeof(harp_ctx));
  if (!c) return HARP_E_NOMEM;
  c->device = device;
  c->max_N = max_N;
  c->max_nrhs = max_nrhs;
  c->lu_prec = -1;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->smem_optin = (size_t)optin;

  const size_t NN = (size_t)max_N * max_N;
  const size_t NR = (size_t)max_N * max_nrhs;
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (!ok) return;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      ok = false;
      cudaGetLastError();
    }
  };
  alloc((void**)&c->z64, NN * sizeof(double2));
  c->ld64 = max_N;
  alloc(&c->lu_re, NN * sizeof(double));
  alloc(&c->lu_im, NN * sizeof(double));
  c->ld_lu = max_N;
  alloc((void**)&c->ipiv, (size_t)max_N * sizeof(int));
  alloc((void**)&c->perm, (size_t)max_N * sizeof(int));
  const size_t ndinv = 2 * (((size_t)max_N + 63) / 64) * 4096;
  alloc(&c->dinv_re, ndinv * sizeof(double));
  alloc(&c->dinv_im, ndinv * sizeof(double));
  alloc(&c->w_re, NR * sizeof(double));
  alloc(&c->w_im, NR * sizeof(double));
  alloc((void**)&c->x_re, NR * sizeof(double));
  alloc((void**)&c->x_im, NR * sizeof(double));
  alloc((void**)&c->r_re, NR * sizeof(double));
  alloc((void**)&c->r_im, NR * sizeof(double));
  alloc((void**)&c->v_re, NR * sizeof(double));
  alloc((void**)&c->v_im, NR * sizeof(double));
  alloc(&c->t_re, NR * sizeof(double));
  alloc(&c->t_im, NR * sizeof(double));
  alloc((void**)&c->zff, 4 * NN * sizeof(float));
  alloc((void**)&c->xff, 4 * NR * sizeof(float));
  alloc((void**)&c->rowsum, (size_t)max_N * sizeof(float));
  alloc((void**)&c->rpart, 2 * 8 * NR * sizeof(double));
  const size_t kp = ((size_t)max_N + 31) / 32 * 32;
  c->tc_a_floats = 4 * (size_t)max_N * kp;
  c->tc_b_floats = 4 * (size_t)std::max(max_N, max_nrhs) * kp;
  alloc((void**)&c->tc_a, c->tc_a_floats * sizeof(float));
  alloc((void**)&c->tc_b, c->tc_b_floats * sizeof(float));
  const size_t nred = 16 + 2 * (size_t)max_nrhs;
  alloc((void**)&c->red, nred * sizeof(double));
  alloc((void**)&c->dstatus, 4 * sizeof(int));
  alloc((void**)&c->blk_uinv, 2 * 64 * 64 * sizeof(float));
  alloc((void**)&c->zbuf, NN * sizeof(float2));
  alloc((void**)&c->finv, 4 * NN * sizeof(float));
  alloc((void**)&c->finv_tmp, 2 * NN * sizeof(float));
  c->finv_split_floats = 4 * (size_t)max_N * kp;
  alloc((void**)&c->finv_split, 2 * c->finv_split_floats * sizeof(float));
  c->finv_split_mode = -1;
  if (ok) {
    // Tensor-core residual buffers: optional (the float-float residual
    // serves when they do not fit).
    const int S = oz_groups(max_N, oz_resid_bits(max_N), 1.0) - 1;
    const size_t kp = ((size_t)max_N + 63) / 64 * 64, np = ((size_t)max_N + 127) / 128 * 128;
    const size_t rp = ((size_t)max_nrhs + 63) / 64 * 64;
    const size_t per_pair = 2 * NR * sizeof(int);
    int slots = (int)std::min<size_t>(oz_pairs(S + 1), std::max<size_t>(S, (1536u << 20) / per_pair));
    bool oz_ok = true;
    auto oalloc = [&](void** p, size_t bytes) {
      if (!oz_ok) return;
      if (cudaMalloc(p, bytes) != cudaSuccess) {
        oz_ok = false;
        cudaGetLastError();
      }
    };
    oalloc(&c->oz_a, 2 * (size_t)S * np * kp * 2);
    oalloc(&c->oz_y, 2 * (size_t)S * rp * kp * 2);
    oalloc((void**)&c->oz_slots, (size_t)slots * per_pair);
    oalloc((void**)&c->oz_acc, 2 * NR * sizeof(double));
    oalloc((void**)&c->oz_rexp, (size_t)max_N * sizeof(int));
    oalloc((void**)&c->oz_cexp, (size_t)max_nrhs * sizeof(int));
    oalloc((void**)&c->oz_part, 32 * (size_t)max_N * sizeof(double));
    oalloc((void**)&c->oz_znorm, sizeof(double));
    if (oz_ok) {
      c->oz_max_slices = S;
      c->oz_slot_pairs = slots;
    } else {
      void* op[] = {c->oz_a,    c->oz_y,    c->oz_slots, c->oz_acc,
                    c->oz_rexp, c->oz_cexp, c->oz_part,  c->oz_znorm};
      for (void* p : op)
        if (p) cudaFree(p);
      c->oz_a = c->oz_y = nullptr;
      c->oz_slots = c->oz_rexp = c->oz_cexp = nullptr;
      c->oz_acc = c->oz_part = c->oz_znorm = nullptr;
    }
    c->oz_N = -1;
    c->z64_ticket = 0;
    c->oz_ticket = -1;
    c->residual_mode = HARP_RESIDUAL_SLICES;
  }
  c->panel_rows = 192;
  c->fill_chunk = 0;
  c->splitk_max = 8;
  if (ok && cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) ok = false;
  // stream priorities: the factorisation's panel chain first, then its far
  // trailing updates; the background Z64 fill and the inverse chains last
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
    cudaGetLastError();
    prio_least = prio_greatest = 0;
  }
  const int prio_mid = (prio_least + prio_greatest) / 2;
  if (ok && cudaStreamCreateWithPriority(&c->lu_stream, cudaStreamNonBlocking, prio_greatest) !=
                cudaSuccess)
    ok = false;
  if (ok && (cudaEventCreateWithFlags(&c->ev_lu_fork, cudaEventDisableTiming) != cudaSuccess ||
             cudaEventCreateWithFlags(&c->ev_lu_join, cudaEventDisableTiming) != cudaSuccess))
    ok = false;
  if (ok && cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_mid) != cudaSuccess)
    ok = false;
  if (ok && cudaStreamCreateWithPriority(&c->fill_stream, cudaStreamNonBlocking, prio_least) !=
                cudaSuccess)
    ok = false;
  if (ok && (cudaEventCreateWithFlags(&c->ev_fill_fork, cudaEventDisableTiming) != cudaSuccess ||
             cudaEventCreateWithFlags(&c->ev_z64, cudaEventDisableTiming) != cudaSuccess))
    ok = false;
  for (int q = 0; ok && q < 2; ++q)
    if (cudaStreamCreateWithPriority(&c->inv_stream[q], cudaStreamNonBlocking, prio_least) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_inv[q], cudaEventDisableTiming) != cudaSuccess)
      ok = false;
  c->finv_incremental = 0;
  c->inv_beside = 1;
  c->inv_policy = 2;
  c->fill_clusters = 0;
  c->fill64 = 2;
  c->adj_g = 1;
  c->fill64_now = 0;
  c->lu_fork = 1;
  if (ok) {
    c->n_events = max_N / 16 + 2;
    if (cudaMalloc((void**)&c->pmap, (size_t)c->n_events * kPmapInts * sizeof(int)) != cudaSuccess)
      ok = false;
    c->ev_fac = (cudaEvent_t*)calloc(c->n_events, sizeof(cudaEvent_t));
    c->ev_big = (cudaEvent_t*)calloc(c->n_events, sizeof(cudaEvent_t));
    if (!c->ev_fac || !c->ev_big) ok = false;
    for (int e = 0; ok && e < c->n_events; ++e)
      if (cudaEventCreateWithFlags(&c->ev_fac[e], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_big[e], cudaEventDisableTiming) != cudaSuccess)
        ok = false;
  }
  if (ok && cudaMallocHost((void**)&c->red_host, nred * sizeof(double)) != cudaSuccess) ok = false;
  if (ok && cudaMallocHost((void**)&c->hstatus, 4 * sizeof(int)) != cudaSuccess) ok = false;
  if (!ok) {
    cudaGetLastError();
    free_all(c);
    free(c);
    return HARP_E_NOMEM;
  }
  int init[4] = {0, INT_MAX, 0, 0};
  if (cudaMemcpy(c->dstatus, init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess) {
    int s = cuda_status(cudaGetLastError());
    free_all(c);
    free(c);
    return s;
  }
  *out = c;
  return HARP_OK;
}

extern "C" int harp_ctx_destroy(harp_ctx* c) {
  if (!c) return -1;
  {
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    free_all(c);
  }
  free(c);
  return HARP_OK;
}

extern "C" int harp_ctx_z64(harp_ctx* c, void** z64, int* ld) {
  if (!c) return -1;
  if (!z64) return -2;
  if (!ld) return -3;
  // the caller may write Z64 now: slices made from a fill's Z64 no longer
  // stand for it; a mixed fill may still be writing it on the fill stream
  c->oz_ticket = -1;
  {
    DeviceGuard g(c->device);
    if (c->ev_z64) HARP_CUDA(cudaEventSynchronize(c->ev_z64));
  }
  *z64 = c->z64;
  *ld = c->ld64;
  return HARP_OK;
}

namespace harp {
int take_pending_status(harp_ctx* c, const int* h, cudaStream_t st);
}

extern "C" int harp_ctx_sync(harp_ctx* c, void* stream) {
  if (!c) return -1;
  DeviceGuard g(c->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t st = (cudaStream_t)stream;
  // the background Z64 fill of a mixed harp_fill runs on the fill stream
  if (c->ev_z64) HARP_CUDA(cudaStreamWaitEvent(st, c->ev_z64, 0));
  HARP_CUDA(cudaMemcpyAsync(c->hstatus, c->dstatus, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
  HARP_CUDA(cudaStreamSynchronize(st));
  const int s = take_pending_status(c, c->hstatus, st);
  HARP_CUDA(cudaStreamSynchronize(st));
  return s;
}
