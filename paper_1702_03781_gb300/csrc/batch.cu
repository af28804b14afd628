// batch.cu -- scheduler for many independent fill + solve problems (the
// wideband case: one problem per frequency, uneven sizes).
//
// Each context is a worker: one host thread and the context's own stream.
// Workers take problems from a shared atomic counter, largest first (the
// caller's order), and run harp_fill + mbf_solve on their stream. Problems
// on different workers overlap on the GPU: the latency-bound parts of one
// (the pivoted panels, the host round trip of each refinement step) run
// while the others' fills, GEMMs and residuals occupy the remaining SMs.
// No CUDA call here allocates; the contexts own all workspace.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace harp;

namespace {

void run_worker(harp_ctx* ctx, harp_problem* probs, int n, std::atomic<int>* next, int prec,
                double tol, int max_iter, cudaEvent_t ev0, cudaEvent_t ev1, int* used) {
  *used = 0;
  for (;;) {
    const int i = next->fetch_add(1);
    if (i >= n) {
      if (*used) {
        DeviceGuard g(ctx->device);
        cudaEventRecord(ev1, ctx->stream);
      }
      return;
    }
    if (!*used) {
      DeviceGuard g(ctx->device);
      cudaEventRecord(ev0, ctx->stream);
      *used = 1;
    }
    harp_problem& p = probs[i];
    const int N = p.Na * p.Nm;
    int s;
    if (N > ctx->max_N || p.Na > ctx->max_nrhs) {
      s = HARP_E_UNSUPPORTED;
    } else {
      const int fill_prec = (prec == HARP_FP64) ? HARP_FP64 : HARP_MIXED_3XTF32;
      // FP64 fills straight into the context's FP64 matrix; the mixed modes
      // write Z64 there and the c64 copy into the worker's buffer.
      void* Z = (prec == HARP_FP64) ? (void*)ctx->z64 : (void*)ctx->zbuf;
      const int ldz = (prec == HARP_FP64) ? ctx->ld64 : N;
      s = harp_fill(ctx, p.Na, p.Nm, p.P, p.Q, p.pos, p.freq_hz, p.coef, p.self_blocks,
                    p.self_stride, Z, ldz, fill_prec, ctx->stream);
      if (s == HARP_OK)
        s = mbf_solve(ctx, N, Z, ldz, nullptr, N, p.Na, p.X, p.ldx, 'N', prec, tol, max_iter,
                      &p.iters, &p.resid, ctx->stream);
    }
    p.status = s;
  }
}

}  // namespace

extern "C" int harp_solve_batch(harp_ctx** ctxs, int n_ctx, harp_problem* probs, int n_probs,
                                int prec, double tol, int max_iter) {
  if (!ctxs || n_ctx < 1) return -1;
  for (int c = 0; c < n_ctx; ++c)
    if (!ctxs[c]) return -1;
  if (n_ctx > 64) return -2;
  if (!probs || n_probs < 0) return -3;
  if (prec != HARP_FP64 && prec != HARP_MIXED_3XTF32 && prec != HARP_MIXED_TF32) return -5;
  if (max_iter < 0) return -7;
  for (int i = 0; i < n_probs; ++i) {
    probs[i].status = HARP_E_STATE;
    probs[i].iters = 0;
    probs[i].resid = -1.0;
  }
  std::atomic<int> next{0};
  std::vector<std::thread> workers;
  workers.reserve(n_ctx);
  // Where each worker builds its factor inverses (HARP_OPT_INVERSES): by
  // default after its factorisation when several workers run (their
  // factorisations overlap one another and leave few idle SMs), beside it
  // for a single worker; the autotuner measures both.
  // With several workers each factorisation's chain also stays on its
  // worker's stream instead of the context's high-priority one: the workers'
  // chains would otherwise all outrank the other work (measured on the 64
  // wideband frequencies with 4 workers: 13.9 ms per frequency instead of
  // 13.4).
  // The background FP64 fill: digit products on the tensor cores by default
  // when several workers run (the whole GPU is busy anyway, and they take a
  // quarter of the float-float kernel's time: 64 wideband frequencies with 4
  // workers, 12.9 -> 11.3 ms per frequency).
  std::vector<int> beside(n_ctx), fork(n_ctx), f64(n_ctx);
  for (int c = 0; c < n_ctx; ++c) {
    beside[c] = ctxs[c]->inv_beside;
    fork[c] = ctxs[c]->lu_fork;
    f64[c] = ctxs[c]->fill64_now;
    const int pol = ctxs[c]->inv_policy;
    ctxs[c]->inv_beside = (pol == 1 || (pol == 2 && n_ctx == 1)) ? 1 : 0;
    if (n_ctx > 1) ctxs[c]->lu_fork = 0;
    const int fp = ctxs[c]->fill64;
    ctxs[c]->fill64_now = (fp == 1 || (fp == 2 && n_ctx > 1)) ? 1 : 0;
  }
  // device time of the batch: an event pair on every worker's stream
  std::vector<cudaEvent_t> ev(2 * n_ctx, nullptr);
  std::vector<int> used(n_ctx, 0);
  for (int c = 0; c < n_ctx; ++c) {
    DeviceGuard g(ctxs[c]->device);
    HARP_CUDA(cudaEventCreate(&ev[2 * c]));
    HARP_CUDA(cudaEventCreate(&ev[2 * c + 1]));
  }
  struct Destroy {
    std::vector<cudaEvent_t>* v;
    ~Destroy() {
      for (cudaEvent_t e : *v)
        if (e) cudaEventDestroy(e);
    }
  } destroy{&ev};
  for (int c = 0; c < n_ctx; ++c)
    workers.emplace_back(run_worker, ctxs[c], probs, n_probs, &next, prec, tol, max_iter,
                         ev[2 * c], ev[2 * c + 1], &used[c]);
  for (auto& w : workers) w.join();
  for (int c = 0; c < n_ctx; ++c) {
    ctxs[c]->inv_beside = beside[c];
    ctxs[c]->lu_fork = fork[c];
    ctxs[c]->fill64_now = f64[c];
  }
  for (int c = 0; c < n_ctx; ++c) {
    DeviceGuard g(ctxs[c]->device);
    HARP_CUDA(cudaStreamSynchronize(ctxs[c]->stream));
  }
  {
    // first start to last end, relative to any worker's start
    int ref = -1;
    for (int c = 0; c < n_ctx; ++c)
      if (used[c]) {
        ref = c;
        break;
      }
    double lo = 0.0, hi = 0.0;
    if (ref >= 0) {
      for (int c = 0; c < n_ctx; ++c) {
        if (!used[c]) continue;
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, ev[2 * ref], ev[2 * c]) != cudaSuccess ||
            cudaEventElapsedTime(&b, ev[2 * ref], ev[2 * c + 1]) != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        lo = std::min(lo, (double)a);
        hi = std::max(hi, (double)b);
      }
    }
    ctxs[0]->batch_device_us = 1e3 * (hi - lo);
  }
  int first_bad = HARP_OK;
  for (int i = 0; i < n_probs; ++i)
    if (probs[i].status != HARP_OK && first_bad == HARP_OK) first_bad = probs[i].status;
  return first_bad;
}
