// solve.cu -- mbf_solve: the direct solve of the reduced MBF system for every
// port excitation (Section II-B), in FP64, in FP32, or in mixed precision
// with FP64-accurate iterative refinement.
//
// Mixed refinement (classical iterative refinement, Wilkinson/Moler; the
// stopping rule follows LAPACK's zcgesv):
//   X0 = (LU32)^{-1} V, R0 = V - Z64 X0 (FP64-accurate: exact integer
//   slices on the tensor cores, ozaki.cu, or float-float, resid.cu)
//   repeat: stop when, for every column j, max_i |R_ij| <= tol ||Z64||_inf
//           max_i |X_ij| (|z| = |re| + |im|); D = (LU32)^{-1} R; X += D;
//           R -= Z64 D (an update accurate relative to |Z64||D|).
// The LU factors live in the context so that an adjoint solve (trans 'T')
// reuses them.
#include <cmath>
#include <algorithm>
#include <climits>

#include "dense.cuh"
#include "prof.cuh"
#include "ozaki.cuh"

namespace harp {

__global__ void set_int_kernel(int* p, int v) { *p = v; }

static int gemm_mode(int prec) {
  if (prec == HARP_MIXED_TF32) return GEMM_TC_TF32;
  if (prec == HARP_MIXED_3XTF32 || prec == HARP_FP32) return GEMM_TC_3XTF32;
  return GEMM_SIMT;
}
// Factorisations are shared between the modes that store the same type.
static int lu_class(int prec) { return prec == HARP_FP64 ? 0 : 1; }

// L^-1 as a view of the L slot of finv, which holds (L^-1)^T when the
// inverses were built beside the factorisation.
static CView<float> linv_view(const harp_ctx* c) {
  const size_t NN = (size_t)c->max_N * c->max_N;
  const CView<float> v = planes<float>(c->finv, c->finv + NN, c->max_N);
  return c->finv_incremental ? v.t() : v;
}

static bool use_slices(const harp_ctx* c) {
  return c->oz_a && c->residual_mode == HARP_RESIDUAL_SLICES;
}

// Copy the right-hand sides (or the port excitations) into FP64 planes.
static int load_rhs(harp_ctx* c, int N, int nrhs, const double* V, int ldv, double* re, double* im,
                    cudaStream_t st) {
  if (V)
    return interleaved_to_planes<double, double>(N, nrhs, V, ldv, re, im, c->max_N, st,
                                                 c->dstatus);
  return port_rhs_planes<double>(N, nrhs, N / nrhs, re, im, c->max_N, st);
}

bool profiling_active();

// The status a caller must see from the context's device words (host
// mirror h, read after a synchronisation): a bounded wait that gave up, then
// the pending flags of the last fill or of this solve's input check
// (coincident antennas, non-finite entries). Clears what it reports.
int take_pending_status(harp_ctx* c, const int* h, cudaStream_t st) {
  if (h[2]) {
    HARP_CUDA(cudaMemsetAsync(c->dstatus + 2, 0, sizeof(int), st));
    return HARP_E_TIMEOUT;
  }
  if (h[0] & (ST_COINCIDENT | ST_NONFINITE)) {
    HARP_CUDA(cudaMemsetAsync(c->dstatus, 0, sizeof(int), st));
    return (h[0] & ST_COINCIDENT) ? HARP_E_COINCIDENT : HARP_E_NONFINITE;
  }
  return HARP_OK;
}

// The first FP32 solve with the port right-hand sides V = E (column m has
// its unit entry in row m s): L^-1 P V is column c_m of L^-1, where
// perm[c_m] = m s, so that product is a gather (CTA m: find c_m, copy the
// column).
__global__ void port_linv_gather_kernel(int N, int s, const int* __restrict__ perm,
                                        CView<float> Li, float* wre, float* wim, long ldw) {
  __shared__ int col;
  const int m = blockIdx.x;
  if (threadIdx.x == 0) col = -1;
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    if (perm[i] == m * s) col = i;
  __syncthreads();
  const int c = col;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    wre[r + (size_t)m * ldw] = (c >= 0) ? Li.r(r, c) : 0.f;
    wim[r + (size_t)m * ldw] = (c >= 0) ? Li.m(r, c) : 0.f;
  }
}

// The FP32 triangular solves of one refinement call: the first runs
// directly; later ones replay a CUDA graph of the same sequence (captured
// once per context and (N, nrhs, mode, trans), on the context's own stream,
// and launched on the caller's stream). The graph reads the context's
// buffers, which never move, so it stays valid across factorisations.
static int solve32(harp_ctx* ctx, int N, int nrhs, char trans, int mode, bool first,
                   cudaStream_t st) {
  const long ldw = ctx->max_N;
  float* wre = (float*)ctx->w_re;
  float* wim = (float*)ctx->w_im;
  float* tre = (float*)ctx->t_re;
  float* tim = (float*)ctx->t_im;
  const int g = (trans == 'T') ? 1 : 0;
  const bool keyed = ctx->solve_graph[g] && ctx->solve_key[g][0] == N &&
                     ctx->solve_key[g][1] == nrhs && ctx->solve_key[g][2] == mode &&
                     ctx->solve_key[g][3] == ctx->finv_incremental;
  const size_t NN = (size_t)ctx->max_N * ctx->max_N;
  const float* fi = ctx->finv;
  const bool pre = (ctx->finv_split_mode == mode);
  const float* lsp = pre ? ctx->finv_split : nullptr;
  const float* usp = pre ? ctx->finv_split + ctx->finv_split_floats : nullptr;
  const CView<float> Li = linv_view(ctx), Ui = planes<float>(const_cast<float*>(fi) + 2 * NN,
                                                             const_cast<float*>(fi) + 3 * NN,
                                                             ctx->max_N);
  auto run = [&](cudaStream_t s) {
    return lu_solve_inv<float>(N, nrhs, Li, Ui, ctx->perm, wre, wim, ldw, tre, tim, trans, mode,
                               s, lsp, usp);
  };
  if (profiling_active() || (first && !keyed)) return run(st);
  if (!keyed) {
    if (ctx->solve_graph[g]) {
      cudaGraphExecDestroy(ctx->solve_graph[g]);
      ctx->solve_graph[g] = nullptr;
    }
    cudaGraph_t graph = nullptr;
    HARP_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const int s = run(ctx->stream);
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (s != HARP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    HARP_CUDA(e);
    const cudaError_t ei = cudaGraphInstantiate(&ctx->solve_graph[g], graph, 0);
    cudaGraphDestroy(graph);
    HARP_CUDA(ei);
    ctx->solve_key[g][0] = N;
    ctx->solve_key[g][1] = nrhs;
    ctx->solve_key[g][2] = mode;
    ctx->solve_key[g][3] = ctx->finv_incremental;
  }
  HARP_CUDA(cudaGraphLaunch(ctx->solve_graph[g], st));
  return HARP_OK;
}

// One of the refinement's per-correction segments (body(s) enqueues it on
// s): the first time a key is seen it runs directly; the second time it is
// captured on the context's stream and instantiated; afterwards the graph
// is replayed on st. Bodies read and write only the context's buffers,
// which never move, so a graph stays valid for its key. Nothing is captured
// while the profiler records launches.
template <typename F>
static int replay_segment(harp_ctx* ctx, int slot, const int* key, F&& body, cudaStream_t st) {
  if (profiling_active()) return body(st);
  bool same = ctx->ref_seen[slot] != 0;
  for (int q = 0; q < 6 && same; ++q) same = (ctx->ref_key[slot][q] == key[q]);
  if (!same) {
    if (ctx->ref_graph[slot]) {
      cudaGraphExecDestroy(ctx->ref_graph[slot]);
      ctx->ref_graph[slot] = nullptr;
    }
    for (int q = 0; q < 6; ++q) ctx->ref_key[slot][q] = key[q];
    ctx->ref_seen[slot] = 1;
    return body(st);
  }
  if (!ctx->ref_graph[slot]) {
    cudaGraph_t graph = nullptr;
    HARP_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const int s = body(ctx->stream);
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (s != HARP_OK) {
      if (graph) cudaGraphDestroy(graph);
      ctx->ref_seen[slot] = 0;
      return s;
    }
    HARP_CUDA(e);
    const cudaError_t ei = cudaGraphInstantiate(&ctx->ref_graph[slot], graph, 0);
    cudaGraphDestroy(graph);
    HARP_CUDA(ei);
  }
  HARP_CUDA(cudaGraphLaunch(ctx->ref_graph[slot], st));
  return HARP_OK;
}

// The FP32 triangular solves of one correction without the solve graph
// (for capture inside a segment).
static int solve32_direct(harp_ctx* ctx, int N, int nrhs, char trans, int mode, cudaStream_t st) {
  const long ldw = ctx->max_N;
  const size_t NN = (size_t)ctx->max_N * ctx->max_N;
  const float* fi = ctx->finv;
  const bool pre = (ctx->finv_split_mode == mode);
  const float* lsp = pre ? ctx->finv_split : nullptr;
  const float* usp = pre ? ctx->finv_split + ctx->finv_split_floats : nullptr;
  const CView<float> Li = linv_view(ctx), Ui = planes<float>(const_cast<float*>(fi) + 2 * NN,
                                                             const_cast<float*>(fi) + 3 * NN,
                                                             ctx->max_N);
  return lu_solve_inv<float>(N, nrhs, Li, Ui, ctx->perm, (float*)ctx->w_re, (float*)ctx->w_im,
                             ldw, (float*)ctx->t_re, (float*)ctx->t_im, trans, mode, st, lsp, usp);
}

}  // namespace harp

using namespace harp;

// Factorise Z (c64, or c128 when z_c128; trans 'N' solves) into the
// context: PZ = LU with the context's pivot rule (FP32 modes) or partial
// pivoting (FP64), the diagonal-block inverses and, in the FP32 modes, the
// explicit factor inverses. Returns +i on an exactly zero pivot in column i,
// or the pending status (coincident antennas, non-finite entries).
static int factorise(harp_ctx* ctx, int N, const void* Z, int ldz, bool z_c128, int prec,
                     int mode, cudaStream_t st) {
  ctx->lu_valid = 0;
  {
    set_int_kernel<<<1, 1, 0, st>>>(ctx->dstatus + 1, INT_MAX);
    HARP_LAUNCHED();
    if (lu_class(prec) == 0) {
      double* re = (double*)ctx->lu_re;
      double* im = (double*)ctx->lu_im;
      HARP_TRY(interleaved_to_planes<double, double>(N, N, (const double*)Z, ldz, re, im,
                                                     ctx->ld_lu, st, ctx->dstatus));
      HARP_TRY(lu_factor<double>(ctx, N, re, im, ctx->ld_lu, ctx->ipiv, ctx->perm,
                                 ctx->dstatus + 1, mode, st));
      const size_t nb = (size_t)((N + 63) / 64) * 4096;
      double* dr = (double*)ctx->dinv_re;
      double* di = (double*)ctx->dinv_im;
      HARP_TRY(diag_inverses<double>(N, planes<double>(re, im, ctx->ld_lu), dr, di, dr + nb,
                                     di + nb, st));
    } else {
      float* re = (float*)ctx->lu_re;
      float* im = (float*)ctx->lu_im;
      if (z_c128)  // the FP32 copy of an FP64 matrix (the context's Z64)
        HARP_TRY(interleaved_to_planes<double, float>(N, N, (const double*)Z, ldz, re, im,
                                                      ctx->ld_lu, st, ctx->dstatus));
      else
        HARP_TRY(interleaved_to_planes<float, float>(N, N, (const float*)Z, ldz, re, im,
                                                     ctx->ld_lu, st, ctx->dstatus));
      ctx->finv_incremental = 0;
      HARP_TRY(lu_factor<float>(ctx, N, re, im, ctx->ld_lu, ctx->ipiv, ctx->perm,
                                ctx->dstatus + 1, mode, st));
      const size_t nb = (size_t)((N + 63) / 64) * 4096;
      float* dr = (float*)ctx->dinv_re;
      float* di = (float*)ctx->dinv_im;
      HARP_TRY(diag_inverses<float>(N, planes<float>(re, im, ctx->ld_lu), dr, di, dr + nb, di + nb,
                                    st));
      const size_t NN = (size_t)ctx->max_N * ctx->max_N;
      float* fi = ctx->finv;
      ctx->finv_split_mode = -1;
      if (ctx->finv_incremental) {
        // built beside the factorisation: U^-1 with its split, and (L^-1)^T,
        // whose transpose is split here
        if (tc_split_operand(N, N, planes<float>(fi, fi + NN, ctx->max_N).t(), ctx->finv_split,
                             ctx->finv_split_floats, mode, st) == HARP_OK)
          ctx->finv_split_mode = mode;
      } else {
        HARP_TRY(factor_inverses(N, planes<float>(re, im, ctx->ld_lu), dr, di, fi, fi + NN,
                                 fi + 2 * NN, fi + 3 * NN, ctx->max_N, ctx->finv_tmp,
                                 ctx->finv_tmp + NN, mode, st, ctx->side, ctx->ev_fac[0],
                                 ctx->ev_big[0]));
      }
      // the inverses as tensor-core operands, once for all forward solves
      if (mode != GEMM_SIMT && !ctx->finv_incremental) {
        const size_t fs = ctx->finv_split_floats;
        const long ldi = ctx->max_N;
        if (tc_split_operand(N, N, planes<float>(fi, fi + NN, ldi), ctx->finv_split, fs, mode,
                             st) == HARP_OK &&
            tc_split_operand(N, N, planes<float>(fi + 2 * NN, fi + 3 * NN, ldi),
                             ctx->finv_split + fs, fs, mode, st) == HARP_OK)
          ctx->finv_split_mode = mode;
      }
    }
    HARP_CUDA(cudaMemcpyAsync(ctx->hstatus, ctx->dstatus, 3 * sizeof(int),
                              cudaMemcpyDeviceToHost, st));
    HARP_CUDA(cudaStreamSynchronize(st));
    HARP_TRY(take_pending_status(ctx, ctx->hstatus, st));
    if (ctx->hstatus[1] != INT_MAX) return ctx->hstatus[1];
    ctx->lu_N = N;
    ctx->lu_prec = lu_class(prec);
    ctx->lu_pivot = (lu_class(prec) == 0) ? HARP_PIVOT_PARTIAL : ctx->pivot_mode;
    ctx->lu_valid = 1;
  }
  return HARP_OK;
}


// Solve with the cached factors (FP64: substitution; FP32: the explicit
// inverses; mixed: refinement against Z64). With stall_exit the refinement
// stops as soon as a correction contracts the backward error by less than
// half (the factors of restricted pivoting are then not worth refining) and
// *stalled is set.
static int solve_factored(harp_ctx* ctx, int N, const double* V, int ldv, int nrhs, double* X,
                          int ldx, bool tr, int prec, int mode, double tol, int max_iter,
                          int* iters_out, double* resid_out, cudaStream_t st, bool stall_exit,
                          bool* stalled) {
  const long ldw = ctx->max_N;
  *stalled = false;
  if (iters_out) *iters_out = 0;
  if (resid_out) *resid_out = -1.0;
  // ---- FP64: direct solve
  if (prec == HARP_FP64) {
    double* wre = (double*)ctx->w_re;
    double* wim = (double*)ctx->w_im;
    HARP_TRY(load_rhs(ctx, N, nrhs, V, ldv, wre, wim, st));
    HARP_TRY(lu_solve<double>(N, nrhs, (double*)ctx->lu_re, (double*)ctx->lu_im, ctx->ld_lu,
                              ctx->perm, wre, wim, ldw, (double*)ctx->t_re, (double*)ctx->t_im,
                              tr ? 'T' : 'N', (const double*)ctx->dinv_re,
                              (const double*)ctx->dinv_im, mode, st));
    HARP_TRY(planes_to_interleaved(N, nrhs, wre, wim, ldw, X, ldx, st));
    return HARP_OK;
  }

  float* wre = (float*)ctx->w_re;
  float* wim = (float*)ctx->w_im;
  float* tre = (float*)ctx->t_re;
  float* tim = (float*)ctx->t_im;
  HARP_TRY(load_rhs(ctx, N, nrhs, V, ldv, ctx->v_re, ctx->v_im, st));
  const size_t NNi = (size_t)ctx->max_N * ctx->max_N;
  if (!V && !tr && N % nrhs == 0 && ctx->finv_split_mode == mode) {
    // port right-hand sides: the L^-1 product is a column gather, then U^-1
    {
      ProfScope ps(HARP_K_OTHER, 0.0, st);
      port_linv_gather_kernel<<<nrhs, 256, 0, st>>>(N, N / nrhs, ctx->perm, linv_view(ctx), wre,
                                                    wim, ldw);
      HARP_LAUNCHED();
    }
    int su = cgemm_tc_f32_asplit(N, nrhs, N, 1.f, ctx->finv_split + ctx->finv_split_floats,
                                 planes<float>(wre, wim, ldw), 0.f, planes<float>(tre, tim, ldw),
                                 mode, st, 0, 0, true, 1);  // U^-1 upper triangular
    if (su == HARP_E_UNSUPPORTED)  // shapes the tensor-core product does not take
      su = cgemm<float>(N, nrhs, N, 1.f,
                        planes<float>(ctx->finv + 2 * NNi, ctx->finv + 3 * NNi, ctx->max_N),
                        planes<float>(wre, wim, ldw), 0.f, planes<float>(tre, tim, ldw), mode, st);
    HARP_TRY(su);
    HARP_TRY(planes_to_planes<float, float>(N, nrhs, tre, tim, ldw, wre, wim, ldw, st));
  } else {
    HARP_TRY(planes_to_planes<double, float>(N, nrhs, ctx->v_re, ctx->v_im, ldw, wre, wim, ldw, st));
    HARP_TRY(solve32(ctx, N, nrhs, tr ? 'T' : 'N', mode, true, st));
  }
  HARP_TRY(planes_to_planes<float, double>(N, nrhs, wre, wim, ldw, ctx->x_re, ctx->x_im, ldw, st));

  // ---- FP32: no refinement
  if (prec == HARP_FP32) {
    HARP_TRY(planes_to_interleaved(N, nrhs, ctx->x_re, ctx->x_im, ldw, X, ldx, st));
    HARP_CUDA(cudaMemcpyAsync(ctx->hstatus, ctx->dstatus, 3 * sizeof(int),
                              cudaMemcpyDeviceToHost, st));
    HARP_CUDA(cudaStreamSynchronize(st));
    return take_pending_status(ctx, ctx->hstatus, st);
  }

  // ---- mixed: FP64-accurate residual against the context's FP64 matrix,
  // by exact integer slices on the tensor cores (ozaki.cu) or in
  // float-float on the FP32 pipe (resid.cu).
  const size_t NN = (size_t)ctx->max_N * ctx->max_N;
  const size_t NR = (size_t)ctx->max_N * ctx->max_nrhs;
  float* zhl[4] = {ctx->zff, ctx->zff + NN, ctx->zff + 2 * NN, ctx->zff + 3 * NN};
  float* xhl[4] = {ctx->xff, ctx->xff + NR, ctx->xff + 2 * NR, ctx->xff + 3 * NR};
  // element (i, k) of op(Z): (1, ld) for Z, (ld, 1) for Z^T
  const long ars = tr ? ldw : 1, acs = tr ? 1 : ldw;
  const bool slices = use_slices(ctx);
  // Z64 may still be filling on the context's fill stream (mixed harp_fill)
  HARP_CUDA(cudaStreamWaitEvent(st, ctx->ev_z64, 0));
  if (slices) {
    // the slices of the last mixed fill's Z64, when it made them for trans
    // 'N' (the wait above covers them), else made here
    if (!tr && ctx->oz_ticket == ctx->z64_ticket && ctx->oz_ticket > 0 && ctx->oz_N == N)
      HARP_CUDA(cudaMemcpyAsync(ctx->red + 0, ctx->oz_znorm, sizeof(double),
                                cudaMemcpyDeviceToDevice, st));
    else
      HARP_TRY(oz_prepare(ctx, N, ctx->z64, ctx->ld64, tr, ctx->red + 0, st));
  } else {
    HARP_TRY(split_c128(N, N, (const double*)ctx->z64, ctx->ld64, zhl, ldw, st));
    HARP_TRY(norm_inf_planes_f32(N, N, zhl[0], zhl[1], ars, acs, ctx->rowsum, ctx->red + 0, st));
  }
  if (tol <= 0.0) tol = std::sqrt((double)N) * std::ldexp(1.0, -53);
  double* colmax_r = ctx->red + 16;
  double* colmax_x = ctx->red + 16 + nrhs;
  // R_0 = V - Z X_0 with the three-float accumulator (X_0 is the FP32
  // solution, exact as hi with lo = 0). Later residuals are updated,
  // R_{k+1} = R_k - Z D_k, whose error only has to be small against
  // |Z||D_k|: with rho = max_j max|D_kj| / max|X_j| <= kDot2Rho the
  // double-float accumulator (~1e-14 of sum |z||d|) keeps the update error
  // below 2^-53 |Z||X|, otherwise the three-float one is used.
  // With slices the update forms only the digit groups that the size of D
  // against X leaves above the FP64 rounding of the residual.
  constexpr double kDot2Rho = 1e-2;
  if (slices) {
    HARP_TRY(oz_residual(ctx, N, nrhs, wre, wim, ldw, ctx->v_re, ctx->v_im, ctx->r_re, ctx->r_im,
                         ldw, 1.0, HARP_K_RESIDUAL, st));
  } else {
    HARP_TRY(split_f32_planes(N, nrhs, wre, wim, ldw, xhl, st));
    HARP_TRY(residual_ff(N, nrhs, zhl, ars, acs, xhl, ldw, ctx->v_re, ctx->v_im, ctx->r_re,
                         ctx->r_im, ldw, ctx->rpart, ctx->rpart + 8 * NR, 8, ctx->num_sms, st,
                         true));
  }
  // X (the caller's buffer) receives every iterate that improves on the
  // best backward error so far, so that it holds the best iterate when the
  // tolerance is not met; a converged iterate is written after the loop.
  double bwd = INFINITY, best = INFINITY;
  int it = 0;
  bool converged = false;
  // the stopping test's inputs for the first residual; after a correction
  // the update segment forms them (X's column maxima are then those formed
  // for the size of the correction: X has not changed since)
  HARP_TRY(colmax_cabs1(N, nrhs, ctx->r_re, ctx->r_im, ldw, colmax_r, st));
  HARP_TRY(colmax_cabs1(N, nrhs, ctx->x_re, ctx->x_im, ldw, colmax_x, st));
  HARP_CUDA(cudaMemcpyAsync(ctx->red_host, ctx->red, sizeof(double) * (16 + 2 * (size_t)nrhs),
                            cudaMemcpyDeviceToHost, st));
  for (;;) {
    HARP_CUDA(cudaStreamSynchronize(st));
    const double* h = ctx->red_host;
    const double znorm = h[0];
    bwd = 0.0;
    for (int j = 0; j < nrhs; ++j) {
      const double rj = h[16 + j], xj = h[16 + nrhs + j];
      const double bj = (rj == 0.0) ? 0.0 : rj / (znorm * xj);
      if (!(bj == bj)) {  // reported here: the pending flag of the input check goes with it
        HARP_CUDA(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), st));
        HARP_CUDA(cudaStreamSynchronize(st));
        return HARP_E_NONFINITE;
      }
      bwd = std::max(bwd, bj);
    }
    if (bwd <= tol) {
      converged = true;
      break;
    }
    const double prev = best;
    if (bwd < best || it == 0) {
      best = bwd;
      HARP_TRY(planes_to_interleaved(N, nrhs, ctx->x_re, ctx->x_im, ldw, X, ldx, st));
    }
    if (stall_exit && it > 0 && !(bwd <= 0.5 * prev)) {
      *stalled = true;
      break;
    }
    if (it >= max_iter) break;
    // correction segment: D = (LU32)^{-1} R; X += D; the size of the
    // correction against the iterate (which picks the update's digit groups
    // or accumulator) to the host
    {
      const char tch = tr ? 'T' : 'N';
      const int key[6] = {N, nrhs, mode, tr ? 1 : 0, ctx->finv_split_mode == mode ? 1 : 0,
                          ctx->finv_incremental};
      HARP_TRY(replay_segment(ctx, tr ? 1 : 0, key, [&](cudaStream_t s) {
        HARP_TRY(planes_to_planes<double, float>(N, nrhs, ctx->r_re, ctx->r_im, ldw, wre, wim, ldw,
                                                 s));
        HARP_TRY(solve32_direct(ctx, N, nrhs, tch, mode, s));
        HARP_TRY(add_planes<float>(N, nrhs, ctx->x_re, ctx->x_im, ldw, wre, wim, ldw, s));
        HARP_TRY(colmax_cabs1_f32(N, nrhs, wre, wim, ldw, colmax_r, s));
        HARP_TRY(colmax_cabs1(N, nrhs, ctx->x_re, ctx->x_im, ldw, colmax_x, s));
        HARP_CUDA(cudaMemcpyAsync(ctx->red_host + 16, colmax_r, sizeof(double) * 2 * (size_t)nrhs,
                                  cudaMemcpyDeviceToHost, s));
        return (int)HARP_OK;
      }, st));
    }
    HARP_CUDA(cudaStreamSynchronize(st));
    double rho = 0.0;
    for (int j = 0; j < nrhs; ++j) {
      const double dj = h[16 + j], xj = h[16 + nrhs + j];
      rho = std::max(rho, (dj == 0.0) ? 0.0 : dj / xj);
    }
    // update segment: R -= Z D, then the stopping test's inputs to the host
    {
      const int variant = slices ? std::min(oz_groups(N, ctx->oz_bits, rho), ctx->oz_slices + 1)
                                 : (rho <= kDot2Rho ? 14 : 15);
      const int slot = 2 + std::max(0, std::min(variant, 15));
      const int key[6] = {N, nrhs, variant, slices ? 1 : 0, tr ? 1 : 0, 0};
      HARP_TRY(replay_segment(ctx, slot, key, [&](cudaStream_t s) {
        if (slices) {
          HARP_TRY(oz_residual(ctx, N, nrhs, wre, wim, ldw, ctx->r_re, ctx->r_im, ctx->r_re,
                               ctx->r_im, ldw, rho, HARP_K_RESID_UPDATE, s));
        } else {
          HARP_TRY(split_f32_planes(N, nrhs, wre, wim, ldw, xhl, s));
          HARP_TRY(residual_ff(N, nrhs, zhl, ars, acs, xhl, ldw, ctx->r_re, ctx->r_im, ctx->r_re,
                               ctx->r_im, ldw, ctx->rpart, ctx->rpart + 8 * NR, 8, ctx->num_sms,
                               s, !(rho <= kDot2Rho)));
        }
        HARP_TRY(colmax_cabs1(N, nrhs, ctx->r_re, ctx->r_im, ldw, colmax_r, s));
        HARP_CUDA(cudaMemcpyAsync(ctx->red_host, ctx->red, sizeof(double) * (16 + 2 * (size_t)nrhs),
                                  cudaMemcpyDeviceToHost, s));
        return (int)HARP_OK;
      }, st));
    }
    ++it;
  }
  if (converged) HARP_TRY(planes_to_interleaved(N, nrhs, ctx->x_re, ctx->x_im, ldw, X, ldx, st));
  if (iters_out) *iters_out = it;
  if (resid_out) *resid_out = converged ? bwd : best;
  HARP_CUDA(cudaMemcpyAsync(ctx->hstatus, ctx->dstatus, 3 * sizeof(int),
                            cudaMemcpyDeviceToHost, st));
  HARP_CUDA(cudaStreamSynchronize(st));
  HARP_TRY(take_pending_status(ctx, ctx->hstatus, st));
  return converged ? HARP_OK : HARP_E_NOCONV;
}

extern "C" int mbf_solve(harp_ctx* ctx, int N, const void* Z, int ldz, const double* V, int ldv,
                         int nrhs, double* X, int ldx, char trans, int prec, double tol,
                         int max_iter, int* iters_out, double* resid_out, void* stream) {
  if (!ctx) return -1;
  if (N < 1 || N > ctx->max_N) return -2;
  const bool tr = (trans == 'T' || trans == 't');
  if (!tr && trans != 'N' && trans != 'n') return -10;
  if (!tr && !Z) return -3;
  if (!tr && ldz < N) return -4;
  if (V && ldv < N) return -6;
  if (nrhs < 1 || nrhs > ctx->max_nrhs || nrhs > 65535) return -7;
  if (!V && (N % nrhs) != 0) return -5;
  if (!X) return -8;
  if (ldx < N) return -9;
  if (prec != HARP_FP64 && prec != HARP_MIXED_3XTF32 && prec != HARP_MIXED_TF32 && prec != HARP_FP32)
    return -11;
  if (!(tol == tol)) return -12;
  if (max_iter < 0) return -13;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t st = (cudaStream_t)stream;
  const int mode = gemm_mode(prec);
  if (iters_out) *iters_out = 0;
  if (resid_out) *resid_out = -1.0;

  // Tensor-core GEMM scratch for this call; cleared timeout flag.
  tc_set_workspace(ctx->tc_a, ctx->tc_a_floats, ctx->tc_b, ctx->tc_b_floats, ctx->dstatus + 2);
  tc_set_splitk_max(ctx->splitk_max);
  HARP_CUDA(cudaMemsetAsync(ctx->dstatus + 2, 0, sizeof(int), st));
  struct Unset {
    ~Unset() {
      tc_set_workspace(nullptr, 0, nullptr, 0, nullptr);
      tc_set_splitk_max(8);
    }
  } unset_on_return;

  // Pivoting restricted to the diagonal blocks gives factors only the
  // refinement can vouch for: the FP32 mode (no refinement) uses partial
  // pivoting instead, and a factorisation that meets a zero pivot or whose
  // refinement stalls is redone with partial pivoting.
  const int rule = ctx->pivot_mode;
  struct Restore {
    harp_ctx* c;
    int rule;
    ~Restore() { c->pivot_mode = rule; }
  } restore{ctx, rule};
  const bool refined = (prec == HARP_MIXED_3XTF32 || prec == HARP_MIXED_TF32);
  if (rule == HARP_PIVOT_BLOCK && !refined) ctx->pivot_mode = HARP_PIVOT_PARTIAL;
  auto fall_back = [&]() {
    ++ctx->pivot_fallbacks;
    ctx->pivot_mode = HARP_PIVOT_PARTIAL;
  };
  if (!tr) {
    int s = factorise(ctx, N, Z, ldz, false, prec, mode, st);
    if (s >= 1 && s <= N && ctx->pivot_mode == HARP_PIVOT_BLOCK) {
      fall_back();
      s = factorise(ctx, N, Z, ldz, false, prec, mode, st);
    }
    if (s != HARP_OK) return s;
  } else if (!ctx->lu_valid || ctx->lu_N != N || ctx->lu_prec != lu_class(prec)) {
    return HARP_E_STATE;
  }
  bool stalled = false;
  const bool check = (ctx->lu_pivot == HARP_PIVOT_BLOCK);
  int s = solve_factored(ctx, N, V, ldv, nrhs, X, ldx, tr, prec, mode, tol, max_iter, iters_out,
                         resid_out, st, check, &stalled);
  if (check && stalled) {
    // refactor with partial pivoting (for 'T' from the context's Z64, the
    // matrix the refinement converges to) and solve again
    fall_back();
    if (!tr) {
      s = factorise(ctx, N, Z, ldz, false, prec, mode, st);
    } else {
      HARP_CUDA(cudaStreamWaitEvent(st, ctx->ev_z64, 0));
      s = factorise(ctx, N, ctx->z64, ctx->ld64, true, prec, mode, st);
    }
    if (s != HARP_OK) return s;
    s = solve_factored(ctx, N, V, ldv, nrhs, X, ldx, tr, prec, mode, tol, max_iter, iters_out,
                       resid_out, st, false, &stalled);
  }
  return s;
}

extern "C" int harp_ctx_set_option(harp_ctx* ctx, int option, int value) {
  if (!ctx) return -1;
  if (option == HARP_OPT_PANEL_ROWS) {
    if (value < 32 || value > 384) return -3;
    ctx->panel_rows = value;
    return HARP_OK;
  }
  if (option == HARP_OPT_FILL_CHUNK) {
    if (value < 0) return -3;
    ctx->fill_chunk = value;
    return HARP_OK;
  }
  if (option == HARP_OPT_ADJOINT_G) {
    if (value < 0 || value > 1) return -3;
    ctx->adj_g = value;
    return HARP_OK;
  }
  if (option == HARP_OPT_FILL64) {
    if (value < 0 || value > 2) return -3;
    ctx->fill64 = value;
    ctx->fill64_now = (value == 1) ? 1 : 0;
    return HARP_OK;
  }
  if (option == HARP_OPT_FILL_CLUSTERS) {
    if (value < 0 || value > 64) return -3;
    ctx->fill_clusters = value;
    return HARP_OK;
  }
  if (option == HARP_OPT_INVERSES) {
    if (value < 0 || value > 2) return -3;
    ctx->inv_policy = value;
    ctx->inv_beside = (value != 0) ? 1 : 0;
    return HARP_OK;
  }
  if (option == HARP_OPT_SPLITK_MAX) {
    if (value < 1 || value > 8) return -3;
    ctx->splitk_max = value;
    return HARP_OK;
  }
  if (option == HARP_OPT_PIVOT) {
    if (value != HARP_PIVOT_PARTIAL && value != HARP_PIVOT_TOURNAMENT &&
        value != HARP_PIVOT_BLOCK)
      return -3;
    ctx->pivot_mode = value;
    return HARP_OK;
  }
  if (option != HARP_OPT_RESIDUAL) return -2;
  if (value != HARP_RESIDUAL_SLICES && value != HARP_RESIDUAL_FF) return -3;
  if (value == HARP_RESIDUAL_SLICES && !ctx->oz_a) return HARP_E_UNSUPPORTED;
  ctx->residual_mode = value;
  return HARP_OK;
}

extern "C" int harp_ctx_get_option(harp_ctx* ctx, int option, int* value) {
  if (!ctx) return -1;
  if (!value) return -3;
  switch (option) {
    case HARP_OPT_PANEL_ROWS: *value = ctx->panel_rows; return HARP_OK;
    case HARP_OPT_FILL_CHUNK: *value = ctx->fill_chunk; return HARP_OK;
    case HARP_OPT_SPLITK_MAX: *value = ctx->splitk_max; return HARP_OK;
    case HARP_OPT_INVERSES: *value = ctx->inv_policy; return HARP_OK;
    case HARP_OPT_FILL_CLUSTERS: *value = ctx->fill_clusters; return HARP_OK;
    case HARP_OPT_FILL64: *value = ctx->fill64; return HARP_OK;
    case HARP_OPT_ADJOINT_G: *value = ctx->adj_g; return HARP_OK;
    case HARP_OPT_TC_FALLBACKS:
      *value = (int)std::min<long>(tc_fallbacks(), 2147483647L);
      return HARP_OK;
    case HARP_OPT_BATCH_DEVICE_US:
      *value = (int)std::min(ctx->batch_device_us + 0.5, 2147483647.0);
      return HARP_OK;
    default: break;
  }
  if (option != HARP_OPT_RESIDUAL && option != HARP_OPT_PIVOT &&
      option != HARP_OPT_PIVOT_FALLBACKS)
    return -2;
  if (option == HARP_OPT_PIVOT)
    *value = ctx->pivot_mode;
  else if (option == HARP_OPT_PIVOT_FALLBACKS)
    *value = (int)std::min<long long>(ctx->pivot_fallbacks, INT_MAX);
  else
    *value = use_slices(ctx) ? HARP_RESIDUAL_SLICES : HARP_RESIDUAL_FF;
  return HARP_OK;
}

extern "C" int harp_residual(harp_ctx* ctx, int N, const double* Z, int ldz, const float* X,
                             int ldx, const double* V, int ldv, int nrhs, double* R, int ldr,
                             char trans, void* stream) {
  if (!ctx) return -1;
  if (N < 1 || N > ctx->max_N) return -2;
  if (!Z) return -3;
  if (ldz < N) return -4;
  if (!X) return -5;
  if (ldx < N) return -6;
  if (!V) return -7;
  if (ldv < N) return -8;
  if (nrhs < 1 || nrhs > ctx->max_nrhs || nrhs > 65535) return -9;
  if (!R) return -10;
  if (ldr < N) return -11;
  const bool tr = (trans == 'T' || trans == 't');
  if (!tr && trans != 'N' && trans != 'n') return -12;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t st = (cudaStream_t)stream;
  const long ldw = ctx->max_N;
  const size_t NN = (size_t)ctx->max_N * ctx->max_N;
  const size_t NR = (size_t)ctx->max_N * ctx->max_nrhs;
  float* wre = (float*)ctx->w_re;
  float* wim = (float*)ctx->w_im;
  HARP_CUDA(cudaMemsetAsync(ctx->dstatus + 2, 0, sizeof(int), st));
  HARP_TRY(interleaved_to_planes<float, float>(N, nrhs, X, ldx, wre, wim, ldw, st));
  HARP_TRY(interleaved_to_planes<double, double>(N, nrhs, V, ldv, ctx->v_re, ctx->v_im, ldw, st));
  if (use_slices(ctx)) {
    HARP_TRY(oz_prepare(ctx, N, (const double2*)Z, ldz, tr, ctx->red + 0, st));
    HARP_TRY(oz_residual(ctx, N, nrhs, wre, wim, ldw, ctx->v_re, ctx->v_im, ctx->r_re, ctx->r_im,
                         ldw, 1.0, HARP_K_RESIDUAL, st));
  } else {
    float* zhl[4] = {ctx->zff, ctx->zff + NN, ctx->zff + 2 * NN, ctx->zff + 3 * NN};
    float* xhl[4] = {ctx->xff, ctx->xff + NR, ctx->xff + 2 * NR, ctx->xff + 3 * NR};
    HARP_TRY(split_c128(N, N, Z, ldz, zhl, ldw, st));
    HARP_TRY(split_f32_planes(N, nrhs, wre, wim, ldw, xhl, st));
    const long ars = tr ? ldw : 1, acs = tr ? 1 : ldw;
    HARP_TRY(residual_ff(N, nrhs, zhl, ars, acs, xhl, ldw, ctx->v_re, ctx->v_im, ctx->r_re,
                         ctx->r_im, ldw, ctx->rpart, ctx->rpart + 8 * NR, 8, ctx->num_sms, st,
                         true));
  }
  HARP_TRY(planes_to_interleaved(N, nrhs, ctx->r_re, ctx->r_im, ldw, R, ldr, st));
  HARP_CUDA(cudaMemcpyAsync(ctx->hstatus + 2, ctx->dstatus + 2, sizeof(int),
                            cudaMemcpyDeviceToHost, st));
  HARP_CUDA(cudaStreamSynchronize(st));
  return ctx->hstatus[2] ? HARP_E_TIMEOUT : HARP_OK;
}
