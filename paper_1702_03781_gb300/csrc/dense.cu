// dense.cu -- dense complex linear algebra for the MBF solve: LU with partial
// pivoting (the direct solve of Section II-B), triangular solves for every
// port excitation, a CUDA-core complex GEMM, conversions and norms.
//
// Storage inside the solver is split planes (real plane, imaginary plane,
// column-major, common leading dimension) so that the same buffers feed the
// tensor-core contraction in lu_tc.cu.
//
// LU structure (blocked right-looking, panel width kNB):
//   for each panel k:  factor A[k:N, k:k+nb] (recursive in-panel LU whose
//                      leaves of <= 8 columns run in one CTA from shared
//                      memory with a block-wide pivot search);
//                      apply the panel's row swaps to the other columns
//                      and to the running permutation;
//                      A12 <- L11^{-1} A12 (triangular solve);
//                      A22 <- A22 - A21 A12 (GEMM).
// The row interchanges of one panel are at most kNB long, so the
// column-parallel swap kernel never runs a long dependency chain; the
// solve phase applies the net permutation once, as a gather.
#include <algorithm>
#include <climits>

#include "dense.cuh"
#include "prof.cuh"

namespace harp {

constexpr int kNB = 64;            // outer panel width
constexpr int kLeafMax = 8;        // widest in-panel leaf
constexpr int kLeafThreads = 512;  // threads of the leaf kernel
constexpr int kTrsmLeaf = 64;      // largest triangle solved by one kernel
constexpr int kTrsmCols = 8;       // right-hand sides per CTA in the leaf

// ---------------------------------------------------------------------------
// GEMM on CUDA cores: C = beta*C + alpha*A*B, 64 x 64 tile, 8-deep k step,
// 16 x 16 threads, 4 x 4 complex register tile per thread.
template <typename R>
__global__ void __launch_bounds__(256) cgemm_simt_kernel(int M, int N, int K, R alpha, CView<R> A,
                                                         CView<R> B, R beta, CView<R> C) {
  __shared__ R As_r[8][64], As_i[8][64], Bs_r[8][64], Bs_i[8][64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  R cr[4][4], ci[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) cr[a][b] = ci[a][b] = 0;
  for (int k0 = 0; k0 < K; k0 += 8) {
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const int e = threadIdx.x + 256 * l;
      const int i = e & 63, kk = e >> 6;
      const bool in = (i0 + i < M) && (k0 + kk < K);
      As_r[kk][i] = in ? A.r(i0 + i, k0 + kk) : (R)0;
      As_i[kk][i] = in ? A.m(i0 + i, k0 + kk) : (R)0;
      const int kb = e & 7, j = e >> 3;
      const bool inb = (k0 + kb < K) && (j0 + j < N);
      Bs_r[kb][j] = inb ? B.r(k0 + kb, j0 + j) : (R)0;
      Bs_i[kb][j] = inb ? B.m(k0 + kb, j0 + j) : (R)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      R ar[4], ai[4], br[4], bi[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ar[a] = As_r[kk][ty + 16 * a];
        ai[a] = As_i[kk][ty + 16 * a];
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        br[b] = Bs_r[kk][tx + 16 * b];
        bi[b] = Bs_i[kk][tx + 16 * b];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          cr[a][b] = fma(ar[a], br[b], cr[a][b]);
          cr[a][b] = fma(-ai[a], bi[b], cr[a][b]);
          ci[a][b] = fma(ar[a], bi[b], ci[a][b]);
          ci[a][b] = fma(ai[a], br[b], ci[a][b]);
        }
    }
    __syncthreads();
  }
  // Epilogue: every C load is issued before any store (the planes could
  // alias as far as the compiler knows, which would serialise the loads).
  R old_r[4][4], old_i[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      const bool in = (beta != (R)0) && (i < M) && (j < N);
      old_r[a][b] = in ? C.r(i, j) : (R)0;
      old_i[a][b] = in ? C.m(i, j) : (R)0;
    }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
    if (i >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      if (j >= N) continue;
      C.r(i, j) = fma(beta, old_r[a][b], alpha * cr[a][b]);
      C.m(i, j) = fma(beta, old_i[a][b], alpha * ci[a][b]);
    }
  }
}

template <typename R>
int cgemm_simt(int M, int N, int K, R alpha, CView<R> A, CView<R> B, R beta, CView<R> C,
               cudaStream_t st, int kind = HARP_K_GEMM) {
  if (M <= 0 || N <= 0) return HARP_OK;
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  ProfScope ps(kind, 8.0 * M * N * (double)K, st);
  cgemm_simt_kernel<R><<<grid, 256, 0, st>>>(M, N, K, alpha, A, B, beta, C);
  HARP_LAUNCHED();
  return HARP_OK;
}

// Tensor-core path (lu_tc.cu). Returns HARP_E_UNSUPPORTED when the shapes
// or strides do not suit it; the caller then uses the CUDA-core kernel.
int cgemm_tc_f32(int M, int N, int K, float alpha, CView<float> A, CView<float> B, float beta,
                 CView<float> C, int mode, cudaStream_t st);

template <>
int cgemm<float>(int M, int N, int K, float alpha, CView<float> A, CView<float> B, float beta,
                 CView<float> C, int mode, cudaStream_t st) {
  if (mode != GEMM_SIMT && K > 0) {
    int s = cgemm_tc_f32(M, N, K, alpha, A, B, beta, C, mode, st);
    if (s != HARP_E_UNSUPPORTED) return s;
  }
  return cgemm_simt<float>(M, N, K, alpha, A, B, beta, C, st);
}
template <>
int cgemm<double>(int M, int N, int K, double alpha, CView<double> A, CView<double> B, double beta,
                  CView<double> C, int, cudaStream_t st) {
  return cgemm_simt<double>(M, N, K, alpha, A, B, beta, C, st);
}

int residual_fp64(int N, int nrhs, CView<double> Z, CView<double> X, CView<double> R,
                  cudaStream_t st) {
  return cgemm_simt<double>(N, nrhs, N, -1.0, Z, X, 1.0, R, st, HARP_K_RESIDUAL);
}

// ---------------------------------------------------------------------------
// In-panel LU leaf: columns j0 .. j0+w-1, rows j0 .. j0+M-1, one CTA. The
// slab is copied to shared memory when it fits (use_smem), else worked on
// in place. Per column: block-wide search for the entry of largest modulus
// (compared as |z|^2, first index on ties), row swap inside the slab,
// scaling of the column below the pivot and rank-1 update of the slab's
// remaining columns.
template <typename R>
__global__ void __launch_bounds__(kLeafThreads) lu_leaf_kernel(R* Are, R* Aim, long lda, int j0,
                                                               int M, int w, int* ipiv,
                                                               int* zero_col, int use_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // Pivot magnitudes |z|^2 in the working precision: FP64 runs at 1/64 of
  // the FP32 rate on this GPU, and FP32 squares order the candidates
  // correctly except on near-ties, where either choice is a valid pivot.
  __shared__ R red_v[kLeafThreads / 32];
  __shared__ int red_i[kLeafThreads / 32];
  __shared__ int s_piv;
  __shared__ R s_best;
  R* gre = Are + (size_t)j0 + (size_t)j0 * lda;
  R* gim = Aim + (size_t)j0 + (size_t)j0 * lda;
  R *sre, *sim;
  long cs;
  if (use_smem) {
    sre = reinterpret_cast<R*>(smem_raw);
    sim = sre + (size_t)w * M;
    cs = M;
    for (int c = 0; c < w; ++c)
      for (int r = threadIdx.x; r < M; r += blockDim.x) {
        sre[(size_t)c * M + r] = gre[r + (size_t)c * lda];
        sim[(size_t)c * M + r] = gim[r + (size_t)c * lda];
      }
  } else {
    sre = gre;
    sim = gim;
    cs = lda;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  for (int c = 0; c < w; ++c) {
    R* cr = sre + (size_t)c * cs;
    R* ci = sim + (size_t)c * cs;
    R best = -1;
    int bi = INT_MAX;
    for (int r = c + threadIdx.x; r < M; r += blockDim.x) {
      const R vr = cr[r], vi = ci[r];
      const R v = vr * vr + vi * vi;
      if (v > best) {
        best = v;
        bi = r;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const R ob = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      red_v[warp] = best;
      red_i[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      best = lane < nwarps ? red_v[lane] : (R)-1;
      bi = lane < nwarps ? red_i[lane] : INT_MAX;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const R ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_best = best;
        s_piv = bi;
      }
    }
    __syncthreads();
    const int piv = s_piv;
    if (!(s_best > (R)0) || piv >= M) {  // exactly zero (or non-finite) column
      if (threadIdx.x == 0) {
        ipiv[j0 + c] = j0 + c;
        atomicMin(zero_col, j0 + c + 1);
      }
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) ipiv[j0 + c] = j0 + piv;
    if (piv != c) {
      for (int t = threadIdx.x; t < w; t += blockDim.x) {
        R* xr = sre + (size_t)t * cs;
        R* xi = sim + (size_t)t * cs;
        const R ar = xr[c], ai = xi[c];
        xr[c] = xr[piv];
        xi[c] = xi[piv];
        xr[piv] = ar;
        xi[piv] = ai;
      }
    }
    __syncthreads();
    const R pr = cr[c], pi = ci[c];
    const R den = pr * pr + pi * pi;
    const R ir = pr / den, ii = -pi / den;
    for (int r = c + 1 + threadIdx.x; r < M; r += blockDim.x) {
      const R ar = cr[r], ai = ci[r];
      const R lr = ar * ir - ai * ii, li = ar * ii + ai * ir;
      cr[r] = lr;
      ci[r] = li;
      for (int cc = c + 1; cc < w; ++cc) {
        R* xr = sre + (size_t)cc * cs;
        R* xi = sim + (size_t)cc * cs;
        const R ur = xr[c], ui = xi[c];
        xr[r] = fma(-lr, ur, fma(li, ui, xr[r]));
        xi[r] = fma(-lr, ui, fma(-li, ur, xi[r]));
      }
    }
    __syncthreads();
  }
  if (use_smem) {
    for (int c = 0; c < w; ++c)
      for (int r = threadIdx.x; r < M; r += blockDim.x) {
        gre[r + (size_t)c * lda] = sre[(size_t)c * M + r];
        gim[r + (size_t)c * lda] = sim[(size_t)c * M + r];
      }
  }
}

// Apply the row swaps ipiv[k1..k2) (in order) to the columns [a0, a1) and
// [b0, b1), one thread per column, and to perm (as one more column) when
// perm != nullptr.
template <typename R>
__global__ void laswp_kernel(R* Are, R* Aim, long lda, const int* ipiv, int k1, int k2, int a0,
                             int a1, int b0, int b1, int* perm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int na = a1 - a0, nb = b1 - b0;
  if (t < na + nb) {
    const int col = (t < na) ? a0 + t : b0 + (t - na);
    R* cr = Are + (size_t)col * lda;
    R* ci = Aim + (size_t)col * lda;
    for (int k = k1; k < k2; ++k) {
      const int p = ipiv[k];
      if (p != k) {
        const R xr = cr[k], xi = ci[k];
        cr[k] = cr[p];
        ci[k] = ci[p];
        cr[p] = xr;
        ci[p] = xi;
      }
    }
  } else if (t == na + nb && perm) {
    for (int k = k1; k < k2; ++k) {
      const int p = ipiv[k];
      if (p != k) {
        const int x = perm[k];
        perm[k] = perm[p];
        perm[p] = x;
      }
    }
  }
}

template <typename R>
static int laswp(R* re, R* im, long ld, const int* ipiv, int k1, int k2, int a0, int a1, int b0,
                 int b1, int* perm, cudaStream_t st) {
  const int n = std::max(0, a1 - a0) + std::max(0, b1 - b0) + (perm ? 1 : 0);
  if (n == 0 || k2 <= k1) return HARP_OK;
  const int threads = 128;
  ProfScope ps(HARP_K_SWAP, 0.0, st);
  laswp_kernel<R><<<(n + threads - 1) / threads, threads, 0, st>>>(
      re, im, ld, ipiv, k1, k2, a0, std::max(a0, a1), b0, std::max(b0, b1), perm);
  HARP_LAUNCHED();
  return HARP_OK;
}

__global__ void iota_kernel(int* p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}

// ---------------------------------------------------------------------------
// Triangular solve leaf: T X = B for an n x n (n <= 64) triangle given as a
// view T (already transposed when the caller solves with op(A) = A^T),
// kTrsmCols right-hand sides per CTA. One barrier per eliminated row.
template <typename R, bool LOWER, bool UNIT>
__global__ void __launch_bounds__(kTrsmLeaf* kTrsmCols) trsm_leaf_kernel(int n, int ncols,
                                                                          CView<R> T, CView<R> B) {
  // Dynamic shared memory (the FP64 tiles exceed the static 48 KB limit).
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typedef R TRow[kTrsmLeaf + 1];
  typedef R BRow[kTrsmCols];
  TRow* Tr = reinterpret_cast<TRow*>(smem_raw);
  TRow* Ti = Tr + kTrsmLeaf;
  BRow* Br = reinterpret_cast<BRow*>(Ti + kTrsmLeaf);
  BRow* Bi = Br + kTrsmLeaf;
  BRow* Xr = Bi + kTrsmLeaf;
  BRow* Xi = Xr + kTrsmLeaf;
  const int i = threadIdx.x, c = threadIdx.y;
  const int col = blockIdx.x * kTrsmCols + c;
  const int tid = threadIdx.y * kTrsmLeaf + threadIdx.x;
  for (int e = tid; e < n * n; e += kTrsmLeaf * kTrsmCols) {
    const int r = e % n, k = e / n;
    const bool need = LOWER ? (r >= k) : (r <= k);
    Tr[r][k] = need ? T.r(r, k) : (R)0;
    Ti[r][k] = need ? T.m(r, k) : (R)0;
  }
  const bool act = (i < n) && (col < ncols);
  R br = 0, bi = 0;
  if (act) {
    br = B.r(i, col);
    bi = B.m(i, col);
  }
  Br[i][c] = br;
  Bi[i][c] = bi;
  __syncthreads();
  for (int s = 0; s < n; ++s) {
    const int k = LOWER ? s : n - 1 - s;
    R xr = Br[k][c], xi = Bi[k][c];
    if (!UNIT) {
      const R dr = Tr[k][k], di = Ti[k][k];
      const R den = dr * dr + di * di;
      const R qr = (xr * dr + xi * di) / den, qi = (xi * dr - xr * di) / den;
      xr = qr;
      xi = qi;
    }
    const bool upd = LOWER ? (i > k) : (i < k);
    if (upd) {
      const R tr = Tr[i][k], ti = Ti[i][k];
      Br[i][c] = fma(-tr, xr, fma(ti, xi, Br[i][c]));
      Bi[i][c] = fma(-tr, xi, fma(-ti, xr, Bi[i][c]));
    }
    if (i == k) {
      Xr[k][c] = xr;
      Xi[k][c] = xi;
    }
    __syncthreads();
  }
  if (act) {
    B.r(i, col) = Xr[i][c];
    B.m(i, col) = Xi[i][c];
  }
}

template <typename R>
static int trsm_leaf(bool lower, bool unit, int n, int ncols, CView<R> T, CView<R> B,
                     cudaStream_t st) {
  dim3 block(kTrsmLeaf, kTrsmCols);
  dim3 grid((ncols + kTrsmCols - 1) / kTrsmCols);
  const size_t smem = sizeof(R) * (2 * kTrsmLeaf * (kTrsmLeaf + 1) + 4 * kTrsmLeaf * kTrsmCols);
  void (*kern)(int, int, CView<R>, CView<R>) =
      lower ? (unit ? trsm_leaf_kernel<R, true, true> : trsm_leaf_kernel<R, true, false>)
            : (unit ? trsm_leaf_kernel<R, false, true> : trsm_leaf_kernel<R, false, false>);
  HARP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope ps(HARP_K_TRSM, 4.0 * n * (double)n * ncols, st);
  kern<<<grid, block, smem, st>>>(n, ncols, T, B);
  HARP_LAUNCHED();
  return HARP_OK;
}

// T X = B with T (n x n) the effective triangle (lower or upper), B n x ncols,
// recursive halving down to kTrsmLeaf with GEMM updates in between.
template <typename R>
static int trsm(bool lower, bool unit, int n, int ncols, CView<R> T, CView<R> B, int mode,
                cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return HARP_OK;
  if (n <= kTrsmLeaf) return trsm_leaf<R>(lower, unit, n, ncols, T, B, st);
  const int n1 = ((n / 2) + 31) / 32 * 32;
  const int n2 = n - n1;
  CView<R> B1 = B, B2 = B.sub(n1, 0);
  if (lower) {
    HARP_TRY(trsm<R>(true, unit, n1, ncols, T, B1, mode, st));
    HARP_TRY(cgemm<R>(n2, ncols, n1, (R)-1, T.sub(n1, 0), B1, (R)1, B2, mode, st));
    HARP_TRY(trsm<R>(true, unit, n2, ncols, T.sub(n1, n1), B2, mode, st));
  } else {
    HARP_TRY(trsm<R>(false, unit, n2, ncols, T.sub(n1, n1), B2, mode, st));
    HARP_TRY(cgemm<R>(n1, ncols, n2, (R)-1, T.sub(0, n1), B2, (R)1, B1, mode, st));
    HARP_TRY(trsm<R>(false, unit, n1, ncols, T, B1, mode, st));
  }
  return HARP_OK;
}

// ---------------------------------------------------------------------------
// LU driver.
template <typename R>
static int leaf_width(const harp_ctx* ctx, int M, int want, int* use_smem) {
  const size_t budget = std::min<size_t>(ctx->smem_optin, 200 * 1024);
  for (int w = std::min(want, kLeafMax); w >= 1; w >>= 1)
    if ((size_t)2 * M * w * sizeof(R) <= budget) {
      *use_smem = 1;
      return w;
    }
  *use_smem = 0;
  return std::min(want, kLeafMax);
}

template <typename R>
static int panel(harp_ctx* ctx, int N, CView<R> A, R* re, R* im, long ld, int j0, int w,
                 int* ipiv, int* zero_col, int mode, cudaStream_t st) {
  const int M = N - j0;
  int use_smem = 0;
  const int lw = leaf_width<R>(ctx, M, w, &use_smem);
  if (w <= lw) {
    const size_t smem = use_smem ? (size_t)2 * M * w * sizeof(R) : 0;
    HARP_CUDA(cudaFuncSetAttribute(lu_leaf_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)std::max<size_t>(smem, 0)));
    ProfScope ps(HARP_K_PANEL, 4.0 * M * w * (double)(w - 1) + 6.0 * M * w, st);
    lu_leaf_kernel<R><<<1, kLeafThreads, smem, st>>>(re, im, ld, j0, M, w, ipiv, zero_col,
                                                     use_smem);
    HARP_LAUNCHED();
    return HARP_OK;
  }
  const int w1 = w / 2, w2 = w - w1;
  HARP_TRY(panel<R>(ctx, N, A, re, im, ld, j0, w1, ipiv, zero_col, mode, st));
  HARP_TRY(laswp<R>(re, im, ld, ipiv, j0, j0 + w1, j0 + w1, j0 + w, 0, 0, nullptr, st));
  HARP_TRY(trsm<R>(true, true, w1, w2, A.sub(j0, j0), A.sub(j0, j0 + w1), mode, st));
  HARP_TRY(cgemm<R>(M - w1, w2, w1, (R)-1, A.sub(j0 + w1, j0), A.sub(j0, j0 + w1), (R)1,
                    A.sub(j0 + w1, j0 + w1), mode, st));
  HARP_TRY(panel<R>(ctx, N, A, re, im, ld, j0 + w1, w2, ipiv, zero_col, mode, st));
  HARP_TRY(laswp<R>(re, im, ld, ipiv, j0 + w1, j0 + w, j0, j0 + w1, 0, 0, nullptr, st));
  return HARP_OK;
}

template <typename R>
int lu_factor(harp_ctx* ctx, int N, R* re, R* im, long ld, int* ipiv, int* perm, int* zero_col,
              int mode, cudaStream_t st) {
  ProfScope ps_o(HARP_K_OTHER, 0.0, st);
  iota_kernel<<<(N + 255) / 256, 256, 0, st>>>(perm, N);
  HARP_LAUNCHED();
  CView<R> A = planes<R>(re, im, ld);
  for (int k = 0; k < N; k += kNB) {
    const int nb = std::min(kNB, N - k);
    HARP_TRY(panel<R>(ctx, N, A, re, im, ld, k, nb, ipiv, zero_col, mode, st));
    HARP_TRY(laswp<R>(re, im, ld, ipiv, k, k + nb, 0, k, k + nb, N, perm, st));
    if (k + nb < N) {
      HARP_TRY(trsm<R>(true, true, nb, N - k - nb, A.sub(k, k), A.sub(k, k + nb), mode, st));
      HARP_TRY(cgemm<R>(N - k - nb, N - k - nb, nb, (R)-1, A.sub(k + nb, k), A.sub(k, k + nb), (R)1,
                        A.sub(k + nb, k + nb), mode, st));
    }
  }
  return HARP_OK;
}

// ---------------------------------------------------------------------------
// Row gather / scatter with the net permutation, then the two triangular
// solves.
template <typename R>
__global__ void permute_rows_kernel(int N, int nrhs, const int* perm, const R* sre, const R* sim,
                                    R* dre, R* dim, long ld, int scatter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= N) return;
  const int p = perm[i];
  const size_t off = (size_t)c * ld;
  if (!scatter) {
    dre[off + i] = sre[off + p];
    dim[off + i] = sim[off + p];
  } else {
    dre[off + p] = sre[off + i];
    dim[off + p] = sim[off + i];
  }
}

template <typename R>
int lu_solve(int N, int nrhs, R* lre, R* lim, long ld, const int* perm, R* bre, R* bim, long ldb,
             R* tre, R* tim, char trans, int mode, cudaStream_t st) {
  CView<R> L = planes<R>(lre, lim, ld);
  dim3 grid((N + 255) / 256, nrhs);
  if (trans == 'N' || trans == 'n') {
    {
      ProfScope ps(HARP_K_OTHER, 0.0, st);
      permute_rows_kernel<R><<<grid, 256, 0, st>>>(N, nrhs, perm, bre, bim, tre, tim, ldb, 0);
    }
    HARP_LAUNCHED();
    CView<R> Tm = planes<R>(tre, tim, ldb);
    HARP_TRY(trsm<R>(true, true, N, nrhs, L, Tm, mode, st));
    HARP_TRY(trsm<R>(false, false, N, nrhs, L, Tm, mode, st));
    HARP_TRY(planes_to_planes<R, R>(N, nrhs, tre, tim, ldb, bre, bim, ldb, st));
  } else {
    CView<R> Bm = planes<R>(bre, bim, ldb);
    HARP_TRY(trsm<R>(true, false, N, nrhs, L.t(), Bm, mode, st));  // U^T y = b
    HARP_TRY(trsm<R>(false, true, N, nrhs, L.t(), Bm, mode, st));  // L^T z = y
    {
      ProfScope ps(HARP_K_OTHER, 0.0, st);
      permute_rows_kernel<R><<<grid, 256, 0, st>>>(N, nrhs, perm, bre, bim, tre, tim, ldb, 1);
    }
    HARP_LAUNCHED();
    HARP_TRY(planes_to_planes<R, R>(N, nrhs, tre, tim, ldb, bre, bim, ldb, st));
  }
  return HARP_OK;
}

// ---------------------------------------------------------------------------
// Conversions, RHS, norms.
template <typename Rin, typename Rout>
__global__ void i2p_kernel(int M, int N, const Rin* src, long lds, Rout* re, Rout* im, long ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= M) return;
  const Rin* s = src + 2 * ((size_t)i + (size_t)j * lds);
  re[i + (size_t)j * ldd] = (Rout)s[0];
  im[i + (size_t)j * ldd] = (Rout)s[1];
}
template <typename Rin, typename Rout>
int interleaved_to_planes(int M, int N, const Rin* src, long lds, Rout* re, Rout* im, long ldd,
                          cudaStream_t st) {
  if (M <= 0 || N <= 0) return HARP_OK;
  dim3 grid((M + 255) / 256, N);
  ProfScope ps_o(HARP_K_OTHER, 0.0, st);
  i2p_kernel<Rin, Rout><<<grid, 256, 0, st>>>(M, N, src, lds, re, im, ldd);
  HARP_LAUNCHED();
  return HARP_OK;
}

template <typename Rin, typename Rout>
__global__ void p2p_kernel(int M, int N, const Rin* sre, const Rin* sim, long lds, Rout* dre,
                           Rout* dim, long ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= M) return;
  dre[i + (size_t)j * ldd] = (Rout)sre[i + (size_t)j * lds];
  dim[i + (size_t)j * ldd] = (Rout)sim[i + (size_t)j * lds];
}
template <typename Rin, typename Rout>
int planes_to_planes(int M, int N, const Rin* sre, const Rin* sim, long lds, Rout* dre, Rout* dim,
                     long ldd, cudaStream_t st) {
  if (M <= 0 || N <= 0) return HARP_OK;
  dim3 grid((M + 255) / 256, N);
  ProfScope ps_o(HARP_K_OTHER, 0.0, st);
  p2p_kernel<Rin, Rout><<<grid, 256, 0, st>>>(M, N, sre, sim, lds, dre, dim, ldd);
  HARP_LAUNCHED();
  return HARP_OK;
}

__global__ void p2i_kernel(int M, int N, const double* re, const double* im, long lds, double* dst,
                           long ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= M) return;
  double2 v = make_double2(re[i + (size_t)j * lds], im[i + (size_t)j * lds]);
  reinterpret_cast<double2*>(dst)[i + (size_t)j * ldd] = v;
}
int planes_to_interleaved(int M, int N, const double* re, const double* im, long lds, double* dst,
                          long ldd, cudaStream_t st) {
  if (M <= 0 || N <= 0) return HARP_OK;
  dim3 grid((M + 255) / 256, N);
  ProfScope ps_o(HARP_K_OTHER, 0.0, st);
  p2i_kernel<<<grid, 256, 0, st>>>(M, N, re, im, lds, dst, ldd);
  HARP_LAUNCHED();
  return HARP_OK;
}

template <typename R>
__global__ void port_rhs_kernel(int M, int N, int Nm, R* re, R* im, long ld) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= M) return;
  re[i + (size_t)j * ld] = (i == j * Nm) ? (R)1 : (R)0;
  im[i + (size_t)j * ld] = (R)0;
}
template <typename R>
int port_rhs_planes(int M, int N, int Nm, R* re, R* im, long ld, cudaStream_t st) {
  dim3 grid((M + 255) / 256, N);
  ProfScope ps_o(HARP_K_OTHER, 0.0, st);
  port_rhs_kernel<R><<<grid, 256, 0, st>>>(M, N, Nm, re, im, ld);
  HARP_LAUNCHED();
  return HARP_OK;
}

template <typename R>
__global__ void add_planes_kernel(int M, int N, double* xre, double* xim, long ldx, const R* dre,
                                  const R* dim, long ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= M) return;
  xre[i + (size_t)j * ldx] += (double)dre[i + (size_t)j * ldd];
  xim[i + (size_t)j * ldx] += (double)dim[i + (size_t)j * ldd];
}
template <typename R>
int add_planes(int M, int N, double* xre, double* xim, long ldx, const R* dre, const R* dim,
               long ldd, cudaStream_t st) {
  dim3 grid((M + 255) / 256, N);
  ProfScope ps_o(HARP_K_OTHER, 0.0, st);
  add_planes_kernel<R><<<grid, 256, 0, st>>>(M, N, xre, xim, ldx, dre, dim, ldd);
  HARP_LAUNCHED();
  return HARP_OK;
}

template <typename R>
__global__ void norm_inf_kernel(int M, int N, CView<R> A, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < M)
    for (int j = 0; j < N; ++j) {
      const double a = (double)A.r(i, j), b = (double)A.m(i, j);
      s += sqrt(a * a + b * b);
    }
  if (!(s == s)) s = __longlong_as_double(0x7ff0000000000000LL);  // NaN -> +Inf
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, off));
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(s));
}
template <typename R>
int norm_inf(int M, int N, CView<R> A, double* out, cudaStream_t st) {
  if (M <= 0) return HARP_OK;
  ProfScope ps_o(HARP_K_OTHER, 0.0, st);
  norm_inf_kernel<R><<<(M + 255) / 256, 256, 0, st>>>(M, N, A, out);
  HARP_LAUNCHED();
  return HARP_OK;
}

int zero_doubles(double* p, int n, cudaStream_t st) {
  HARP_CUDA(cudaMemsetAsync(p, 0, sizeof(double) * n, st));
  return HARP_OK;
}

// ---------------------------------------------------------------------------
// Explicit instantiations.
template int lu_factor<float>(harp_ctx*, int, float*, float*, long, int*, int*, int*, int,
                              cudaStream_t);
template int lu_factor<double>(harp_ctx*, int, double*, double*, long, int*, int*, int*, int,
                               cudaStream_t);
template int lu_solve<float>(int, int, float*, float*, long, const int*, float*, float*, long,
                             float*, float*, char, int, cudaStream_t);
template int lu_solve<double>(int, int, double*, double*, long, const int*, double*, double*, long,
                              double*, double*, char, int, cudaStream_t);
template int interleaved_to_planes<float, float>(int, int, const float*, long, float*, float*, long,
                                                 cudaStream_t);
template int interleaved_to_planes<double, double>(int, int, const double*, long, double*, double*,
                                                   long, cudaStream_t);
template int interleaved_to_planes<double, float>(int, int, const double*, long, float*, float*,
                                                  long, cudaStream_t);
template int planes_to_planes<double, float>(int, int, const double*, const double*, long, float*,
                                             float*, long, cudaStream_t);
template int planes_to_planes<double, double>(int, int, const double*, const double*, long, double*,
                                              double*, long, cudaStream_t);
template int planes_to_planes<float, double>(int, int, const float*, const float*, long, double*,
                                             double*, long, cudaStream_t);
template int planes_to_planes<float, float>(int, int, const float*, const float*, long, float*,
                                            float*, long, cudaStream_t);
template int port_rhs_planes<float>(int, int, int, float*, float*, long, cudaStream_t);
template int port_rhs_planes<double>(int, int, int, double*, double*, long, cudaStream_t);
template int add_planes<float>(int, int, double*, double*, long, const float*, const float*, long,
                               cudaStream_t);
template int add_planes<double>(int, int, double*, double*, long, const double*, const double*,
                                long, cudaStream_t);
template int norm_inf<double>(int, int, CView<double>, double*, cudaStream_t);
template int norm_inf<float>(int, int, CView<float>, double*, cudaStream_t);

}  // namespace harp
