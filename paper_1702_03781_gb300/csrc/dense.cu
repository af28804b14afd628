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
#include <atomic>
#include <array>
#include <climits>
#include <type_traits>
#include <vector>

#include "dense.cuh"
#include "prof.cuh"

namespace harp {

constexpr int kNB = 64;            // outer panel width
constexpr int kLeafMax = 8;        // widest in-panel leaf
constexpr int kLeafThreads = 512;  // threads of the leaf kernel
constexpr int kLeafSmem = 200 * 1024;  // shared-memory budget of the leaf
constexpr int kTrsmLeaf = 64;      // largest triangle solved by one kernel
constexpr int kTrsmCols = 8;       // right-hand sides per CTA in the leaf

// ---------------------------------------------------------------------------
// GEMM on CUDA cores: C = beta*C + alpha*A*B, 64 x 64 tile, 8-deep k step,
// 16 x 16 threads, 4 x 4 complex register tile per thread.
template <typename R>
__global__ void __launch_bounds__(256) cgemm_simt_kernel(int M, int N, int K, R alpha, CView<R> A,
                                                         CView<R> B, R beta, CView<R> C, long sA,
                                                         long sB, long sC) {
  __shared__ R As_r[8][64], As_i[8][64], Bs_r[8][64], Bs_i[8][64];
  // batch z: every operand moved by its element stride
  A.re += blockIdx.z * sA;
  A.im += blockIdx.z * sA;
  B.re += blockIdx.z * sB;
  B.im += blockIdx.z * sB;
  C.re += blockIdx.z * sC;
  C.im += blockIdx.z * sC;
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
               cudaStream_t st, int kind = HARP_K_GEMM, long sA = 0, long sB = 0, long sC = 0,
               int batch = 1) {
  if (M <= 0 || N <= 0 || batch <= 0) return HARP_OK;
  if (batch > 65535) return HARP_E_UNSUPPORTED;
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  ProfScope ps(kind, 8.0 * M * N * (double)K * batch, st);
  cgemm_simt_kernel<R><<<grid, 256, 0, st>>>(M, N, K, alpha, A, B, beta, C, sA, sB, sC);
  HARP_LAUNCHED();
  return HARP_OK;
}

// Tensor-core path (lu_tc.cu). Returns HARP_E_UNSUPPORTED when the shapes
// or strides do not suit it; the caller then uses the CUDA-core kernel.
int cgemm_tc_f32(int M, int N, int K, float alpha, CView<float> A, CView<float> B, float beta,
                 CView<float> C, int mode, cudaStream_t st, long sA, long sB, long sC, int batch);

template <>
int cgemm<float>(int M, int N, int K, float alpha, CView<float> A, CView<float> B, float beta,
                 CView<float> C, int mode, cudaStream_t st) {
  return cgemm_batched(M, N, K, alpha, A, 0, B, 0, beta, C, 0, 1, mode, st);
}

// Tensor-core-sized FP32 products that ran on the CUDA cores instead.
static std::atomic<long> g_tc_fallbacks{0};

long tc_fallbacks() { return g_tc_fallbacks.load(); }

int cgemm_batched(int M, int N, int K, float alpha, CView<float> A, long sA, CView<float> B,
                  long sB, float beta, CView<float> C, long sC, int batch, int mode,
                  cudaStream_t st) {
  if (mode != GEMM_SIMT && K > 0) {
    int s = cgemm_tc_f32(M, N, K, alpha, A, B, beta, C, mode, st, sA, sB, sC, batch);
    if (s != HARP_E_UNSUPPORTED) return s;
    if (M >= 64 && N >= 64 && K >= 32) g_tc_fallbacks.fetch_add(1);
  }
  return cgemm_simt<float>(M, N, K, alpha, A, B, beta, C, st, HARP_K_GEMM, sA, sB, sC, batch);
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
// In-panel LU leaf: columns j0 .. j0+w-1, rows j0 .. j0+M-1, one CTA. With
// SMEM the slab is copied to shared memory (loads batched into registers
// first so they overlap), else it is worked on in place. Per column: a
// block-wide search for the entry of largest modulus (|z|^2 in the working
// precision, first index on ties; every thread reduces the per-warp
// candidates itself, so one barrier suffices), the row swap inside the
// slab, then scaling of the column below the pivot and the rank-1 update
// of the slab's remaining columns.
template <typename R, bool SMEM>
__global__ void __launch_bounds__(kLeafThreads) lu_leaf_kernel(R* Are, R* Aim, long lda, int j0,
                                                               int M, int w, int* ipiv,
                                                               int* zero_col) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R red_v[kLeafThreads / 32];
  __shared__ int red_i[kLeafThreads / 32];
  R* gre = Are + (size_t)j0 + (size_t)j0 * lda;
  R* gim = Aim + (size_t)j0 + (size_t)j0 * lda;
  R* sre = SMEM ? reinterpret_cast<R*>(smem_raw) : gre;
  R* sim = SMEM ? sre + (size_t)w * M : gim;
  const long cs = SMEM ? (long)M : lda;
  constexpr int kB = 8;  // rows per thread per batch
  if (SMEM) {
    for (int c = 0; c < w; ++c)
      for (int r0 = 0; r0 < M; r0 += kB * kLeafThreads) {
        R vr[kB], vi[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          const int r = r0 + threadIdx.x + u * kLeafThreads;
          vr[u] = (r < M) ? gre[r + (size_t)c * lda] : (R)0;
          vi[u] = (r < M) ? gim[r + (size_t)c * lda] : (R)0;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          const int r = r0 + threadIdx.x + u * kLeafThreads;
          if (r < M) {
            sre[(size_t)c * M + r] = vr[u];
            sim[(size_t)c * M + r] = vi[u];
          }
        }
      }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nwarps = kLeafThreads / 32;
  for (int c = 0; c < w; ++c) {
    R* cr = sre + (size_t)c * cs;
    R* ci = sim + (size_t)c * cs;
    R best = -1;
    int bi = INT_MAX;
    for (int r = c + threadIdx.x; r < M; r += kLeafThreads) {
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
    best = red_v[0];
    bi = red_i[0];
#pragma unroll
    for (int q = 1; q < nwarps; ++q) {
      const R ob = red_v[q];
      const int oi = red_i[q];
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    const int piv = bi;
    if (!(best > (R)0) || piv >= M) {  // exactly zero (or non-finite) column
      if (threadIdx.x == 0) {
        ipiv[j0 + c] = j0 + c;
        atomicMin(zero_col, j0 + c + 1);
      }
      __syncthreads();  // red_v reuse
      continue;
    }
    if (threadIdx.x == 0) ipiv[j0 + c] = j0 + piv;
    if (piv != c && threadIdx.x < w) {
      R* xr = sre + (size_t)threadIdx.x * cs;
      R* xi = sim + (size_t)threadIdx.x * cs;
      const R ar = xr[c], ai = xi[c];
      xr[c] = xr[piv];
      xi[c] = xi[piv];
      xr[piv] = ar;
      xi[piv] = ai;
    }
    __syncthreads();
    const R pr = cr[c], pi = ci[c];
    const R den = pr * pr + pi * pi;
    const R ir = pr / den, ii = -pi / den;
    R ur[kLeafMax], ui[kLeafMax];
#pragma unroll
    for (int cc = 0; cc < kLeafMax; ++cc) {
      if (cc > c && cc < w) {
        ur[cc] = sre[(size_t)cc * cs + c];
        ui[cc] = sim[(size_t)cc * cs + c];
      }
    }
    for (int r = c + 1 + threadIdx.x; r < M; r += kLeafThreads) {
      const R ar = cr[r], ai = ci[r];
      const R lr = ar * ir - ai * ii, li = ar * ii + ai * ir;
      cr[r] = lr;
      ci[r] = li;
#pragma unroll
      for (int cc = 0; cc < kLeafMax; ++cc) {
        if (cc > c && cc < w) {
          R* xr = sre + (size_t)cc * cs;
          R* xi = sim + (size_t)cc * cs;
          xr[r] = fma(-lr, ur[cc], fma(li, ui[cc], xr[r]));
          xi[r] = fma(-lr, ui[cc], fma(-li, ur[cc], xi[r]));
        }
      }
    }
    __syncthreads();
  }
  if (SMEM) {
    for (int c = 0; c < w; ++c)
      for (int r = threadIdx.x; r < M; r += kLeafThreads) {
        gre[r + (size_t)c * lda] = sre[(size_t)c * M + r];
        gim[r + (size_t)c * lda] = sim[(size_t)c * M + r];
      }
  }
}

// Apply the row swaps ipiv[k1..k2) (in order, k2 - k1 <= kNB) to the columns
// [a0, a1) and [b0, b1), and to perm (as one more column of ints) when perm
// != nullptr. Each CTA first composes the swaps into the net permutation of
// the touched rows (rows k1..k2 and the distinct pivot rows below them, at
// most 2*kNB): warp 0 runs the swaps on row labels in shared memory. A pivot
// outside [k1 + u, nrows) (left unset by a panel that gave up) is taken as
// no swap, so every access stays inside the nrows x lda matrix.
// Every column is then a gather by one warp -- all loads of the touched rows
// (from their source rows) before all stores -- with no dependency chain.
constexpr int kSwapWarps = 8;
template <typename R>
__global__ void __launch_bounds__(kSwapWarps * 32) laswp_kernel(R* Are, R* Aim, long lda,
                                                                int nrows, const int* ipiv, int k1,
                                                                int k2, int a0, int a1, int b0,
                                                                int b1, int* perm) {
  __shared__ int piv[kNB], row[2 * kNB], src[2 * kNB], nt_s;
  const int nsw = k2 - k1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < nsw) {
    const int p = ipiv[k1 + tid];
    piv[tid] = (p >= k1 + tid && p < nrows) ? p : k1 + tid;
  }
  __syncthreads();
  if (warp == 0) {
    // slots 0..nsw-1: rows k1..k2-1; then one slot per distinct pivot row >= k2
    for (int u = lane; u < nsw; u += 32) {
      row[u] = k1 + u;
      src[u] = k1 + u;
    }
    __syncwarp();
    int nt = nsw;
    for (int u = 0; u < nsw; ++u) {
      const int p = piv[u];
      int sl = -1;
      if (p < k2) {
        sl = p - k1;
      } else {
        for (int v0 = nsw; v0 < nt && sl < 0; v0 += 32) {
          const int v = v0 + lane;
          const unsigned hit = __ballot_sync(0xffffffffu, v < nt && row[v] == p);
          if (hit) sl = v0 + __ffs(hit) - 1;
        }
        if (sl < 0) {
          sl = nt++;
          if (lane == 0) {
            row[sl] = p;
            src[sl] = p;
          }
        }
      }
      // run swap u on the labels: afterwards slot v holds original row src[v]
      if (lane == 0 && sl != u) {
        const int t = src[u];
        src[u] = src[sl];
        src[sl] = t;
      }
      __syncwarp();
    }
    if (lane == 0) nt_s = nt;
  }
  __syncthreads();
  const int nt = nt_s;
  const int na = a1 - a0, nb = b1 - b0;
  const int ncols = na + nb + (perm ? 1 : 0);
  for (int c = blockIdx.x * kSwapWarps + warp; c < ncols; c += gridDim.x * kSwapWarps) {
    constexpr int kPer = (2 * kNB + 31) / 32;
    if (c < na + nb) {
      const int col = (c < na) ? a0 + c : b0 + (c - na);
      R* cr = Are + (size_t)col * lda;
      R* ci = Aim + (size_t)col * lda;
      R vr[kPer], vi[kPer];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int t = lane + 32 * q;
        if (t < nt) {
          vr[q] = cr[src[t]];
          vi[q] = ci[src[t]];
        }
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int t = lane + 32 * q;
        if (t < nt) {
          cr[row[t]] = vr[q];
          ci[row[t]] = vi[q];
        }
      }
    } else {
      int v[kPer];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int t = lane + 32 * q;
        if (t < nt) v[q] = perm[src[t]];
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int t = lane + 32 * q;
        if (t < nt) perm[row[t]] = v[q];
      }
    }
  }
}

template <typename R>
static int laswp(R* re, R* im, long ld, int nrows, const int* ipiv, int k1, int k2, int a0, int a1,
                 int b0, int b1, int* perm, cudaStream_t st) {
  const int n = std::max(0, a1 - a0) + std::max(0, b1 - b0) + (perm ? 1 : 0);
  if (n == 0 || k2 <= k1) return HARP_OK;
  if (k2 - k1 > kNB || k2 > nrows || k1 < 0) return HARP_E_UNSUPPORTED;
  const int blocks = std::min((n + kSwapWarps - 1) / kSwapWarps, 4 * 152);
  ProfScope ps(HARP_K_SWAP, 0.0, st);
  laswp_kernel<R><<<blocks, kSwapWarps * 32, 0, st>>>(re, im, ld, nrows, ipiv, k1, k2, a0,
                                                      std::max(a0, a1), b0, std::max(b0, b1),
                                                      perm);
  HARP_LAUNCHED();
  return HARP_OK;
}

// The row interchanges of a cluster-factored panel on the columns [a0, a1)
// and [b0, b1) (and perm, as one more column, when given), from the panel's
// exported row map: rmap[0] = n entries, then pairs (destination row, source
// row), every destination taking the old content of its source. One warp
// per column: all loads, then all stores.
template <typename R>
__global__ void __launch_bounds__(kSwapWarps * 32) laswp_map_kernel(R* Are, R* Aim, long lda,
                                                                    const int* rmap, int a0, int a1,
                                                                    int b0, int b1, int* perm) {
  __shared__ int dst[2 * kNB], src[2 * kNB];
  __shared__ int nt_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) nt_s = min(rmap[0], 2 * kNB);
  __syncthreads();
  const int nt = nt_s;
  for (int t = tid; t < nt; t += blockDim.x) {
    dst[t] = rmap[1 + 2 * t];
    src[t] = rmap[2 + 2 * t];
  }
  __syncthreads();
  const int na = a1 - a0, nb = b1 - b0;
  const int ncols = na + nb + (perm ? 1 : 0);
  constexpr int kPer = (2 * kNB + 31) / 32;
  for (int c = blockIdx.x * kSwapWarps + warp; c < ncols; c += gridDim.x * kSwapWarps) {
    if (c < na + nb) {
      const int col = (c < na) ? a0 + c : b0 + (c - na);
      R* cr = Are + (size_t)col * lda;
      R* ci = Aim + (size_t)col * lda;
      R vr[kPer], vi[kPer];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int t = lane + 32 * q;
        if (t < nt) {
          vr[q] = cr[src[t]];
          vi[q] = ci[src[t]];
        }
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int t = lane + 32 * q;
        if (t < nt) {
          cr[dst[t]] = vr[q];
          ci[dst[t]] = vi[q];
        }
      }
    } else {
      int v[kPer];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int t = lane + 32 * q;
        if (t < nt) v[q] = perm[src[t]];
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int t = lane + 32 * q;
        if (t < nt) perm[dst[t]] = v[q];
      }
    }
  }
}

template <typename R>
static int laswp_map(R* re, R* im, long ld, const int* rmap, int a0, int a1, int b0, int b1,
                     int* perm, cudaStream_t st) {
  const int n = std::max(0, a1 - a0) + std::max(0, b1 - b0) + (perm ? 1 : 0);
  if (n == 0) return HARP_OK;
  const int blocks = std::min((n + kSwapWarps - 1) / kSwapWarps, 4 * 152);
  ProfScope ps(HARP_K_SWAP, 0.0, st);
  laswp_map_kernel<R><<<blocks, kSwapWarps * 32, 0, st>>>(re, im, ld, rmap, a0, std::max(a0, a1),
                                                          b0, std::max(b0, b1), perm);
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
                                                                          CView<R> T, CView<R> B,
                                                                          int batch_n, long t_step,
                                                                          long b_step) {
  // blockIdx.y selects a problem of a batch: the triangle and the right-hand
  // sides move by t_step / b_step elements, the last one may be smaller.
  if (blockIdx.y > 0) {
    T.re += t_step * blockIdx.y;
    T.im += t_step * blockIdx.y;
    B.re += b_step * blockIdx.y;
    B.im += b_step * blockIdx.y;
  }
  n = min(n, batch_n - (int)blockIdx.y * n);
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
  void (*kern)(int, int, CView<R>, CView<R>, int, long, long) =
      lower ? (unit ? trsm_leaf_kernel<R, true, true> : trsm_leaf_kernel<R, true, false>)
            : (unit ? trsm_leaf_kernel<R, false, true> : trsm_leaf_kernel<R, false, false>);
  HARP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope ps(HARP_K_TRSM, 4.0 * n * (double)n * ncols, st);
  kern<<<grid, block, smem, st>>>(n, ncols, T, B, n, 0, 0);
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
// Inverses of the 64 x 64 diagonal blocks of the factors, for the solves of
// the refinement (the factors are reused by every solve of a call, so a
// triangular leaf becomes one small parallel product). Block b of a triangle
// is inverted by solving T_bb X = I with the leaf kernel (batched over
// blocks); the last block may be smaller. The inverse of a leading
// principal block of a triangular matrix is the leading block of its
// inverse, which is what the 64-aligned recursion below uses.
template <typename R>
__global__ void identity_blocks_kernel(R* re, R* im, int nblk) {
  const int b = blockIdx.y;
  for (int e = threadIdx.x; e < kTrsmLeaf * kTrsmLeaf; e += blockDim.x) {
    const int i = e % kTrsmLeaf, j = e / kTrsmLeaf;
    re[(size_t)b * kTrsmLeaf * kTrsmLeaf + e] = (i == j) ? (R)1 : (R)0;
    im[(size_t)b * kTrsmLeaf * kTrsmLeaf + e] = (R)0;
  }
}

// Triangle blocks of at most 64 rows, inverted by one warp per column with
// shuffles. The block is held by columns in shared memory (Tr/Ti[p * 65 +
// row], zeros outside the triangle); column c of the inverse solves
// T x = e_c by substitution, lane l holding rows l and l + 32.
__device__ __forceinline__ void tri64_load(int n, const CView<float>& T, bool upper, float* Tr,
                                           float* Ti, int tid) {
  float vr[16], vi[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int e = tid + 256 * q, p = e >> 6, row = e & 63;
    const bool in = row < n && p < n && (upper ? row <= p : row > p);
    vr[q] = in ? T.r(row, p) : 0.f;
    vi[q] = in ? T.m(row, p) : 0.f;
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int e = tid + 256 * q;
    Tr[(e >> 6) * 65 + (e & 63)] = vr[q];
    Ti[(e >> 6) * 65 + (e & 63)] = vi[q];
  }
}

// Unit lower (upper = false) or upper triangle; for c >= n the column of the
// identity (a block of n < 64 rows embedded in the identity).
__device__ __forceinline__ void tri64_inv_column(int n, const float* Tr, const float* Ti, bool upper,
                                                 int c, int lane, float& x0r, float& x0i,
                                                 float& x1r, float& x1i) {
  x0r = (lane == c) ? 1.f : 0.f;
  x1r = (lane + 32 == c) ? 1.f : 0.f;
  x0i = x1i = 0.f;
  if (c >= n) return;
  if (!upper) {
    for (int p = c; p + 1 < n; ++p) {  // rows above c stay zero
      const float pr = __shfl_sync(0xffffffffu, p < 32 ? x0r : x1r, p & 31);
      const float pi = __shfl_sync(0xffffffffu, p < 32 ? x0i : x1i, p & 31);
      const float l0r = Tr[p * 65 + lane], l0i = Ti[p * 65 + lane];
      const float l1r = Tr[p * 65 + lane + 32], l1i = Ti[p * 65 + lane + 32];
      x0r = fmaf(-l0r, pr, fmaf(l0i, pi, x0r));
      x0i = fmaf(-l0r, pi, fmaf(-l0i, pr, x0i));
      x1r = fmaf(-l1r, pr, fmaf(l1i, pi, x1r));
      x1i = fmaf(-l1r, pi, fmaf(-l1i, pr, x1i));
    }
    return;
  }
  for (int p = c; p >= 0; --p) {  // rows below c stay zero
    // the owner of row p divides by the diagonal, then everyone subtracts
    const bool own0 = (lane == p), own1 = (lane + 32 == p);
    if (own0 || own1) {
      const float dr = Tr[p * 65 + p], di = Ti[p * 65 + p];
      const float den = dr * dr + di * di;
      const float xr = own0 ? x0r : x1r, xi = own0 ? x0i : x1i;
      const float qr = (xr * dr + xi * di) / den, qi = (xi * dr - xr * di) / den;
      if (own0) {
        x0r = qr;
        x0i = qi;
      } else {
        x1r = qr;
        x1i = qi;
      }
    }
    const float pr = __shfl_sync(0xffffffffu, p < 32 ? x0r : x1r, p & 31);
    const float pi = __shfl_sync(0xffffffffu, p < 32 ? x0i : x1i, p & 31);
    const float u0r = (lane < p) ? Tr[p * 65 + lane] : 0.f;
    const float u0i = (lane < p) ? Ti[p * 65 + lane] : 0.f;
    const float u1r = (lane + 32 < p) ? Tr[p * 65 + lane + 32] : 0.f;
    const float u1i = (lane + 32 < p) ? Ti[p * 65 + lane + 32] : 0.f;
    x0r = fmaf(-u0r, pr, fmaf(u0i, pi, x0r));
    x0i = fmaf(-u0r, pi, fmaf(-u0i, pr, x0i));
    x1r = fmaf(-u1r, pr, fmaf(u1i, pi, x1r));
    x1i = fmaf(-u1r, pi, fmaf(-u1i, pr, x1i));
  }
}

// FP32 inverses of the 64 x 64 diagonal blocks of the unit-lower L (z = 0)
// and the upper U (z = 1) of an LU: block b = blockIdx.x, its columns
// 8 blockIdx.y .. + 7 (a warp each); a last block of n < 64 rows is embedded
// in the identity. Output by blocks of 64 x 64, column-major.
__global__ void __launch_bounds__(256) diag_inv_f32_kernel(int N, CView<float> A, float* lre,
                                                           float* lim, float* ure, float* uim) {
  __shared__ float Tr[64 * 65], Ti[64 * 65];
  const int b = blockIdx.x, upper = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = min(64, N - 64 * b);
  tri64_load(n, A.sub(64L * b, 64L * b), upper, Tr, Ti, tid);
  __syncthreads();
  const int c = blockIdx.y * 8 + warp;
  float x0r, x0i, x1r, x1i;
  tri64_inv_column(n, Tr, Ti, upper, c, lane, x0r, x0i, x1r, x1i);
  float* ore = (upper ? ure : lre) + (size_t)b * 4096 + (size_t)c * 64;
  float* oim = (upper ? uim : lim) + (size_t)b * 4096 + (size_t)c * 64;
  ore[lane] = x0r;
  oim[lane] = x0i;
  ore[lane + 32] = x1r;
  oim[lane + 32] = x1i;
}

// The inverse of one triangle block T (n <= 64 rows; unit lower or upper)
// into the n x n block O, transposed when trans_out; 8 CTAs of 8 warps.
__global__ void __launch_bounds__(256) tri64_inv_kernel(int n, CView<float> T, int upper,
                                                        CView<float> O, int trans_out) {
  __shared__ float Tr[64 * 65], Ti[64 * 65];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  tri64_load(n, T, upper, Tr, Ti, tid);
  __syncthreads();
  const int c = blockIdx.x * 8 + warp;
  if (c >= n) return;
  float x0r, x0i, x1r, x1i;
  tri64_inv_column(n, Tr, Ti, upper, c, lane, x0r, x0i, x1r, x1i);
  if (lane < n) {
    const long o = trans_out ? c * O.rs + lane * O.cs : lane * O.rs + c * O.cs;
    O.re[o] = x0r;
    O.im[o] = x0i;
  }
  if (lane + 32 < n) {
    const long o = trans_out ? c * O.rs + (lane + 32) * O.cs : (lane + 32) * O.rs + c * O.cs;
    O.re[o] = x1r;
    O.im[o] = x1i;
  }
}

template <typename R>
int diag_inverses(int N, CView<R> A, R* lre, R* lim, R* ure, R* uim, cudaStream_t st) {
  const int nblk = (N + kTrsmLeaf - 1) / kTrsmLeaf;
  const long bs = (long)kTrsmLeaf * kTrsmLeaf;
  if constexpr (std::is_same<R, float>::value) {
    static_assert(kTrsmLeaf == 64, "diagonal blocks of 64");
    ProfScope ps(HARP_K_TRSM, 8.0 * kTrsmLeaf * (double)kTrsmLeaf * kTrsmLeaf * nblk, st);
    diag_inv_f32_kernel<<<dim3(nblk, 8, 2), 256, 0, st>>>(N, A, lre, lim, ure, uim);
    HARP_LAUNCHED();
    return HARP_OK;
  }
  {
    ProfScope ps(HARP_K_OTHER, 0.0, st);
    identity_blocks_kernel<R><<<dim3(1, nblk), 256, 0, st>>>(lre, lim, nblk);
    HARP_LAUNCHED();
    identity_blocks_kernel<R><<<dim3(1, nblk), 256, 0, st>>>(ure, uim, nblk);
    HARP_LAUNCHED();
  }
  dim3 block(kTrsmLeaf, kTrsmCols);
  dim3 grid(kTrsmLeaf / kTrsmCols, nblk);
  const size_t smem = sizeof(R) * (2 * kTrsmLeaf * (kTrsmLeaf + 1) + 4 * kTrsmLeaf * kTrsmCols);
  const long tstep = (long)kTrsmLeaf * (A.rs + A.cs);
  HARP_CUDA(cudaFuncSetAttribute(trsm_leaf_kernel<R, true, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  HARP_CUDA(cudaFuncSetAttribute(trsm_leaf_kernel<R, false, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope ps(HARP_K_TRSM, 8.0 * kTrsmLeaf * (double)kTrsmLeaf * kTrsmLeaf * nblk, st);
  trsm_leaf_kernel<R, true, true><<<grid, block, smem, st>>>(
      kTrsmLeaf, kTrsmLeaf, A, planes<R>(lre, lim, kTrsmLeaf), N, tstep, bs);
  HARP_LAUNCHED();
  trsm_leaf_kernel<R, false, false><<<grid, block, smem, st>>>(
      kTrsmLeaf, kTrsmLeaf, A, planes<R>(ure, uim, kTrsmLeaf), N, tstep, bs);
  HARP_LAUNCHED();
  return HARP_OK;
}

// B <- D B for an n x n (n <= 64) block D (any view) and B n x ncols, in
// place: the block and kTrsmCols columns of B are staged in shared memory.
template <typename R>
__global__ void __launch_bounds__(kTrsmLeaf* kTrsmCols) leaf_inv_kernel(int n, int ncols,
                                                                         CView<R> D, CView<R> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typedef R TRow[kTrsmLeaf + 1];
  typedef R BRow[kTrsmCols];
  TRow* Dr = reinterpret_cast<TRow*>(smem_raw);
  TRow* Di = Dr + kTrsmLeaf;
  BRow* Br = reinterpret_cast<BRow*>(Di + kTrsmLeaf);
  BRow* Bi = Br + kTrsmLeaf;
  const int i = threadIdx.x, c = threadIdx.y;
  const int col = blockIdx.x * kTrsmCols + c;
  const int tid = threadIdx.y * kTrsmLeaf + threadIdx.x;
  for (int e = tid; e < n * n; e += kTrsmLeaf * kTrsmCols) {
    const int r = e % n, k = e / n;
    Dr[r][k] = D.r(r, k);
    Di[r][k] = D.m(r, k);
  }
  const bool act = (i < n) && (col < ncols);
  Br[i][c] = act ? B.r(i, col) : (R)0;
  Bi[i][c] = act ? B.m(i, col) : (R)0;
  __syncthreads();
  R xr = 0, xi = 0;
  for (int k = 0; k < n; ++k) {
    const R dr = Dr[i][k], di = Di[i][k], br = Br[k][c], bi = Bi[k][c];
    xr = fma(dr, br, fma(-di, bi, xr));
    xi = fma(dr, bi, fma(di, br, xi));
  }
  if (act) {
    B.r(i, col) = xr;
    B.m(i, col) = xi;
  }
}

// T X = B for the effective triangle T of a solve (rows row0.. of the whole
// system), with the inverses of its 64-blocks (block b at dre/dim + b*4096,
// column-major 64 x 64; transposed when dtrans). Splits at multiples of 64
// so every leaf is a leading part of one block.
template <typename R>
static int trsm_inv(bool lower, int n, int ncols, CView<R> T, CView<R> B, int row0,
                    const R* dre, const R* dim, bool dtrans, int mode, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return HARP_OK;
  if (n <= kTrsmLeaf) {
    const long off = (long)(row0 / kTrsmLeaf) * kTrsmLeaf * kTrsmLeaf;
    CView<R> D = planes<R>(const_cast<R*>(dre) + off, const_cast<R*>(dim) + off, kTrsmLeaf);
    if (dtrans) D = D.t();
    dim3 block(kTrsmLeaf, kTrsmCols);
    dim3 grid((ncols + kTrsmCols - 1) / kTrsmCols);
    const size_t smem = sizeof(R) * (2 * kTrsmLeaf * (kTrsmLeaf + 1) + 2 * kTrsmLeaf * kTrsmCols);
    static bool attr_set = false;
    if (!attr_set) {
      HARP_CUDA(cudaFuncSetAttribute(leaf_inv_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
      attr_set = true;
    }
    ProfScope ps(HARP_K_TRSM, 8.0 * n * (double)n * ncols, st);
    leaf_inv_kernel<R><<<grid, block, smem, st>>>(n, ncols, D, B);
    HARP_LAUNCHED();
    return HARP_OK;
  }
  const int n1 = ((n / 2) + kTrsmLeaf - 1) / kTrsmLeaf * kTrsmLeaf;
  const int n2 = n - n1;
  CView<R> B1 = B, B2 = B.sub(n1, 0);
  if (lower) {
    HARP_TRY(trsm_inv<R>(true, n1, ncols, T, B1, row0, dre, dim, dtrans, mode, st));
    HARP_TRY(cgemm<R>(n2, ncols, n1, (R)-1, T.sub(n1, 0), B1, (R)1, B2, mode, st));
    HARP_TRY(trsm_inv<R>(true, n2, ncols, T.sub(n1, n1), B2, row0 + n1, dre, dim, dtrans, mode, st));
  } else {
    HARP_TRY(trsm_inv<R>(false, n2, ncols, T.sub(n1, n1), B2, row0 + n1, dre, dim, dtrans, mode, st));
    HARP_TRY(cgemm<R>(n1, ncols, n2, (R)-1, T.sub(0, n1), B2, (R)1, B1, mode, st));
    HARP_TRY(trsm_inv<R>(false, n1, ncols, T, B1, row0, dre, dim, dtrans, mode, st));
  }
  return HARP_OK;
}

// ---------------------------------------------------------------------------
// LU driver.
template <typename R>
static int leaf_width(const harp_ctx* ctx, int M, int want, int* use_smem) {
  const size_t budget = std::min<size_t>(ctx->smem_optin, kLeafSmem);
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
    ProfScope ps(HARP_K_PANEL, 4.0 * M * w * (double)(w - 1) + 6.0 * M * w, st);
    if (use_smem) {
      static bool attr_set = false;  // per instantiation
      if (!attr_set) {
        HARP_CUDA(cudaFuncSetAttribute(lu_leaf_kernel<R, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kLeafSmem));
        attr_set = true;
      }
      const size_t smem = (size_t)2 * M * w * sizeof(R);
      lu_leaf_kernel<R, true><<<1, kLeafThreads, smem, st>>>(re, im, ld, j0, M, w, ipiv, zero_col);
    } else {
      lu_leaf_kernel<R, false><<<1, kLeafThreads, 0, st>>>(re, im, ld, j0, M, w, ipiv, zero_col);
    }
    HARP_LAUNCHED();
    return HARP_OK;
  }
  const int w1 = w / 2, w2 = w - w1;
  HARP_TRY(panel<R>(ctx, N, A, re, im, ld, j0, w1, ipiv, zero_col, mode, st));
  HARP_TRY(laswp<R>(re, im, ld, N, ipiv, j0, j0 + w1, j0 + w1, j0 + w, 0, 0, nullptr, st));
  HARP_TRY(trsm<R>(true, true, w1, w2, A.sub(j0, j0), A.sub(j0, j0 + w1), mode, st));
  HARP_TRY(cgemm<R>(M - w1, w2, w1, (R)-1, A.sub(j0 + w1, j0), A.sub(j0, j0 + w1), (R)1,
                    A.sub(j0 + w1, j0 + w1), mode, st));
  HARP_TRY(panel<R>(ctx, N, A, re, im, ld, j0 + w1, w2, ipiv, zero_col, mode, st));
  HARP_TRY(laswp<R>(re, im, ld, N, ipiv, j0 + w1, j0 + w, j0, j0 + w1, 0, 0, nullptr, st));
  return HARP_OK;
}

// Cluster panels, FP32 only: partial pivoting (panel_cluster.cu) and
// tournament pivoting (panel_calu.cu).
int panel_cluster_plan(const harp_ctx* ctx, int M, int want_nb, int* csize, int* Mb);
int panel_cluster(const harp_ctx* ctx, float* re, float* im, long ld, int k0, int M, int nb,
                  int C, int Mb, int* ipiv, int* zero_col, cudaStream_t st, int* rmap);
int panel_calu_plan(const harp_ctx* ctx, int M, int want_nb, int* csize, int* Mb);
int panel_calu(const harp_ctx* ctx, float* re, float* im, long ld, int k0, int M, int nb, int C,
               int Mb, int* ipiv, int* zero_col, cudaStream_t st, int* rmap, int restricted = 0);
bool panel_block_plan(const harp_ctx* ctx, int M, int nb, int* csize, int* Mb);

// How the FP32 panel at M remaining rows is factored: kind 3 pivoting
// restricted to the diagonal block, 2 tournament cluster panel, 1
// partial-pivoting cluster panel, 0 the recursive panel; returns the width.
static int plan_panel_f32(const harp_ctx* ctx, int M, int want, int* kind, int* C, int* Mb) {
  if (ctx->pivot_mode == HARP_PIVOT_BLOCK && want % 16 == 0 && want <= 64 && M >= want &&
      ctx->blk_uinv) {
    *kind = 3;
    *C = 1;
    *Mb = want;
    return want;
  }
  if (ctx->pivot_mode == HARP_PIVOT_TOURNAMENT) {
    const int w = panel_calu_plan(ctx, M, want, C, Mb);
    if (w > 0) {
      *kind = 2;
      return w;
    }
  }
  const int w = panel_cluster_plan(ctx, M, want, C, Mb);
  if (w > 0) {
    *kind = 1;
    return w;
  }
  *kind = 0;
  return want;
}

// The panel at column k with pivoting restricted to its diagonal block
// (defined with the look-ahead kernels below).
static int panel_block_local(harp_ctx* ctx, int N, CView<float> A, float* re, float* im, long ld,
                             int k, int nb, int* ipiv, int* zero_col, cudaStream_t st, int* rmap);

// Factor the panel at column k (rows k..N); returns the width used in *nb.
// rmap (optional): where a cluster panel exports its row map; *mapped
// tells whether it did.
template <typename R>
static int factor_panel(harp_ctx* ctx, int N, CView<R> A, R* re, R* im, long ld, int k,
                        int want, int* ipiv, int* zero_col, int mode, cudaStream_t st, int* nb,
                        int* rmap = nullptr, bool* mapped = nullptr) {
  if (mapped) *mapped = false;
  if constexpr (std::is_same<R, float>::value) {
    // the plans only offer clusters that can be resident
    int kind = 0, C = 0, Mb = 0;
    const int w = plan_panel_f32(ctx, N - k, want, &kind, &C, &Mb);
    if (kind > 0) {
      *nb = w;
      if (mapped) *mapped = (rmap != nullptr);
      if (kind == 3) return panel_block_local(ctx, N, A, re, im, ld, k, w, ipiv, zero_col, st, rmap);
      if (kind == 2)
        return panel_calu(ctx, re, im, ld, k, N - k, w, C, Mb, ipiv, zero_col, st, rmap);
      return panel_cluster(ctx, re, im, ld, k, N - k, w, C, Mb, ipiv, zero_col, st, rmap);
    }
  }
  *nb = want;
  return panel<R>(ctx, N, A, re, im, ld, k, want, ipiv, zero_col, mode, st);
}

// ---------------------------------------------------------------------------
// The look-ahead update of the next panel's columns (at most 64 of them) by
// the current panel (width n <= 64): U12 = L11^-1 A12 in place, then
// A22 -= L21 U12. Both are latency-bound at these sizes, so each is one
// launch that stages everything it reads at once.

// U12 = L11^-1 A12, L11 unit lower: warp w of CTA b solves column 8 b + w,
// lane l holding rows l and l + 32; row p is final after step p and reaches
// the other lanes by shuffle. L11 by columns in shared memory (zeros on and
// above the diagonal).
__global__ void __launch_bounds__(256) la_trsm_kernel(int n, int ncols, const float* __restrict__ lre,
                                                      const float* __restrict__ lim, float* bre,
                                                      float* bim, long ld) {
  __shared__ float Lr[64 * 65], Li[64 * 65];  // [p][row], row stride 1, column stride 65
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = blockIdx.x * 8 + warp;
  const bool col = c < ncols;
  float* br = bre + (size_t)(col ? c : 0) * ld;
  float* bi = bim + (size_t)(col ? c : 0) * ld;
  // every load (the triangle and this warp's column) issued before any use
  float x0r = (col && lane < n) ? br[lane] : 0.f, x0i = (col && lane < n) ? bi[lane] : 0.f;
  float x1r = (col && lane + 32 < n) ? br[lane + 32] : 0.f;
  float x1i = (col && lane + 32 < n) ? bi[lane + 32] : 0.f;
  {
    float vr[16], vi[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = tid + 256 * q, p = e >> 6, row = e & 63;
      const bool in = row < n && p < n && row > p;
      vr[q] = in ? lre[row + (size_t)p * ld] : 0.f;
      vi[q] = in ? lim[row + (size_t)p * ld] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = tid + 256 * q, p = e >> 6, row = e & 63;
      Lr[p * 65 + row] = vr[q];
      Li[p * 65 + row] = vi[q];
    }
  }
  __syncthreads();
  if (!col) return;
  for (int p = 0; p + 1 < n; ++p) {
    const float pr = __shfl_sync(0xffffffffu, p < 32 ? x0r : x1r, p & 31);
    const float pi = __shfl_sync(0xffffffffu, p < 32 ? x0i : x1i, p & 31);
    const float l0r = Lr[p * 65 + lane], l0i = Li[p * 65 + lane];
    const float l1r = Lr[p * 65 + lane + 32], l1i = Li[p * 65 + lane + 32];
    x0r = fmaf(-l0r, pr, fmaf(l0i, pi, x0r));
    x0i = fmaf(-l0r, pi, fmaf(-l0i, pr, x0i));
    x1r = fmaf(-l1r, pr, fmaf(l1i, pi, x1r));
    x1i = fmaf(-l1r, pi, fmaf(-l1i, pr, x1i));
  }
  if (lane < n) {
    br[lane] = x0r;
    bi[lane] = x0i;
  }
  if (lane + 32 < n) {
    br[lane + 32] = x1r;
    bi[lane + 32] = x1i;
  }
}

// C -= A B (NEG) or C += A B for C M x ncols, A M x n, B n x ncols (n, ncols
// <= 64), column-major planes with leading dimensions lda, ldb, ldc (TA: A
// given by its transpose, element (r, k) at a[k + r lda]; ZC: C starts from
// zero instead of being read): 32 rows of C per CTA, lane l row l, warp w
// columns 8 w .. 8 w + 7; the CTA's rows of A and all of B are staged in
// shared memory by one round of loads, so C may be A itself (same rows).
template <bool TA, bool ZC, bool NEG = true>
__global__ void __launch_bounds__(256) la_gemm_kernel(int M, int n, int ncols,
                                                      const float* __restrict__ are,
                                                      const float* __restrict__ aim, long lda,
                                                      const float* __restrict__ bre,
                                                      const float* __restrict__ bim, long ldb,
                                                      float* cre, float* cim, long ldc) {
  __shared__ __align__(16) float Ar[64 * 32], Ai[64 * 32];  // [k][row]
  __shared__ __align__(16) float Br[64 * 64], Bi[64 * 64];  // [k][col]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = blockIdx.x * 32;
  const int row = i0 + lane, c0 = warp * 8;
  float accr[8], acci[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const bool in = !ZC && (row < M) && (c0 + j < ncols);
    accr[j] = in ? cre[row + (size_t)(c0 + j) * ldc] : 0.f;
    acci[j] = in ? cim[row + (size_t)(c0 + j) * ldc] : 0.f;
  }
  {
    float vr[8], vi[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q, r = e & 31, k = e >> 5;
      const bool in = (i0 + r < M) && (k < n);
      const size_t o = TA ? (size_t)k + (size_t)(i0 + r) * lda : (size_t)(i0 + r) + (size_t)k * lda;
      vr[q] = in ? are[o] : 0.f;
      vi[q] = in ? aim[o] : 0.f;
    }
    float wr[16], wi[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = tid + 256 * q, c = e & 63, k = e >> 6;
      const bool in = (k < n) && (c < ncols);
      wr[q] = in ? bre[k + (size_t)c * ldb] : 0.f;
      wi[q] = in ? bim[k + (size_t)c * ldb] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q;
      Ar[e] = vr[q];
      Ai[e] = vi[q];
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = tid + 256 * q;
      Br[e] = wr[q];
      Bi[e] = wi[q];
    }
  }
  __syncthreads();
#pragma unroll 4
  for (int k = 0; k < n; ++k) {
    const float ar = Ar[k * 32 + lane], ai = Ai[k * 32 + lane];
    const float4 b0r = *reinterpret_cast<const float4*>(&Br[k * 64 + c0]);
    const float4 b1r = *reinterpret_cast<const float4*>(&Br[k * 64 + c0 + 4]);
    const float4 b0i = *reinterpret_cast<const float4*>(&Bi[k * 64 + c0]);
    const float4 b1i = *reinterpret_cast<const float4*>(&Bi[k * 64 + c0 + 4]);
    const float bR[8] = {b0r.x, b0r.y, b0r.z, b0r.w, b1r.x, b1r.y, b1r.z, b1r.w};
    const float bI[8] = {b0i.x, b0i.y, b0i.z, b0i.w, b1i.x, b1i.y, b1i.z, b1i.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (NEG) {
        accr[j] = fmaf(-ar, bR[j], fmaf(ai, bI[j], accr[j]));
        acci[j] = fmaf(-ar, bI[j], fmaf(-ai, bR[j], acci[j]));
      } else {
        accr[j] = fmaf(ar, bR[j], fmaf(-ai, bI[j], accr[j]));
        acci[j] = fmaf(ar, bI[j], fmaf(ai, bR[j], acci[j]));
      }
    }
  }
  if (row < M) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (c0 + j < ncols) {
        cre[row + (size_t)(c0 + j) * ldc] = accr[j];
        cim[row + (size_t)(c0 + j) * ldc] = acci[j];
      }
  }
}

// The look-ahead update of columns [k1, k1 + nb1) by the panel at k (width
// nb): U12 = L11^-1 A12, A22 -= L21 U12 (planes, leading dimension ld).
static int lookahead_update(float* re, float* im, long ld, int N, int k, int nb, int k1, int nb1,
                            cudaStream_t st) {
  const size_t d = (size_t)k + (size_t)k * ld, u = (size_t)k + (size_t)k1 * ld;
  {
    ProfScope ps(HARP_K_TRSM, 4.0 * nb * (double)nb * nb1, st);
    la_trsm_kernel<<<(nb1 + 7) / 8, 256, 0, st>>>(nb, nb1, re + d, im + d, re + u, im + u, ld);
    HARP_LAUNCHED();
  }
  const int M = N - k1;
  if (M <= 0) return HARP_OK;
  const size_t l = (size_t)k1 + (size_t)k * ld, c = (size_t)k1 + (size_t)k1 * ld;
  ProfScope ps(HARP_K_TRSM, 8.0 * M * (double)nb1 * nb, st);
  la_gemm_kernel<false, false><<<(M + 31) / 32, 256, 0, st>>>(
      M, nb, nb1, re + l, im + l, ld, re + u, im + u, ld, re + c, im + c, ld);
  HARP_LAUNCHED();
  return HARP_OK;
}

// The panel at column k with pivoting restricted to its nb x nb diagonal
// block (the refinement's factors only; see HARP_PIVOT_BLOCK). Usually one
// cluster launch: CTA 0 pivots the block, every CTA eliminates its rows
// below against the block's U (the tournament kernel without its
// tournament). Panels too tall for one cluster: the block alone (one CTA),
// then L21 = A21 U11^-1 through the explicit inverse of U11 (one warp per
// column) and one CUDA-core product in place.
static int panel_block_local(harp_ctx* ctx, int N, CView<float> A, float* re, float* im, long ld,
                             int k, int nb, int* ipiv, int* zero_col, cudaStream_t st, int* rmap) {
  int C = 0, Mb = 0;
  if (panel_block_plan(ctx, N - k, nb, &C, &Mb))
    return panel_calu(ctx, re, im, ld, k, N - k, nb, C, Mb, ipiv, zero_col, st, rmap, 1);
  HARP_TRY(panel_calu(ctx, re, im, ld, k, nb, nb, 1, nb, ipiv, zero_col, st, rmap));
  const int M2 = N - k - nb;
  if (M2 <= 0) return HARP_OK;
  const CView<float> Ui = planes<float>(ctx->blk_uinv, ctx->blk_uinv + 64 * 64, 64);
  {
    ProfScope ps(HARP_K_TRSM, 8.0 * nb * (double)nb * nb, st);
    tri64_inv_kernel<<<(nb + 7) / 8, 256, 0, st>>>(nb, A.sub(k, k), 1, Ui, 0);
    HARP_LAUNCHED();
  }
  const CView<float> L = A.sub(k + nb, k);
  ProfScope ps(HARP_K_PANEL, 4.0 * M2 * (double)nb * nb, st);
  la_gemm_kernel<false, true, false><<<(M2 + 31) / 32, 256, 0, st>>>(
      M2, nb, nb, L.re, L.im, L.cs, Ui.re, Ui.im, 64, L.re, L.im, L.cs);
  HARP_LAUNCHED();
  return HARP_OK;
}

// The factor inverses built beside the look-ahead LU, one panel at a time,
// on ctx->inv_stream. X = U^-1 and V = (L^-1)^T = (L^T)^-1 are upper
// triangular; after the panel at k (width nb):
//   X[k:k+nb, k:k+nb] = U_kk^-1,
//   X[0:k, k:k+nb] = X[0:k, 0:k] (-U[0:k, k:k+nb] U_kk^-1),
// and V likewise from L^T, whose block column is row block k of L. Block
// column k of U is final once the panel is factored, and row block k of L
// once the panel's interchanges reached the L columns (later panels swap only
// rows below it). Each product takes X[0:k, 0:k] (V[0:k, 0:k]) from
// persistent TF32 split planes, to which every new block column is appended.
struct IncInverse {
  CView<float> T;  // planes of U^-1 (upper) or of (L^-1)^T
  CView<float> W;  // a k x 64 scratch (column-major, leading dimension ldw)
  float* sp;       // split planes of T (N rows, row stride Kp, plane stride N Kp)
  long Kp;
  size_t plane;
  bool lower;      // T is (L^-1)^T, built from the row blocks of L
  float* wa;       // tensor-core workspace of this chain
  size_t na;
  float* wb;
  size_t nbf;
};

static int inc_inverse_step(const IncInverse& I, CView<float> A, int k, int nb, int mode, int* err,
                            cudaStream_t s) {
  const CView<float> T = I.T;
  {
    ProfScope ps(HARP_K_TRSM, 8.0 * nb * (double)nb * nb, s);
    tri64_inv_kernel<<<(nb + 7) / 8, 256, 0, s>>>(nb, A.sub(k, k), I.lower ? 0 : 1, T.sub(k, k),
                                                   I.lower ? 1 : 0);
    HARP_LAUNCHED();
  }
  if (k > 0) {
    // W = -(U[0:k, k:k+nb] or L[k:k+nb, 0:k]^T) T[k:k+nb, k:k+nb]
    {
      ProfScope ps(HARP_K_TRSM, 8.0 * k * (double)nb * nb, s);
      const CView<float> D = T.sub(k, k);
      if (I.lower) {
        const CView<float> Lr = A.sub(k, 0);  // its transpose is the k x nb operand
        la_gemm_kernel<true, true><<<(k + 31) / 32, 256, 0, s>>>(
            k, nb, nb, Lr.re, Lr.im, Lr.cs, D.re, D.im, D.cs, I.W.re, I.W.im, I.W.cs);
      } else {
        const CView<float> Uc = A.sub(0, k);
        la_gemm_kernel<false, true><<<(k + 31) / 32, 256, 0, s>>>(
            k, nb, nb, Uc.re, Uc.im, Uc.cs, D.re, D.im, D.cs, I.W.re, I.W.im, I.W.cs);
      }
      HARP_LAUNCHED();
    }
    tc_set_workspace(I.wa, I.na, I.wb, I.nbf, err);
    int r = cgemm_tc_f32_asplit(k, nb, k, 1.f, I.sp, I.W, 0.f, T.sub(0, k), mode, s, I.Kp,
                                I.plane, true, 1);  // T[0:k, 0:k] upper triangular
    if (r == HARP_E_UNSUPPORTED) r = cgemm<float>(k, nb, k, 1.f, T, I.W, 0.f, T.sub(0, k), mode, s);
    HARP_TRY(r);
  }
  return tc_split_block(k + nb, nb, T.sub(0, k), I.sp + k, I.Kp, I.plane, mode, s);
}

// FP32 LU with a look-ahead of one panel. Main stream: the update of the
// next panel's columns by the current panel (row swaps, U12, CUDA-core
// GEMM), then the next panel's factorisation -- the critical path. Side
// stream: the rest of the current panel's update (row swaps of the other
// columns and of the permutation, U12 and the tensor-core GEMM of the far
// trailing matrix), which overlaps the next panel. Events order the two:
// the side stream starts a panel's update once that panel is factored, and
// the main stream touches columns of panel i+2 only after panel i's far
// update (which covers them) is done. The side stream and the inverse
// stream (the factor inverses, panel by panel, once a panel's far update is
// done) use separate halves of the tensor-core GEMM workspace.
static int lu_factor_lookahead(harp_ctx* ctx, int N, float* re, float* im, long ld, int* ipiv,
                               int* perm, int* zero_col, int mode, cudaStream_t st) {
  CView<float> A = planes<float>(re, im, ld);
  cudaStream_t s2 = ctx->side;
  float *wa = nullptr, *wb = nullptr;
  size_t na = 0, nbf = 0;
  int* werr = nullptr;
  tc_get_workspace(&wa, &na, &wb, &nbf, &werr);
  struct Restore {
    float *a, *b;
    size_t na, nb;
    int* e;
    ~Restore() { tc_set_workspace(a, na, b, nb, e); }
  } restore{wa, wb, na, nbf, werr};
  // the factor inverses beside the factorisation (L^-1 on one inverse
  // stream, U^-1 on the other), when the workspaces and streams are there;
  // the tensor-core workspace is split in three (side stream, two chains)
  ctx->finv_incremental = 0;
  cudaStream_t si[2] = {ctx->inv_stream[0], ctx->inv_stream[1]};
  bool inc = ctx->inv_beside && si[0] && si[1] && wa && wb && ctx->finv && ctx->finv_split &&
             ctx->finv_tmp;
  IncInverse I[2];
  // thirds rounded down to 256 bytes: each third is the base of TMA
  // tensor maps, which must be 16-byte aligned
  const size_t wa3 = (na / 3) & ~(size_t)63, wb3 = (nbf / 3) & ~(size_t)63;
  if (inc) {
    const size_t NN = (size_t)ctx->max_N * ctx->max_N;
    const long ldi = ctx->max_N;
    for (int c = 0; c < 2; ++c) {
      I[c].lower = (c == 0);
      I[c].T = planes<float>(ctx->finv + 2 * c * NN, ctx->finv + (2 * c + 1) * NN, ldi);
      // the scratch: 64 columns each, side by side
      I[c].W = planes<float>(ctx->finv_tmp + (size_t)c * 64 * ldi,
                             ctx->finv_tmp + NN + (size_t)c * 64 * ldi, ldi);
      I[c].Kp = (N + 31) / 32 * 32;
      I[c].plane = (size_t)N * I[c].Kp;
      I[c].sp = ctx->finv_split + c * ctx->finv_split_floats;
      I[c].wa = wa + (1 + c) * wa3;
      I[c].na = wa3;
      I[c].wb = wb + (1 + c) * wb3;
      I[c].nbf = wb3;
    }
    inc = (mode == GEMM_TC_3XTF32 ? 4 : 2) * I[0].plane <= ctx->finv_split_floats &&
          (size_t)128 * ldi <= NN;
  }
  if (inc) {
    // after the caller's earlier work: zero each inverse and its split
    const size_t NN = (size_t)ctx->max_N * ctx->max_N;
    const size_t np = (mode == GEMM_TC_3XTF32 ? 4 : 2) * I[0].plane;
    HARP_CUDA(cudaEventRecord(ctx->ev_inv[0], st));
    for (int c = 0; c < 2; ++c) {
      HARP_CUDA(cudaStreamWaitEvent(si[c], ctx->ev_inv[0], 0));
      HARP_CUDA(cudaMemsetAsync(ctx->finv + 2 * c * NN, 0, 2 * NN * sizeof(float), si[c]));
      HARP_CUDA(cudaMemsetAsync(I[c].sp, 0, np * sizeof(float), si[c]));
    }
  }
  std::vector<int> ks, nbs;
  std::vector<char> maps;  // panel i exported its row map to pmap(i)
  auto pmap = [&](int i) { return ctx->pmap + (size_t)i * kPmapInts; };
  int k = 0, nb = 0;
  bool mp = false;
  HARP_TRY(factor_panel<float>(ctx, N, A, re, im, ld, 0, std::min(kNB, N), ipiv, zero_col, mode,
                               st, &nb, pmap(0), &mp));
  ks.push_back(0);
  nbs.push_back(nb);
  maps.push_back(mp);
  for (int i = 0;; ++i) {
    if (i + 1 >= ctx->n_events) return HARP_E_UNSUPPORTED;
    k = ks[i];
    nb = nbs[i];
    const int k1 = k + nb;  // first column after panel i
    HARP_CUDA(cudaEventRecord(ctx->ev_fac[i], st));
    // main stream: update and factor panel i+1
    int nb1 = 0;
    if (k1 < N) {
      const int want = std::min(kNB, N - k1);
      // the width of panel i+1 is only known after planning; plan it now
      int kind = 0, C = 0, Mb = 0;
      nb1 = plan_panel_f32(ctx, N - k1, want, &kind, &C, &Mb);
      if (maps[i])
        HARP_TRY(laswp_map<float>(re, im, ld, pmap(i), k1, k1 + nb1, 0, 0, nullptr, st));
      else
        HARP_TRY(laswp<float>(re, im, ld, N, ipiv, k, k1, k1, k1 + nb1, 0, 0, nullptr, st));
      if (nb <= 64 && nb1 <= 64) {
        HARP_TRY(lookahead_update(re, im, ld, N, k, nb, k1, nb1, st));
      } else {
        HARP_TRY(trsm<float>(true, true, nb, nb1, A.sub(k, k), A.sub(k, k1), GEMM_SIMT, st));
        HARP_TRY(cgemm<float>(N - k1, nb1, nb, -1.f, A.sub(k1, k), A.sub(k, k1), 1.f,
                              A.sub(k1, k1), GEMM_SIMT, st));
      }
      int used = 0;
      HARP_TRY(factor_panel<float>(ctx, N, A, re, im, ld, k1, nb1, ipiv, zero_col, mode, st,
                                   &used, pmap(i + 1), &mp));
      nb1 = used;
      ks.push_back(k1);
      nbs.push_back(nb1);
      maps.push_back(mp);
    }
    // side stream: the rest of panel i's update
    const int k2 = k1 + nb1;  // first column past panel i+1
    HARP_CUDA(cudaStreamWaitEvent(s2, ctx->ev_fac[i], 0));
    if (maps[i])
      HARP_TRY(laswp_map<float>(re, im, ld, pmap(i), 0, k, k2, N, perm, s2));
    else
      HARP_TRY(laswp<float>(re, im, ld, N, ipiv, k, k1, 0, k, k2, N, perm, s2));
    if (k2 < N) {
      if (nb <= 64) {
        const size_t d = (size_t)k + (size_t)k * ld, u = (size_t)k + (size_t)k2 * ld;
        ProfScope ps(HARP_K_TRSM, 4.0 * nb * (double)nb * (N - k2), s2);
        la_trsm_kernel<<<(N - k2 + 7) / 8, 256, 0, s2>>>(nb, N - k2, re + d, im + d, re + u, im + u,
                                                         ld);
        HARP_LAUNCHED();
      } else {
        HARP_TRY(trsm<float>(true, true, nb, N - k2, A.sub(k, k), A.sub(k, k2), mode, s2));
      }
      if (inc) tc_set_workspace(wa, wa3, wb, wb3, werr);
      HARP_TRY(cgemm<float>(N - k1, N - k2, nb, -1.f, A.sub(k1, k), A.sub(k, k2), 1.f,
                            A.sub(k1, k2), mode, s2));
    }
    HARP_CUDA(cudaEventRecord(ctx->ev_big[i], s2));
    HARP_CUDA(cudaStreamWaitEvent(st, ctx->ev_big[i], 0));
    // inverse stream: panel i's block columns of the factor inverses (every
    // panel but the last must be kNB wide, so that the block columns stay
    // on the tensor cores' 32-wide K tiles)
    if (inc && (nb != kNB && k1 < N)) inc = false;
    if (inc) {
      for (int c = 0; c < 2; ++c) {
        HARP_CUDA(cudaStreamWaitEvent(si[c], ctx->ev_big[i], 0));
        HARP_TRY(inc_inverse_step(I[c], A, k, nb, mode, werr, si[c]));
      }
    }
    if (k1 >= N) break;
  }
  if (si[0] && si[1] && ctx->finv) {
    // the caller's stream continues once both inverse streams are done
    for (int c = 0; c < 2; ++c) {
      HARP_CUDA(cudaEventRecord(ctx->ev_inv[c], si[c]));
      HARP_CUDA(cudaStreamWaitEvent(st, ctx->ev_inv[c], 0));
    }
  }
  ctx->finv_incremental = inc ? 1 : 0;
  return HARP_OK;
}

template <typename R>
int lu_factor(harp_ctx* ctx, int N, R* re, R* im, long ld, int* ipiv, int* perm, int* zero_col,
              int mode, cudaStream_t st) {
  {
    ProfScope ps_o(HARP_K_OTHER, 0.0, st);
    iota_kernel<<<(N + 255) / 256, 256, 0, st>>>(perm, N);
    HARP_LAUNCHED();
  }
  if constexpr (std::is_same<R, float>::value) {
    if (ctx->side && mode != GEMM_SIMT) {
      if (!ctx->lu_stream || !ctx->lu_fork)
        return lu_factor_lookahead(ctx, N, re, im, ld, ipiv, perm, zero_col, mode, st);
      // the chain on the context's highest-priority stream, after the
      // caller's work and before anything the caller enqueues next
      HARP_CUDA(cudaEventRecord(ctx->ev_lu_fork, st));
      HARP_CUDA(cudaStreamWaitEvent(ctx->lu_stream, ctx->ev_lu_fork, 0));
      const int s =
          lu_factor_lookahead(ctx, N, re, im, ld, ipiv, perm, zero_col, mode, ctx->lu_stream);
      HARP_CUDA(cudaEventRecord(ctx->ev_lu_join, ctx->lu_stream));
      HARP_CUDA(cudaStreamWaitEvent(st, ctx->ev_lu_join, 0));
      return s;
    }
  }
  CView<R> A = planes<R>(re, im, ld);
  for (int k = 0, nb = 0; k < N; k += nb) {
    HARP_TRY(factor_panel<R>(ctx, N, A, re, im, ld, k, std::min(kNB, N - k), ipiv, zero_col, mode,
                             st, &nb));
    HARP_TRY(laswp<R>(re, im, ld, N, ipiv, k, k + nb, 0, k, k + nb, N, perm, st));
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

// ---------------------------------------------------------------------------
// Explicit inverses of the triangular factors (FP32 path), so that every
// solve of the refinement is two dense products. Recursive on 64-aligned
// halves: for lower T = [T11 0; T21 T22],
//   inv(T) = [inv(T11) 0; -inv(T22) T21 inv(T11)  inv(T22)],
// for upper T = [T11 T12; 0 T22],
//   inv(T) = [inv(T11)  -inv(T11) T12 inv(T22); 0 inv(T22)],
// the leaves being leading parts of the 64 x 64 block inverses.
template <typename R>
__global__ void copy_block_kernel(int n, const R* sre, const R* sim, long lds, R* dre, R* dim,
                                  long ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n || j >= n) return;
  dre[i + (size_t)j * ldd] = sre[i + (size_t)j * lds];
  dim[i + (size_t)j * ldd] = sim[i + (size_t)j * lds];
}

// The diagonal-block inverses (64 x 64 at dre + b * 4096, the last block
// possibly smaller) copied onto the diagonal of Ti: block b, column c.
template <typename R>
__global__ void copy_diag_blocks_kernel(int N, const R* __restrict__ dre,
                                        const R* __restrict__ dim, R* tre, R* tim, long ld) {
  const int b = blockIdx.x, c = blockIdx.y, r = threadIdx.x;
  const int nb = min(kTrsmLeaf, N - b * kTrsmLeaf);
  if (c >= nb || r >= nb) return;
  const size_t s = (size_t)b * kTrsmLeaf * kTrsmLeaf + r + (size_t)c * kTrsmLeaf;
  const size_t d = (size_t)b * kTrsmLeaf + r + ((size_t)b * kTrsmLeaf + c) * ld;
  tre[d] = dre[s];
  tim[d] = dim[s];
}

// Nodes of the halving recursion over a triangle of n rows at off: each
// splits into n1 (a multiple of the 64-row leaf) + n2; listed per depth in
// increasing offset.
static void inv_nodes(int off, int n, int depth, std::vector<std::vector<std::array<int, 3>>>& lv) {
  if (n <= kTrsmLeaf) return;
  const int n1 = ((n / 2) + kTrsmLeaf - 1) / kTrsmLeaf * kTrsmLeaf;
  const int n2 = n - n1;
  if ((int)lv.size() <= depth) lv.resize(depth + 1);
  lv[depth].push_back({off, n1, n2});
  inv_nodes(off, n1, depth + 1, lv);
  inv_nodes(off + n1, n2, depth + 1, lv);
}

// Ti = T^-1 for the unit-lower (lower) or upper triangle of T, bottom-up by
// depth: for a node [T11 0; T21 T22], inv21 = -inv(T22) (T21 inv(T11)); for
// [T11 T12; 0 T22], inv12 = -inv(T11) (T12 inv(T22)). The nodes of one depth
// with the same split and a constant offset step are one batched product
// (their blocks lie at a constant stride along the diagonal). tmp holds the
// intermediate product at the block's own position (strictly lower blocks
// for L, strictly upper for U, so both triangles can share it).
static int tri_inv(bool lower, int N, CView<float> T, CView<float> Ti, CView<float> tmp,
                   const float* dre, const float* dim, int mode, cudaStream_t st) {
  if (N <= 0) return HARP_OK;
  {
    ProfScope ps(HARP_K_OTHER, 0.0, st);
    const int nblk = (N + kTrsmLeaf - 1) / kTrsmLeaf;
    copy_diag_blocks_kernel<float><<<dim3(nblk, kTrsmLeaf), kTrsmLeaf, 0, st>>>(N, dre, dim, Ti.re,
                                                                                Ti.im, Ti.cs);
    HARP_LAUNCHED();
  }
  std::vector<std::vector<std::array<int, 3>>> lv;
  inv_nodes(0, N, 0, lv);
  for (int d = (int)lv.size() - 1; d >= 0; --d) {
    const auto& nodes = lv[d];
    size_t i = 0;
    while (i < nodes.size()) {
      const int off = nodes[i][0], n1 = nodes[i][1], n2 = nodes[i][2];
      size_t j = i + 1;
      long step = 0;
      if (j < nodes.size() && nodes[j][1] == n1 && nodes[j][2] == n2) {
        step = nodes[j][0] - off;
        ++j;
        while (j < nodes.size() && nodes[j][1] == n1 && nodes[j][2] == n2 &&
               nodes[j][0] - nodes[j - 1][0] == step)
          ++j;
      }
      const int cnt = (int)(j - i);
      auto so = [&](const CView<float>& v) { return step * (v.rs + v.cs); };
      if (lower) {
        HARP_TRY(cgemm_batched(n2, n1, n1, 1.f, T.sub(off + n1, off), so(T), Ti.sub(off, off),
                               so(Ti), 0.f, tmp.sub(off + n1, off), so(tmp), cnt, mode, st));
        HARP_TRY(cgemm_batched(n2, n1, n2, -1.f, Ti.sub(off + n1, off + n1), so(Ti),
                               tmp.sub(off + n1, off), so(tmp), 0.f, Ti.sub(off + n1, off), so(Ti),
                               cnt, mode, st));
      } else {
        HARP_TRY(cgemm_batched(n1, n2, n2, 1.f, T.sub(off, off + n1), so(T),
                               Ti.sub(off + n1, off + n1), so(Ti), 0.f, tmp.sub(off, off + n1),
                               so(tmp), cnt, mode, st));
        HARP_TRY(cgemm_batched(n1, n2, n1, -1.f, Ti.sub(off, off), so(Ti), tmp.sub(off, off + n1),
                               so(tmp), 0.f, Ti.sub(off, off + n1), so(Ti), cnt, mode, st));
      }
      i = j;
    }
  }
  return HARP_OK;
}

int factor_inverses(int N, CView<float> A, const float* dinv_re, const float* dinv_im,
                    float* linv_re, float* linv_im, float* uinv_re, float* uinv_im, long ldi,
                    float* tre, float* tim, int mode, cudaStream_t st, cudaStream_t side,
                    cudaEvent_t fork, cudaEvent_t join) {
  const long nblk = (N + kTrsmLeaf - 1) / kTrsmLeaf;
  const long bs = (long)kTrsmLeaf * kTrsmLeaf;
  for (float* p : {linv_re, linv_im, uinv_re, uinv_im})
    HARP_CUDA(cudaMemsetAsync(p, 0, sizeof(float) * (size_t)ldi * N, st));
  CView<float> tmp = planes<float>(tre, tim, ldi);
  if (!side) {
    HARP_TRY(tri_inv(true, N, A, planes<float>(linv_re, linv_im, ldi), tmp, dinv_re, dinv_im,
                     mode, st));
    return tri_inv(false, N, A, planes<float>(uinv_re, uinv_im, ldi), tmp, dinv_re + nblk * bs,
                   dinv_im + nblk * bs, mode, st);
  }
  // L^-1 on st and U^-1 on the side stream, each with half of the
  // tensor-core operand workspace (the largest product, a half-size block,
  // needs a quarter of it).
  float *wa, *wb;
  size_t na, nb;
  int* err;
  tc_get_workspace(&wa, &na, &wb, &nb, &err);
  HARP_CUDA(cudaEventRecord(fork, st));
  HARP_CUDA(cudaStreamWaitEvent(side, fork, 0));
  tc_set_workspace(wa, na / 2, wb, nb / 2, err);
  int s1 = tri_inv(true, N, A, planes<float>(linv_re, linv_im, ldi), tmp, dinv_re, dinv_im, mode,
                   st);
  tc_set_workspace(wa ? wa + na / 2 : nullptr, na / 2, wb ? wb + nb / 2 : nullptr, nb / 2, err);
  int s2 = (s1 == HARP_OK)
               ? tri_inv(false, N, A, planes<float>(uinv_re, uinv_im, ldi), tmp,
                         dinv_re + nblk * bs, dinv_im + nblk * bs, mode, side)
               : HARP_OK;
  tc_set_workspace(wa, na, wb, nb, err);
  // join even after an error, so that st never runs ahead of queued side work
  HARP_CUDA(cudaEventRecord(join, side));
  HARP_CUDA(cudaStreamWaitEvent(st, join, 0));
  return s1 != HARP_OK ? s1 : s2;
}

// Solve op(A) X = B with the explicit factor inverses: two dense products
// and the row permutation. B (N x nrhs planes, ld ldb) is overwritten; tmp
// has room for N x nrhs.
template <typename R>
int lu_solve_inv(int N, int nrhs, CView<R> Li, CView<R> Ui, const int* perm, R* bre, R* bim,
                 long ldb, R* tre, R* tim, char trans, int mode, cudaStream_t st,
                 const float* li_split, const float* ui_split) {
  CView<R> Bm = planes<R>(bre, bim, ldb), Tm = planes<R>(tre, tim, ldb);
  dim3 grid((N + 255) / 256, nrhs);
  if (trans == 'N' || trans == 'n') {
    {
      ProfScope ps(HARP_K_OTHER, 0.0, st);
      permute_rows_kernel<R><<<grid, 256, 0, st>>>(N, nrhs, perm, bre, bim, tre, tim, ldb, 0);
      HARP_LAUNCHED();
    }
    // B = L^-1 P b, T = U^-1 B (the inverses pre-split when given)
    int s1 = HARP_E_UNSUPPORTED, s2 = HARP_E_UNSUPPORTED;
    if constexpr (std::is_same<R, float>::value)
      if (li_split)  // L^-1 is lower triangular: each row tile skips its zero k-tiles
        s1 = cgemm_tc_f32_asplit(N, nrhs, N, 1.f, li_split, Tm, 0.f, Bm, mode, st, 0, 0, true, 2);
    if (s1 == HARP_E_UNSUPPORTED) s1 = cgemm<R>(N, nrhs, N, (R)1, Li, Tm, (R)0, Bm, mode, st);
    HARP_TRY(s1);
    if constexpr (std::is_same<R, float>::value)
      if (ui_split)  // and U^-1 upper triangular
        s2 = cgemm_tc_f32_asplit(N, nrhs, N, 1.f, ui_split, Bm, 0.f, Tm, mode, st, 0, 0, true, 1);
    if (s2 == HARP_E_UNSUPPORTED) s2 = cgemm<R>(N, nrhs, N, (R)1, Ui, Bm, (R)0, Tm, mode, st);
    HARP_TRY(s2);
    HARP_TRY(planes_to_planes<R, R>(N, nrhs, tre, tim, ldb, bre, bim, ldb, st));
  } else {
    HARP_TRY(cgemm<R>(N, nrhs, N, (R)1, Ui.t(), Bm, (R)0, Tm, mode, st));  // T = U^-T b
    HARP_TRY(cgemm<R>(N, nrhs, N, (R)1, Li.t(), Tm, (R)0, Bm, mode, st));  // B = L^-T T
    {
      ProfScope ps(HARP_K_OTHER, 0.0, st);
      permute_rows_kernel<R><<<grid, 256, 0, st>>>(N, nrhs, perm, bre, bim, tre, tim, ldb, 1);
      HARP_LAUNCHED();
    }
    HARP_TRY(planes_to_planes<R, R>(N, nrhs, tre, tim, ldb, bre, bim, ldb, st));
  }
  return HARP_OK;
}

template <typename R>
int lu_solve(int N, int nrhs, R* lre, R* lim, long ld, const int* perm, R* bre, R* bim, long ldb,
             R* tre, R* tim, char trans, const R* dinv_re, const R* dinv_im, int mode,
             cudaStream_t st) {
  CView<R> L = planes<R>(lre, lim, ld);
  const long nblk = (N + kTrsmLeaf - 1) / kTrsmLeaf;
  const R* linv_r = dinv_re;
  const R* linv_i = dinv_im;
  const R* uinv_r = dinv_re + nblk * kTrsmLeaf * kTrsmLeaf;
  const R* uinv_i = dinv_im + nblk * kTrsmLeaf * kTrsmLeaf;
  dim3 grid((N + 255) / 256, nrhs);
  if (trans == 'N' || trans == 'n') {
    {
      ProfScope ps(HARP_K_OTHER, 0.0, st);
      permute_rows_kernel<R><<<grid, 256, 0, st>>>(N, nrhs, perm, bre, bim, tre, tim, ldb, 0);
      HARP_LAUNCHED();
    }
    CView<R> Tm = planes<R>(tre, tim, ldb);
    HARP_TRY(trsm_inv<R>(true, N, nrhs, L, Tm, 0, linv_r, linv_i, false, mode, st));
    HARP_TRY(trsm_inv<R>(false, N, nrhs, L, Tm, 0, uinv_r, uinv_i, false, mode, st));
    HARP_TRY(planes_to_planes<R, R>(N, nrhs, tre, tim, ldb, bre, bim, ldb, st));
  } else {
    CView<R> Bm = planes<R>(bre, bim, ldb);
    // U^T y = b (lower), then L^T z = y (upper): inverses are the transposes
    HARP_TRY(trsm_inv<R>(true, N, nrhs, L.t(), Bm, 0, uinv_r, uinv_i, true, mode, st));
    HARP_TRY(trsm_inv<R>(false, N, nrhs, L.t(), Bm, 0, linv_r, linv_i, true, mode, st));
    {
      ProfScope ps(HARP_K_OTHER, 0.0, st);
      permute_rows_kernel<R><<<grid, 256, 0, st>>>(N, nrhs, perm, bre, bim, tre, tim, ldb, 1);
      HARP_LAUNCHED();
    }
    HARP_TRY(planes_to_planes<R, R>(N, nrhs, tre, tim, ldb, bre, bim, ldb, st));
  }
  return HARP_OK;
}

// ---------------------------------------------------------------------------
// Conversions, RHS, norms.
template <typename Rin, typename Rout>
__global__ void i2p_kernel(int M, int N, const Rin* src, long lds, Rout* re, Rout* im, long ldd,
                           int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= M) return;
  const Rin* s = src + 2 * ((size_t)i + (size_t)j * lds);
  const Rin a = s[0], b = s[1];
  re[i + (size_t)j * ldd] = (Rout)a;
  im[i + (size_t)j * ldd] = (Rout)b;
  if (flag && !(isfinite(a) && isfinite(b))) atomicOr(flag, ST_NONFINITE);
}
template <typename Rin, typename Rout>
int interleaved_to_planes(int M, int N, const Rin* src, long lds, Rout* re, Rout* im, long ldd,
                          cudaStream_t st, int* nonfinite_flag) {
  if (M <= 0 || N <= 0) return HARP_OK;
  dim3 grid((M + 255) / 256, N);
  ProfScope ps_o(HARP_K_OTHER, 0.0, st);
  i2p_kernel<Rin, Rout><<<grid, 256, 0, st>>>(M, N, src, lds, re, im, ldd, nonfinite_flag);
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
                             float*, float*, char, const float*, const float*, int, cudaStream_t);
template int lu_solve<double>(int, int, double*, double*, long, const int*, double*, double*, long,
                              double*, double*, char, const double*, const double*, int,
                              cudaStream_t);
template int diag_inverses<float>(int, CView<float>, float*, float*, float*, float*, cudaStream_t);
template int lu_solve_inv<float>(int, int, CView<float>, CView<float>, const int*, float*, float*,
                                 long, float*, float*, char, int, cudaStream_t, const float*,
                                 const float*);
template int diag_inverses<double>(int, CView<double>, double*, double*, double*, double*,
                                   cudaStream_t);
template int interleaved_to_planes<float, float>(int, int, const float*, long, float*, float*, long,
                                                 cudaStream_t, int*);
template int interleaved_to_planes<double, double>(int, int, const double*, long, double*, double*,
                                                   long, cudaStream_t, int*);
template int interleaved_to_planes<double, float>(int, int, const double*, long, float*, float*,
                                                  long, cudaStream_t, int*);
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
