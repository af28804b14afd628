// resid.cu -- FP64-accurate refinement residual R = V - Z X on the FP32 pipe.
//
// GB300 runs FP64 FMAs at 1/64 of the FP32 rate, so the residual of the
// mixed-precision refinement is formed with error-free transformations on
// the FP32 pipe (each FP64 operand split as hi + lo, hi = fl32(x),
// lo = fl32(x - hi)):
//   product   a*b ~ p + e,  p = ah*bh, e = fma(ah,bh,-p) + ah*bl + al*bh
//             (Dekker's exact product via FMA plus the first-order cross
//             terms; the dropped al*bl and the roundings in e are ~2^-48 |p|);
//   sum       a three-float accumulator (S, s1, s2): S += p by Knuth's
//             TwoSum; its exact error t and the product error e are each
//             added to s1 by TwoSum, and those errors go to s2.
// Every rounding left is relative to a single term (~2^-48), not to the
// running sum, so the result is as accurate as an FP64 dot product, which
// is what limits the accuracy the refinement can reach.
//
// Also here: the hi/lo splits, and the norms of the stopping test
// (LAPACK zcgesv style: per column max |r|, max |x| with |z| = |re| + |im|,
// and the matrix infinity norm of Z from its hi part).
#include <algorithm>
#include <cmath>

#include "dense.cuh"
#include "ff.cuh"
#include "prof.cuh"

namespace harp {

constexpr int kRBM = 64, kRBN = 32, kRBK = 16;

// R[i, c] = V[i, c] - sum_k A[i, k] X[k, c]; A as 4 float planes (hi/lo of
// re/im, element (i,k) at i*ars + k*acs), X as 4 float planes (ld ldx).
// With split-K (gridDim.z > 1) each z-slice sums its own K range and writes
// its FP64 partial to P[z] (no V); resid_combine_kernel then forms V - sum.
// FFF selects the three-float accumulator (FP64-accurate); otherwise the
// double-float one (for updates R - Z D with a small correction D).
template <bool FFF>
__global__ void __launch_bounds__(256) resid_ff_kernel(
    int N, int nrhs, const float* __restrict__ Ahr, const float* __restrict__ Ahi,
    const float* __restrict__ Alr, const float* __restrict__ Ali, long ars, long acs,
    const float* __restrict__ Bhr, const float* __restrict__ Bhi, const float* __restrict__ Blr,
    const float* __restrict__ Bli, long ldb, const double* __restrict__ Vr,
    const double* __restrict__ Vi, double* __restrict__ Rr, double* __restrict__ Ri, long ldr,
    int kchunk, double* __restrict__ Pr, double* __restrict__ Pi, long pstride) {
  __shared__ __align__(16) float As[4][kRBK][kRBM];
  __shared__ __align__(16) float Bs[4][kRBK][kRBN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * kRBM, j0 = blockIdx.x * kRBN;
  // outputs: rows ty*4 + a (a < 4), cols tx*2 + b (b < 2); three-float
  // accumulators for the real and imaginary parts
  float Sr[4][2], s1r[4][2], s2r[4][2], Si[4][2], s1i[4][2], s2i[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) Sr[a][b] = s1r[a][b] = s2r[a][b] = Si[a][b] = s1i[a][b] = s2i[a][b] = 0.f;
  const float* Ap[4] = {Ahr, Ahi, Alr, Ali};
  const float* Bp[4] = {Bhr, Bhi, Blr, Bli};
  const int kbeg = blockIdx.z * kchunk, kend = min(N, kbeg + kchunk);
  for (int k0 = kbeg; k0 < kend; k0 += kRBK) {
    // A tile: kRBM x kRBK per plane (1024 elements, 4 per thread per plane)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = threadIdx.x + 256 * l;
      // lanes run along the contiguous dimension of A (rows, or k when A is
      // a transposed view)
      const int i = (acs == 1) ? e / kRBK : e % kRBM;
      const int kk = (acs == 1) ? e % kRBK : e / kRBM;
      const bool in = (i0 + i < N) && (k0 + kk < kend);
      const long off = (long)(i0 + i) * ars + (long)(k0 + kk) * acs;
#pragma unroll
      for (int q = 0; q < 4; ++q) As[q][kk][i] = in ? Ap[q][off] : 0.f;
    }
    // B tile: kRBK x kRBN per plane (512 elements, 2 per thread per plane)
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const int e = threadIdx.x + 256 * l;
      const int kk = e % kRBK, j = e / kRBK;
      const bool in = (k0 + kk < kend) && (j0 + j < nrhs);
      const long off = (long)(k0 + kk) + (long)(j0 + j) * ldb;
#pragma unroll
      for (int q = 0; q < 4; ++q) Bs[q][kk][j] = in ? Bp[q][off] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kRBK; ++kk) {
      const float4 ahr = *reinterpret_cast<const float4*>(&As[0][kk][ty * 4]);
      const float4 ahi = *reinterpret_cast<const float4*>(&As[1][kk][ty * 4]);
      const float4 alr = *reinterpret_cast<const float4*>(&As[2][kk][ty * 4]);
      const float4 ali = *reinterpret_cast<const float4*>(&As[3][kk][ty * 4]);
      const float2 bhr = *reinterpret_cast<const float2*>(&Bs[0][kk][tx * 2]);
      const float2 bhi = *reinterpret_cast<const float2*>(&Bs[1][kk][tx * 2]);
      const float2 blr = *reinterpret_cast<const float2*>(&Bs[2][kk][tx * 2]);
      const float2 bli = *reinterpret_cast<const float2*>(&Bs[3][kk][tx * 2]);
      const float ar_h[4] = {ahr.x, ahr.y, ahr.z, ahr.w}, ai_h[4] = {ahi.x, ahi.y, ahi.z, ahi.w};
      const float ar_l[4] = {alr.x, alr.y, alr.z, alr.w}, ai_l[4] = {ali.x, ali.y, ali.z, ali.w};
      const float br_h[2] = {bhr.x, bhr.y}, bi_h[2] = {bhi.x, bhi.y};
      const float br_l[2] = {blr.x, blr.y}, bi_l[2] = {bli.x, bli.y};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          // re += ar*br - ai*bi ; im += ar*bi + ai*br
          if (FFF) {
            fff_mac(Sr[a][b], s1r[a][b], s2r[a][b], ar_h[a], ar_l[a], br_h[b], br_l[b]);
            fff_mac(Sr[a][b], s1r[a][b], s2r[a][b], -ai_h[a], -ai_l[a], bi_h[b], bi_l[b]);
            fff_mac(Si[a][b], s1i[a][b], s2i[a][b], ar_h[a], ar_l[a], bi_h[b], bi_l[b]);
            fff_mac(Si[a][b], s1i[a][b], s2i[a][b], ai_h[a], ai_l[a], br_h[b], br_l[b]);
          } else {
            ff2_mac(Sr[a][b], s1r[a][b], ar_h[a], ar_l[a], br_h[b], br_l[b]);
            ff2_mac(Sr[a][b], s1r[a][b], -ai_h[a], -ai_l[a], bi_h[b], bi_l[b]);
            ff2_mac(Si[a][b], s1i[a][b], ar_h[a], ar_l[a], bi_h[b], bi_l[b]);
            ff2_mac(Si[a][b], s1i[a][b], ai_h[a], ai_l[a], br_h[b], br_l[b]);
          }
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty * 4 + a;
    if (i >= N) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int j = j0 + tx * 2 + b;
      if (j >= nrhs) continue;
      const long o = (long)i + (long)j * ldr;
      const double dr = (double)Sr[a][b] + ((double)s1r[a][b] + (double)s2r[a][b]);
      const double di = (double)Si[a][b] + ((double)s1i[a][b] + (double)s2i[a][b]);
      if (gridDim.z == 1) {
        Rr[o] = Vr[o] - dr;
        Ri[o] = Vi[o] - di;
      } else {
        Pr[blockIdx.z * pstride + o] = dr;
        Pi[blockIdx.z * pstride + o] = di;
      }
    }
  }
}

// Interleaved c128 (M x N, ld) -> hi/lo float planes (ld ldp).
__global__ void split_c128_kernel(int M, int N, const double2* __restrict__ Z, long ldz,
                                  float* hr, float* hi, float* lr, float* li, long ldp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= M) return;
  const double2 z = Z[(size_t)i + (size_t)j * ldz];
  float a, b;
  const size_t o = (size_t)i + (size_t)j * ldp;
  ff_split(z.x, a, b);
  hr[o] = a;
  lr[o] = b;
  ff_split(z.y, a, b);
  hi[o] = a;
  li[o] = b;
}

// FP64 planes (M x N, ld) -> hi/lo float planes (same ld).
__global__ void split_planes_kernel(int M, int N, const double* __restrict__ xr,
                                    const double* __restrict__ xi, long ld, float* hr, float* hi,
                                    float* lr, float* li) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= M) return;
  const size_t o = (size_t)i + (size_t)j * ld;
  float a, b;
  ff_split(xr[o], a, b);
  hr[o] = a;
  lr[o] = b;
  ff_split(xi[o], a, b);
  hi[o] = a;
  li[o] = b;
}

// FP32 planes (M x N, ld) -> hi/lo float planes: hi = value, lo = 0.
__global__ void split_f32_planes_kernel(int M, int N, const float* __restrict__ xr,
                                        const float* __restrict__ xi, long ld, float* hr,
                                        float* hi, float* lr, float* li) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= M) return;
  const size_t o = (size_t)i + (size_t)j * ld;
  hr[o] = xr[o];
  hi[o] = xi[o];
  lr[o] = 0.f;
  li[o] = 0.f;
}

// Per-column max of |re| + |im| of FP32 planes -> colmax[j] (zeroed before).
__global__ void colmax_cabs1_f32_kernel(int M, int N, const float* __restrict__ xr,
                                        const float* __restrict__ xi, long ld, double* colmax) {
  const int j = blockIdx.y;
  float m = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const size_t o = (size_t)i + (size_t)j * ld;
    const float v = fabsf(xr[o]) + fabsf(xi[o]);
    m = (v == v) ? fmaxf(m, v) : __int_as_float(0x7f800000);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(colmax + j),
              (unsigned long long)__double_as_longlong((double)m));
}

// Per-column max of |re| + |im| over FP64 planes -> colmax[j] (zeroed before).
__global__ void colmax_cabs1_kernel(int M, int N, const double* __restrict__ xr,
                                    const double* __restrict__ xi, long ld, double* colmax) {
  const int j = blockIdx.y;
  float m = 0.f;  // FP32 magnitude is ample for a stopping test
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const size_t o = (size_t)i + (size_t)j * ld;
    const float v = fabsf((float)xr[o]) + fabsf((float)xi[o]);
    m = (v == v) ? fmaxf(m, v) : __int_as_float(0x7f800000);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(colmax + j),
              (unsigned long long)__double_as_longlong((double)m));
}

// Row sums of |re| + |im| of float planes (M x N): atomics into rowsum (zeroed).
__global__ void rowsum_cabs1_kernel(int M, int N, const float* __restrict__ re,
                                    const float* __restrict__ im, long rs, long cs,
                                    float* rowsum) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = blockIdx.y * 64;
  if (i >= M) return;
  float s = 0.f;
  const int j1 = min(N, j0 + 64);
  for (int j = j0; j < j1; ++j) {
    const size_t o = (size_t)i * rs + (size_t)j * cs;
    s += fabsf(re[o]) + fabsf(im[o]);
  }
  atomicAdd(rowsum + i, s);
}

__global__ void max_floats_kernel(int n, const float* __restrict__ v, double* out) {
  float m = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, v[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
    if (threadIdx.x == 0) *out = (double)m;
  }
}

int split_c128(int M, int N, const double* Z, long ldz, float* const hl[4], long ldp,
               cudaStream_t st) {
  dim3 grid((M + 255) / 256, N);
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  split_c128_kernel<<<grid, 256, 0, st>>>(M, N, reinterpret_cast<const double2*>(Z), ldz, hl[0],
                                          hl[1], hl[2], hl[3], ldp);
  HARP_LAUNCHED();
  return HARP_OK;
}

int split_planes(int M, int N, const double* xr, const double* xi, long ld, float* const hl[4],
                 cudaStream_t st) {
  dim3 grid((M + 255) / 256, N);
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  split_planes_kernel<<<grid, 256, 0, st>>>(M, N, xr, xi, ld, hl[0], hl[1], hl[2], hl[3]);
  HARP_LAUNCHED();
  return HARP_OK;
}

// R = V - sum_z P[z], the slices added in a fixed order in FP64.
__global__ void resid_combine_kernel(int N, int nrhs, int nz, const double* __restrict__ Pr,
                                     const double* __restrict__ Pi, long pstride,
                                     const double* __restrict__ Vr, const double* __restrict__ Vi,
                                     double* __restrict__ Rr, double* __restrict__ Ri, long ld) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= N) return;
  const long o = (long)i + (long)j * ld;
  double sr = 0.0, si = 0.0;
  for (int z = 0; z < nz; ++z) {
    sr += Pr[z * pstride + o];
    si += Pi[z * pstride + o];
  }
  Rr[o] = Vr[o] - sr;
  Ri[o] = Vi[o] - si;
}

int residual_ff(int N, int nrhs, const float* const A[4], long ars, long acs,
                const float* const B[4], long ldb, const double* vr, const double* vi, double* rr,
                double* ri, long ldr, double* pr, double* pi, int max_split, int num_sms,
                cudaStream_t st, bool fff) {
  const int tiles = ((nrhs + kRBN - 1) / kRBN) * ((N + kRBM - 1) / kRBM);
  // split K so that the CTAs (two resident per SM) fill whole waves
  const double slots = 2.0 * num_sms;
  int ks = 1;
  double best = 0.0;
  for (int k = 1; k <= max_split; ++k) {
    if ((long)k * kRBK > N) break;
    const double waves = tiles * k / slots;
    const double eff = waves / std::ceil(waves);
    if (eff > best + 0.02) {
      best = eff;
      ks = k;
    }
  }
  int kchunk = (N + ks - 1) / ks;
  kchunk = (kchunk + kRBK - 1) / kRBK * kRBK;
  ks = (N + kchunk - 1) / kchunk;
  dim3 grid((nrhs + kRBN - 1) / kRBN, (N + kRBM - 1) / kRBM, ks);
  const long pstride = (long)ldr * nrhs;
  {
    ProfScope ps(fff ? HARP_K_RESIDUAL : HARP_K_RESID_UPDATE, 8.0 * N * (double)N * nrhs, st);
    auto kern = fff ? resid_ff_kernel<true> : resid_ff_kernel<false>;
    kern<<<grid, 256, 0, st>>>(N, nrhs, A[0], A[1], A[2], A[3], ars, acs, B[0], B[1], B[2], B[3],
                               ldb, vr, vi, rr, ri, ldr, kchunk, pr, pi, pstride);
    HARP_LAUNCHED();
  }
  if (ks > 1) {
    ProfScope ps(HARP_K_OTHER, 0.0, st);
    resid_combine_kernel<<<dim3((N + 255) / 256, nrhs), 256, 0, st>>>(N, nrhs, ks, pr, pi, pstride,
                                                                      vr, vi, rr, ri, ldr);
    HARP_LAUNCHED();
  }
  return HARP_OK;
}

int colmax_cabs1(int M, int N, const double* xr, const double* xi, long ld, double* colmax,
                 cudaStream_t st) {
  HARP_CUDA(cudaMemsetAsync(colmax, 0, sizeof(double) * N, st));
  dim3 grid(std::min(16, (M + 255) / 256), N);
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  colmax_cabs1_kernel<<<grid, 256, 0, st>>>(M, N, xr, xi, ld, colmax);
  HARP_LAUNCHED();
  return HARP_OK;
}

int split_f32_planes(int M, int N, const float* xr, const float* xi, long ld, float* const hl[4],
                     cudaStream_t st) {
  dim3 grid((M + 255) / 256, N);
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  split_f32_planes_kernel<<<grid, 256, 0, st>>>(M, N, xr, xi, ld, hl[0], hl[1], hl[2], hl[3]);
  HARP_LAUNCHED();
  return HARP_OK;
}

int colmax_cabs1_f32(int M, int N, const float* xr, const float* xi, long ld, double* colmax,
                     cudaStream_t st) {
  HARP_CUDA(cudaMemsetAsync(colmax, 0, sizeof(double) * N, st));
  dim3 grid(std::min(16, (M + 255) / 256), N);
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  colmax_cabs1_f32_kernel<<<grid, 256, 0, st>>>(M, N, xr, xi, ld, colmax);
  HARP_LAUNCHED();
  return HARP_OK;
}

int norm_inf_planes_f32(int M, int N, const float* re, const float* im, long rs, long cs,
                        float* rowsum, double* out, cudaStream_t st) {
  HARP_CUDA(cudaMemsetAsync(rowsum, 0, sizeof(float) * M, st));
  dim3 grid((M + 255) / 256, (N + 63) / 64);
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  rowsum_cabs1_kernel<<<grid, 256, 0, st>>>(M, N, re, im, rs, cs, rowsum);
  HARP_LAUNCHED();
  max_floats_kernel<<<1, 1024, 0, st>>>(M, rowsum, out);
  HARP_LAUNCHED();
  return HARP_OK;
}

}  // namespace harp
