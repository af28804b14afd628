// ri.cu -- the reduced matrix under a radius of influence (Section II-D,
// Section IV-A): interactions are kept only between antennas closer than
// RI, so the matrix is block sparse. The structure is a block-CSR list of
// the kept blocks of every block row (the diagonal block always, the
// columns in increasing order); the values are the blocks of Eq. 3 and 4
// (and the self blocks), computed for the kept pairs only. The solve runs
// on the matrix scattered into dense storage (zeros outside RI), through
// the dense LU; RI -> infinity gives back the full matrix.
//
// The pair test r^2 < RI^2 uses plain IEEE FP64 with every product and sum
// rounded separately (no fused multiply-add), so that the kept pairs are
// reproducible bit for bit.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace harp {

constexpr double kPiR = 3.14159265358979323846;
constexpr double kC0R = 299792458.0;
constexpr int kRiThreads = 128;

__device__ __forceinline__ bool ri_keep(const double* pos, int m, int n, double R2) {
  if (m == n) return true;
  const double dx = __dsub_rn(pos[2 * m], pos[2 * n]);
  const double dy = __dsub_rn(pos[2 * m + 1], pos[2 * n + 1]);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < R2;
}

// Kept blocks of block row m (one thread per row): the count, or the
// columns at row_ptr[m] in increasing order.
__global__ void ri_rows_kernel(int Na, const double* __restrict__ pos, double R2, int count,
                               long* __restrict__ cnt, const long* __restrict__ row_ptr,
                               int* __restrict__ col_idx) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= Na) return;
  long c = 0;
  for (int n = 0; n < Na; ++n)
    if (ri_keep(pos, m, n, R2)) {
      if (!count) col_idx[row_ptr[m] + c] = n;
      ++c;
    }
  if (count) cnt[m] = c;
}

// One CTA per kept block (m, n): the self block, or Eq. 3 in Eq. 4 with the
// basis e^{-jkr} e^{j p alpha} d^q formed once per pair (FP64 geometry and
// phase, powers by repeated multiplication) and contracted with the
// coefficients in the precision R. Values: block b column-major Nm x Nm.
template <typename R>
__global__ void __launch_bounds__(kRiThreads) ri_fill_kernel(
    int Na, int Nm, int P, int Q, const double* __restrict__ pos, double k,
    const double2* __restrict__ coef, const double2* __restrict__ sb, long self_stride,
    const long* __restrict__ row_ptr, const int* __restrict__ col_idx,
    cplx_t<R>* __restrict__ vals, int* flag) {
  using C = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char ri_raw[];
  C* phi = reinterpret_cast<C*>(ri_raw);  // [K]
  __shared__ int s_m;
  const long b = blockIdx.x;
  const int nq = Q + 1, K = (2 * P + 1) * nq, nm2 = Nm * Nm;
  if (threadIdx.x == 0) {  // block row: the last m with row_ptr[m] <= b
    int lo = 0, hi = Na - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (row_ptr[mid] <= b) lo = mid;
      else hi = mid - 1;
    }
    s_m = lo;
  }
  __syncthreads();
  const int m = s_m, n = col_idx[b];
  C* out = vals + (size_t)b * nm2;
  if (m == n) {
    for (int e = threadIdx.x; e < nm2; e += kRiThreads) {
      const double2 v = sb[(size_t)m * self_stride + e];
      out[e] = mk<R>((R)v.x, (R)v.y);
    }
    return;
  }
  const double dx = pos[2 * m] - pos[2 * n], dy = pos[2 * m + 1] - pos[2 * n + 1];
  const double r = hypot(dx, dy);
  const bool coincident = (r == 0.0);
  if (threadIdx.x == 0) {
    if (coincident) {
      for (int kk = 0; kk < K; ++kk) phi[kk] = mk<R>(0, 0);
      atomicOr(flag, ST_COINCIDENT);
    } else {
      const double d = 1.0 / r;
      double s, c;
      sincos(k * r, &s, &c);
      const C ph = mk<R>((R)c, (R)(-s));            // e^{-jkr}
      const C z = mk<R>((R)(dx * d), (R)(dy * d));  // e^{j alpha}
      const R dR = (R)d;
      C zp = mk<R>(1, 0);
      for (int p = 0; p <= P; ++p) {
        const C bp = cmul(ph, zp), bn = cmul(ph, cconj(zp));
        R dq = 1;
        for (int q = 0; q <= Q; ++q) {
          phi[(P + p) * nq + q] = mk<R>(bp.x * dq, bp.y * dq);
          if (p > 0) phi[(P - p) * nq + q] = mk<R>(bn.x * dq, bn.y * dq);
          dq *= dR;
        }
        zp = cmul(zp, z);
      }
    }
  }
  __syncthreads();
  bool bad = false;
  for (int e = threadIdx.x; e < nm2; e += kRiThreads) {
    const int T = e % Nm, S = e / Nm;  // column-major block entry (T, S)
    const double2* cc = coef + ((size_t)T * Nm + S) * K;
    C acc = mk<R>(0, 0);
    for (int kk = 0; kk < K; ++kk) {
      const double2 cv = cc[kk];
      cfma(acc, mk<R>((R)cv.x, (R)cv.y), phi[kk]);
    }
    bad |= !(isfinite(acc.x) && isfinite(acc.y));
    out[e] = acc;
  }
  if (bad) atomicOr(flag, ST_NONFINITE);
}

// Dense column-major storage of a block-sparse matrix: a zeroing pass,
// then one CTA per kept block writing its entries.
template <typename C>
__global__ void ri_zero_kernel(long N, C* Z, long ldz) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    C z;
    z.x = 0;
    z.y = 0;
    Z[i + (size_t)blockIdx.y * ldz] = z;
  }
}

template <typename C>
__global__ void ri_scatter_kernel(int Na, int Nm, const long* __restrict__ row_ptr,
                                  const int* __restrict__ col_idx, const C* __restrict__ vals,
                                  C* Z, long ldz) {
  __shared__ int s_m;
  const long b = blockIdx.x;
  if (threadIdx.x == 0) {
    int lo = 0, hi = Na - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (row_ptr[mid] <= b) lo = mid;
      else hi = mid - 1;
    }
    s_m = lo;
  }
  __syncthreads();
  const int m = s_m, n = col_idx[b], nm2 = Nm * Nm;
  for (int e = threadIdx.x; e < nm2; e += blockDim.x) {
    const int T = e % Nm, S = e / Nm;
    Z[(size_t)m * Nm + T + ((size_t)n * Nm + S) * ldz] = vals[(size_t)b * nm2 + e];
  }
}

}  // namespace harp

using namespace harp;

extern "C" int harp_ri_pairs(int Na, const double* pos, double RI, long cap, long* row_ptr,
                             int* col_idx, long* nnzb, void* stream) {
  if (Na < 1) return -1;
  if (!pos) return -2;
  if (!(RI >= 0.0)) return -3;
  if (cap < 0) return -4;
  if (!row_ptr) return -5;
  if (!col_idx) return -6;
  if (!nnzb) return -7;
  cudaStream_t st = (cudaStream_t)stream;
  const double R2 = RI * RI;
  long* cnt = nullptr;
  HARP_CUDA(cudaMallocAsync(&cnt, sizeof(long) * (size_t)Na, st));
  struct Free {
    long* p;
    cudaStream_t s;
    ~Free() { cudaFreeAsync(p, s); }
  } f{cnt, st};
  ri_rows_kernel<<<(Na + 127) / 128, 128, 0, st>>>(Na, pos, R2, 1, cnt, nullptr, nullptr);
  HARP_LAUNCHED();
  std::vector<long> h(Na), rp(Na + 1, 0);
  HARP_CUDA(cudaMemcpyAsync(h.data(), cnt, sizeof(long) * (size_t)Na, cudaMemcpyDeviceToHost, st));
  HARP_CUDA(cudaStreamSynchronize(st));
  for (int m = 0; m < Na; ++m) rp[m + 1] = rp[m] + h[m];
  *nnzb = rp[Na];
  if (rp[Na] > cap || rp[Na] > 2147483647L) return HARP_E_UNSUPPORTED;
  HARP_CUDA(cudaMemcpyAsync(row_ptr, rp.data(), sizeof(long) * (Na + 1), cudaMemcpyHostToDevice, st));
  ri_rows_kernel<<<(Na + 127) / 128, 128, 0, st>>>(Na, pos, R2, 0, nullptr, row_ptr, col_idx);
  HARP_LAUNCHED();
  HARP_CUDA(cudaStreamSynchronize(st));
  return HARP_OK;
}

extern "C" int harp_ri_fill(int Na, int Nm, int P, int Q, const double* pos, double freq_hz,
                            const double* coef, const double* self_blocks, long self_stride,
                            const long* row_ptr, const int* col_idx, long nnzb, void* values,
                            int prec, int* flag, void* stream) {
  if (Na < 1) return -1;
  if (Nm < 1) return -2;
  if (P < 0 || P > 64) return -3;
  if (Q < 0 || Q > 64) return -4;
  if (!pos) return -5;
  if (!(freq_hz > 0.0) || freq_hz > 1e15) return -6;
  if (!coef) return -7;
  if (!self_blocks) return -8;
  if (self_stride < 0) return -9;
  if (!row_ptr) return -10;
  if (!col_idx) return -11;
  if (nnzb < Na || nnzb > 2147483647L) return -12;
  if (!values) return -13;
  if (prec != HARP_FP64 && prec != HARP_MIXED_3XTF32 && prec != HARP_MIXED_TF32 && prec != HARP_FP32)
    return -14;
  if (!flag) return -15;
  cudaStream_t st = (cudaStream_t)stream;
  const int K = (2 * P + 1) * (Q + 1);
  const double k = 2.0 * kPiR * freq_hz / kC0R;
  const double2* c = reinterpret_cast<const double2*>(coef);
  const double2* s = reinterpret_cast<const double2*>(self_blocks);
  ProfScope ps(HARP_K_FILL, 8.0 * Nm * (double)Nm * K * (double)(nnzb - Na), st);
  if (prec == HARP_FP64) {
    const size_t smem = (size_t)K * sizeof(double2);
    if (smem > 200 * 1024) return HARP_E_UNSUPPORTED;
    HARP_CUDA(cudaFuncSetAttribute(ri_fill_kernel<double>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ri_fill_kernel<double><<<(unsigned)nnzb, kRiThreads, smem, st>>>(
        Na, Nm, P, Q, pos, k, c, s, self_stride, row_ptr, col_idx,
        static_cast<double2*>(values), flag);
  } else {
    const size_t smem = (size_t)K * sizeof(float2);
    HARP_CUDA(cudaFuncSetAttribute(ri_fill_kernel<float>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ri_fill_kernel<float><<<(unsigned)nnzb, kRiThreads, smem, st>>>(
        Na, Nm, P, Q, pos, k, c, s, self_stride, row_ptr, col_idx, static_cast<float2*>(values),
        flag);
  }
  HARP_LAUNCHED();
  return HARP_OK;
}

extern "C" int harp_bsr_to_dense(int Na, int Nm, const long* row_ptr, const int* col_idx,
                                 long nnzb, const void* values, int prec, void* Z, int ldz,
                                 void* stream) {
  if (Na < 1) return -1;
  if (Nm < 1) return -2;
  if (!row_ptr) return -3;
  if (!col_idx) return -4;
  if (nnzb < 1 || nnzb > 2147483647L) return -5;
  if (!values) return -6;
  if (prec != HARP_FP64 && prec != HARP_MIXED_3XTF32 && prec != HARP_MIXED_TF32 && prec != HARP_FP32)
    return -7;
  if (!Z) return -8;
  const long N = (long)Na * Nm;
  if (ldz < N) return -9;
  if (N > 65535) return HARP_E_UNSUPPORTED;  // one grid row per dense column
  cudaStream_t st = (cudaStream_t)stream;
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  const dim3 gz((unsigned)((N + 255) / 256), (unsigned)N);
  if (prec == HARP_FP64) {
    ri_zero_kernel<double2><<<gz, 256, 0, st>>>(N, static_cast<double2*>(Z), ldz);
    HARP_LAUNCHED();
    ri_scatter_kernel<double2><<<(unsigned)nnzb, 128, 0, st>>>(
        Na, Nm, row_ptr, col_idx, static_cast<const double2*>(values), static_cast<double2*>(Z),
        ldz);
  } else {
    ri_zero_kernel<float2><<<gz, 256, 0, st>>>(N, static_cast<float2*>(Z), ldz);
    HARP_LAUNCHED();
    ri_scatter_kernel<float2><<<(unsigned)nnzb, 128, 0, st>>>(
        Na, Nm, row_ptr, col_idx, static_cast<const float2*>(values), static_cast<float2*>(Z),
        ldz);
  }
  HARP_LAUNCHED();
  return HARP_OK;
}
