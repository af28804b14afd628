// model.cu -- HARP model construction (Section II-A, Eq. 2-3; Section II-B
// for the sampling grid and the DFT): the coefficients c_pq of
//   B_TS(d, alpha) = sum_{p=-P..P} e^{j p alpha} sum_{q=0..Q} c_pq^{TS} d^q
// from samples of B on a polar grid regular in alpha (alpha_a = 2 pi a /
// N_alpha) and in d = 1/r (caller's d_l). For every MBF pair (one CTA each):
//   1. the DFT over alpha gives the radial samples of each harmonic,
//        b_p(d_l) = (1 / N_alpha) sum_a B(d_l, alpha_a) e^{-j p alpha_a}
//      (exact for a model band-limited to |p| <= P when N_alpha >= 2P + 1);
//   2. a least-squares polynomial in d fits each harmonic: c_p = R^-1 Q^T
//      b_p with V = QR the thin QR factorisation of the Vandermonde matrix
//      V[l, q] = d_l^q (modified Gram-Schmidt, each column orthogonalised
//      twice), so the fit does not square V's condition number;
//   3. the root-mean-square residual of the fitted model on the samples.
// Everything in FP64: the samples are few (Nd x N_alpha per pair) and the
// Vandermonde matrix is ill conditioned.
#include <cmath>

#include "common.cuh"
#include "prof.cuh"

namespace harp {

constexpr int kModelThreads = 128;
constexpr int kModelMaxQ1 = 16;  // Q + 1

// Dynamic shared memory: the pair's samples (Nd x Na c128), the harmonic
// samples b (Nd x np c128), the Q factor (Nd x nq) and R (nq x nq), a
// reduction buffer.
static size_t model_smem(int Nd, int Na, int np, int nq) {
  return sizeof(double2) * ((size_t)Nd * Na + (size_t)Nd * np) +
         sizeof(double) * ((size_t)Nd * nq + (size_t)nq * nq + kModelThreads);
}

__global__ void __launch_bounds__(kModelThreads) model_fit_kernel(
    int Nm, int P, int Q, int Nd, int Na, const double* __restrict__ dv,
    const double2* __restrict__ B, double2* __restrict__ coef, double* __restrict__ rms) {
  extern __shared__ __align__(16) unsigned char model_raw[];
  const int np = 2 * P + 1, nq = Q + 1;
  double2* Bs = reinterpret_cast<double2*>(model_raw);  // [l][a]
  double2* bs = Bs + (size_t)Nd * Na;                    // [l][p]
  double* Qf = reinterpret_cast<double*>(bs + (size_t)Nd * np);  // [q][l]
  double* Rf = Qf + (size_t)nq * Nd;                              // [i][q]
  double* red = Rf + nq * nq;
  const int ts = blockIdx.x, tid = threadIdx.x;
  const double2* Bp = B + (size_t)ts * Nd * Na;
  for (int e = tid; e < Nd * Na; e += kModelThreads) Bs[e] = Bp[e];
  // thin QR of V (warp 0): column q starts as d^q, is orthogonalised twice
  // against the earlier columns, then normalised
  if (tid < 32) {
    const int lane = tid;
    for (int e = lane; e < nq * nq; e += 32) Rf[e] = 0.0;
    __syncwarp();
    for (int q = 0; q < nq; ++q) {
      for (int l = lane; l < Nd; l += 32) Qf[q * Nd + l] = pow(dv[l], (double)q);
      __syncwarp();
      for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < q; ++i) {
          double s = 0.0;
          for (int l = lane; l < Nd; l += 32) s += Qf[i * Nd + l] * Qf[q * Nd + l];
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
          for (int l = lane; l < Nd; l += 32) Qf[q * Nd + l] -= s * Qf[i * Nd + l];
          if (lane == 0) Rf[i * nq + q] += s;
          __syncwarp();
        }
      double s = 0.0;
      for (int l = lane; l < Nd; l += 32) s += Qf[q * Nd + l] * Qf[q * Nd + l];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      const double nrm = sqrt(s);
      const double inv = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      for (int l = lane; l < Nd; l += 32) Qf[q * Nd + l] *= inv;
      if (lane == 0) Rf[q * nq + q] = nrm;
      __syncwarp();
    }
  }
  __syncthreads();
  // DFT over alpha: e^{-j p alpha_a} = cos, -sin of pi (2 ((p a) mod Na) / Na)
  for (int e = tid; e < Nd * np; e += kModelThreads) {
    const int l = e / np, pi = e - l * np, p = pi - P;
    double sr = 0.0, si = 0.0;
    for (int a = 0; a < Na; ++a) {
      const int m = (int)((((long)p * a) % Na + Na) % Na);
      double s, c;
      sincospi(2.0 * m / Na, &s, &c);
      const double2 v = Bs[l * Na + a];
      sr += v.x * c + v.y * s;  // v e^{-j theta}
      si += v.y * c - v.x * s;
    }
    bs[l * np + pi] = make_double2(sr / Na, si / Na);
  }
  __syncthreads();
  // c_p = R^-1 Q^T b_p, one thread per harmonic
  double2* cout = coef + (size_t)ts * np * nq;
  for (int pi = tid; pi < np; pi += kModelThreads) {
    double2 y[kModelMaxQ1];
    for (int q = 0; q < nq; ++q) {
      double yr = 0.0, yi = 0.0;
      for (int l = 0; l < Nd; ++l) {
        const double qv = Qf[q * Nd + l];
        yr += qv * bs[l * np + pi].x;
        yi += qv * bs[l * np + pi].y;
      }
      y[q] = make_double2(yr, yi);
    }
    for (int q = nq - 1; q >= 0; --q) {
      double yr = y[q].x, yi = y[q].y;
      for (int i = q + 1; i < nq; ++i) {
        yr -= Rf[q * nq + i] * y[i].x;
        yi -= Rf[q * nq + i] * y[i].y;
      }
      const double rq = Rf[q * nq + q];
      y[q] = (rq != 0.0) ? make_double2(yr / rq, yi / rq) : make_double2(0.0, 0.0);
    }
    for (int q = 0; q < nq; ++q) cout[pi * nq + q] = y[q];
  }
  __syncthreads();
  if (!rms) return;
  // the fitted model at every sample against the sample
  double acc = 0.0;
  for (int e = tid; e < Nd * Na; e += kModelThreads) {
    const int l = e / Na, a = e - l * Na;
    double mr = 0.0, mi = 0.0;
    for (int pi = 0; pi < np; ++pi) {
      double wr = 0.0, wi = 0.0, dq = 1.0;
      for (int q = 0; q < nq; ++q) {
        wr += cout[pi * nq + q].x * dq;
        wi += cout[pi * nq + q].y * dq;
        dq *= dv[l];
      }
      const int m = (int)((((long)(pi - P) * a) % Na + Na) % Na);
      double s, c;
      sincospi(2.0 * m / Na, &s, &c);
      mr += wr * c - wi * s;
      mi += wr * s + wi * c;
    }
    const double2 v = Bs[e];
    acc += (v.x - mr) * (v.x - mr) + (v.y - mi) * (v.y - mi);
  }
  red[tid] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int i = 0; i < kModelThreads; ++i) t += red[i];
    rms[ts] = sqrt(t / ((double)Nd * Na));
  }
}

}  // namespace harp

using namespace harp;

extern "C" int harp_model_fit(int Nm, int P, int Q, int Nd, int Nalpha, const double* d,
                              const double* B, double* coef, double* rms, void* stream) {
  if (Nm < 1) return -1;
  if (P < 0 || P > 64) return -2;
  if (Q < 0) return -3;
  if (Nd < Q + 1) return -4;
  if (Nalpha < 2 * P + 1) return -5;
  if (!d) return -6;
  if (!B) return -7;
  if (!coef) return -8;
  if (Q + 1 > kModelMaxQ1) return HARP_E_UNSUPPORTED;
  if ((long)Nm * Nm > 2147483647L) return HARP_E_UNSUPPORTED;
  const size_t smem = model_smem(Nd, Nalpha, 2 * P + 1, Q + 1);
  int dev = 0, optin = 0;
  HARP_CUDA(cudaGetDevice(&dev));
  HARP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)optin) return HARP_E_UNSUPPORTED;
  HARP_CUDA(cudaFuncSetAttribute(model_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  cudaStream_t st = (cudaStream_t)stream;
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  model_fit_kernel<<<Nm * Nm, kModelThreads, smem, st>>>(
      Nm, P, Q, Nd, Nalpha, d, reinterpret_cast<const double2*>(B),
      reinterpret_cast<double2*>(coef), rms);
  HARP_LAUNCHED();
  return HARP_OK;
}
