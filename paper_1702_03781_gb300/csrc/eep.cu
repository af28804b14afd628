// eep.cu -- embedded element patterns of every port (Section II-C, Eq. 5
// and 6) and the pattern error of Eq. 8.
//
// For the currents X of the port excitations (column m of X: the MBF
// coefficients c_ij = X[i*Nm + j, m] for excitation at port m) the pattern
// of port m in direction u is Eq. 5 with the sums swapped as in Eq. 6:
//   E_m(u) = sum_j F_j(u) AF_jm(u),   AF_jm(u) = sum_i X[i*Nm + j, m] e^{jk u.x_i},
// u.x_i = u_x x_i + u_y y_i (planar array). The array factors of all MBFs
// and ports form one dense contraction over the antennas,
//   AF[d, (j, m)] = sum_i A[d, i] B[i, (j, m)],   A[d, i] = e^{jk u_d.x_i},
// which runs on the tensor cores (three-term TF32 products, FP32
// accumulation: FP32-level accuracy over the Na-term sums) against the
// phase matrix A, generated for a chunk of directions at a time. The
// patterns F_j then weight the array factors of each port and direction:
// Nm complex products per output, a pass over AF at memory speed.
#include <algorithm>
#include <cmath>

#include "dense.cuh"
#include "prof.cuh"

namespace harp {

constexpr double kPiE = 3.14159265358979323846;
constexpr double kC0E = 299792458.0;

// A[d, i] = e^{j k (ux_d x_i + uy_d y_i)} as FP32 planes (Dc x Na, column-
// major, ld Dc). The phase (up to a few hundred radians) is formed and
// reduced to a fraction of a turn in FP64; sin and cos of pi times twice
// that fraction are then taken in FP32, so each entry carries FP32-level
// error whatever the size of the array.
__global__ void eep_phase_kernel(int Dc, int Na, const double* __restrict__ ux,
                                 const double* __restrict__ uy, const double* __restrict__ pos,
                                 double k, float* __restrict__ are, float* __restrict__ aim) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (d >= Dc) return;
  const double ph = k * (ux[d] * pos[2 * i] + uy[d] * pos[2 * i + 1]);
  double t = ph * (1.0 / (2.0 * kPiE));  // turns
  t -= rint(t);                           // in [-1/2, 1/2]
  float s, c;
  sincospif((float)(2.0 * t), &s, &c);
  are[d + (size_t)Dc * i] = c;
  aim[d + (size_t)Dc * i] = s;
}

// B[i, j + Nm m] = X[i Nm + j, m]: the currents by MBF (FP32 planes, Na x
// Nm nports, ld Na).
__global__ void eep_currents_kernel(int Na, int Nm, const double2* __restrict__ X, long ldx,
                                    float* __restrict__ bre, float* __restrict__ bim) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int col = blockIdx.y, m = col / Nm, j = col - m * Nm;
  if (i >= Na) return;
  const double2 v = X[(size_t)i * Nm + j + (size_t)m * ldx];
  bre[i + (size_t)Na * col] = (float)v.x;
  bim[i + (size_t)Na * col] = (float)v.y;
}

// E[c, m, d0 + d] = sum_j F[c, d0 + d, j] AF[d, j + Nm m] for the chunk of
// directions d0 .. d0 + Dc - 1 (c = 0 theta, 1 phi).
__global__ void eep_combine_kernel(int Dc, int d0, int D, int Nm, int nports,
                                   const float* __restrict__ afr, const float* __restrict__ afi,
                                   const double2* __restrict__ F, float2* __restrict__ E) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (d >= Dc) return;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const double2* f = F + ((size_t)c * D + d0 + d) * Nm;
    float sr = 0.f, si = 0.f;
    for (int j = 0; j < Nm; ++j) {
      const double2 fj = f[j];
      const size_t o = d + (size_t)Dc * (j + (size_t)Nm * m);
      const float ar = afr[o], ai = afi[o], fr = (float)fj.x, fi = (float)fj.y;
      sr = fmaf(fr, ar, fmaf(-fi, ai, sr));
      si = fmaf(fr, ai, fmaf(fi, ar, si));
    }
    E[((size_t)c * nports + m) * D + d0 + d] = make_float2(sr, si);
  }
}

// eps[q] = sqrt(|E_theta - Eref_theta|^2 + |E_phi - Eref_phi|^2) / norm.
__global__ void pattern_error_kernel(long n, const float2* __restrict__ E,
                                     const float2* __restrict__ Er, float inv_norm,
                                     float* __restrict__ eps) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float2 a = E[q], ar = Er[q], b = E[n + q], br = Er[n + q];
  const float xr = a.x - ar.x, xi = a.y - ar.y, yr = b.x - br.x, yi = b.y - br.y;
  eps[q] = sqrtf(xr * xr + xi * xi + yr * yr + yi * yi) * inv_norm;
}

}  // namespace harp

using namespace harp;

extern "C" int harp_eep(harp_ctx* ctx, int Na, int Nm, const double* pos, double freq_hz,
                        const double* X, int ldx, int nports, int D, const double* ux,
                        const double* uy, const double* F, float* E, void* stream) {
  if (!ctx) return -1;
  if (Na < 1) return -2;
  if (Nm < 1) return -3;
  if (!pos) return -4;
  if (!(freq_hz > 0.0) || freq_hz > 1e15) return -5;
  if (!X) return -6;
  if ((long)ldx < (long)Na * Nm) return -7;
  if (nports < 1) return -8;
  if (D < 1) return -9;
  if (!ux) return -10;
  if (!uy) return -11;
  if (!F) return -12;
  if (!E) return -13;
  if (Na > 65535 || (long)Nm * nports > 65535 || nports > 65535) return HARP_E_UNSUPPORTED;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t st = (cudaStream_t)stream;
  const long ncol = (long)Nm * nports;
  // directions per chunk: the tensor-core workspace holds the split phase
  // matrix (4 planes of Dc x Kp), and the chunk's array factors stay below
  // 512 MB
  const long Kp = ((long)Na + 31) / 32 * 32;
  long Dc = std::min<long>(D, 8192);
  Dc = std::min<long>(Dc, (long)(ctx->tc_a_floats / (4 * (size_t)Kp)));
  Dc = std::min<long>(Dc, (512L << 20) / (8 * ncol));
  if (Dc < 1) Dc = 1;
  const size_t need = sizeof(float) * (2 * (size_t)Na * ncol + 2 * (size_t)Dc * Na +
                                       2 * (size_t)Dc * ncol);
  if (ctx->eep_bytes < need) {
    HARP_CUDA(cudaStreamSynchronize(st));
    if (ctx->eep_ws) cudaFree(ctx->eep_ws);
    ctx->eep_ws = nullptr;
    ctx->eep_bytes = 0;
    if (cudaMalloc(&ctx->eep_ws, need) != cudaSuccess) {
      cudaGetLastError();
      return HARP_E_NOMEM;
    }
    ctx->eep_bytes = need;
  }
  float* bre = static_cast<float*>(ctx->eep_ws);
  float* bim = bre + (size_t)Na * ncol;
  float* are = bim + (size_t)Na * ncol;
  float* aim = are + (size_t)Dc * Na;
  float* afr = aim + (size_t)Dc * Na;
  float* afi = afr + (size_t)Dc * ncol;
  tc_set_workspace(ctx->tc_a, ctx->tc_a_floats, ctx->tc_b, ctx->tc_b_floats, ctx->dstatus + 2);
  struct Unset {
    ~Unset() { tc_set_workspace(nullptr, 0, nullptr, 0, nullptr); }
  } unset_on_return;
  const double k = 2.0 * kPiE * freq_hz / kC0E;
  {
    ProfScope ps(HARP_K_OTHER, 0.0, st);
    eep_currents_kernel<<<dim3((Na + 255) / 256, (unsigned)ncol), 256, 0, st>>>(
        Na, Nm, reinterpret_cast<const double2*>(X), ldx, bre, bim);
    HARP_LAUNCHED();
  }
  for (long d0 = 0; d0 < D; d0 += Dc) {
    const int dc = (int)std::min<long>(Dc, D - d0);
    {
      ProfScope ps(HARP_K_OTHER, 0.0, st);
      eep_phase_kernel<<<dim3((dc + 255) / 256, Na), 256, 0, st>>>(dc, Na, ux + d0, uy + d0, pos,
                                                                   k, are, aim);
      HARP_LAUNCHED();
    }
    // AF = A B: Dc x (Nm nports) x Na, three-term TF32 on the tensor cores
    HARP_TRY(cgemm<float>(dc, (int)ncol, Na, 1.f, planes<float>(are, aim, dc),
                          planes<float>(bre, bim, Na), 0.f, planes<float>(afr, afi, dc),
                          GEMM_TC_3XTF32, st));
    {
      ProfScope ps(HARP_K_OTHER, 0.0, st);
      eep_combine_kernel<<<dim3((dc + 255) / 256, nports), 256, 0, st>>>(
          dc, (int)d0, D, Nm, nports, afr, afi, reinterpret_cast<const double2*>(F),
          reinterpret_cast<float2*>(E));
      HARP_LAUNCHED();
    }
  }
  return HARP_OK;
}

extern "C" int harp_pattern_error(long n, const float* E, const float* Eref, double norm,
                                  float* eps, void* stream) {
  if (n < 1) return -1;
  if (!E) return -2;
  if (!Eref) return -3;
  if (!(norm > 0.0)) return -4;
  if (!eps) return -5;
  cudaStream_t st = (cudaStream_t)stream;
  pattern_error_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      n, reinterpret_cast<const float2*>(E), reinterpret_cast<const float2*>(Eref),
      (float)(1.0 / norm), eps);
  HARP_LAUNCHED();
  return HARP_OK;
}
