// port.cu -- the port objective of the synthesis workload:
//   P = E^T X (Na x Na: row m*Nm of every column of X, MBF 0 of antenna m),
//   J = sum_mn |P_mn|^2,
//   W = E conj(P) (N x Na: conj(P_mn) at row m*Nm of column n, zero elsewhere),
// W being the right-hand side of the adjoint solve Z^T Lambda = W.
// J is reduced by one CTA in a fixed order (deterministic).
#include "common.cuh"
#include "prof.cuh"

namespace harp {

constexpr int kPortThreads = 1024;

__global__ void __launch_bounds__(kPortThreads) port_objective_kernel(int Na, int Nm,
                                                                      const double2* X, long ldx,
                                                                      double2* P, double* J) {
  __shared__ double red[kPortThreads / 32];
  double s = 0.0;
  const long n2 = (long)Na * Na;
  for (long e = threadIdx.x; e < n2; e += kPortThreads) {
    const int m = (int)(e % Na), n = (int)(e / Na);
    const double2 v = X[(size_t)m * Nm + (size_t)n * ldx];
    if (P) P[e] = v;
    s += v.x * v.x + v.y * v.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = red[threadIdx.x];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) *J = s;
  }
}

__global__ void port_adjoint_rhs_kernel(int Na, int Nm, const double2* X, long ldx, double2* W,
                                        long ldw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // row of W
  const int n = blockIdx.y;                             // column
  const int N = Na * Nm;
  if (i >= N) return;
  double2 v = make_double2(0.0, 0.0);
  if (i % Nm == 0) {
    const double2 x = X[(size_t)i + (size_t)n * ldx];
    v = make_double2(x.x, -x.y);
  }
  W[(size_t)i + (size_t)n * ldw] = v;
}

// C = alpha op(A) op(B) for small complex FP64 matrices (n x n, the port
// response's size): op(X) = X or X^H. 16 x 16 output tiles, K in 16-wide
// shared-memory chunks.
constexpr int kZt = 16;
__global__ void zgemm_small_kernel(int n, int ha, const double2* __restrict__ A, long lda, int hb,
                                   const double2* __restrict__ B, long ldb, double alpha,
                                   double2* __restrict__ C, long ldc) {
  __shared__ double2 As[kZt][kZt + 1], Bs[kZt][kZt + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.y * kZt + ty, j = blockIdx.x * kZt + tx;
  double cr = 0.0, ci = 0.0;
  for (int k0 = 0; k0 < n; k0 += kZt) {
    {  // As[ty][tx] = op(A)(i, k0 + tx)
      const int k = k0 + tx;
      double2 v = make_double2(0.0, 0.0);
      if (i < n && k < n) {
        v = ha ? A[(size_t)k + (size_t)i * lda] : A[(size_t)i + (size_t)k * lda];
        if (ha) v.y = -v.y;
      }
      As[ty][tx] = v;
    }
    {  // Bs[ty][tx] = op(B)(k0 + ty, j)
      const int k = k0 + ty;
      double2 v = make_double2(0.0, 0.0);
      if (k < n && j < n) {
        v = hb ? B[(size_t)j + (size_t)k * ldb] : B[(size_t)k + (size_t)j * ldb];
        if (hb) v.y = -v.y;
      }
      Bs[ty][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kZt; ++kk) {
      const double2 a = As[ty][kk], b = Bs[kk][tx];
      cr += a.x * b.x - a.y * b.y;
      ci += a.x * b.y + a.y * b.x;
    }
    __syncthreads();
  }
  if (i < n && j < n) C[(size_t)i + (size_t)j * ldc] = make_double2(alpha * cr, alpha * ci);
}

// W = E conj(G): conj(G_mn) at row m*Nm of column n, zero elsewhere.
__global__ void port_impedance_rhs_kernel(int Na, int Nm, const double2* G, long ldg, double2* W,
                                          long ldw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // row of W
  const int n = blockIdx.y;                             // column
  if (i >= Na * Nm) return;
  double2 v = make_double2(0.0, 0.0);
  if (i % Nm == 0) {
    const double2 g = G[(size_t)(i / Nm) + (size_t)n * ldg];
    v = make_double2(g.x, -g.y);
  }
  W[(size_t)i + (size_t)n * ldw] = v;
}

}  // namespace harp

using namespace harp;

extern "C" int harp_port_impedance(harp_ctx* ctx, int Na, int Nm, const double* P, int ldp,
                                   double* Y, int ldy, double* J, double* G, int ldg, double* W,
                                   int ldw, void* stream) {
  if (!ctx) return -1;
  if (Na < 1) return -2;
  if (Nm < 1) return -3;
  if (!P) return -4;
  if (ldp < Na) return -5;
  if (!Y) return -6;
  if (ldy < Na) return -7;
  if (!J) return -8;
  if (!G) return -9;
  if (ldg < Na) return -10;
  if (!W) return -11;
  if (ldw < (long)Na * Nm) return -12;
  if (Na > 65535) return HARP_E_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  // Y = P^-1: the FP64 solve of P Y = I (the identity is the port
  // excitation of a system with one basis function per port)
  int iters = 0;
  double resid = 0.0;
  const int s = mbf_solve(ctx, Na, P, ldp, nullptr, Na, Na, Y, ldy, 'N', HARP_FP64, 0.0, 0,
                          &iters, &resid, stream);
  if (s != HARP_OK) return s;
  const dim3 blk(kZt, kZt), grid((Na + kZt - 1) / kZt, (Na + kZt - 1) / kZt);
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  port_objective_kernel<<<1, kPortThreads, 0, st>>>(Na, 1, reinterpret_cast<const double2*>(Y), ldy,
                                                    nullptr, J);  // J = sum |Y|^2
  HARP_LAUNCHED();
  // T = Y^H Y in W's storage (W is written last), then G = -T Y^H
  double2* T = reinterpret_cast<double2*>(W);
  const double2* Yc = reinterpret_cast<const double2*>(Y);
  zgemm_small_kernel<<<grid, blk, 0, st>>>(Na, 1, Yc, ldy, 0, Yc, ldy, 1.0, T, ldw);
  HARP_LAUNCHED();
  zgemm_small_kernel<<<grid, blk, 0, st>>>(Na, 0, T, ldw, 1, Yc, ldy, -1.0,
                                           reinterpret_cast<double2*>(G), ldg);
  HARP_LAUNCHED();
  port_impedance_rhs_kernel<<<dim3(((long)Na * Nm + 255) / 256, Na), 256, 0, st>>>(
      Na, Nm, reinterpret_cast<const double2*>(G), ldg, reinterpret_cast<double2*>(W), ldw);
  HARP_LAUNCHED();
  return HARP_OK;
}

extern "C" int harp_port_objective(int Na, int Nm, const double* X, int ldx, double* P, double* J,
                                   double* W, int ldw, void* stream) {
  if (Na < 1) return -1;
  if (Nm < 1) return -2;
  if (!X) return -3;
  if (ldx < (long)Na * Nm) return -4;
  if (!J) return -6;
  if (W && ldw < (long)Na * Nm) return -8;
  if (Na > 65535) return HARP_E_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  {
    ProfScope ps(HARP_K_OTHER, 0.0, st);
    port_objective_kernel<<<1, kPortThreads, 0, st>>>(Na, Nm, reinterpret_cast<const double2*>(X),
                                                      ldx, reinterpret_cast<double2*>(P), J);
    HARP_LAUNCHED();
  }
  if (W) {
    ProfScope ps(HARP_K_OTHER, 0.0, st);
    dim3 grid(((long)Na * Nm + 255) / 256, Na);
    port_adjoint_rhs_kernel<<<grid, 256, 0, st>>>(Na, Nm, reinterpret_cast<const double2*>(X),
                                                  ldx, reinterpret_cast<double2*>(W), ldw);
    HARP_LAUNCHED();
  }
  return HARP_OK;
}
