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

}  // namespace harp

using namespace harp;

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
