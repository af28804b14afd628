// lu_tc.cu -- tensor-core (tcgen05) complex GEMM for the FP32 LU trailing
// updates and triangular-solve updates. Placeholder until the tcgen05
// kernel lands: reports the shape as unsupported so the CUDA-core kernel
// runs.
#include "dense.cuh"

namespace harp {

int cgemm_tc_f32(int, int, int, float, CView<float>, CView<float>, float, CView<float>, int,
                 cudaStream_t) {
  return HARP_E_UNSUPPORTED;
}

}  // namespace harp
