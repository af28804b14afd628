// dense.cuh -- internal interface of the dense complex kernels (LU with
// partial pivoting, triangular solves, GEMM, conversions, norms).
#pragma once

#include "common.cuh"

namespace harp {

// How the FP32 contractions of the mixed path run.
enum GemmMode : int {
  GEMM_SIMT = 0,       // CUDA-core FMA (FP32 or FP64 by type)
  GEMM_TC_3XTF32 = 1,  // tcgen05 kind::tf32, hi/lo split, three products
  GEMM_TC_TF32 = 2,    // tcgen05 kind::tf32, one product
};

// C = beta*C + alpha*A*B for complex views (A: M x K, B: K x N).
template <typename R>
int cgemm(int M, int N, int K, R alpha, CView<R> A, CView<R> B, R beta, CView<R> C, int mode,
          cudaStream_t st);
template <>
int cgemm<float>(int M, int N, int K, float alpha, CView<float> A, CView<float> B, float beta,
                 CView<float> C, int mode, cudaStream_t st);
template <>
int cgemm<double>(int M, int N, int K, double alpha, CView<double> A, CView<double> B, double beta,
                  CView<double> C, int mode, cudaStream_t st);

// batch products C_z = beta*C_z + alpha*A_z*B_z, z < batch, operand z at
// element offset z*sA (z*sB, z*sC) from the given views (same offset for the
// real and imaginary planes).
int cgemm_batched(int M, int N, int K, float alpha, CView<float> A, long sA, CView<float> B,
                  long sB, float beta, CView<float> C, long sC, int batch, int mode,
                  cudaStream_t st);

// R = R - Z X in FP64 (the refinement residual; R holds V on entry).
int residual_fp64(int N, int nrhs, CView<double> Z, CView<double> X, CView<double> R,
                  cudaStream_t st);

// Scratch and timeout flag used by the tensor-core GEMM of this thread's
// current solve (lu_tc.cu); a null workspace selects the CUDA-core GEMM.
void tc_set_workspace(float* a, size_t a_floats, float* b, size_t b_floats, int* err);
void tc_get_workspace(float** a, size_t* a_floats, float** b, size_t* b_floats, int** err);
// Cap (1..8) on the K splits of this thread's tensor-core products.
void tc_set_splitk_max(int s);
// FP32 products of tensor-core shape that fell back to the CUDA cores.
long tc_fallbacks();

// Float-float refinement pieces (resid.cu).
int split_c128(int M, int N, const double* Z, long ldz, float* const hl[4], long ldp,
               cudaStream_t st);
int split_planes(int M, int N, const double* xr, const double* xi, long ld, float* const hl[4],
                 cudaStream_t st);
// pr/pi: scratch for up to max_split FP64 partials of ldr * nrhs entries.
// fff: three-float accumulator (FP64-accurate) or double-float (updates).
int residual_ff(int N, int nrhs, const float* const A[4], long ars, long acs,
                const float* const B[4], long ldb, const double* vr, const double* vi, double* rr,
                double* ri, long ldr, double* pr, double* pi, int max_split, int num_sms,
                cudaStream_t st, bool fff);
int split_f32_planes(int M, int N, const float* xr, const float* xi, long ld, float* const hl[4],
                     cudaStream_t st);
int colmax_cabs1_f32(int M, int N, const float* xr, const float* xi, long ld, double* colmax,
                     cudaStream_t st);
int colmax_cabs1(int M, int N, const double* xr, const double* xi, long ld, double* colmax,
                 cudaStream_t st);
int norm_inf_planes_f32(int M, int N, const float* re, const float* im, long rs, long cs,
                        float* rowsum, double* out, cudaStream_t st);

// PA = LU in place on split planes (N x N, leading dimension ld).
// ipiv[k] = row swapped with row k (0-based, global). The smallest
// 1-based column with an exactly zero pivot is atomically min-ed into
// *zero_col (device). perm (device, N ints) receives the net row
// permutation: row i of PA is row perm[i] of A.
template <typename R>
int lu_factor(harp_ctx* ctx, int N, R* re, R* im, long ld, int* ipiv, int* perm, int* zero_col,
              int mode, cudaStream_t st);

// Inverses of the 64 x 64 diagonal blocks of L (unit lower) and U (upper)
// of a factorisation held in A (N x N): block b of each at b*4096 elements
// (column-major 64 x 64) of the given planes.
template <typename R>
int diag_inverses(int N, CView<R> A, R* lre, R* lim, R* ure, R* uim, cudaStream_t st);

// Explicit inverses of the factors held in A (FP32 path): L^-1 and U^-1 as
// planes (ld ldi), built from the diagonal-block inverses; t planes are
// scratch of ldi x N. With a side stream (and two events to fork and join)
// U^-1 is built there while L^-1 is built on st.
int factor_inverses(int N, CView<float> A, const float* dinv_re, const float* dinv_im,
                    float* linv_re, float* linv_im, float* uinv_re, float* uinv_im, long ldi,
                    float* tre, float* tim, int mode, cudaStream_t st, cudaStream_t side,
                    cudaEvent_t fork, cudaEvent_t join);
// Solve op(A) X = B with the explicit factor inverses (two products).
// li_split / ui_split (optional): L^-1 and U^-1 already split into
// tensor-core operand planes (tc_split_operand, same mode), used by the
// 'N' products.
template <typename R>
int lu_solve_inv(int N, int nrhs, CView<R> Li, CView<R> Ui, const int* perm, R* bre, R* bim,
                 long ldb, R* tre, R* tim, char trans, int mode, cudaStream_t st,
                 const float* li_split = nullptr, const float* ui_split = nullptr);

// K-major tensor-core operand planes of V (R x K) for repeated use, and the
// product that takes them as its A operand (lu_tc.cu).
int tc_split_operand(int R, int K, CView<float> V, float* out, size_t out_floats, int mode,
                     cudaStream_t st);
// a_ld > 0: A is a block of larger split planes, row stride a_ld, plane
// stride a_plane (K then a multiple of 32). split_k: K may be split to fill
// the SMs. a_tri: A is upper (1: row i zero for k < i) or lower (2: zero for
// k > i) triangular, and the zero k-tiles of each row tile are skipped.
int cgemm_tc_f32_asplit(int M, int N, int K, float alpha, const float* a_split, CView<float> B,
                        float beta, CView<float> C, int mode, cudaStream_t st, long a_ld = 0,
                        size_t a_plane = 0, bool split_k = true, int a_tri = 0);
// The TF32 planes of V (R x Kc) into a block of larger split planes
// (element (r, k) at out[p * plane + r * ldo + k]).
int tc_split_block(int R, int Kc, CView<float> V, float* out, long ldo, size_t plane, int mode,
                   cudaStream_t st);

// Solve op(A) X = B with the factors of lu_factor and their diagonal-block
// inverses (dinv planes: the L blocks, then the U blocks); B (N x nrhs split
// planes, leading dimension ldb) is overwritten. tmp has room for N x nrhs
// (leading dimension ldb) of each plane.
template <typename R>
int lu_solve(int N, int nrhs, R* lre, R* lim, long ld, const int* perm, R* bre, R* bim, long ldb,
             R* tre, R* tim, char trans, const R* dinv_re, const R* dinv_im, int mode,
             cudaStream_t st);

// Elementwise conversions between interleaved complex storage and planes.
// nonfinite_flag (optional, device): ST_NONFINITE is or-ed into it when an
// entry read is NaN or infinite.
template <typename Rin, typename Rout>
int interleaved_to_planes(int M, int N, const Rin* src, long lds, Rout* re, Rout* im, long ldd,
                          cudaStream_t st, int* nonfinite_flag = nullptr);
template <typename Rin, typename Rout>
int planes_to_planes(int M, int N, const Rin* sre, const Rin* sim, long lds, Rout* dre, Rout* dim,
                     long ldd, cudaStream_t st);
int planes_to_interleaved(int M, int N, const double* re, const double* im, long lds, double* dst,
                          long ldd, cudaStream_t st);
// dst (planes, M x N) = E: unit entry at row c*Nm of column c.
template <typename R>
int port_rhs_planes(int M, int N, int Nm, R* re, R* im, long ld, cudaStream_t st);
// X += D (FP64 planes += R planes)
template <typename R>
int add_planes(int M, int N, double* xre, double* xim, long ldx, const R* dre, const R* dim,
               long ldd, cudaStream_t st);
// out[slot] = max_i sum_j |A_ij| (matrix infinity norm), A given as a view.
// out must be zeroed first (zero_doubles).
template <typename R>
int norm_inf(int M, int N, CView<R> A, double* out, cudaStream_t st);
int zero_doubles(double* p, int n, cudaStream_t st);

}  // namespace harp
