// ozaki.cuh -- internal interface of the tensor-core refinement residual
// (exact integer slices, ozaki.cu).
#pragma once

#include "common.cuh"

namespace harp {

constexpr int kOzMaxG = 13;  // largest slice-group index t + u formed
constexpr int kOzMaxPairs = kOzMaxG * (kOzMaxG - 1) / 2;

// Digit width for a K-long product (exact FP32 accumulation, bf16 digits).
int oz_digit_bits(int K);
// The residual's digit width (its products split K into exact chunks).
int oz_resid_bits(int K);
// Groups G needed for a residual whose correction is rho times the iterate.
int oz_groups(int K, int b, double rho);
int oz_pairs(int G);

// Row exponents, ||op(Z)||_inf (|re| + |im|, into *znorm on the device) and
// the digits of op(Z), Z the N x N c128 matrix (ld) -- once per solve.
int oz_prepare(harp_ctx* ctx, int N, const double2* z, long ld, bool trans, double* znorm,
               cudaStream_t st);
// R = S - op(Z) Y for FP32 planes Y (ldy); S, R FP64 planes (ldr, may alias).
// rho: max_j max|Y_j| / max|X_j| of the iterate X the residual belongs to
// (1 for a full residual).
int oz_residual(harp_ctx* ctx, int N, int nrhs, const float* yr, const float* yi, long ldy,
                const double* sr, const double* si, double* rr, double* ri, long ldr, double rho,
                int prof_kind, cudaStream_t st);

// The FP64-accurate fill of Z (Eq. 3 in Eq. 4) on the tensor cores by exact
// digit products: Z64's pair blocks and self blocks, coincident antennas or-ed
// into *status. HARP_E_UNSUPPORTED when it does not apply (the caller falls
// back to the float-float kernel).
int oz_fill_z64(harp_ctx* ctx, int Na, int Nm, int P, int Q, const double* pos, double kw,
                const double2* coef, const double2* self, long self_stride, double2* Z, long ldz,
                int* status, cudaStream_t st);

// G = Lambda X^T (N x nrhs operands, column-major; G's columns are rows of
// X) as exact digit products on the tensor cores, FP64-accurate: prepare
// slices Lambda into the residual's A buffer (resetting its Z64 slices) and
// takes the row exponents of both; each chunk then forms columns
// j0 .. j0 + ncols - 1 of G (at most oz_gram_max_cols, 0 when the buffers do
// not serve) into G[i + jj ldg] (the caller's N x ncols buffer).
// HARP_E_UNSUPPORTED when it does not apply.
int oz_gram_max_cols(const harp_ctx* ctx, int N, int nrhs);
int oz_gram_prepare(harp_ctx* ctx, int N, int nrhs, const double2* Lam, long ldl,
                    const double2* X, long ldx, cudaStream_t st);
int oz_gram_chunk(harp_ctx* ctx, int N, int nrhs, const double2* X, long ldx, int j0, int ncols,
                  double2* G, long ldg, cudaStream_t st);

// The adjoint's coefficient contraction as exact digit products: for the
// pairs (m, n0 + nl), m < Na, nl < nn, H[(m + Na nl) + k ldh] = sum_TS
// G^{mn}_TS c_k^{TS} with G's columns of those antennas as oz_gram_chunk
// leaves them (G[i + (nl Nm + S) ldg]). The work buffer (oz_adj_h_bytes, 0
// when it does not apply: K <= 128, Nm^2 <= 1024, the slots hold the
// chunk) keeps the table's digits between prepare and the chunks.
size_t oz_adj_h_bytes(const harp_ctx* ctx, int Na, int Nm, int K, int nn);
int oz_adj_h_prepare(harp_ctx* ctx, int Na, int Nm, int K, int nn, const double2* coef,
                     void* work, cudaStream_t st);
int oz_adj_h_chunk(harp_ctx* ctx, int Na, int Nm, int K, int nn, const double2* G, long ldg,
                   void* work, double2* H, long ldh, cudaStream_t st);

}  // namespace harp
