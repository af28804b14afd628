// ozaki.cu -- FP64-accurate refinement residual on the tensor cores by exact
// integer slices (Ozaki's error-free splitting of a matrix product):
//
//   R = S - op(Z) Y,   Z: N x N FP64 (the context's matrix), Y: N x nrhs FP32
//   (the FP32 solution X_0 or a correction D_k), S = V or the previous R.
//
// Scaling and slices. Each row i of A = op(Z) is scaled by 2^-sig_i so that
// its largest real or imaginary part is below 1/2, each column j of Y by
// 2^-tau_j likewise, and the scaled values are cut into signed base-2^b
// digits by repeated round-to-nearest on a 64-bit fixed point:
//   a_ik = 2^sig_i sum_t d_t[i,k] 2^-bt,   y_kj = 2^tau_j sum_u e_u[k,j] 2^-bu,
// with |d|, |e| <= 2^(b-1), so every digit is an integer exact in bf16.
//
// Exact products. For one slice pair (t, u) the four real products
// Re(d_t) Re(e_u), Re(d_t) Im(e_u), Im(d_t) Re(e_u), Im(d_t) Im(e_u) are
// sums over K of integer products of magnitude <= 2^(2b-2); b is the
// largest width with K 2^(2b-2) <= 2^24, so every partial sum is an integer
// an FP32 accumulator holds exactly, and the bf16 tcgen05 product with FP32
// accumulation (kind::f16) is exact. Two MMAs per 16-deep K step produce all
// four: A_re x [Y_re | Y_im] and A_im x [Y_re | Y_im] (N = 2 x 64 columns).
//
// Combination. The pair results of one group g = t + u share the weight
// 2^-bg; they are added exactly in integers (re = rr - ii, im = ri + ir),
// four groups at a time are combined exactly in 64-bit integers, and those
// blocks in FP64 by Horner's rule from the smallest weight up, then scaled
// back by 2^(sig_i + tau_j). Only the pairs with
// t + u <= G are formed; oz_groups picks G from the accuracy the caller
// needs (the dropped groups are below the FP64 rounding of the result).
//
// Kernels: oz_rowexp (row exponents and row sums of |re| + |im| for the
// stopping test, one pass over Z), oz_slice_a (digits of op(Z), K-major),
// oz_colexp_y / oz_slice_y (digits of Y), oz_mma (one CTA per 128 x 64
// output tile and slice pair; TMA into a two-stage ring, tcgen05.mma by one
// thread, integer pair results written out), oz_combine (groups -> FP64).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <vector>

#include "dense.cuh"
#include "ozaki.cuh"
#include "prof.cuh"

namespace harp {

constexpr int OZ_BM = 128;  // output rows per CTA (TMEM lanes)
constexpr int OZ_BN = 64;   // output columns per CTA
constexpr int OZ_BK = 64;   // K per stage: one 128-byte swizzle atom of bf16
constexpr int OZ_STAGES = 2;
constexpr int OZ_THREADS = 128;
constexpr int OZ_A_PLANE = OZ_BM * OZ_BK * 2;  // 16 KB
constexpr int OZ_B_PLANE = OZ_BN * OZ_BK * 2;  //  8 KB
constexpr int OZ_STAGE = 2 * OZ_A_PLANE + 2 * OZ_B_PLANE;
constexpr int OZ_KCH = 32;  // K chunks of the row-exponent pass
constexpr long long OZ_WAIT_CYCLES = 1LL << 30;  // ~0.5 s at 2 GHz
// Exponent of an all-zero row or column: any value below kOzNone (real
// exponents are above -1100); the row pass starts from a byte-filled
// 0x80808080.
constexpr int OZ_NOEXP = INT_MIN;
constexpr int kOzNone = -4000;
__host__ __device__ __forceinline__ bool oz_none(int e) { return e < kOzNone; }

// Exponent e with |v| < 2^e (v != 0), from the bits (no libm).
__device__ __forceinline__ int exp_above(double v) {
  const int eb = (int)((__double_as_longlong(v) >> 52) & 0x7ff);
  return (eb == 0 ? 1 : eb) - 1022;
}
// v != 0 from the bits (an integer test, off the FP64 pipe)
__device__ __forceinline__ bool oz_nz(double v) {
  return (__double_as_longlong(v) & 0x7fffffffffffffffLL) != 0;
}
__device__ __forceinline__ int exp_above_f(float v) {
  const int eb = (int)((__float_as_uint(v) >> 23) & 0xff);
  return (eb == 0 ? 1 : eb) - 126;
}

// ---------------------------------------------------------------------------
// Row exponents of op(Z), N rows of Kd entries (max over the row of the
// exponents of |re|, |im|, atomically max-ed into emax[i], which starts at
// OZ_NOEXP) and, when part is given, partial row sums of |re| + |im| per K
// chunk (part[chunk * N + i]). Element (i, k) of
// op(Z) is z[i * ars + k * acs] (c128 units); lanes run along whichever of
// i and k is contiguous.
__global__ void __launch_bounds__(256) oz_rowexp_kernel(int N, int Kd,
                                                        const double2* __restrict__ z, long ars,
                                                        long acs, int kchunk, int* emax,
                                                        double* part) {
  __shared__ double ssum[8][33];
  __shared__ int sexp[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i0 = blockIdx.x * 32;
  const int kc0 = blockIdx.y * kchunk, kc1 = min(Kd, kc0 + kchunk);
  if (ars == 1) {
    // rows contiguous: lane = row, warps step along k
    const int i = i0 + tx;
    double s = 0.0;
    int e = OZ_NOEXP;
    if (i < N)
      for (int k = kc0 + ty; k < kc1; k += 8) {
        const double2 v = z[(long)i + (long)k * acs];
        s += fabs(v.x) + fabs(v.y);
        if (v.x != 0.0) e = max(e, exp_above(v.x));
        if (v.y != 0.0) e = max(e, exp_above(v.y));
      }
    ssum[ty][tx] = s;
    sexp[ty][tx] = e;
    __syncthreads();
    if (ty == 0 && i < N) {
      double t = 0.0;
      int m = OZ_NOEXP;
      for (int w = 0; w < 8; ++w) {
        t += ssum[w][tx];
        m = max(m, sexp[w][tx]);
      }
      if (part) part[(long)blockIdx.y * N + i] = t;
      if (!oz_none(m)) atomicMax(&emax[i], m);
    }
  } else {
    // k contiguous: a warp walks one row at a time, lanes along k
    for (int l = ty; l < 32; l += 8) {
      const int i = i0 + l;
      if (i >= N) break;
      double s = 0.0;
      int e = OZ_NOEXP;
      for (int k = kc0 + tx; k < kc1; k += 32) {
        const double2 v = z[(long)i * ars + k];
        s += fabs(v.x) + fabs(v.y);
        if (v.x != 0.0) e = max(e, exp_above(v.x));
        if (v.y != 0.0) e = max(e, exp_above(v.y));
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
      }
      if (tx == 0) {
        if (part) part[(long)blockIdx.y * N + i] = s;
        if (!oz_none(e)) atomicMax(&emax[i], e);
      }
    }
  }
}

// ||op(Z)||_inf with |z| = |re| + |im|: the K-chunk partials of each row
// summed in chunk order, then the largest row (out must be zeroed first).
__global__ void oz_rownorm_kernel(int N, int nch, const double* __restrict__ part, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < N)
    for (int c = 0; c < nch; ++c) s += part[(long)c * N + i];
  if (!(s == s)) s = __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, off));
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(s));
}

// Digits of one value of a row (column) whose largest exponent is e
// (|v| < 2^e). The scaled value w = v 2^-(e+1) (|w| < 1/2) is taken to the
// 64-bit fixed point X = round(w 2^63) (|X| <= 2^62; bits below 2^-63 of
// the scale are dropped, ~2^-61 of the row's largest entry), and
// out[t * pstride], t < s, gets the signed base-2^b digits from the top,
// each the round-to-nearest quotient of the remainder by 2^(63 - b(t+1)),
// so |digit| <= 2^(b-1). Integer arithmetic only (the FP64 pipe runs at
// 1/64 rate): X comes from the bits of v, v = +-mant 2^(ef - 1075), so
// X = mant 2^(ef - 1013 - e); as |v| < 2^e the mantissa moves left at most
// 9 places, and a right move rounds half away from zero (within half a
// unit, which is all the digit bound needs). The digits fit an int32.
__device__ __forceinline__ void oz_digits(double v, int e, int b, int s, __nv_bfloat16* out,
                                          size_t pstride) {
  const long long bits = __double_as_longlong(v);
  int ef = (int)((bits >> 52) & 0x7ff);
  unsigned long long mant = (unsigned long long)bits & 0xFFFFFFFFFFFFFull;
  if (ef) mant |= 1ull << 52;
  else ef = 1;
  const int sh = ef - 1013 - e;
  long long X = 0;
  if (!oz_none(e) && mant != 0) {
    if (sh >= 0) X = (long long)(mant << sh);
    else if (sh > -63) X = (long long)((mant + (1ull << (-sh - 1))) >> (-sh));
    if (bits < 0) X = -X;
  }
  int shift = 63;
  for (int t = 0; t < s; ++t) {
    shift -= b;
    long long d;
    if (shift > 0) {
      d = (X + (1LL << (shift - 1))) >> shift;
      X -= d << shift;
    } else {
      d = X << (-shift);
      X = 0;
    }
    out[(size_t)t * pstride] = __float2bfloat16_rn((float)(int)d);
  }
}

// Digits of op(Z) (N rows of Kd entries): out[(2t + p) * plane + i * Kp + k]
// (p = 0 re, 1 im) for rows i < Np, zero for rows N <= i < Np and columns
// Kd <= k < Kp. A 32 x 32
// tile goes through shared memory so that both the reads of Z and the
// K-major writes are coalesced.
__global__ void __launch_bounds__(256) oz_slice_a_kernel(int N, int Kd, int Np, int Kp,
                                                         const double2* __restrict__ z,
                                                         long ars, long acs,
                                                         const int* __restrict__ emax, int b,
                                                         int s, __nv_bfloat16* out, size_t plane) {
  __shared__ double tr[32][33], ti[32][33];  // [i_local][k_local]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  for (int l = ty; l < 32; l += 8) {
    const int il = (ars == 1) ? tx : l, kl = (ars == 1) ? l : tx;
    const int i = i0 + il, k = k0 + kl;
    double2 v = make_double2(0.0, 0.0);
    if (i < N && k < Kd) v = z[(long)i * ars + (long)k * acs];
    tr[il][kl] = v.x;
    ti[il][kl] = v.y;
  }
  __syncthreads();
  const int k = k0 + tx;
  if (k >= Kp) return;
  for (int l = ty; l < 32; l += 8) {
    const int i = i0 + l;
    if (i >= Np) break;
    const int e = (i < N) ? emax[i] : OZ_NOEXP;
    __nv_bfloat16* o = out + (size_t)i * Kp + k;
    oz_digits(tr[l][tx], e, b, s, o, 2 * plane);
    oz_digits(ti[l][tx], e, b, s, o + plane, 2 * plane);
  }
}

// Column exponents of Y (FP32 planes, column j at j * ldy).
__global__ void oz_colexp_y_kernel(int N, const float* __restrict__ yr, const float* __restrict__ yi,
                                   long ldy, int* emax) {
  __shared__ int sm[32];
  const int j = blockIdx.x;
  int e = OZ_NOEXP;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const float a = yr[(long)j * ldy + k], c = yi[(long)j * ldy + k];
    if (a != 0.f) e = max(e, exp_above_f(a));
    if (c != 0.f) e = max(e, exp_above_f(c));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = OZ_NOEXP;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, sm[w]);
    emax[j] = m;
  }
}

// Digits of Y: out[(2u + p) * plane + j * Kp + k] for columns j < gridDim.y,
// zero for columns j >= nrhs and rows N <= k < Kp.
__global__ void oz_slice_y_kernel(int N, int nrhs, int Kp, const float* __restrict__ yr,
                                  const float* __restrict__ yi, long ldy,
                                  const int* __restrict__ emax, int b, int s, __nv_bfloat16* out,
                                  size_t plane) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (k >= Kp) return;
  const bool in = (j < nrhs) && (k < N);
  const int e = (j < nrhs) ? emax[j] : OZ_NOEXP;
  const double a = in ? (double)yr[(long)j * ldy + k] : 0.0;
  const double c = in ? (double)yi[(long)j * ldy + k] : 0.0;
  __nv_bfloat16* o = out + (size_t)j * Kp + k;
  oz_digits(a, e, b, s, o, 2 * plane);
  oz_digits(c, e, b, s, o + plane, 2 * plane);
}

// ---------------------------------------------------------------------------
// Tensor-core pair products.
__device__ __forceinline__ uint32_t oz_su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void oz_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void oz_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool oz_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the error flag set) when the clock budget runs out.
__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity, int* err) {
  const long long t0 = clock64();
  while (!oz_try_wait(bar, parity)) {
    if (clock64() - t0 > OZ_WAIT_CYCLES) {
      atomicOr(err, 1);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void oz_tma_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                          int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
// K-major operand, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t oz_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor: kind::f16 with bf16 A and B, FP32 accumulate,
// K-major operands.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void oz_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void oz_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

#define OZ_LD16(taddr, v)                                                                         \
  asm volatile(                                                                                   \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14," \
      "%15}, [%16];"                                                                              \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),      \
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),  \
        "=r"(v[14]), "=r"(v[15])                                                                  \
      : "r"(taddr))

struct OzArgs {
  int N, nrhs, nk, tiles_m;
  int* err;
  int* slots;        // [slot][plane][j][i], i contiguous (N), j < nrhs
  long slot_stride;  // 2 * nrhs * N
  unsigned char pt[kOzMaxPairs], pu[kOzMaxPairs];  // slice t, u of each pair
  // product y sums the pairs pfirst[y] .. pfirst[y+1]-1 in its accumulators
  // (exact while their count times K 2^(2b-2) stays within 2^24) and
  // writes slot ps[y]
  unsigned char pfirst[kOzMaxPairs + 1], ps[kOzMaxPairs];
};

// grid (tiles_m * tiles_n, nproducts): blockIdx.y picks the product (one
// slice pair, or several of one group), so the CTAs of one product run
// together and share its A slices in L2.
__global__ void __launch_bounds__(OZ_THREADS, 2)
    oz_mma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const __grid_constant__ OzArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[OZ_STAGES], bar_empty[OZ_STAGES], bar_done;
  __shared__ uint32_t tmem_slot;
  if (*reinterpret_cast<volatile int*>(a.err)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (oz_su32(smem_raw) + 1023u) & ~1023u;
  const int tm = blockIdx.x % a.tiles_m, tn = blockIdx.x / a.tiles_m;
  const int i0 = tm * OZ_BM, j0 = tn * OZ_BN;
  const int y = blockIdx.y;
  const int q0 = a.pfirst[y], nl = (a.pfirst[y + 1] - q0) * a.nk;  // k tiles over the pairs

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      oz_mbar_init(oz_su32(&bar_full[s]), 1);
      oz_mbar_init(oz_su32(&bar_empty[s]), 1);
    }
    oz_mbar_init(oz_su32(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     oz_su32(&tmem_slot)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // d0: A_re x [Y_re | Y_im] -> columns 0..63 rr, 64..127 ri
  // d1: A_im x [Y_re | Y_im] -> columns 0..63 ir, 64..127 ii
  const uint32_t d0 = tmem, d1 = tmem + 128;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      int issued = 0;
      for (int L = 0; L < nl; ++L) {
        const int s = L % OZ_STAGES, use = L / OZ_STAGES;
        if (use > 0 && !oz_wait(oz_su32(&bar_empty[s]), (use - 1) & 1, a.err)) break;
        const int qi = L / a.nk, kt = L - qi * a.nk;
        const int t = a.pt[q0 + qi], u = a.pu[q0 + qi];
        const uint32_t st = base + s * OZ_STAGE;
        const uint32_t fb = oz_su32(&bar_full[s]);
        oz_expect_tx(fb, OZ_STAGE);
        oz_tma_3d(st, &tmA, fb, kt * OZ_BK, i0, 2 * t);
        oz_tma_3d(st + OZ_A_PLANE, &tmA, fb, kt * OZ_BK, i0, 2 * t + 1);
        oz_tma_3d(st + 2 * OZ_A_PLANE, &tmB, fb, kt * OZ_BK, j0, 2 * u);
        oz_tma_3d(st + 2 * OZ_A_PLANE + OZ_B_PLANE, &tmB, fb, kt * OZ_BK, j0, 2 * u + 1);
        issued = L + 1;
      }
      for (int kt = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); kt < issued; ++kt)
        oz_wait(oz_su32(&bar_full[kt % OZ_STAGES]), (kt / OZ_STAGES) & 1, a.err);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer (single thread)
      constexpr uint32_t ID = bf16_idesc(OZ_BM, 2 * OZ_BN);
      for (int kt = 0; kt < nl; ++kt) {
        const int s = kt % OZ_STAGES, use = kt / OZ_STAGES;
        if (!oz_wait(oz_su32(&bar_full[s]), use & 1, a.err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = base + s * OZ_STAGE;
#pragma unroll
        for (int j = 0; j < OZ_BK / 16; ++j) {
          const uint32_t ko = 32u * j;  // 16 bf16 = 32 bytes along K inside the atom
          const uint64_t are = oz_desc(st + ko);
          const uint64_t aim = oz_desc(st + OZ_A_PLANE + ko);
          const uint64_t by = oz_desc(st + 2 * OZ_A_PLANE + ko);  // 128 rows: Y_re then Y_im
          const uint32_t acc = (kt == 0 && j == 0) ? 0u : 1u;
          oz_mma(d0, are, by, ID, acc);
          oz_mma(d1, aim, by, ID, acc);
        }
        oz_commit(oz_su32(&bar_empty[s]));
      }
      oz_commit(oz_su32(&bar_done));
    }
    __syncwarp();
  }

  // ---- epilogue: exact integer pair results -> slots
  const bool ok = oz_wait(oz_su32(&bar_done), 0, a.err);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int gi = i0 + warp * 32 + lane;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
  int* sre = a.slots + (long)a.ps[y] * a.slot_stride;
  int* sim = sre + (long)a.nrhs * a.N;
#pragma unroll 1
  for (int c0 = 0; c0 < OZ_BN; c0 += 16) {
    uint32_t rr[16], ri[16], ir[16], ii[16];
    OZ_LD16(d0 + lane_off + c0, rr);
    OZ_LD16(d0 + lane_off + OZ_BN + c0, ri);
    OZ_LD16(d1 + lane_off + c0, ir);
    OZ_LD16(d1 + lane_off + OZ_BN + c0, ii);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (ok && gi < a.N) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int j = j0 + c0 + c;
        if (j < a.nrhs) {
          const long o = (long)j * a.N + gi;
          sre[o] = __float2int_rn(__uint_as_float(rr[c])) - __float2int_rn(__uint_as_float(ii[c]));
          sim[o] = __float2int_rn(__uint_as_float(ri[c])) + __float2int_rn(__uint_as_float(ir[c]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// K-split pair products, for K above the exact range of one FP32 sum. K runs
// in chunks of kc k-tiles whose digit products stay below 2^24 in the FP32
// accumulators (kc 64 2^(2b-2) <= 2^24: 16 k-tiles at b = 8), so the digits
// can stay 8 bits wide at any K, which needs fewer digit pairs than
// narrowing them (at K = 3072: 36 pairs instead of 45; at K = 16384, 36
// instead of 66). Persistent: CTA c takes tiles c, c + gridDim.x, ... (the
// non-persistent kernel's order: blockIdx.x fastest, then the product), and
// the chunks of all its tiles alternate between two TMEM regions (512
// columns, one CTA per SM): the MMA warp fills one while the four epilogue
// warps move the other's exact integers into int32 register sums (at most
// 2 K 2^14 < 2^31), so a tile's slot writes overlap the next tile's
// products. Warps: 0-3 epilogue (TMEM lanes 32 w ..), 4 TMA producer, 5 MMA
// issuer; four smem stages. Every wait is bounded; after a failed wait the
// warps leave their loops (warp-uniformly around the collective TMEM
// loads) and the error flag stays set.
constexpr int OZK_STAGES = 4;
constexpr int OZK_THREADS = 192;

// Unit `tile` of the persistent kernel -> (output tile bx, product y). order
// 0: bx fastest, then the product; order 1 (products that mix A slices):
// row block of A slowest, then the product, then the column block, so that
// the A slices of a few row blocks are all that is live in L2.
__device__ __forceinline__ void oz_unit(int tile, int tiles_xy, int tiles_m, int nprod, int order,
                                        int* bx, int* y) {
  if (order == 0) {
    *bx = tile % tiles_xy;
    *y = tile / tiles_xy;
  } else {
    const int tiles_n = tiles_xy / tiles_m;
    const int rb = tile / (nprod * tiles_n), rem = tile - rb * (nprod * tiles_n);
    *y = rem / tiles_n;
    *bx = rb + (rem - *y * tiles_n) * tiles_m;
  }
}

__global__ void __launch_bounds__(OZK_THREADS, 1)
    oz_mma_ks_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ OzArgs a, int kc, int tiles_xy, int ntiles,
                     int order) {
  const int nprod = ntiles / tiles_xy;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[OZK_STAGES], bar_empty[OZK_STAGES], bar_tfull[2],
      bar_tempty[2];
  __shared__ uint32_t tmem_slot;
  if (*reinterpret_cast<volatile int*>(a.err)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (oz_su32(smem_raw) + 1023u) & ~1023u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZK_STAGES; ++s) {
      oz_mbar_init(oz_su32(&bar_full[s]), 1);
      oz_mbar_init(oz_su32(&bar_empty[s]), 1);
    }
    for (int r = 0; r < 2; ++r) {
      oz_mbar_init(oz_su32(&bar_tfull[r]), 1);
      oz_mbar_init(oz_su32(&bar_tempty[r]), 4);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     oz_su32(&tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 4) {
    if (lane == 0) {
      // ---- TMA producer: every k-tile of every tile, one ring
      long issued = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int bx, y;
        oz_unit(tile, tiles_xy, a.tiles_m, nprod, order, &bx, &y);
        const int i0 = (bx % a.tiles_m) * OZ_BM, j0 = (bx / a.tiles_m) * OZ_BN;
        const int q0 = a.pfirst[y], nl = (a.pfirst[y + 1] - q0) * a.nk;
        for (int L = 0; L < nl; ++L) {
          const int s = (int)(issued % OZK_STAGES);
          const long use = issued / OZK_STAGES;
          if (use > 0 && !oz_wait(oz_su32(&bar_empty[s]), (uint32_t)((use - 1) & 1), a.err)) {
            ok = false;
            break;
          }
          const int qi = L / a.nk, kt = L - qi * a.nk;
          const int t = a.pt[q0 + qi], u = a.pu[q0 + qi];
          const uint32_t st = base + s * OZ_STAGE;
          const uint32_t fb = oz_su32(&bar_full[s]);
          oz_expect_tx(fb, OZ_STAGE);
          oz_tma_3d(st, &tmA, fb, kt * OZ_BK, i0, 2 * t);
          oz_tma_3d(st + OZ_A_PLANE, &tmA, fb, kt * OZ_BK, i0, 2 * t + 1);
          oz_tma_3d(st + 2 * OZ_A_PLANE, &tmB, fb, kt * OZ_BK, j0, 2 * u);
          oz_tma_3d(st + 2 * OZ_A_PLANE + OZ_B_PLANE, &tmB, fb, kt * OZ_BK, j0, 2 * u + 1);
          ++issued;
        }
      }
      // the copies still in flight land before the CTA leaves
      for (long L = (issued > OZK_STAGES ? issued - OZK_STAGES : 0); L < issued; ++L)
        oz_wait(oz_su32(&bar_full[L % OZK_STAGES]), (uint32_t)((L / OZK_STAGES) & 1), a.err);
    }
    __syncwarp();
  } else if (warp == 5) {
    if (lane == 0) {
      // ---- MMA issuer: chunk gc (counted over the CTA's tiles) into TMEM
      // region gc & 1
      constexpr uint32_t ID = bf16_idesc(OZ_BM, 2 * OZ_BN);
      bool ok = true;
      long gL = 0, gc = 0;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int bx, y;
        oz_unit(tile, tiles_xy, a.tiles_m, nprod, order, &bx, &y);
        const int nl = (a.pfirst[y + 1] - a.pfirst[y]) * a.nk;
        for (int c0 = 0; c0 < nl && ok; c0 += kc, ++gc) {
          const int r = (int)(gc & 1);
          if (gc >= 2 &&
              !oz_wait(oz_su32(&bar_tempty[r]), (uint32_t)(((gc >> 1) - 1) & 1), a.err)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d0 = tmem + 256u * r, d1 = d0 + 128;
          const int L1 = min(nl, c0 + kc);
          for (int L = c0; L < L1; ++L, ++gL) {
            const int s = (int)(gL % OZK_STAGES);
            if (!oz_wait(oz_su32(&bar_full[s]), (uint32_t)((gL / OZK_STAGES) & 1), a.err)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = base + s * OZ_STAGE;
#pragma unroll
            for (int j = 0; j < OZ_BK / 16; ++j) {
              const uint32_t ko = 32u * j;
              const uint64_t are = oz_desc(st + ko);
              const uint64_t aim = oz_desc(st + OZ_A_PLANE + ko);
              const uint64_t by = oz_desc(st + 2 * OZ_A_PLANE + ko);
              const uint32_t acc = (L == c0 && j == 0) ? 0u : 1u;
              oz_mma(d0, are, by, ID, acc);
              oz_mma(d1, aim, by, ID, acc);
            }
            oz_commit(oz_su32(&bar_empty[s]));
          }
          if (ok) oz_commit(oz_su32(&bar_tfull[r]));
        }
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue warps: each tile's chunks -> exact int32 sums -> slots
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    bool ok = true;
    long gc = 0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      int bx, y;
      oz_unit(tile, tiles_xy, a.tiles_m, nprod, order, &bx, &y);
      const int i0 = (bx % a.tiles_m) * OZ_BM, j0 = (bx / a.tiles_m) * OZ_BN;
      const int nl = (a.pfirst[y + 1] - a.pfirst[y]) * a.nk;
      int sre_acc[OZ_BN], sim_acc[OZ_BN];
#pragma unroll
      for (int c = 0; c < OZ_BN; ++c) sre_acc[c] = sim_acc[c] = 0;
      for (int c0 = 0; c0 < nl; c0 += kc, ++gc) {
        const int r = (int)(gc & 1);
        ok = __all_sync(0xffffffffu,
                        oz_wait(oz_su32(&bar_tfull[r]), (uint32_t)((gc >> 1) & 1), a.err));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d0 = tmem + 256u * r + lane_off, d1 = d0 + 128;
#pragma unroll
        for (int c1 = 0; c1 < OZ_BN; c1 += 16) {
          uint32_t rr[16], ri[16], ir[16], ii[16];
          OZ_LD16(d0 + c1, rr);
          OZ_LD16(d0 + OZ_BN + c1, ri);
          OZ_LD16(d1 + c1, ir);
          OZ_LD16(d1 + OZ_BN + c1, ii);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            sre_acc[c1 + k] += __float2int_rn(__uint_as_float(rr[k])) -
                               __float2int_rn(__uint_as_float(ii[k]));
            sim_acc[c1 + k] += __float2int_rn(__uint_as_float(ri[k])) +
                               __float2int_rn(__uint_as_float(ir[k]));
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(oz_su32(&bar_tempty[r]))
                       : "memory");
      }
      const int gi = i0 + warp * 32 + lane;
      if (ok && gi < a.N) {
        int* sre = a.slots + (long)a.ps[y] * a.slot_stride;
        int* sim = sre + (long)a.nrhs * a.N;
#pragma unroll
        for (int c = 0; c < OZ_BN; ++c) {
          const int j = j0 + c;
          if (j < a.nrhs) {
            const long o = (long)j * a.N + gi;
            sre[o] = sre_acc[c];
            sim[o] = sim_acc[c];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// The double nearest to a 2^x (a a signed 128-bit integer; ties to even),
// by integer operations: the bit length, the top 53 bits rounded on the
// bits below them, the exponent and sign put in place. Results outside the
// normal range (not met by Z's entries) go through ldexp.
__device__ __forceinline__ double oz_i128_to_double(__int128 a, int x) {
  if (a == 0) return 0.0;
  const unsigned long long sign = (a < 0) ? (1ull << 63) : 0ull;
  const unsigned __int128 u = (a < 0) ? (unsigned __int128)(-a) : (unsigned __int128)a;
  const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
  const int nb = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
  unsigned long long mant;
  int ex = x;  // |a| 2^x = mant 2^ex
  if (nb <= 53) {
    mant = lo << (53 - nb);
    ex -= 53 - nb;
  } else {
    const int sh = nb - 53;
    mant = (unsigned long long)(u >> sh);
    const unsigned __int128 rem = u & ((((unsigned __int128)1) << sh) - 1);
    const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) ++mant;
    ex += sh;
    if (mant >> 53) {
      mant >>= 1;
      ++ex;
    }
  }
  const int ef = ex + 52 + 1023;  // mant in [2^52, 2^53)
  if (ef >= 1 && ef <= 2046)
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)ef << 52) | (mant & 0xFFFFFFFFFFFFFull)));
  const double v = ldexp((double)mant, ex);
  return sign ? -v : v;
}

// Groups -> FP64. The pair results of a chunk of groups (descending g, from
// g_hi to g_lo) are loaded 16 at a time (independent loads in flight) and
// summed exactly in a 128-bit integer in units of the chunk's smallest
// weight, unit(g_hi): pair p of group g enters times 2^shift[p], shift =
// b (g_hi - g) (at most 78 pairs of |v| < 2^26 and shifts up to 88: below
// 2^121). A single chunk (the usual case) is rounded once, straight to
// R = S - I 2^((sig_i + 1) + (tau_j + 1) - b g_hi); with several, the
// running sum acc (units of the last chunk's g_lo) is carried in FP64,
// acc = acc 2^-(span + b) + I 2^-span, span = b (g_hi - g_lo), and the
// last chunk (g_lo = 2) writes R = S - acc 2^((sig_i + 1) + (tau_j + 1) - 2b).
struct OzCombine {
  int np;                              // pairs in this chunk
  int span;                            // b (g_hi - g_lo)
  unsigned char slot[kOzMaxPairs];     // slot of pair p
  unsigned char shift[kOzMaxPairs];    // b (g_hi - g) of pair p's group
};

__global__ void oz_combine_kernel(int N, int nrhs, const int* __restrict__ slots, long slot_stride,
                                  const __grid_constant__ OzCombine c, int b, int ghi, int first,
                                  int last, double* __restrict__ acc_re, double* __restrict__ acc_im,
                                  const int* __restrict__ rexp, const int* __restrict__ cexp,
                                  const double* sr, const double* si, double* rr, double* ri,
                                  long ldr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= N) return;
  const long o = (long)j * N + i;
  __int128 ar = 0, ai = 0;
  for (int p0 = 0; p0 < c.np; p0 += 16) {
    int vre[16], vim[16];
#pragma unroll
    for (int y = 0; y < 16; ++y) {
      vre[y] = 0;
      vim[y] = 0;
      if (p0 + y < c.np) {
        const int* sl = slots + (long)c.slot[p0 + y] * slot_stride;
        vre[y] = sl[o];
        vim[y] = sl[(long)nrhs * N + o];
      }
    }
#pragma unroll
    for (int y = 0; y < 16; ++y) {
      if (p0 + y < c.np) {
        const int sh = c.shift[p0 + y];
        ar += (__int128)((unsigned __int128)(__int128)vre[y] << sh);
        ai += (__int128)((unsigned __int128)(__int128)vim[y] << sh);
      }
    }
  }
  const int er = rexp[i], ec = cexp[j];
  const bool none = oz_none(er) || oz_none(ec);
  double vr = 0.0, vi = 0.0;
  if (first && last) {
    if (!none) {
      const int x = (er + 1) + (ec + 1) - b * ghi;
      vr = oz_i128_to_double(ar, x);
      vi = oz_i128_to_double(ai, x);
    }
  } else {
    double cr = oz_i128_to_double(ar, -c.span), ci = oz_i128_to_double(ai, -c.span);
    if (!first) {
      const double w = ldexp(1.0, -(c.span + b));
      cr = fma(acc_re[o], w, cr);
      ci = fma(acc_im[o], w, ci);
    }
    if (!last) {
      acc_re[o] = cr;
      acc_im[o] = ci;
      return;
    }
    if (!none) {
      const int e = (er + 1) + (ec + 1) - 2 * b;
      vr = ldexp(cr, e);
      vi = ldexp(ci, e);
    }
  }
  const long r = (long)j * ldr + i;
  rr[r] = sr[r] - vr;
  ri[r] = si[r] - vi;
}

// ---------------------------------------------------------------------------
// The FP64-accurate fill (Eq. 3 in Eq. 4) as an exact-slice product on the
// tensor cores. Per ordered antenna pair (m, n), m != n,
//   Z^{mn}_TS = sum_k C[i][k] Phi[k][j],  i = T + Nm S,  j = m + Na n,
// with C[i][k] = c_{pq}^{TS} (k = (p + P)(Q + 1) + q, the table's order) and
// Phi[k][j] = e^{-jkr} e^{j p alpha} d^q of the pair: a product of
// Nm^2 x K by K x Na^2, cut into digits like the residual's (rows of C and
// columns of Phi scaled by their largest exponent), the pair products
// formed by oz_mma_kernel, the groups combined exactly and written to Z64's
// blocks. The basis is never stored: the digit kernel forms each column in
// FP64 from the pair's geometry.

// Digits of C: out[(2t + p) * plane + i * Kp + k] for rows i < Np (zero from
// Nm^2) and k < Kp (zero from K); rexp[i] the row's exponent. One warp per
// row.
__global__ void oz_fill_slice_c_kernel(int Nm, int K, int Kp, int Np,
                                       const double2* __restrict__ coef, int b, int s,
                                       int* rexp, __nv_bfloat16* out, size_t plane) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= Np) return;
  const int Nm2 = Nm * Nm;
  const int T = i % Nm, S = i / Nm;
  const double2* row = coef + ((size_t)T * Nm + S) * K;
  int e = OZ_NOEXP;
  if (i < Nm2)
    for (int k = lane; k < K; k += 32) {
      const double2 v = row[k];
      if (v.x != 0.0) e = max(e, exp_above(v.x));
      if (v.y != 0.0) e = max(e, exp_above(v.y));
    }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
  if (lane == 0) rexp[i] = e;
  for (int k = lane; k < Kp; k += 32) {
    const double2 v = (i < Nm2 && k < K) ? row[k] : make_double2(0.0, 0.0);
    __nv_bfloat16* o = out + (size_t)i * Kp + k;
    oz_digits(v.x, e, b, s, o, 2 * plane);
    oz_digits(v.y, e, b, s, o + plane, 2 * plane);
  }
}

// Digits of Phi for the pair columns j0 .. j0 + nc - 1 (padded to ncp with
// zero columns): out[(2u + p) * plane + jj * Kp + k], cexp[jj] the column's
// exponent. A block of 4 warps takes kPhiCols = 16 columns. First lanes
// 0..15 of warp 0 form one column's factors each in FP64 (Eq. 3, 4): the
// geometry, E_p = e^{-jkr} e^{j p alpha} for |p| <= P and d^q for q <= Q,
// into shared memory (one warp for all: the FP64 pipe's cost is per warp
// instruction; 16 columns a block so that several blocks share an SM and
// one block's FP64 chain overlaps the others' digits). Then each warp takes
// 4 of the columns: its lanes form the
// basis values phi_{p,q} = E_p d^q of their k (k = lane + 32 i, at most 4
// when K <= 128), the warp their largest exponent, and the digits
// (coalesced along k). Diagonal pairs (m == n) are zero columns (the self
// blocks are written apart); coincident antennas are flagged and give zero
// columns. Shared memory: 16 columns of (2P + 1) complex and (Q + 1) real
// factors.
constexpr int kPhiCols = 16;
__global__ void __launch_bounds__(128) oz_fill_slice_phi_kernel(
    int Na, int P, int Q, int K, int Kp, const double* __restrict__ pos, double kw, int j0, int nc,
    int ncp, int b, int s, int* status, int* cexp, __nv_bfloat16* out, size_t plane) {
  extern __shared__ double2 oz_fac[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ne = 2 * P + 1, nq = Q + 1;
  const int per_col = ne + (nq + 1) / 2;  // double2 slots per column
  double2* E = oz_fac;
  const int jb = blockIdx.x * kPhiCols;  // first column of the block
  if (warp == 0 && lane < kPhiCols) {
    const int jj = jb + lane;
    const int j = j0 + jj;
    const int m = j % Na, n = j / Na;
    bool valid = (jj < nc) && (n < Na) && (m != n);
    double r = 0.0, dx = 0.0, dy = 0.0;
    if (valid) {
      dx = pos[2 * m] - pos[2 * n];
      dy = pos[2 * m + 1] - pos[2 * n + 1];
      r = hypot(dx, dy);
      if (r == 0.0) {
        atomicOr(status, ST_COINCIDENT);
        valid = false;
      }
    }
    double2* Ec = E + (size_t)lane * per_col;
    double* Dc = reinterpret_cast<double*>(Ec + ne);
    if (valid) {
      const double d = 1.0 / r;
      const double zr = dx * d, zi = dy * d;
      double sn, cs;
      sincos(kw * r, &sn, &cs);
      const double phr = cs, phi = -sn;
      Ec[P] = make_double2(phr, phi);
      double pr = 1.0, pi = 0.0;  // (e^{j alpha})^p
      for (int p = 1; p <= P; ++p) {
        const double tr = pr * zr - pi * zi;
        pi = pr * zi + pi * zr;
        pr = tr;
        Ec[P + p] = make_double2(phr * pr - phi * pi, phr * pi + phi * pr);
        Ec[P - p] = make_double2(phr * pr + phi * pi, phi * pr - phr * pi);
      }
      double dq = 1.0;
      for (int q = 0; q < nq; ++q) {
        Dc[q] = dq;
        dq *= d;
      }
    } else {
      for (int p = 0; p < ne; ++p) Ec[p] = make_double2(0.0, 0.0);
      for (int q = 0; q < nq; ++q) Dc[q] = 0.0;
    }
  }
  __syncthreads();
  constexpr int kPer = 4;
  int kp[kPer], kq[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int k = lane + 32 * i;
    kp[i] = (k < K) ? k / nq : -1;
    kq[i] = (k < K) ? k - (k / nq) * nq : 0;
  }
  for (int c = warp; c < kPhiCols; c += (blockDim.x >> 5)) {
    const double2* Ec = E + (size_t)c * per_col;
    const double* Dc = reinterpret_cast<const double*>(Ec + ne);
    double vr[kPer], vi[kPer];
    int e = OZ_NOEXP;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      vr[i] = 0.0;
      vi[i] = 0.0;
      if (kp[i] >= 0) {
        const double2 ep = Ec[kp[i]];
        const double dd = Dc[kq[i]];
        vr[i] = ep.x * dd;
        vi[i] = ep.y * dd;
      }
      if (oz_nz(vr[i])) e = max(e, exp_above(vr[i]));
      if (oz_nz(vi[i])) e = max(e, exp_above(vi[i]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
    const int jj = jb + c;
    if (lane == 0) cexp[jj] = e;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int k = lane + 32 * i;
      if (k >= Kp) break;
      __nv_bfloat16* o = out + (size_t)jj * Kp + k;
      oz_digits(vr[i], e, b, s, o, 2 * plane);
      oz_digits(vi[i], e, b, s, o + plane, 2 * plane);
    }
  }
}

// Groups -> the pair blocks of Z64 for the chunk's columns, one round (every
// product in the slots). Block jj takes pair column jj, thread i = T + Nm S
// of its Nm^2 entries (the slots' layout: coalesced reads, the block's
// columns written in runs of Nm). All product results are loaded first
// (independent loads in flight), then summed exactly in units of the
// smallest group's weight: product y of group ordinal g (counted from
// g_max) enters times 2^(b g), into one of three int64 parts by
// 32-bit steps of that shift (each part below 16 2^26 2^31 = 2^61), and
// the parts are joined in a 128-bit integer (at most 2^26 2^88 16 < 2^118)
// and rounded once to FP64 with the scale 2^((er + 1) + (ec + 1) - b g_max):
// integer work only, off the FP64 pipe.
constexpr int kOzFillMaxProd = 16;
struct OzFillCombine {
  int np;                               // products
  unsigned char slot[kOzFillMaxProd];   // slot of product y
  unsigned char shift[kOzFillMaxProd];  // b times its group ordinal (< 96)
};

__global__ void oz_fill_combine_kernel(int Na, int Nm, int j0, int nc, const int* __restrict__ slots,
                                       long slot_stride, const __grid_constant__ OzFillCombine c,
                                       int b, int gmax, const int* __restrict__ rexp,
                                       const int* __restrict__ cexp, double2* Z, long ldz) {
  const int Nm2 = Nm * Nm;
  const int jj = blockIdx.x, i = threadIdx.x;
  if (i >= Nm2) return;
  const int j = j0 + jj, n = j / Na, m = j - n * Na;
  if (m == n || n >= Na) return;
  const long idx = (long)jj * Nm2 + i;
  const int er = rexp[i], ec = cexp[jj];
  double vr = 0.0, vi = 0.0;
  if (!oz_none(er) && !oz_none(ec)) {
    int vre[kOzFillMaxProd], vim[kOzFillMaxProd];
#pragma unroll
    for (int y = 0; y < kOzFillMaxProd; ++y) {
      vre[y] = 0;
      vim[y] = 0;
      if (y < c.np) {
        const int* sl = slots + (long)c.slot[y] * slot_stride;
        vre[y] = sl[idx];
        vim[y] = sl[(long)nc * Nm2 + idx];
      }
    }
    long long r0 = 0, r1 = 0, r2 = 0, i0 = 0, i1 = 0, i2 = 0;
#pragma unroll
    for (int y = 0; y < kOzFillMaxProd; ++y) {
      if (y < c.np) {
        const int sh = c.shift[y], s5 = sh & 31;
        const long long tr = (long long)vre[y] * (1LL << s5);
        const long long ti = (long long)vim[y] * (1LL << s5);
        if (sh < 32) {
          r0 += tr;
          i0 += ti;
        } else if (sh < 64) {
          r1 += tr;
          i1 += ti;
        } else {
          r2 += tr;
          i2 += ti;
        }
      }
    }
    const __int128 ar = (__int128)r0 + (__int128)r1 * ((__int128)1 << 32) +
                        (__int128)r2 * ((__int128)1 << 64);
    const __int128 ai = (__int128)i0 + (__int128)i1 * ((__int128)1 << 32) +
                        (__int128)i2 * ((__int128)1 << 64);
    const int x = (er + 1) + (ec + 1) - b * gmax;
    vr = oz_i128_to_double(ar, x);
    vi = oz_i128_to_double(ai, x);
  }
  const int S = i / Nm, T = i - S * Nm;
  Z[(size_t)m * Nm + T + ((size_t)n * Nm + S) * ldz] = make_double2(vr, vi);
}

// ---------------------------------------------------------------------------
// G = Lambda X^T (the adjoint's contraction over the right-hand sides) as
// exact digit products: the rows of Lambda are the A operand (oz_prepare's
// layout, K = nrhs), the rows of X in a chunk of columns of G the B operand.
// Product results -> G[i + jj ldg] (FP64 complex) for i < N, jj < ncols:
// loaded 16 at a time and summed exactly in a 128-bit integer at their
// group's weight, 2^shift[y] with shift = b (g_max - g) (at most 78 products
// of |v| < 2^26 and shifts up to 88: below 2^121), then rounded once with
// the scale 2^((sig_i + 1) + (tau_j + 1) - b g_max).
struct OzGramCombine {
  int np;
  unsigned char slot[kOzMaxPairs];
  unsigned char shift[kOzMaxPairs];
};

__global__ void oz_gram_combine_kernel(int N, int ncols, const int* __restrict__ slots,
                                       long slot_stride, const __grid_constant__ OzGramCombine c,
                                       int b, int gmax, const int* __restrict__ rexp,
                                       const int* __restrict__ cexp, double2* G, long ldg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int jj = blockIdx.y;
  if (i >= N) return;
  const long o = (long)jj * N + i;
  const int er = rexp[i], ec = cexp[jj];
  double vr = 0.0, vi = 0.0;
  if (!oz_none(er) && !oz_none(ec)) {
    __int128 ar = 0, ai = 0;
    for (int p0 = 0; p0 < c.np; p0 += 16) {
      int vre[16], vim[16];
#pragma unroll
      for (int y = 0; y < 16; ++y) {
        vre[y] = 0;
        vim[y] = 0;
        if (p0 + y < c.np) {
          const int* sl = slots + (long)c.slot[p0 + y] * slot_stride;
          vre[y] = sl[o];
          vim[y] = sl[(long)ncols * N + o];
        }
      }
#pragma unroll
      for (int y = 0; y < 16; ++y) {
        if (p0 + y < c.np) {
          const int sh = c.shift[p0 + y];
          ar += (__int128)((unsigned __int128)(__int128)vre[y] << sh);
          ai += (__int128)((unsigned __int128)(__int128)vim[y] << sh);
        }
      }
    }
    const int x = (er + 1) + (ec + 1) - b * gmax;
    vr = oz_i128_to_double(ar, x);
    vi = oz_i128_to_double(ai, x);
  }
  G[(long)jj * ldg + i] = make_double2(vr, vi);
}

// ---------------------------------------------------------------------------
// The adjoint's coefficient contraction H[(m, n)][k] = sum_TS G^{mn}_TS c_k^{TS}
// as exact digit products: the A operand is G pair-major (row r = m + Na nl
// of the chunk's source antennas n = n0 + nl, K index ts = T Nm + S, the
// table's order), the B operand the coefficient table transposed (row k, K
// index ts: oz_slice_a with the table's own strides). One warp per A row: the row's largest
// exponent, then its digits out[(2t + p) plane + r Kp + ts].
__global__ void oz_slice_gpm_kernel(int Na, int Nm, int rows, int Rp, int Kp,
                                    const double2* __restrict__ G, long ldg, int b, int s,
                                    int* rexp, __nv_bfloat16* out, size_t plane) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= Rp) return;
  const int Nm2 = Nm * Nm;
  const int m = r % Na, nl = r / Na;
  const bool in = r < rows;
  const double2* g0 = G + (size_t)m * Nm + (size_t)nl * Nm * ldg;
  int e = OZ_NOEXP;
  if (in)
    for (int ts = lane; ts < Nm2; ts += 32) {
      const int T = ts / Nm, S = ts - T * Nm;  // the table's order, T S
      const double2 v = g0[T + (size_t)S * ldg];
      if (oz_nz(v.x)) e = max(e, exp_above(v.x));
      if (oz_nz(v.y)) e = max(e, exp_above(v.y));
    }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, off));
  if (lane == 0) rexp[r] = e;
  for (int ts = lane; ts < Kp; ts += 32) {
    double2 v = make_double2(0.0, 0.0);
    if (in && ts < Nm2) {
      const int T = ts / Nm, S = ts - T * Nm;
      v = g0[T + (size_t)S * ldg];
    }
    __nv_bfloat16* o = out + (size_t)r * Kp + ts;
    oz_digits(v.x, e, b, s, o, 2 * plane);
    oz_digits(v.y, e, b, s, o + plane, 2 * plane);
  }
}

// The self blocks onto the diagonal blocks of Z64: thread (e, m), e = T + Nm S.
__global__ void oz_fill_self_kernel(int Na, int Nm, const double2* __restrict__ self,
                                    long self_stride, double2* Z, long ldz) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (e >= Nm * Nm) return;
  const int T = e % Nm, S = e / Nm;
  Z[(size_t)m * Nm + T + ((size_t)m * Nm + S) * ldz] =
      self[(size_t)m * self_stride + T + (size_t)S * Nm];
}

// ---------------------------------------------------------------------------
// Host side.

// The digit-product kernel's shared-memory limit, set once per device (the
// attribute belongs to the current device; contexts on several devices and
// the batch's worker threads call this concurrently).
static int oz_mma_attr() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  HARP_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load() & bit) return HARP_OK;
  HARP_CUDA(cudaFuncSetAttribute(oz_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 OZ_STAGES * OZ_STAGE + 1024));
  HARP_CUDA(cudaFuncSetAttribute(oz_mma_ks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 OZK_STAGES * OZ_STAGE + 1024));
  done.fetch_or(bit);
  return HARP_OK;
}
static PFN_cuTensorMapEncodeTiled_v12000 oz_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// 3-D map over bf16 planes [np][rows][Kp], box (64, box_rows, 1), 128B swizzle.
static bool oz_map(CUtensorMap* m, void* base, int rows, int Kp, int np, int box_rows) {
  auto enc = oz_encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)np};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * (cuuint64_t)rows};
  cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int ceil_log2(long v) {
  int c = 0;
  while ((1L << c) < v) ++c;
  return c;
}

// The products of a round: the persistent K-split kernel where its chunks
// are exact (8-bit digits: 16 k-tiles, 64 2^14 16 = 2^24, whatever the
// pairs a product sums) and `persistent` asks for it, else one CTA per tile
// and product (two per SM; the better of the two for the fill's short
// products: 1.37 against 1.49 ms at the station).
static int launch_pair_products(const harp_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb,
                                const OzArgs& a, int tiles_xy, int nprod, int b, bool persistent,
                                cudaStream_t st) {
  if (b == 8 && persistent) {
    const int ntiles = tiles_xy * nprod;
    oz_mma_ks_kernel<<<std::min(ntiles, ctx->num_sms), OZK_THREADS, OZK_STAGES * OZ_STAGE + 1024,
                       st>>>(ma, mb, a, 16, tiles_xy, ntiles, 0);
  } else {
    oz_mma_kernel<<<dim3(tiles_xy, nprod), OZ_THREADS, OZ_STAGES * OZ_STAGE + 1024, st>>>(ma, mb,
                                                                                         a);
  }
  HARP_LAUNCHED();
  return HARP_OK;
}

int oz_digit_bits(int K) {
  // K 2^(2b-2) <= 2^24, and |digit| <= 2^(b-1) <= 128 exact in bf16
  const int b = (24 - ceil_log2(std::max(K, 1))) / 2 + 1;
  return std::min(8, b);
}

// The residual's digits: 8 bits at any K, the products running in K chunks
// of kOzSplitTiles k-tiles (64 2^14 16 = 2^24) when K is longer
// (oz_mma_ks_kernel).
int oz_resid_bits(int K) {
  (void)K;
  return 8;
}
constexpr int kOzSplitTiles = 16;

int oz_groups(int K, int b, double rho) {
  // Smallest G with b (G - 1) >= 53 + log2(sqrt K) + log2 G + log2 rho. The
  // first dropped group (G pair sums of digits below 2^(b-1), weight
  // 2^-b(G+1)) is below G 2^(-b(G-1)-2) of 2^(sig+tau) per term; over K terms
  // of random sign, sqrt(K) times that, i.e. below 2^-55 of 2^(sig+tau) <=
  // 16 ||op(Z)||_inf max|X_j|: under 2^-51 of the stopping test's scale,
  // about the FP64 rounding of one residual entry. rho scales the
  // correction's columns against the iterate's.
  const double lr = (rho > 0.0) ? std::log2(std::min(rho, 1.0)) : -1100.0;
  for (int G = 2; G <= kOzMaxG; ++G)
    if (b * (G - 1) >= 53.0 + 0.5 * std::log2((double)std::max(K, 1)) + std::log2((double)G) + lr)
      return G;
  return kOzMaxG;
}

int oz_pairs(int G) { return G * (G - 1) / 2; }

int oz_prepare(harp_ctx* ctx, int N, const double2* z, long ld, bool trans, double* znorm,
               cudaStream_t st) {
  if (!ctx->oz_a) return HARP_E_UNSUPPORTED;
  ctx->oz_ticket = -1;  // the caller marks slices made from a fill's Z64
  const int b = oz_resid_bits(N);
  const int s = oz_groups(N, b, 1.0) - 1;
  if (s > ctx->oz_max_slices) return HARP_E_UNSUPPORTED;
  const int Kp = (N + OZ_BK - 1) / OZ_BK * OZ_BK;
  const int Np = (N + OZ_BM - 1) / OZ_BM * OZ_BM;
  const long ars = trans ? ld : 1, acs = trans ? 1 : ld;
  const int kchunk = (N + OZ_KCH - 1) / OZ_KCH;
  const int nch = (N + kchunk - 1) / kchunk;
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  HARP_CUDA(cudaMemsetAsync(ctx->oz_rexp, 0x80, sizeof(int) * N, st));  // "no entry"
  oz_rowexp_kernel<<<dim3((N + 31) / 32, nch), 256, 0, st>>>(N, N, z, ars, acs, kchunk,
                                                            ctx->oz_rexp, ctx->oz_part);
  HARP_LAUNCHED();
  HARP_CUDA(cudaMemsetAsync(znorm, 0, sizeof(double), st));
  oz_rownorm_kernel<<<(N + 255) / 256, 256, 0, st>>>(N, nch, ctx->oz_part, znorm);
  HARP_LAUNCHED();
  const size_t plane = (size_t)Np * Kp;
  oz_slice_a_kernel<<<dim3(Kp / 32, Np / 32), 256, 0, st>>>(
      N, N, Np, Kp, z, ars, acs, ctx->oz_rexp, b, s, (__nv_bfloat16*)ctx->oz_a, plane);
  HARP_LAUNCHED();
  ctx->oz_N = N;
  ctx->oz_bits = b;
  ctx->oz_slices = s;
  ctx->oz_Kp = Kp;
  ctx->oz_Np = Np;
  return HARP_OK;
}

int oz_residual(harp_ctx* ctx, int N, int nrhs, const float* yr, const float* yi, long ldy,
                const double* sr, const double* si, double* rr, double* ri, long ldr, double rho,
                int prof_kind, cudaStream_t st) {
  if (!ctx->oz_a || ctx->oz_N != N) return HARP_E_STATE;
  if (nrhs < 1 || nrhs > ctx->max_nrhs) return HARP_E_UNSUPPORTED;
  const int b = ctx->oz_bits, Kp = ctx->oz_Kp, Np = ctx->oz_Np;
  const int G = std::min(oz_groups(N, b, rho), ctx->oz_slices + 1);
  const int sy = G - 1;
  const int nrhs_p = (nrhs + OZ_BN - 1) / OZ_BN * OZ_BN;
  const size_t plane_y = (size_t)nrhs_p * Kp;
  {
    ProfScope ps(HARP_K_OTHER, 0.0, st);
    oz_colexp_y_kernel<<<nrhs, 256, 0, st>>>(N, yr, yi, ldy, ctx->oz_cexp);
    HARP_LAUNCHED();
    oz_slice_y_kernel<<<dim3((Kp + 255) / 256, nrhs_p), 256, 0, st>>>(
        N, nrhs, Kp, yr, yi, ldy, ctx->oz_cexp, b, sy, (__nv_bfloat16*)ctx->oz_y, plane_y);
    HARP_LAUNCHED();
  }
  // the operands are zero padded to whole tiles, so no box leaves its tensor
  CUtensorMap ma, mb;
  if (!oz_map(&ma, ctx->oz_a, Np, Kp, 2 * ctx->oz_slices, OZ_BM) ||
      !oz_map(&mb, ctx->oz_y, nrhs_p, Kp, 2 * sy, OZ_BN))
    return HARP_E_UNSUPPORTED;
  HARP_TRY(oz_mma_attr());
  const int tiles_m = Np / OZ_BM, tiles_n = nrhs_p / OZ_BN;
  const long slot_stride = 2L * nrhs * N;
  // Groups in descending g, cut into chunks that the slot buffer holds. With
  // K above one exact FP32 sum the products run on the K-split kernel. When
  // the digit pairs do not fit the slots in one round (large N x nrhs), it
  // also sums up to `run` pairs of a group in one slot (at most what int32
  // holds, and at most 3 so that the persistent CTAs' units stay even),
  // with the units ordered by row block of A: config 5's forward step 854
  // -> 759 ms. Otherwise one pair a product, ordered by A slice (at the
  // station the grouped form took 0.56-0.64 ms for the first residual
  // instead of 0.52).
  const bool split = (Kp / OZ_BK > kOzSplitTiles);
  int all_pairs = 0;
  for (int gg = G; gg >= 2; --gg)
    all_pairs += std::max(0, std::min(gg - 1, ctx->oz_slices) - std::max(1, gg - sy) + 1);
  const bool group = split && all_pairs > ctx->oz_slot_pairs;
  const int run = group ? (int)std::min<long>(
                              3, std::max<long>(1, (long)(0x7fffffff /
                                                          ((long)2 * Kp << (2 * b - 2)))))
                        : 1;
  int g = G;
  bool first = true;
  while (g >= 2) {
    OzArgs a;
    OzCombine c;
    a.N = N;
    a.nrhs = nrhs;
    a.nk = Kp / OZ_BK;
    a.tiles_m = tiles_m;
    a.err = ctx->dstatus + 2;
    a.slots = ctx->oz_slots;
    a.slot_stride = slot_stride;
    int np = 0;
    const int ghi = g;
    if (split) {
      // one product per run of a group's pairs: the K-split kernel sums them
      // exactly in its int32 registers (each pair's real parts below
      // 2 N 2^(2b-2)); one slot per product
      int nprod = 0;
      a.pfirst[0] = 0;
      while (g >= 2) {
        const int tlo = std::max(1, g - sy), thi = std::min(g - 1, ctx->oz_slices);
        const int cnt = std::max(0, thi - tlo + 1);
        const int prods = (cnt + run - 1) / run;
        if (nprod > 0 && nprod + prods > ctx->oz_slot_pairs) break;
        if (prods > ctx->oz_slot_pairs || np + cnt > kOzMaxPairs) return HARP_E_UNSUPPORTED;
        for (int t = tlo; t <= thi; ++t) {
          a.pt[np] = (unsigned char)(t - 1);
          a.pu[np] = (unsigned char)(g - t - 1);
          ++np;
          if (t == thi || np - a.pfirst[nprod] == run) {
            a.ps[nprod] = (unsigned char)nprod;
            c.slot[nprod] = (unsigned char)nprod;
            c.shift[nprod] = (unsigned char)(b * (ghi - g));
            a.pfirst[++nprod] = (unsigned char)np;
          }
        }
        --g;
      }
      c.np = nprod;
      c.span = b * (ghi - (g + 1));
      if (c.span > 88) return HARP_E_UNSUPPORTED;
      const bool last = (g < 2);
      if (nprod > 0) {
        if (!group) {
          // one pair a product: order them by A slice so that one slice is
          // live in L2 at a time (a product's slot stays its own)
          std::vector<int> ord(nprod);
          for (int k = 0; k < nprod; ++k) ord[k] = k;
          std::stable_sort(ord.begin(), ord.end(),
                           [&](int x, int y) { return a.pt[x] < a.pt[y]; });
          unsigned char pt[kOzMaxPairs], pu[kOzMaxPairs], psl[kOzMaxPairs];
          for (int k = 0; k < nprod; ++k) {
            pt[k] = a.pt[ord[k]];
            pu[k] = a.pu[ord[k]];
            psl[k] = a.ps[ord[k]];
          }
          for (int k = 0; k < nprod; ++k) {
            a.pt[k] = pt[k];
            a.pu[k] = pu[k];
            a.ps[k] = psl[k];
          }
        }
        // grouped products mix A slices: units ordered by row block of A
        ProfScope ps(prof_kind, 8.0 * np * (double)N * N * nrhs, st);
        const int ntiles = tiles_m * tiles_n * nprod;
        oz_mma_ks_kernel<<<std::min(ntiles, ctx->num_sms), OZK_THREADS,
                           OZK_STAGES * OZ_STAGE + 1024, st>>>(
            ma, mb, a, kOzSplitTiles, tiles_m * tiles_n, ntiles, group ? 1 : 0);
        HARP_LAUNCHED();
      }
      {
        ProfScope ps(HARP_K_OTHER, 0.0, st);
        oz_combine_kernel<<<dim3((N + 255) / 256, nrhs), 256, 0, st>>>(
            N, nrhs, ctx->oz_slots, slot_stride, c, b, ghi, first ? 1 : 0, last ? 1 : 0,
            ctx->oz_acc, ctx->oz_acc + (size_t)N * nrhs, ctx->oz_rexp, ctx->oz_cexp, sr, si, rr,
            ri, ldr);
        HARP_LAUNCHED();
      }
      first = false;
      continue;
    }
    while (g >= 2) {
      const int tlo = std::max(1, g - sy), thi = std::min(g - 1, ctx->oz_slices);
      const int cnt = std::max(0, thi - tlo + 1);
      if (np > 0 && np + cnt > ctx->oz_slot_pairs) break;
      if (cnt > ctx->oz_slot_pairs || np + cnt > kOzMaxPairs) return HARP_E_UNSUPPORTED;
      for (int t = tlo; t <= thi; ++t) {
        c.slot[np] = (unsigned char)np;
        c.shift[np] = (unsigned char)(b * (ghi - g));
        a.pt[np] = (unsigned char)(t - 1);
        a.pu[np] = (unsigned char)(g - t - 1);
        a.ps[np] = (unsigned char)np;
        ++np;
      }
      --g;
    }
    c.np = np;
    c.span = b * (ghi - (g + 1));
    if (c.span > 88) return HARP_E_UNSUPPORTED;
    const bool last = (g < 2);
    if (np > 0) {
      // order the products by A slice so that one slice is live in L2 at a time
      std::vector<int> ord(np);
      for (int k = 0; k < np; ++k) ord[k] = k;
      std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return a.pt[x] < a.pt[y]; });
      unsigned char pt[kOzMaxPairs], pu[kOzMaxPairs], psl[kOzMaxPairs];
      for (int k = 0; k < np; ++k) {
        pt[k] = a.pt[ord[k]];
        pu[k] = a.pu[ord[k]];
        psl[k] = a.ps[ord[k]];
      }
      for (int k = 0; k < np; ++k) {
        a.pt[k] = pt[k];
        a.pu[k] = pu[k];
        a.ps[k] = psl[k];
        a.pfirst[k] = (unsigned char)k;
      }
      a.pfirst[np] = (unsigned char)np;
      ProfScope ps(prof_kind, 8.0 * np * (double)N * N * nrhs, st);
      oz_mma_kernel<<<dim3(tiles_m * tiles_n, np), OZ_THREADS, OZ_STAGES * OZ_STAGE + 1024, st>>>(
          ma, mb, a);
      HARP_LAUNCHED();
    }
    {
      ProfScope ps(HARP_K_OTHER, 0.0, st);
      oz_combine_kernel<<<dim3((N + 255) / 256, nrhs), 256, 0, st>>>(
          N, nrhs, ctx->oz_slots, slot_stride, c, b, ghi, first ? 1 : 0, last ? 1 : 0, ctx->oz_acc,
          ctx->oz_acc + (size_t)N * nrhs, ctx->oz_rexp, ctx->oz_cexp, sr, si, rr, ri, ldr);
      HARP_LAUNCHED();
    }
    first = false;
  }
  return HARP_OK;
}

// The FP64-accurate fill on the tensor cores (see oz_fill_slice_c_kernel
// and what follows): HARP_E_UNSUPPORTED when the residual's buffers are
// absent or too small for it, or the model is outside the kernels' limits
// (K <= 128, P, Q < 32); the caller then uses the float-float kernel.
int oz_fill_z64(harp_ctx* ctx, int Na, int Nm, int P, int Q, const double* pos, double kw,
                const double2* coef, const double2* self, long self_stride, double2* Z, long ldz,
                int* status, cudaStream_t st) {
  if (!ctx->oz_a || !ctx->oz_y || !ctx->oz_slots || !ctx->oz_rexp || !ctx->oz_part)
    return HARP_E_UNSUPPORTED;
  const int K = (2 * P + 1) * (Q + 1);
  if (K > 128 || P > 31 || Q > 31) return HARP_E_UNSUPPORTED;
  const int Nm2 = Nm * Nm;
  if (Na > 65535) return HARP_E_UNSUPPORTED;  // grid rows of the self-block kernel
  const int b = oz_digit_bits(K);
  const int G = oz_groups(K, b, 1.0);
  const int sl = G - 1;
  if (sl > ctx->oz_max_slices) return HARP_E_UNSUPPORTED;
  const int Kp = (K + OZ_BK - 1) / OZ_BK * OZ_BK;
  const int Np = (Nm2 + OZ_BM - 1) / OZ_BM * OZ_BM;
  if (Np > ctx->max_N) return HARP_E_UNSUPPORTED;  // row exponents in oz_rexp
  // buffer capacities (bf16 elements, ints), as ctx.cu sizes them
  const size_t kpN = ((size_t)ctx->max_N + 63) / 64 * 64, npN = ((size_t)ctx->max_N + 127) / 128 * 128;
  const size_t rpN = ((size_t)ctx->max_nrhs + 63) / 64 * 64;
  const size_t a_cap = 2 * (size_t)ctx->oz_max_slices * npN * kpN;
  const size_t y_cap = 2 * (size_t)ctx->oz_max_slices * rpN * kpN;
  const size_t slot_cap = (size_t)ctx->oz_slot_pairs * 2 * (size_t)ctx->max_N * ctx->max_nrhs;
  const size_t cexp_cap = 2 * 32 * (size_t)ctx->max_N;  // oz_part as ints
  if (2 * (size_t)sl * Np * Kp > a_cap) return HARP_E_UNSUPPORTED;
  // The pairs (t, u), t + u = g, in descending groups, one round. The pairs
  // of a group add up in one product's FP32 accumulators while the sum stays
  // an exact integer: each pair's real products are below K 2^(2b-2), so
  // runs of up to 2^24 / (K 2^(2b-2)) pairs (10 at K = 102, b = 8).
  const long run = std::max<long>(1, (1L << 24) / ((long)K << (2 * b - 2)));
  OzArgs a;
  OzFillCombine c;
  int np = 0, nprod = 0;
  a.pfirst[0] = 0;
  for (int g = G; g >= 2; --g) {
    const int tlo = std::max(1, g - sl), thi = std::min(g - 1, sl);
    for (int t = tlo; t <= thi; ++t) {
      if (np >= kOzMaxPairs) return HARP_E_UNSUPPORTED;
      a.pt[np] = (unsigned char)(t - 1);
      a.pu[np] = (unsigned char)(g - t - 1);
      ++np;
      if (t == thi || np - a.pfirst[nprod] == run) {
        if (nprod >= kOzFillMaxProd) return HARP_E_UNSUPPORTED;
        a.ps[nprod] = (unsigned char)nprod;
        c.slot[nprod] = (unsigned char)nprod;
        c.shift[nprod] = (unsigned char)(b * (G - g));
        a.pfirst[++nprod] = (unsigned char)np;
      }
    }
  }
  c.np = nprod;
  // one combine block per pair column (Nm^2 threads)
  if (nprod < 1 || b * (G - 2) > 88 || Nm2 > 1024) return HARP_E_UNSUPPORTED;
  // pair columns per round: up to 8192 (enough basis blocks to spread the
  // FP64 geometry over the SMs; the round's products, ~75 MB at 144 MBF
  // pairs, mostly stay in L2), within the digit and slot buffers
  long chunk = 8192;
  chunk = std::min<long>(chunk, (long)(y_cap / (2 * (size_t)sl * Kp)) / OZ_BN * OZ_BN);
  chunk = std::min<long>(chunk, (long)(slot_cap / ((size_t)nprod * 2 * Nm2)) / OZ_BN * OZ_BN);
  chunk = std::min<long>(chunk, (long)cexp_cap / OZ_BN * OZ_BN);
  if (chunk < OZ_BN) return HARP_E_UNSUPPORTED;
  __nv_bfloat16* adig = (__nv_bfloat16*)ctx->oz_a;
  __nv_bfloat16* ydig = (__nv_bfloat16*)ctx->oz_y;
  const size_t plane_a = (size_t)Np * Kp;
  int* cexp = reinterpret_cast<int*>(ctx->oz_part);
  {
    ProfScope ps(HARP_K_OTHER, 0.0, st);
    oz_fill_slice_c_kernel<<<(Np + 7) / 8, 256, 0, st>>>(Nm, K, Kp, Np, coef, b, sl, ctx->oz_rexp,
                                                         adig, plane_a);
    HARP_LAUNCHED();
    oz_fill_self_kernel<<<dim3((Nm2 + 127) / 128, Na), 128, 0, st>>>(Na, Nm, self, self_stride, Z,
                                                                      ldz);
    HARP_LAUNCHED();
  }
  HARP_TRY(oz_mma_attr());
  // the basis kernel's factor table: kPhiCols columns
  const size_t phi_smem = kPhiCols * (size_t)(2 * P + 1 + (Q + 2) / 2) * sizeof(double2);
  if (phi_smem > 48 * 1024)
    HARP_CUDA(cudaFuncSetAttribute(oz_fill_slice_phi_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)phi_smem));
  CUtensorMap ma;
  if (!oz_map(&ma, adig, Np, Kp, 2 * sl, OZ_BM)) return HARP_E_UNSUPPORTED;
  const long npairs = (long)Na * Na;
  const int tiles_m = Np / OZ_BM;
  ProfScope ps(HARP_K_FILL_FF, 8.0 * Nm2 * (double)K * Na * (Na - 1), st);
  for (long j0 = 0; j0 < npairs; j0 += chunk) {
    const int nc = (int)std::min<long>(chunk, npairs - j0);
    const int ncp = (nc + OZ_BN - 1) / OZ_BN * OZ_BN;
    const size_t plane_y = (size_t)ncp * Kp;
    oz_fill_slice_phi_kernel<<<ncp / kPhiCols, 128, phi_smem, st>>>(
        Na, P, Q, K, Kp, pos, kw, (int)j0, nc, ncp, b, sl, status, cexp, ydig, plane_y);
    HARP_LAUNCHED();
    CUtensorMap mb;
    if (!oz_map(&mb, ydig, ncp, Kp, 2 * sl, OZ_BN)) return HARP_E_UNSUPPORTED;
    a.N = Nm2;
    a.nrhs = nc;
    a.nk = Kp / OZ_BK;
    a.tiles_m = tiles_m;
    a.err = ctx->dstatus + 2;
    a.slots = ctx->oz_slots;
    a.slot_stride = 2L * nc * Nm2;
    HARP_TRY(launch_pair_products(ctx, ma, mb, a, tiles_m * (ncp / OZ_BN), nprod, b, false, st));
    oz_fill_combine_kernel<<<nc, (Nm2 + 31) / 32 * 32, 0, st>>>(
        Na, Nm, (int)j0, nc, ctx->oz_slots, 2L * nc * Nm2, c, b, G, ctx->oz_rexp, cexp, Z, ldz);
    HARP_LAUNCHED();
  }
  return HARP_OK;
}

// ---------------------------------------------------------------------------
// G = Lambda X^T by exact digit products (oz_gram_combine_kernel). The
// operands are N x nrhs, column-major; K = nrhs.
struct OzGramPlan {
  int b, G, s, Kp, Np, nprod;
  OzArgs a;           // pairs and products (N, nrhs, slots filled per chunk)
  OzGramCombine c;
};

static int oz_gram_plan(const harp_ctx* ctx, int N, int nrhs, OzGramPlan* pl) {
  if (!ctx->oz_a || !ctx->oz_y || !ctx->oz_slots || !ctx->oz_rexp || !ctx->oz_part)
    return HARP_E_UNSUPPORTED;
  if (N < 1 || nrhs < 1 || N > ctx->max_N) return HARP_E_UNSUPPORTED;
  pl->b = oz_digit_bits(nrhs);
  pl->G = oz_groups(nrhs, pl->b, 1.0);
  pl->s = pl->G - 1;
  if (pl->s > ctx->oz_max_slices) return HARP_E_UNSUPPORTED;
  pl->Kp = (nrhs + OZ_BK - 1) / OZ_BK * OZ_BK;
  pl->Np = (N + OZ_BM - 1) / OZ_BM * OZ_BM;
  const size_t kpN = ((size_t)ctx->max_N + 63) / 64 * 64, npN = ((size_t)ctx->max_N + 127) / 128 * 128;
  if (2 * (size_t)pl->s * pl->Np * pl->Kp > 2 * (size_t)ctx->oz_max_slices * npN * kpN)
    return HARP_E_UNSUPPORTED;
  // pairs t + u = g in descending groups; a product sums up to `run` pairs
  // of one group while its FP32 accumulator stays an exact integer
  const int b = pl->b, G = pl->G, sl = pl->s;
  const long run = std::max<long>(1, (1L << 24) / ((long)nrhs << (2 * b - 2)));
  int np = 0, nprod = 0;
  pl->a.pfirst[0] = 0;
  for (int g = G; g >= 2; --g) {
    const int tlo = std::max(1, g - sl), thi = std::min(g - 1, sl);
    for (int t = tlo; t <= thi; ++t) {
      if (np >= kOzMaxPairs) return HARP_E_UNSUPPORTED;
      pl->a.pt[np] = (unsigned char)(t - 1);
      pl->a.pu[np] = (unsigned char)(g - t - 1);
      ++np;
      if (t == thi || np - pl->a.pfirst[nprod] == run) {
        pl->a.ps[nprod] = (unsigned char)nprod;
        pl->c.slot[nprod] = (unsigned char)nprod;
        pl->c.shift[nprod] = (unsigned char)(b * (G - g));
        pl->a.pfirst[++nprod] = (unsigned char)np;
      }
    }
  }
  if (nprod < 1 || b * (G - 2) > 88) return HARP_E_UNSUPPORTED;
  pl->nprod = nprod;
  pl->c.np = nprod;
  return HARP_OK;
}

int oz_gram_max_cols(const harp_ctx* ctx, int N, int nrhs) {
  OzGramPlan pl;
  if (oz_gram_plan(ctx, N, nrhs, &pl) != HARP_OK) return 0;
  const size_t kpN = ((size_t)ctx->max_N + 63) / 64 * 64;
  const size_t rpN = ((size_t)ctx->max_nrhs + 63) / 64 * 64;
  const size_t y_cap = 2 * (size_t)ctx->oz_max_slices * rpN * kpN;
  const size_t slot_cap = (size_t)ctx->oz_slot_pairs * 2 * (size_t)ctx->max_N * ctx->max_nrhs;
  size_t cols = y_cap / (2 * (size_t)pl.s * pl.Kp) / OZ_BN * OZ_BN;
  cols = std::min(cols, slot_cap / ((size_t)pl.nprod * 2 * N));
  return (int)std::min<size_t>(cols, 65535);  // grid rows of the combine
}

int oz_gram_prepare(harp_ctx* ctx, int N, int nrhs, const double2* Lam, long ldl,
                    const double2* X, long ldx, cudaStream_t st) {
  OzGramPlan pl;
  HARP_TRY(oz_gram_plan(ctx, N, nrhs, &pl));
  // the A buffer no longer holds the slices of Z64
  ctx->oz_N = -1;
  ctx->oz_ticket = -1;
  int* xexp = reinterpret_cast<int*>(ctx->oz_part);
  HARP_CUDA(cudaMemsetAsync(ctx->oz_rexp, 0x80, sizeof(int) * N, st));  // "no entry"
  HARP_CUDA(cudaMemsetAsync(xexp, 0x80, sizeof(int) * N, st));
  const int kchunk = (nrhs + OZ_KCH - 1) / OZ_KCH;
  const int nch = (nrhs + kchunk - 1) / kchunk;
  oz_rowexp_kernel<<<dim3((N + 31) / 32, nch), 256, 0, st>>>(N, nrhs, Lam, 1, ldl, kchunk,
                                                            ctx->oz_rexp, nullptr);
  HARP_LAUNCHED();
  oz_rowexp_kernel<<<dim3((N + 31) / 32, nch), 256, 0, st>>>(N, nrhs, X, 1, ldx, kchunk, xexp,
                                                            nullptr);
  HARP_LAUNCHED();
  oz_slice_a_kernel<<<dim3(pl.Kp / 32, pl.Np / 32), 256, 0, st>>>(
      N, nrhs, pl.Np, pl.Kp, Lam, 1, ldl, ctx->oz_rexp, pl.b, pl.s, (__nv_bfloat16*)ctx->oz_a,
      (size_t)pl.Np * pl.Kp);
  HARP_LAUNCHED();
  return HARP_OK;
}

int oz_gram_chunk(harp_ctx* ctx, int N, int nrhs, const double2* X, long ldx, int j0, int ncols,
                  double2* G, long ldg, cudaStream_t st) {
  OzGramPlan pl;
  HARP_TRY(oz_gram_plan(ctx, N, nrhs, &pl));
  if (ncols < 1 || ncols > oz_gram_max_cols(ctx, N, nrhs) || j0 < 0 || j0 + ncols > N)
    return HARP_E_UNSUPPORTED;
  const int* xexp = reinterpret_cast<const int*>(ctx->oz_part);
  const int ncp = (ncols + OZ_BN - 1) / OZ_BN * OZ_BN;
  __nv_bfloat16* ydig = (__nv_bfloat16*)ctx->oz_y;
  // digits of the chunk's rows of X (the B operand)
  oz_slice_a_kernel<<<dim3(pl.Kp / 32, ncp / 32), 256, 0, st>>>(
      ncols, nrhs, ncp, pl.Kp, X + j0, 1, ldx, xexp + j0, pl.b, pl.s, ydig, (size_t)ncp * pl.Kp);
  HARP_LAUNCHED();
  HARP_TRY(oz_mma_attr());
  CUtensorMap ma, mb;
  if (!oz_map(&ma, ctx->oz_a, pl.Np, pl.Kp, 2 * pl.s, OZ_BM) ||
      !oz_map(&mb, ydig, ncp, pl.Kp, 2 * pl.s, OZ_BN))
    return HARP_E_UNSUPPORTED;
  OzArgs& a = pl.a;
  a.N = N;
  a.nrhs = ncols;
  a.nk = pl.Kp / OZ_BK;
  a.tiles_m = pl.Np / OZ_BM;
  a.err = ctx->dstatus + 2;
  a.slots = ctx->oz_slots;
  a.slot_stride = 2L * ncols * N;
  HARP_TRY(
      launch_pair_products(ctx, ma, mb, a, a.tiles_m * (ncp / OZ_BN), pl.nprod, pl.b, true, st));
  oz_gram_combine_kernel<<<dim3((N + 255) / 256, ncols), 256, 0, st>>>(
      N, ncols, ctx->oz_slots, 2L * ncols * N, pl.c, pl.b, pl.G, ctx->oz_rexp, xexp + j0, G, ldg);
  HARP_LAUNCHED();
  return HARP_OK;
}

// ---------------------------------------------------------------------------
// H = G_pm C^T (oz_slice_gpm_kernel) in a caller's work buffer, laid out as
// [C^T digits | C^T row exponents | G_pm digits | G_pm row exponents].
struct OzAdjHPlan {
  int b, G, s, Kts, Kn, Rp, nprod;
  size_t off_cexp, off_gdig, off_gexp, bytes;
  OzArgs a;
  OzGramCombine c;
};

static int oz_adj_h_plan(const harp_ctx* ctx, int Na, int Nm, int K, int nn, OzAdjHPlan* pl) {
  if (!ctx->oz_slots) return HARP_E_UNSUPPORTED;
  const int Nm2 = Nm * Nm;
  if (K < 1 || K > 128 || Nm2 > 1024 || nn < 1) return HARP_E_UNSUPPORTED;
  pl->b = 8;  // Nm^2 2^14 <= 2^24
  pl->G = oz_groups(Nm2, pl->b, 1.0);
  pl->s = pl->G - 1;
  pl->Kts = (Nm2 + OZ_BK - 1) / OZ_BK * OZ_BK;
  pl->Kn = 128;  // the K output columns, padded to two 64-wide tiles
  const long rows = (long)Na * nn;
  pl->Rp = (int)((rows + OZ_BM - 1) / OZ_BM * OZ_BM);
  const int b = pl->b, G = pl->G, sl = pl->s;
  const long run = std::max<long>(1, (1L << 24) / ((long)Nm2 << (2 * b - 2)));
  int np = 0, nprod = 0;
  pl->a.pfirst[0] = 0;
  for (int g = G; g >= 2; --g) {
    const int tlo = std::max(1, g - sl), thi = std::min(g - 1, sl);
    for (int t = tlo; t <= thi; ++t) {
      if (np >= kOzMaxPairs) return HARP_E_UNSUPPORTED;
      pl->a.pt[np] = (unsigned char)(t - 1);
      pl->a.pu[np] = (unsigned char)(g - t - 1);
      ++np;
      if (t == thi || np - pl->a.pfirst[nprod] == run) {
        pl->a.ps[nprod] = (unsigned char)nprod;
        pl->c.slot[nprod] = (unsigned char)nprod;
        pl->c.shift[nprod] = (unsigned char)(b * (G - g));
        pl->a.pfirst[++nprod] = (unsigned char)np;
      }
    }
  }
  if (nprod < 1 || b * (G - 2) > 88) return HARP_E_UNSUPPORTED;
  pl->nprod = nprod;
  pl->c.np = nprod;
  const size_t slot_cap = (size_t)ctx->oz_slot_pairs * 2 * (size_t)ctx->max_N * ctx->max_nrhs;
  if ((size_t)nprod * 2 * rows * K > slot_cap) return HARP_E_UNSUPPORTED;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t cdig = 2 * (size_t)sl * pl->Kn * pl->Kts * sizeof(__nv_bfloat16);
  pl->off_cexp = al(cdig);
  pl->off_gdig = al(pl->off_cexp + sizeof(int) * pl->Kn);
  pl->off_gexp = al(pl->off_gdig + 2 * (size_t)sl * pl->Rp * pl->Kts * sizeof(__nv_bfloat16));
  pl->bytes = al(pl->off_gexp + sizeof(int) * (size_t)pl->Rp);
  return HARP_OK;
}

size_t oz_adj_h_bytes(const harp_ctx* ctx, int Na, int Nm, int K, int nn) {
  OzAdjHPlan pl;
  return oz_adj_h_plan(ctx, Na, Nm, K, nn, &pl) == HARP_OK ? pl.bytes : 0;
}

int oz_adj_h_prepare(harp_ctx* ctx, int Na, int Nm, int K, int nn, const double2* coef,
                     void* work, cudaStream_t st) {
  OzAdjHPlan pl;
  HARP_TRY(oz_adj_h_plan(ctx, Na, Nm, K, nn, &pl));
  char* w = static_cast<char*>(work);
  int* cexp = reinterpret_cast<int*>(w + pl.off_cexp);
  const int Nm2 = Nm * Nm;
  HARP_CUDA(cudaMemsetAsync(cexp, 0x80, sizeof(int) * pl.Kn, st));  // "no entry"
  // C^T: row k, entry ts at coef[ts K + k]
  const int kchunk = (Nm2 + OZ_KCH - 1) / OZ_KCH;
  const int nch = (Nm2 + kchunk - 1) / kchunk;
  oz_rowexp_kernel<<<dim3((K + 31) / 32, nch), 256, 0, st>>>(K, Nm2, coef, 1, K, kchunk, cexp,
                                                           nullptr);
  HARP_LAUNCHED();
  oz_slice_a_kernel<<<dim3(pl.Kts / 32, pl.Kn / 32), 256, 0, st>>>(
      K, Nm2, pl.Kn, pl.Kts, coef, 1, K, cexp, pl.b, pl.s, (__nv_bfloat16*)w,
      (size_t)pl.Kn * pl.Kts);
  HARP_LAUNCHED();
  return HARP_OK;
}

int oz_adj_h_chunk(harp_ctx* ctx, int Na, int Nm, int K, int nn, const double2* G, long ldg,
                   void* work, double2* H, long ldh, cudaStream_t st) {
  OzAdjHPlan pl;
  HARP_TRY(oz_adj_h_plan(ctx, Na, Nm, K, nn, &pl));
  char* w = static_cast<char*>(work);
  const int* cexp = reinterpret_cast<const int*>(w + pl.off_cexp);
  __nv_bfloat16* gdig = reinterpret_cast<__nv_bfloat16*>(w + pl.off_gdig);
  int* gexp = reinterpret_cast<int*>(w + pl.off_gexp);
  const int rows = Na * nn;
  oz_slice_gpm_kernel<<<(pl.Rp + 7) / 8, 256, 0, st>>>(Na, Nm, rows, pl.Rp, pl.Kts, G, ldg, pl.b,
                                                       pl.s, gexp, gdig,
                                                       (size_t)pl.Rp * pl.Kts);
  HARP_LAUNCHED();
  HARP_TRY(oz_mma_attr());
  CUtensorMap ma, mb;
  if (!oz_map(&ma, gdig, pl.Rp, pl.Kts, 2 * pl.s, OZ_BM) ||
      !oz_map(&mb, w, pl.Kn, pl.Kts, 2 * pl.s, OZ_BN))
    return HARP_E_UNSUPPORTED;
  OzArgs& a = pl.a;
  a.N = rows;
  a.nrhs = K;
  a.nk = pl.Kts / OZ_BK;
  a.tiles_m = pl.Rp / OZ_BM;
  a.err = ctx->dstatus + 2;
  a.slots = ctx->oz_slots;
  a.slot_stride = 2L * K * rows;
  HARP_TRY(launch_pair_products(ctx, ma, mb, a, a.tiles_m * (pl.Kn / OZ_BN), pl.nprod, pl.b,
                                true, st));
  oz_gram_combine_kernel<<<dim3((rows + 255) / 256, K), 256, 0, st>>>(
      rows, K, ctx->oz_slots, 2L * K * rows, pl.c, pl.b, pl.G, gexp, cexp, H, ldh);
  HARP_LAUNCHED();
  return HARP_OK;
}

}  // namespace harp
