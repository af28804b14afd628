// adjoint.cu -- harp_fill_adjoint: position gradient of a real objective of the
// solution X of Z X = V, with the fill recomputed rather than stored.
//
// With G = Lambda X^T (Lambda the adjoint solution), dJ = -2 Re sum_ij G_ij dZ_ij.
// Block (m, n) of Z depends only on Delta = x_m - x_n through r and alpha
// (Eq. 3, 4), so per ordered pair
//   H_k   = sum_TS G^{mn}_TS c_k^{TS}                 (k = (p, q))
//   dZ/dr contraction     = sum_k H_k phi_k (-j kw - q d)
//   dZ/dalpha contraction = sum_k H_k phi_k (j p)
// with phi_k = e^{-j kw r} e^{j p alpha} d^q, d = 1/r (d d^q/dr = -q d^{q+1}),
// and g = -2 Re(dr_sum Delta/r + dalpha_sum (-Delta_y, Delta_x)/r^2);
// grad[m] += g, grad[n] -= g. Per-pair results go to a buffer and are
// summed in a fixed order, so the gradient is deterministic.
//
// Work item = (source antenna n, tile of BA testing antennas). Per item the
// CTA forms G for the tile (contraction over the right-hand sides, X rows of
// antenna n staged in shared memory in chunks), then H (contraction over
// (T, S) with the coefficient table), then the per-pair derivative sums.
//
// Precision of G: FP64 (HARP_FP64), FP32 (HARP_FP32), or, in the mixed
// modes, exact digit products on the bf16 tensor cores rounded once to FP64
// (ozaki.cu: oz_gram_*, option HARP_OPT_ADJOINT_G, the default where the
// context holds the tensor-core residual's buffers), or double-float on the
// FP32 pipe: Lambda and X are first split into
// float pairs (hi + lo, 48 bits), every product is formed error-free
// (Dekker's product via FMA plus the cross terms) and summed into a
// double-float accumulator (Ogita-Rump-Oishi Dot2), which is FP64-accurate
// for these sums at about five times the FP64 pipe's rate on GB300. H and
// the derivative sums stay in FP64.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "ff.cuh"
#include "ozaki.cuh"
#include "prof.cuh"

namespace harp {

constexpr double kC0a = 299792458.0;
constexpr double kPia = 3.14159265358979323846;
constexpr int kAdjThreads = 256;
constexpr int kRChunk = 16;

struct AdjArgs {
  int Na, Nm, P, Q, K, nq, nrhs;
  const double* pos;
  double k;
  const double2* coef;
  const double2* Lam;
  const double2* X;
  long ld;
  double* gpair;  // [m][n][2]
  int BA, n_mtiles, n_items;
  // double-float G: Lambda and X split into (re_hi, re_lo, im_hi, im_lo),
  // column r of the right-hand sides at r * N; the coefficients likewise
  // ([T][S][k] as coef)
  const float4* Lsp;
  const float4* Xsp;
  const float4* Csp;
  // the source antennas of this launch, n0 .. n0 + nn - 1; with G given
  // (digit products): its columns of those antennas, G[i + (j - n0 Nm) ldg]
  int n0, nn;
  const double2* Gc;
  long ldg;
};

// dst[i] = the float pairs of src[i] (real, then imaginary).
__global__ void split_c128_kernel(long n, const double2* __restrict__ src,
                                  float4* __restrict__ dst) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = src[i];
  float rh, rl, ih, il;
  ff_split(v.x, rh, rl);
  ff_split(v.y, ih, il);
  dst[i] = make_float4(rh, rl, ih, il);
}

// dst[r N + i] = the float pairs of src[i + r ld] (real, then imaginary).
__global__ void adjoint_split_kernel(int N, int nrhs, const double2* __restrict__ src, long ld,
                                     float4* __restrict__ dst) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)N * nrhs) return;
  const long r = e / N, i = e - r * N;
  const double2 v = src[i + r * ld];
  float rh, rl, ih, il;
  ff_split(v.x, rh, rl);
  ff_split(v.y, ih, il);
  dst[e] = make_float4(rh, rl, ih, il);
}

// The per-pair derivative sums (FP64) from H_k (h[k hs]) of the pair whose
// separation is (dx, dy), r = |(dx, dy)|: dZ/dr and dZ/dalpha contracted
// with G, then the chain rule to the separation; (0, 0) for r = 0.
template <typename HV>
__device__ void adj_pair_grad(const AdjArgs& a, double dx, double dy, double r, const HV* h,
                              long hs, double* gx, double* gy) {
  *gx = 0.0;
  *gy = 0.0;
  if (!(r > 0.0)) return;
  const double d = 1.0 / r;
  double s, c;
  sincos(a.k * r, &s, &c);
  const double2 ph = make_double2(c, -s);
  const double2 z = make_double2(dx * d, dy * d);
  double2 zp = make_double2(1.0, 0.0);
  double2 sum_r = make_double2(0, 0), sum_a = make_double2(0, 0);
  for (int p = 0; p <= a.P; ++p) {
    const double2 bp = cmul(ph, zp), bn = cmul(ph, cconj(zp));
    double dq = 1.0;
    for (int q = 0; q <= a.Q; ++q) {
      // weight for dZ/dr: (-j kw - q d); for dZ/dalpha: (j p)
      const double2 wr = make_double2(-(double)q * d, -a.k);
      {
        const HV hv = h[(long)((a.P + p) * a.nq + q) * hs];
        const double2 hp = make_double2((double)hv.x * dq, (double)hv.y * dq);
        const double2 t = cmul(hp, bp);
        const double2 tr = cmul(t, wr);
        sum_r.x += tr.x;
        sum_r.y += tr.y;
        sum_a.x += -(double)p * t.y;  // t * (j p)
        sum_a.y += (double)p * t.x;
      }
      if (p > 0) {
        const HV hv = h[(long)((a.P - p) * a.nq + q) * hs];
        const double2 hp = make_double2((double)hv.x * dq, (double)hv.y * dq);
        const double2 t = cmul(hp, bn);
        const double2 tr = cmul(t, wr);
        sum_r.x += tr.x;
        sum_r.y += tr.y;
        sum_a.x += (double)p * t.y;  // t * (-j p)
        sum_a.y += -(double)p * t.x;
      }
      dq *= d;
    }
    zp = cmul(zp, z);
  }
  // dZ/dDx = dZ/dr dx/r + dZ/dalpha (-dy/r^2); dZ/dDy = dZ/dr dy/r + dZ/dalpha dx/r^2
  *gx = -2.0 * (sum_r.x * (dx * d) + sum_a.x * (-dy * d * d));
  *gy = -2.0 * (sum_r.x * (dy * d) + sum_a.x * (dx * d * d));
}

// The derivative sums of the chunk's pairs (m, n0 + nl) from H as the digit
// products leave it, H[(m + Na nl) + k ldh]: one thread per pair.
__global__ void adjoint_deriv_kernel(AdjArgs a, const double2* __restrict__ H, long ldh) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)a.Na * a.nn) return;
  const int nl = (int)(e / a.Na), m = (int)(e - (long)nl * a.Na);
  const int n = a.n0 + nl;
  if (m == n) return;
  const double dx = a.pos[2 * m] - a.pos[2 * n];
  const double dy = a.pos[2 * m + 1] - a.pos[2 * n + 1];
  const double r = hypot(dx, dy);
  double gx, gy;
  adj_pair_grad(a, dx, dy, r, H + e, ldh, &gx, &gy);
  double* out = a.gpair + 2 * ((size_t)m * a.Na + n);
  out[0] = gx;
  out[1] = gy;
}

template <typename R, bool FF, bool LOADG>
__global__ void __launch_bounds__(kAdjThreads) adjoint_pairs_kernel(AdjArgs a) {
  static_assert(!FF || sizeof(R) == 8, "double-float G feeds the FP64 stages");
  static_assert(!LOADG || FF, "a given G feeds the double-float H sums");
  using C = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nm = a.Nm, Nm2 = Nm * Nm, K = a.K, BA = a.BA;
  C* Gs = reinterpret_cast<C*>(smem_raw);  // [BA][Nm2], entry T + Nm*S
  C* Hs = Gs + (size_t)BA * Nm2;           // [BA][K]
  C* Xs = Hs + (size_t)BA * K;             // [kRChunk][Nm]
  double* geo = reinterpret_cast<double*>(Xs + (size_t)kRChunk * Nm);  // [BA][4]
  // double-float G only: the tile's Lambda rows for one chunk of right-hand
  // sides, [kRChunk][BA * Nm]
  float4* Lf = reinterpret_cast<float4*>(geo + 4 * (size_t)BA);

  for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const int nl = item / a.n_mtiles;
    const int n = a.n0 + nl;
    const int m0 = (item - nl * a.n_mtiles) * BA;
    // G tile = Lambda rows of the tile times X rows of antenna n (transposed)
    // Each thread owns outputs e = tid + j*blockDim (T fastest).
    constexpr int kMaxOut = 24;
    const int nG = BA * Nm2;
    const int nmine = (nG - (int)threadIdx.x + kAdjThreads - 1) / kAdjThreads;
    if constexpr (LOADG) {
      // the tile's G blocks from the digit products, as float pairs
      __syncthreads();  // the previous item's readers of Gs, Hs and geo are done
      for (int e = threadIdx.x; e < nG; e += blockDim.x) {
        const int mi = e / Nm2, ts = e - mi * Nm2;
        const int S = ts / Nm, T = ts - S * Nm;
        const int m = m0 + mi;
        double2 v = make_double2(0.0, 0.0);
        if (m < a.Na) v = a.Gc[(size_t)m * Nm + T + ((size_t)nl * Nm + S) * a.ldg];
        float hr, lr, hi, li;
        ff_split(v.x, hr, lr);
        ff_split(v.y, hi, li);
        reinterpret_cast<float4*>(Gs)[(size_t)mi * Nm2 + T + Nm * S] = make_float4(hr, lr, hi, li);
      }
    } else if constexpr (FF) {
      float4* Xf = reinterpret_cast<float4*>(Xs);  // [kRChunk][Nm], same bytes
      const long N = (long)a.Na * Nm;
      float Sr[kMaxOut], er[kMaxOut], Si[kMaxOut], ei[kMaxOut];
#pragma unroll
      for (int j = 0; j < kMaxOut; ++j) Sr[j] = er[j] = Si[j] = ei[j] = 0.f;
      for (int r0 = 0; r0 < a.nrhs; r0 += kRChunk) {
        const int rc = min(kRChunk, a.nrhs - r0);
        __syncthreads();
        for (int e = threadIdx.x; e < rc * Nm; e += blockDim.x) {
          const int rr = e / Nm, S = e - rr * Nm;
          Xf[rr * Nm + S] = a.Xsp[(size_t)n * Nm + S + (size_t)(r0 + rr) * N];
        }
        {
          const int rows = min(BA, a.Na - m0) * Nm;  // the tile's Lambda rows
          for (int e = threadIdx.x; e < rc * rows; e += blockDim.x) {
            const int rr = e / rows, q = e - rr * rows;
            Lf[rr * BA * Nm + q] = a.Lsp[(size_t)m0 * Nm + q + (size_t)(r0 + rr) * N];
          }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j) {
          if (j >= nmine) break;
          const int e = threadIdx.x + j * kAdjThreads;
          const int T = e % Nm, rest = e / Nm;
          const int S = rest % Nm, mi = rest / Nm;
          const int m = m0 + mi;
          if (m >= a.Na) continue;
          const float4* lrow = Lf + mi * Nm + T;
          float sr = Sr[j], tr = er[j], si = Si[j], ti = ei[j];
          for (int rr = 0; rr < rc; ++rr) {
            const float4 l = lrow[rr * BA * Nm];
            const float4 x = Xf[rr * Nm + S];
            // re += lr xr - li xi, im += lr xi + li xr
            ff2_mac(sr, tr, l.x, l.y, x.x, x.y);
            ff2_mac(sr, tr, -l.z, -l.w, x.z, x.w);
            ff2_mac(si, ti, l.x, l.y, x.z, x.w);
            ff2_mac(si, ti, l.z, l.w, x.x, x.y);
          }
          Sr[j] = sr;
          er[j] = tr;
          Si[j] = si;
          ei[j] = ti;
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kMaxOut; ++j) {
        if (j >= nmine) break;
        const int e = threadIdx.x + j * kAdjThreads;
        const int T = e % Nm, rest = e / Nm;
        const int S = rest % Nm, mi = rest / Nm;
        // G as a normalised float pair (hi + lo = S + e) for the H sums
        const float hr = __fadd_rn(Sr[j], er[j]), lr = __fsub_rn(er[j], __fsub_rn(hr, Sr[j]));
        const float hi = __fadd_rn(Si[j], ei[j]), li = __fsub_rn(ei[j], __fsub_rn(hi, Si[j]));
        reinterpret_cast<float4*>(Gs)[(size_t)mi * Nm2 + T + Nm * S] = make_float4(hr, lr, hi, li);
      }
    } else {
      C acc[kMaxOut];
#pragma unroll
      for (int j = 0; j < kMaxOut; ++j) acc[j] = mk<R>(0, 0);
      for (int r0 = 0; r0 < a.nrhs; r0 += kRChunk) {
        const int rc = min(kRChunk, a.nrhs - r0);
        __syncthreads();
        for (int e = threadIdx.x; e < rc * Nm; e += blockDim.x) {
          const int rr = e / Nm, S = e - rr * Nm;
          const double2 v = a.X[(size_t)n * Nm + S + (size_t)(r0 + rr) * a.ld];
          Xs[rr * Nm + S] = mk<R>((R)v.x, (R)v.y);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j) {
          if (j >= nmine) break;
          const int e = threadIdx.x + j * kAdjThreads;
          const int T = e % Nm, rest = e / Nm;
          const int S = rest % Nm, mi = rest / Nm;
          const int m = m0 + mi;
          if (m >= a.Na) continue;
          const double2* lrow = a.Lam + (size_t)m * Nm + T;
          C s = acc[j];
          for (int rr = 0; rr < rc; ++rr) {
            const double2 l = lrow[(size_t)(r0 + rr) * a.ld];
            cfma(s, mk<R>((R)l.x, (R)l.y), Xs[rr * Nm + S]);
          }
          acc[j] = s;
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kMaxOut; ++j) {
        if (j >= nmine) break;
        const int e = threadIdx.x + j * kAdjThreads;
        const int T = e % Nm, rest = e / Nm;
        const int S = rest % Nm, mi = rest / Nm;
        Gs[(size_t)mi * Nm2 + T + Nm * S] = acc[j];
      }
    }
    // geometry of the tile's pairs
    for (int mi = threadIdx.x; mi < BA; mi += blockDim.x) {
      const int m = m0 + mi;
      double dx = 0, dy = 0, r = 1;
      if (m < a.Na && m != n) {
        dx = a.pos[2 * m] - a.pos[2 * n];
        dy = a.pos[2 * m + 1] - a.pos[2 * n + 1];
        r = hypot(dx, dy);
      }
      geo[4 * mi + 0] = dx;
      geo[4 * mi + 1] = dy;
      geo[4 * mi + 2] = r;
    }
    __syncthreads();
    // H[mi][k] = sum_TS G[mi][TS] c_k^{TS} (double-float with G)
    for (int e = threadIdx.x; e < BA * K; e += blockDim.x) {
      const int mi = e / K, kk = e - mi * K;
      if constexpr (FF) {
        float hr = 0.f, er_ = 0.f, hi = 0.f, ei_ = 0.f;
        const float4* g = reinterpret_cast<const float4*>(Gs) + (size_t)mi * Nm2;
        for (int S = 0; S < Nm; ++S)
          for (int T = 0; T < Nm; ++T) {
            const float4 gv = g[T + Nm * S];
            const float4 c = a.Csp[((size_t)T * Nm + S) * K + kk];
            // re += gr cr - gi ci, im += gr ci + gi cr
            ff2_mac(hr, er_, gv.x, gv.y, c.x, c.y);
            ff2_mac(hr, er_, -gv.z, -gv.w, c.z, c.w);
            ff2_mac(hi, ei_, gv.x, gv.y, c.z, c.w);
            ff2_mac(hi, ei_, gv.z, gv.w, c.x, c.y);
          }
        Hs[(size_t)mi * K + kk] = mk<R>((R)((double)hr + (double)er_), (R)((double)hi + (double)ei_));
      } else {
        C h = mk<R>(0, 0);
        const C* g = Gs + (size_t)mi * Nm2;
        for (int S = 0; S < Nm; ++S)
          for (int T = 0; T < Nm; ++T) {
            const double2 c = a.coef[((size_t)T * Nm + S) * K + kk];
            cfma(h, g[T + Nm * S], mk<R>((R)c.x, (R)c.y));
          }
        Hs[(size_t)mi * K + kk] = h;
      }
    }
    __syncthreads();
    // per-pair derivative sums (FP64), one thread per pair
    for (int mi = threadIdx.x; mi < BA; mi += blockDim.x) {
      const int m = m0 + mi;
      if (m >= a.Na || m == n) continue;
      const double dx = geo[4 * mi], dy = geo[4 * mi + 1], r = geo[4 * mi + 2];
      double gx = 0.0, gy = 0.0;
      adj_pair_grad(a, dx, dy, r, Hs + (size_t)mi * K, 1, &gx, &gy);
      double* out = a.gpair + 2 * ((size_t)m * a.Na + n);
      out[0] = gx;
      out[1] = gy;
    }
  }
}

// grad[m] = sum_n g(m, n) - sum_n g(n, m) in a fixed order (deterministic):
// one warp per antenna m, lane l summing n = l, l + 32, ... in turn, then a
// fixed shuffle tree over the lanes.
__global__ void adjoint_reduce_kernel(int Na, const double* gpair, double* grad) {
  const int lane = threadIdx.x & 31;
  const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (m >= Na) return;
  double gx = 0.0, gy = 0.0;
  for (int n = lane; n < Na; n += 32) {
    if (n == m) continue;
    const double2 a = *reinterpret_cast<const double2*>(gpair + 2 * ((size_t)m * Na + n));
    const double2 b = *reinterpret_cast<const double2*>(gpair + 2 * ((size_t)n * Na + m));
    gx += a.x - b.x;
    gy += a.y - b.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    gx += __shfl_xor_sync(0xffffffffu, gx, off);
    gy += __shfl_xor_sync(0xffffffffu, gy, off);
  }
  if (lane == 0) {
    grad[2 * m] = gx;
    grad[2 * m + 1] = gy;
  }
}

// The pair kernel for the source antennas a.n0 .. a.n0 + a.nn - 1; `prof`:
// record it as the adjoint class (off when the caller records the whole
// digit-product path as one).
template <typename R, bool FF, bool LOADG>
static int launch_adjoint(harp_ctx* ctx, AdjArgs a, cudaStream_t st, bool prof = true) {
  using C = cplx_t<R>;
  const int Nm2 = a.Nm * a.Nm;
  int BA = 32;
  size_t smem = 0;
  for (; BA >= 1; BA /= 2) {
    smem = ((size_t)BA * Nm2 + (size_t)BA * a.K + (size_t)kRChunk * a.Nm) * sizeof(C) +
           (size_t)BA * 4 * sizeof(double) +
           ((FF && !LOADG) ? (size_t)kRChunk * BA * a.Nm * sizeof(float4) : 0);
    if (smem <= std::min<size_t>(ctx->smem_optin, 200 * 1024) && BA * Nm2 <= 24 * kAdjThreads) break;
  }
  if (BA < 1) return HARP_E_UNSUPPORTED;
  a.BA = BA;
  a.n_mtiles = (a.Na + BA - 1) / BA;
  a.n_items = a.nn * a.n_mtiles;
  HARP_CUDA(cudaFuncSetAttribute(adjoint_pairs_kernel<R, FF, LOADG>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjoint_pairs_kernel<R, FF, LOADG>,
                                                kAdjThreads, smem);
  const int grid = std::min(a.n_items, ctx->num_sms * std::max(1, per_sm));
  ProfScope ps(prof ? HARP_K_ADJOINT : -1,
               8.0 * a.Na * (double)(a.Na - 1) * a.Nm * a.Nm * (double)(a.nrhs + a.K), st);
  adjoint_pairs_kernel<R, FF, LOADG><<<grid, kAdjThreads, smem, st>>>(a);
  HARP_LAUNCHED();
  return HARP_OK;
}

}  // namespace harp

using namespace harp;

extern "C" int harp_fill_adjoint(harp_ctx* ctx, int Na, int Nm, int P, int Q, const double* pos,
                                 double freq_hz, const double* coef, const double* Lambda,
                                 const double* X, int ld, int nrhs, double* grad_pos, int prec,
                                 void* stream) {
  if (!ctx) return -1;
  if (Na < 1) return -2;
  if (Nm < 1) return -3;
  if (P < 0 || P > 64) return -4;
  if (Q < 0 || Q > 64) return -5;
  if (!pos) return -6;
  if (!(freq_hz > 0.0) || freq_hz > 1e15) return -7;
  if (!coef) return -8;
  if (!Lambda) return -9;
  if (!X) return -10;
  if (ld < (long)Na * Nm) return -11;
  if (nrhs < 1) return -12;
  if (!grad_pos) return -13;
  if (prec != HARP_FP64 && prec != HARP_MIXED_3XTF32 && prec != HARP_MIXED_TF32 && prec != HARP_FP32)
    return -14;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t st = (cudaStream_t)stream;
  const size_t need = (size_t)Na * Na * 2 * sizeof(double);
  if (ctx->gpair_bytes < need) {
    if (ctx->gpair) cudaFree(ctx->gpair);
    ctx->gpair = nullptr;
    ctx->gpair_bytes = 0;
    if (cudaMalloc((void**)&ctx->gpair, need) != cudaSuccess) {
      cudaGetLastError();
      return HARP_E_NOMEM;
    }
    ctx->gpair_bytes = need;
  }
  AdjArgs a;
  a.Na = Na;
  a.Nm = Nm;
  a.P = P;
  a.Q = Q;
  a.nq = Q + 1;
  a.K = (2 * P + 1) * (Q + 1);
  a.nrhs = nrhs;
  a.pos = pos;
  a.k = 2.0 * kPia * freq_hz / kC0a;
  a.coef = reinterpret_cast<const double2*>(coef);
  a.Lam = reinterpret_cast<const double2*>(Lambda);
  a.X = reinterpret_cast<const double2*>(X);
  a.ld = ld;
  a.gpair = ctx->gpair;
  a.Lsp = nullptr;
  a.Xsp = nullptr;
  a.Csp = nullptr;
  a.n0 = 0;
  a.nn = Na;
  a.Gc = nullptr;
  a.ldg = 0;
  HARP_CUDA(cudaMemsetAsync(ctx->gpair, 0, need, st));
  // mixed modes: G in double-float, the split operands in the context's
  // float-float scratch (Lambda: 4 max_N max_nrhs floats; X: 4 max_N^2)
  const long Nl = (long)Na * Nm;
  const bool ff = (prec == HARP_MIXED_3XTF32 || prec == HARP_MIXED_TF32) && ctx->xff && ctx->zff &&
                  ctx->tc_b && Nl <= ctx->max_N && nrhs <= ctx->max_nrhs &&
                  Nl * nrhs <= (long)ctx->max_N * ctx->max_N &&
                  (size_t)4 * Nm * Nm * a.K <= ctx->tc_b_floats;
  // mixed modes with the tensor-core residual's buffers: G by exact digit
  // products, in chunks of source antennas (columns of G) that the buffers
  // hold, each followed by the pair kernel on those antennas
  const bool mixed = (prec == HARP_MIXED_3XTF32 || prec == HARP_MIXED_TF32);
  const int gcols = (mixed && ctx->adj_g == 1 && ctx->tc_b && Nl <= ctx->max_N &&
                     (size_t)4 * Nm * Nm * a.K <= ctx->tc_b_floats)
                        ? (int)std::min<long>(oz_gram_max_cols(ctx, (int)Nl, nrhs), Nl)
                        : 0;
  int na_chunk = gcols / Nm;
  // H = G C^T by digit products too where its plan fits the slots (fewer
  // source antennas a chunk if need be); its work buffer and H follow G's
  // columns in the context's buffer
  size_t hwork = 0;
  if (na_chunk >= 1) {
    int nnh = na_chunk;
    while (nnh >= 1 && !(hwork = oz_adj_h_bytes(ctx, Na, Nm, a.K, nnh))) nnh /= 2;
    if (hwork) na_chunk = nnh;
  }
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t off_hw = 0, off_h = 0;
  if (na_chunk >= 1) {
    // the context's buffer, grown on demand; without it G's columns go to
    // the residual's accumulator (max_N max_nrhs complex) and H stays on
    // the CUDA cores
    off_hw = al((size_t)Nl * na_chunk * Nm * sizeof(double2));
    off_h = off_hw + (hwork ? al(hwork) : 0);
    const size_t want = off_h + (hwork ? (size_t)Na * na_chunk * a.K * sizeof(double2) : 0);
    if (ctx->gbuf_bytes < want) {
      HARP_CUDA(cudaStreamSynchronize(st));  // a previous call may still use it
      if (ctx->gbuf) cudaFree(ctx->gbuf);
      ctx->gbuf = nullptr;
      ctx->gbuf_bytes = 0;
      if (cudaMalloc(&ctx->gbuf, want) == cudaSuccess) {
        ctx->gbuf_bytes = want;
      } else {
        cudaGetLastError();
        ctx->gbuf = nullptr;
      }
    }
    if (!ctx->gbuf) {
      hwork = 0;
      na_chunk = (int)std::min<long>(na_chunk, (long)ctx->max_N * ctx->max_nrhs / Nl / Nm);
    }
  }
  if (na_chunk >= 1) {
    // after the context's pending background fill, which may still use the
    // residual's buffers (the next solve slices Z64 again)
    if (ctx->ev_z64) HARP_CUDA(cudaStreamWaitEvent(st, ctx->ev_z64, 0));
    ProfScope ps(HARP_K_ADJOINT,
                 8.0 * a.Na * (double)(a.Na - 1) * a.Nm * a.Nm * (double)(a.nrhs + a.K), st);
    char* gb = static_cast<char*>(ctx->gbuf);
    void* hw = hwork ? gb + off_hw : nullptr;
    double2* Hb = hwork ? reinterpret_cast<double2*>(gb + off_h) : nullptr;
    if (hwork) {
      HARP_TRY(oz_adj_h_prepare(ctx, Na, Nm, a.K, na_chunk, a.coef, hw, st));
    } else {
      const long nc = (long)Nm * Nm * a.K;
      split_c128_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(
          nc, a.coef, reinterpret_cast<float4*>(ctx->tc_b));
      HARP_LAUNCHED();
      a.Csp = reinterpret_cast<const float4*>(ctx->tc_b);
    }
    HARP_TRY(oz_gram_prepare(ctx, (int)Nl, nrhs, a.Lam, ld, a.X, ld, st));
    double2* Gc = reinterpret_cast<double2*>(ctx->gbuf ? ctx->gbuf : (void*)ctx->oz_acc);
    for (int n0 = 0; n0 < Na; n0 += na_chunk) {
      const int nn = std::min(na_chunk, Na - n0);
      HARP_TRY(oz_gram_chunk(ctx, (int)Nl, nrhs, a.X, ld, n0 * Nm, nn * Nm, Gc, Nl, st));
      a.n0 = n0;
      a.nn = nn;
      a.Gc = Gc;
      a.ldg = Nl;
      if (hwork) {
        const long ldh = (long)Na * nn;
        HARP_TRY(oz_adj_h_chunk(ctx, Na, Nm, a.K, nn, Gc, Nl, hw, Hb, ldh, st));
        adjoint_deriv_kernel<<<(unsigned)((ldh + 127) / 128), 128, 0, st>>>(a, Hb, ldh);
        HARP_LAUNCHED();
      } else {
        HARP_TRY((launch_adjoint<double, true, true>(ctx, a, st, false)));
      }
    }
  } else if (ff) {
    float4* lsp = reinterpret_cast<float4*>(ctx->xff);
    float4* xsp = reinterpret_cast<float4*>(ctx->zff);
    {
      ProfScope ps(HARP_K_OTHER, 0.0, st);
      const unsigned blocks = (unsigned)((Nl * nrhs + 255) / 256);
      adjoint_split_kernel<<<blocks, 256, 0, st>>>((int)Nl, nrhs, a.Lam, ld, lsp);
      HARP_LAUNCHED();
      adjoint_split_kernel<<<blocks, 256, 0, st>>>((int)Nl, nrhs, a.X, ld, xsp);
      HARP_LAUNCHED();
      // the coefficient table into the (idle) tensor-core B workspace
      const long nc = (long)Nm * Nm * a.K;
      split_c128_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(
          nc, a.coef, reinterpret_cast<float4*>(ctx->tc_b));
      HARP_LAUNCHED();
    }
    a.Lsp = lsp;
    a.Xsp = xsp;
    a.Csp = reinterpret_cast<const float4*>(ctx->tc_b);
    HARP_TRY((launch_adjoint<double, true, false>(ctx, a, st)));
  } else if (prec == HARP_FP32) {
    HARP_TRY((launch_adjoint<float, false, false>(ctx, a, st)));
  } else {
    HARP_TRY((launch_adjoint<double, false, false>(ctx, a, st)));
  }
  adjoint_reduce_kernel<<<(Na + 7) / 8, 256, 0, st>>>(Na, ctx->gpair, grad_pos);
  HARP_LAUNCHED();
  return HARP_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of harp_fill_adjoint.
//
// Some callers cannot call cudaMalloc at all: an application whose device
// memory is owned by its own allocator (or was reserved in full at start-up)
// or code with a fixed memory budget that must not grow. For them the
// per-pair gradient buffer of the adjoint lives in a fixed device array
// declared here, so the call allocates nothing; the caller still passes
// every input and the output.
//
// The array is file-scope device memory: every GPU that loads this library
// holds it (HARP_NOALLOC_MAX_NA^2 * 2 doubles = 4 MiB) until the process
// exits. Host code cannot use the array's name as a device address, so on
// the first call on each device the library asks the runtime for that
// device's address of the array (with the device current) and keeps it.
// All calls share the one array and it keeps the last call's contents: each
// call clears the part it uses first, and calls whose work overlaps on the
// GPU (for example on two streams) race on it.
static __device__ __align__(256) double g_adjoint_scratch[(size_t)HARP_NOALLOC_MAX_NA *
                                                          HARP_NOALLOC_MAX_NA * 2];

namespace harp {
namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= kNoAllocMaxDevices) return HARP_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_adjoint_scratch);
    if (e != cudaSuccess) return cuda_status(e);
    g_noalloc_ptr[device] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[device];
  return HARP_OK;
}

template <typename R>
int launch_adjoint_noalloc(int device, AdjArgs a, cudaStream_t st) {
  using C = cplx_t<R>;
  int optin = 0, sms = 0;
  HARP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  HARP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int Nm2 = a.Nm * a.Nm;
  int BA = 32;
  size_t smem = 0;
  for (; BA >= 1; BA /= 2) {
    smem = ((size_t)BA * Nm2 + (size_t)BA * a.K + (size_t)kRChunk * a.Nm) * sizeof(C) +
           (size_t)BA * 4 * sizeof(double);
    if (smem <= std::min<size_t>((size_t)optin, 200 * 1024) && BA * Nm2 <= 24 * kAdjThreads)
      break;
  }
  if (BA < 1) return HARP_E_UNSUPPORTED;
  a.BA = BA;
  a.n_mtiles = (a.Na + BA - 1) / BA;
  a.n_items = a.Na * a.n_mtiles;
  HARP_CUDA(cudaFuncSetAttribute(adjoint_pairs_kernel<R, false, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 1;
  HARP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm,
                                                          adjoint_pairs_kernel<R, false, false>,
                                                          kAdjThreads, smem));
  const int grid = std::min(a.n_items, sms * std::max(1, per_sm));
  ProfScope ps(HARP_K_ADJOINT,
               8.0 * a.Na * (double)(a.Na - 1) * a.Nm * a.Nm * (double)(a.nrhs + a.K), st);
  adjoint_pairs_kernel<R, false, false><<<grid, kAdjThreads, smem, st>>>(a);
  HARP_LAUNCHED();
  return HARP_OK;
}
}  // namespace
}  // namespace harp

extern "C" int harp_fill_adjoint_noalloc(int Na, int Nm, int P, int Q, const double* pos,
                                         double freq_hz, const double* coef, const double* Lambda,
                                         const double* X, int ld, int nrhs, double* grad_pos,
                                         int prec, void* stream) {
  if (Na < 1) return -1;
  if (Nm < 1) return -2;
  if (P < 0 || P > 64) return -3;
  if (Q < 0 || Q > 64) return -4;
  if (!pos) return -5;
  if (!(freq_hz > 0.0) || freq_hz > 1e15) return -6;
  if (!coef) return -7;
  if (!Lambda) return -8;
  if (!X) return -9;
  if (ld < (long)Na * Nm) return -10;
  if (nrhs < 1) return -11;
  if (!grad_pos) return -12;
  if (prec != HARP_FP64 && prec != HARP_MIXED_3XTF32 && prec != HARP_MIXED_TF32 && prec != HARP_FP32)
    return -13;
  if (Na > HARP_NOALLOC_MAX_NA) return HARP_E_UNSUPPORTED;  // beyond the fixed scratch array
  int device = -1;
  HARP_CUDA(cudaGetDevice(&device));
  double* scratch = nullptr;
  HARP_TRY(noalloc_scratch(device, &scratch));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t used = (size_t)Na * Na * 2 * sizeof(double);
  // a safeguard only: the pair kernel writes every entry (m, n) with m != n
  // and the reduction never reads m == n, so no leftover of an earlier call
  // is read even without it
  HARP_CUDA(cudaMemsetAsync(scratch, 0, used, st));
  AdjArgs a;
  a.Lsp = nullptr;
  a.Xsp = nullptr;
  a.Csp = nullptr;
  a.n0 = 0;
  a.nn = Na;
  a.Gc = nullptr;
  a.ldg = 0;
  a.Na = Na;
  a.Nm = Nm;
  a.P = P;
  a.Q = Q;
  a.nq = Q + 1;
  a.K = (2 * P + 1) * (Q + 1);
  a.nrhs = nrhs;
  a.pos = pos;
  a.k = 2.0 * kPia * freq_hz / kC0a;
  a.coef = reinterpret_cast<const double2*>(coef);
  a.Lam = reinterpret_cast<const double2*>(Lambda);
  a.X = reinterpret_cast<const double2*>(X);
  a.ld = ld;
  a.gpair = scratch;
  if (prec == HARP_FP64)
    HARP_TRY(launch_adjoint_noalloc<double>(device, a, st));
  else
    HARP_TRY(launch_adjoint_noalloc<float>(device, a, st));
  adjoint_reduce_kernel<<<(Na + 7) / 8, 256, 0, st>>>(Na, scratch, grad_pos);
  HARP_LAUNCHED();
  return HARP_OK;
}
