// fill.cu -- the HARP fill of the reduced MBF matrix (Eq. 3 and 4).
//
// For every ordered antenna pair (m, n), m != n, with Delta = x_m - x_n,
// r = |Delta|, e^{j alpha} = Delta / r and d = 1/r:
//   Z^{mn}_TS = sum_k c_k^{TS} phi_k,   phi_{p,q} = e^{-jkr} e^{j p alpha} d^q,
// k running over the K = (2P+1)(Q+1) harmonic/power pairs (Eq. 3 inserted
// in Eq. 4; the far-field term of Eq. 1 arrives folded into q = 1).
//
// Work item = (source antenna n, a tile of 32 testing antennas, a chunk of
// source MBFs S). A CTA stages the coefficient chunk C[k][S,T] in shared
// memory once and loops over work items (persistent grid, one CTA per SM
// at the shared-memory sizes used here). Per item, one warp computes the
// basis phi[k][pair] (geometry and e^{-jkr} in FP64, powers of e^{j alpha}
// and d by repeated multiplication in the kernel's precision), then all 8
// warps run the contraction Z[pair, (S,T)] = sum_k phi[k][pair] C[k][(S,T)]
// with a 4-pair x TN-entry register tile per thread. Lanes run along (S,T)
// with T fastest, so stores are runs of Nm consecutive rows of a column.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"
#include "ff.cuh"
#include "ozaki.cuh"
#include "prof.cuh"

namespace harp {

constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;

struct FillArgs {
  int Na, Nm, P, Q, K, nq;
  const double* pos;
  double k;
  const double2* coef;  // [T][S][p+P][q]
  const double2* self;
  long self_stride;
  void* Z;  // cplx_t<R>, ldz
  long ldz;
  float2* Z32;  // optional rounded copy (dual store), ld32
  long ld32;
  int* status;
  int s_chunk;
  int n_mtiles;
  int n_items;
  int Wp;  // padded row length of the staged coefficient chunk (32*TN)
};

constexpr int kPairsPerTile = 32;
constexpr int kFillThreads = 256;

template <typename R, int TN, bool DUAL>
__global__ void __launch_bounds__(kFillThreads, 1) fill_kernel(FillArgs a) {
  using C = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = a.K, Nm = a.Nm, nq = a.nq, P = a.P, Q = a.Q;
  const int s0 = blockIdx.y * a.s_chunk;
  const int sc = min(a.s_chunk, Nm - s0);
  const int W = sc * Nm;
  const int Wp = a.Wp;
  C* Cs = reinterpret_cast<C*>(smem_raw);  // [K][Wp], entry (S - s0)*Nm + T
  C* Phi = Cs + (size_t)K * Wp;            // [K][32]

  for (int idx = threadIdx.x; idx < K * Wp; idx += blockDim.x) {
    const int kk = idx / Wp, e = idx - kk * Wp;
    C v = mk<R>(0, 0);
    if (e < W) {
      const int sl = e / Nm, T = e - sl * Nm;
      const double2 c = a.coef[((size_t)T * Nm + (s0 + sl)) * K + kk];
      v = mk<R>((R)c.x, (R)c.y);
    }
    Cs[idx] = v;
  }

  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  bool nonfinite = false;  // a stored entry is NaN or infinite
  for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const int n = item / a.n_mtiles;
    const int m0 = (item - n * a.n_mtiles) * kPairsPerTile;
    __syncthreads();  // Cs staged / previous item's Phi consumed
    if (threadIdx.x < kPairsPerTile) {
      const int t = threadIdx.x;
      const int m = m0 + t;
      bool valid = (m < a.Na) && (m != n);
      double dx = 0.0, dy = 0.0, r = 0.0;
      if (valid) {
        dx = a.pos[2 * m] - a.pos[2 * n];
        dy = a.pos[2 * m + 1] - a.pos[2 * n + 1];
        r = hypot(dx, dy);
        if (r == 0.0) {
          atomicOr(a.status, ST_COINCIDENT);
          valid = false;
        }
      }
      if (!valid) {
        for (int kk = 0; kk < K; ++kk) Phi[kk * kPairsPerTile + t] = mk<R>(0, 0);
      } else {
        const double d = 1.0 / r;
        double s, c;
        sincos(a.k * r, &s, &c);  // FP64: kr reaches a few hundred radians
        const C ph = mk<R>((R)c, (R)(-s));             // e^{-jkr}
        const C z = mk<R>((R)(dx * d), (R)(dy * d));  // e^{j alpha}
        const R dR = (R)d;
        C zp = mk<R>(1, 0);
        for (int p = 0; p <= P; ++p) {
          const C bp = cmul(ph, zp);
          const C bn = cmul(ph, cconj(zp));
          R dq = 1;
          for (int q = 0; q <= Q; ++q) {
            Phi[((P + p) * nq + q) * kPairsPerTile + t] = mk<R>(bp.x * dq, bp.y * dq);
            if (p > 0) Phi[((P - p) * nq + q) * kPairsPerTile + t] = mk<R>(bn.x * dq, bn.y * dq);
            dq *= dR;
          }
          zp = cmul(zp, z);
        }
      }
    }
    __syncthreads();

    C acc[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = mk<R>(0, 0);

    const C* phrow = Phi + ty * 4;
#pragma unroll 2
    for (int kk = 0; kk < K; ++kk) {
      C f[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) f[i] = phrow[kk * kPairsPerTile + i];
      const C* crow = Cs + (size_t)kk * Wp + tx;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const C cv = crow[32 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i) cfma(acc[i][j], f[i], cv);
      }
    }

#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + ty * 4 + i;
      if (m >= a.Na) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int e = tx + 32 * j;
        if (e >= W) continue;
        const int sl = e / Nm, T = e - sl * Nm, S = s0 + sl;
        const size_t row = (size_t)m * Nm + T, col = (size_t)n * Nm + S;
        C v = acc[i][j];
        double2 dv = make_double2((double)v.x, (double)v.y);
        if (m == n) {
          dv = a.self[(size_t)m * a.self_stride + T + (size_t)S * Nm];
          v = mk<R>((R)dv.x, (R)dv.y);
        }
        nonfinite |= !(isfinite(v.x) && isfinite(v.y));
        reinterpret_cast<C*>(a.Z)[row + col * a.ldz] = v;
        if (DUAL) a.Z32[row + col * a.ld32] = make_float2((float)dv.x, (float)dv.y);
      }
    }
  }
  if (nonfinite) atomicOr(a.status, ST_NONFINITE);
}

// FP64-accurate fill on the FP32 pipe (mixed modes). Same work split as
// fill_kernel, with the sum of Eq. 4 factored by the order of the basis:
//   Z^{mn}_TS = sum_p E_p W_p,  E_p = e^{-jkr} e^{jp alpha},
//   W_p = sum_q c_pq(T, S) d^q   (d = 1/r real),
// so that the inner sums are complex x real. Coefficients and basis are
// carried as hi/lo float pairs (coefficients as float4 = re_hi, im_hi,
// re_lo, im_lo; E_p likewise; d^q as float2 = hi, lo). Each W_p, Q + 1
// terms of decreasing size, is summed in a double-float accumulator, then
// renormalised to a hi/lo pair; the 2P + 1 products E_p W_p go into the
// three-float accumulator of ff.cuh. Writes the FP64 matrix (Z, c128) and,
// when asked, its rounded c64 copy (Z32).
template <int TN>
__global__ void __launch_bounds__(kFillThreads, 1) fill_ff_kernel(FillArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int K = a.K, Nm = a.Nm, nq = a.nq, P = a.P;
  const int np = 2 * P + 1;
  const int s0 = blockIdx.y * a.s_chunk;
  const int sc = min(a.s_chunk, Nm - s0);
  const int W = sc * Nm;
  const int Wp = a.Wp;
  float4* Cs = reinterpret_cast<float4*>(smem_raw);  // [K][Wp]
  float4* Es = Cs + (size_t)K * Wp;                  // [np][32]
  float2* Ds = reinterpret_cast<float2*>(Es + (size_t)np * kPairsPerTile);  // [nq][32]

  for (int idx = threadIdx.x; idx < K * Wp; idx += blockDim.x) {
    const int kk = idx / Wp, e = idx - kk * Wp;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < W) {
      const int sl = e / Nm, T = e - sl * Nm;
      const double2 c = a.coef[((size_t)T * Nm + (s0 + sl)) * K + kk];
      ff_split(c.x, v.x, v.z);
      ff_split(c.y, v.y, v.w);
    }
    Cs[idx] = v;
  }

  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const int n = item / a.n_mtiles;
    const int m0 = (item - n * a.n_mtiles) * kPairsPerTile;
    __syncthreads();
    if (threadIdx.x < kPairsPerTile) {
      const int t = threadIdx.x;
      const int m = m0 + t;
      bool valid = (m < a.Na) && (m != n);
      double dx = 0.0, dy = 0.0, r = 0.0;
      if (valid) {
        dx = a.pos[2 * m] - a.pos[2 * n];
        dy = a.pos[2 * m + 1] - a.pos[2 * n + 1];
        r = hypot(dx, dy);
        if (r == 0.0) {
          atomicOr(a.status, ST_COINCIDENT);
          valid = false;
        }
      }
      if (!valid) {
        for (int pi = 0; pi < np; ++pi) Es[pi * kPairsPerTile + t] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = 0; q < nq; ++q) Ds[q * kPairsPerTile + t] = make_float2(0.f, 0.f);
      } else {
        // basis factors in FP64 (Eq. 3, 4), then split into hi/lo pairs
        const double d = 1.0 / r;
        double sn, cs;
        sincos(a.k * r, &sn, &cs);
        const double2 ph = make_double2(cs, -sn);
        const double2 z = make_double2(dx * d, dy * d);
        double2 zp = make_double2(1.0, 0.0);
        for (int p = 0; p <= P; ++p) {
          const double2 bp = cmul(ph, zp), bn = cmul(ph, cconj(zp));
          float4 v;
          ff_split(bp.x, v.x, v.z);
          ff_split(bp.y, v.y, v.w);
          Es[(P + p) * kPairsPerTile + t] = v;
          if (p > 0) {
            ff_split(bn.x, v.x, v.z);
            ff_split(bn.y, v.y, v.w);
            Es[(P - p) * kPairsPerTile + t] = v;
          }
          zp = cmul(zp, z);
        }
        double dq = 1.0;
        for (int q = 0; q < nq; ++q) {
          float2 v;
          ff_split(dq, v.x, v.y);
          Ds[q * kPairsPerTile + t] = v;
          dq *= d;
        }
      }
    }
    __syncthreads();

    float Sr[4][TN], s1r[4][TN], s2r[4][TN], Si[4][TN], s1i[4][TN], s2i[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j)
        Sr[i][j] = s1r[i][j] = s2r[i][j] = Si[i][j] = s1i[i][j] = s2i[i][j] = 0.f;
    for (int pi = 0; pi < np; ++pi) {
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        // W_p for this thread's 4 pairs and column j: sum over q of c * d^q
        float wr[4], er[4], wi[4], ei[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) wr[i] = er[i] = wi[i] = ei[i] = 0.f;
        const float4* crow = Cs + (size_t)pi * nq * Wp + tx + 32 * j;
        for (int q = 0; q < nq; ++q) {
          const float4 c = crow[(size_t)q * Wp];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float2 dq = Ds[q * kPairsPerTile + ty * 4 + i];
            ff2_mac(wr[i], er[i], c.x, c.z, dq.x, dq.y);
            ff2_mac(wi[i], ei[i], c.y, c.w, dq.x, dq.y);
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          // renormalise (|e| is far below |w|): hi + lo = w + e
          const float whr = __fadd_rn(wr[i], er[i]);
          const float wlr = __fsub_rn(er[i], __fsub_rn(whr, wr[i]));
          const float whi = __fadd_rn(wi[i], ei[i]);
          const float wli = __fsub_rn(ei[i], __fsub_rn(whi, wi[i]));
          const float4 f = Es[pi * kPairsPerTile + ty * 4 + i];
          // re += fr*wr - fi*wi ; im += fr*wi + fi*wr
          fff_mac(Sr[i][j], s1r[i][j], s2r[i][j], f.x, f.z, whr, wlr);
          fff_mac(Sr[i][j], s1r[i][j], s2r[i][j], -f.y, -f.w, whi, wli);
          fff_mac(Si[i][j], s1i[i][j], s2i[i][j], f.x, f.z, whi, wli);
          fff_mac(Si[i][j], s1i[i][j], s2i[i][j], f.y, f.w, whr, wlr);
        }
      }
    }

#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + ty * 4 + i;
      if (m >= a.Na) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int e = tx + 32 * j;
        if (e >= W) continue;
        const int sl = e / Nm, T = e - sl * Nm, S = s0 + sl;
        const size_t row = (size_t)m * Nm + T, col = (size_t)n * Nm + S;
        double2 dv = make_double2((double)Sr[i][j] + ((double)s1r[i][j] + (double)s2r[i][j]),
                                  (double)Si[i][j] + ((double)s1i[i][j] + (double)s2i[i][j]));
        if (m == n) dv = a.self[(size_t)m * a.self_stride + T + (size_t)S * Nm];
        reinterpret_cast<double2*>(a.Z)[row + col * a.ldz] = dv;
        if (a.Z32) a.Z32[row + col * a.ld32] = make_float2((float)dv.x, (float)dv.y);
      }
    }
  }
}

// How many 16-CTA clusters of this kernel and shared-memory size can be
// resident at once (one per GPC with 16 free SMs), cached; 0 when none.
static int fill_cluster_slots(void (*kern)(FillArgs), size_t smem) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<void*, size_t>, int>> cache;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& e : cache)
    if (e.first.first == (void*)kern && e.first.second == smem) return e.second;
  int n = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16);
  cfg.blockDim = dim3(kFillThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 16;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cache.push_back({{(void*)kern, smem}, n});
  return n;
}

// background: the fill runs beside the factorisation. It is then launched as
// 16-CTA clusters (each occupies one GPC) on half of the GPCs, so that whole
// GPCs stay free for the factorisation's 16-CTA panel clusters; a plain grid
// over all SMs would leave no GPC with 16 free SMs until the fill ends.
static int launch_fill_ff(const harp_ctx* ctx, FillArgs a, int TN, size_t smem, int nchunks,
                          cudaStream_t st, bool background) {
  void (*kern)(FillArgs) = nullptr;
  switch (TN) {
    case 1: kern = fill_ff_kernel<1>; break;
    case 2: kern = fill_ff_kernel<2>; break;
    case 3: kern = fill_ff_kernel<3>; break;
    case 4: kern = fill_ff_kernel<4>; break;
    default: return HARP_E_UNSUPPORTED;
  }
  HARP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope ps(HARP_K_FILL_FF, 8.0 * a.Nm * a.Nm * a.K * (double)a.Na * (a.Na - 1), st);
  const int slots = background ? fill_cluster_slots(kern, smem) : 0;
  if (slots >= 2) {
    // about half of the cluster slots (4 of the 7 a GB300 holds), split over
    // the source chunks
    const int want = (ctx->fill_clusters > 0) ? std::min(ctx->fill_clusters, slots) : (slots + 1) / 2;
    const int q = std::max(1, want / nchunks);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16 * q, nchunks);
    cfg.blockDim = dim3(kFillThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    HARP_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
  } else {
    const int per_chunk = std::max(1, (ctx->num_sms + nchunks - 1) / nchunks);
    dim3 grid(std::min(a.n_items, per_chunk), nchunks);
    kern<<<grid, kFillThreads, smem, st>>>(a);
  }
  HARP_LAUNCHED();
  return HARP_OK;
}

template <typename R, bool DUAL>
static int launch_fill(const harp_ctx* ctx, FillArgs a, int TN, size_t smem, int nchunks,
                       cudaStream_t st) {
  void (*kern)(FillArgs) = nullptr;
  switch (TN) {
    case 1: kern = fill_kernel<R, 1, DUAL>; break;
    case 2: kern = fill_kernel<R, 2, DUAL>; break;
    case 3: kern = fill_kernel<R, 3, DUAL>; break;
    case 4: kern = fill_kernel<R, 4, DUAL>; break;
    case 5: kern = fill_kernel<R, 5, DUAL>; break;
    case 6: kern = fill_kernel<R, 6, DUAL>; break;
    case 7: kern = fill_kernel<R, 7, DUAL>; break;
    case 8: kern = fill_kernel<R, 8, DUAL>; break;
    default: return HARP_E_UNSUPPORTED;
  }
  HARP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int per_chunk = std::max(1, (ctx->num_sms + nchunks - 1) / nchunks);
  dim3 grid(std::min(a.n_items, per_chunk), nchunks);
  ProfScope ps(HARP_K_FILL, 8.0 * a.Nm * a.Nm * a.K * (double)a.Na * (a.Na - 1), st);
  kern<<<grid, kFillThreads, smem, st>>>(a);
  HARP_LAUNCHED();
  return HARP_OK;
}

// Largest source-MBF chunk whose staged coefficients fit in shared memory.
static bool plan_fill(const harp_ctx* ctx, int Nm, int K, size_t csz, int* s_chunk, int* TN,
                      size_t* smem, int max_tn = 8) {
  const int top = (ctx->fill_chunk > 0) ? std::min(ctx->fill_chunk, Nm) : Nm;
  for (int sc = top; sc >= 1; --sc) {
    const int W = sc * Nm;
    const int tn = (W + 31) / 32;
    if (tn > max_tn) continue;
    // staged coefficients, then the per-item basis (the float-float kernel's
    // factors E_p and d^q take at most K + 1 of its 16-byte entries per pair)
    const size_t bytes =
        ((size_t)K * 32 * tn + (size_t)(K + (csz == sizeof(double2) ? 1 : 0)) * kPairsPerTile) *
        csz;
    if (bytes <= ctx->smem_optin) {
      *s_chunk = sc;
      *TN = tn;
      *smem = bytes;
      return true;
    }
  }
  return false;
}

int fill_dispatch(harp_ctx* ctx, int Na, int Nm, int P, int Q, const double* pos, double freq_hz,
                  const double* coef, const double* self_blocks, long self_stride, void* Z,
                  long ldz, float2* Z32, long ld32, int prec_kind, cudaStream_t st,
                  int* status = nullptr, bool background = false) {
  // prec_kind: 0 = FP64 only, 1 = FP64 with rounded c64 copy, 2 = FP32 only
  FillArgs a;
  a.Na = Na;
  a.Nm = Nm;
  a.P = P;
  a.Q = Q;
  a.nq = Q + 1;
  a.K = (2 * P + 1) * (Q + 1);
  a.pos = pos;
  a.k = 2.0 * kPi * freq_hz / kC0;
  a.coef = reinterpret_cast<const double2*>(coef);
  a.self = reinterpret_cast<const double2*>(self_blocks);
  a.self_stride = self_stride;
  a.Z = Z;
  a.ldz = ldz;
  a.Z32 = Z32;
  a.ld32 = ld32;
  a.status = status ? status : ctx->dstatus;
  a.n_mtiles = (Na + kPairsPerTile - 1) / kPairsPerTile;
  a.n_items = Na * a.n_mtiles;
  // prec_kind 1 (mixed): float-float kernel, 16-byte staged entries
  const size_t csz = (prec_kind == 2) ? sizeof(float2) : sizeof(double2);
  int sc, TN;
  size_t smem;
  if (!plan_fill(ctx, Nm, a.K, csz, &sc, &TN, &smem, prec_kind == 1 ? 4 : 8))
    return HARP_E_UNSUPPORTED;
  a.s_chunk = sc;
  a.Wp = 32 * TN;
  const int nchunks = (Nm + sc - 1) / sc;
  if (prec_kind == 2) return launch_fill<float, false>(ctx, a, TN, smem, nchunks, st);
  if (prec_kind == 1) return launch_fill_ff(ctx, a, TN, smem, nchunks, st, background);
  return launch_fill<double, false>(ctx, a, TN, smem, nchunks, st);
}

}  // namespace harp

using namespace harp;

extern "C" int harp_fill(harp_ctx* ctx, int Na, int Nm, int P, int Q, const double* pos,
                         double freq_hz, const double* coef, const double* self_blocks,
                         long self_stride, void* Z, int ldz, int prec, void* stream) {
  if (!ctx) return -1;
  if (Na < 1) return -2;
  if (Nm < 1) return -3;
  if (P < 0 || P > 64) return -4;
  if (Q < 0 || Q > 64) return -5;
  if (!pos) return -6;
  if (!(freq_hz > 0.0) || freq_hz > 1e15) return -7;
  if (!coef) return -8;
  if (!self_blocks) return -9;
  if (self_stride < 0) return -10;
  if (!Z) return -11;
  const long N = (long)Na * Nm;
  if (N > (1L << 30)) return HARP_E_UNSUPPORTED;
  if (ldz < N) return -12;
  if (prec != HARP_FP64 && prec != HARP_MIXED_3XTF32 && prec != HARP_MIXED_TF32 && prec != HARP_FP32)
    return -13;
  const bool mixed = (prec == HARP_MIXED_3XTF32 || prec == HARP_MIXED_TF32);
  if (mixed && N > ctx->max_N) return HARP_E_UNSUPPORTED;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t st = (cudaStream_t)stream;
  // the context's pending status describes the latest fill: coincident
  // antennas and non-finite entries are flagged by the kernels below and
  // reported, without a host synchronisation here, by the next mbf_solve or
  // harp_ctx_sync
  HARP_CUDA(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), st));
  int s;
  if (prec == HARP_FP64)
    s = fill_dispatch(ctx, Na, Nm, P, Q, pos, freq_hz, coef, self_blocks, self_stride, Z, ldz,
                      nullptr, 0, 0, st);
  else if (prec == HARP_FP32)
    s = fill_dispatch(ctx, Na, Nm, P, Q, pos, freq_hz, coef, self_blocks, self_stride, Z, ldz,
                      nullptr, 0, 2, st);
  else  // mixed: the FP32 matrix for the factorisation, here
    s = fill_dispatch(ctx, Na, Nm, P, Q, pos, freq_hz, coef, self_blocks, self_stride, Z, ldz,
                      nullptr, 0, 2, st);
  if (s != HARP_OK) return s;
  if (mixed) {
    // The background fill below runs after this call returns, so it reads
    // context-owned copies of the model inputs, made here on `stream`: the
    // caller may release or reuse its buffers in the order of its stream.
    // The copies wait for the previous background fill, which read the last
    // ones (the refinement waits for it anyway).
    const size_t pos_b = (size_t)Na * 2 * sizeof(double);
    const size_t coef_b = (size_t)Nm * Nm * (2 * P + 1) * (Q + 1) * sizeof(double2);
    const size_t self_b =
        ((size_t)(Na - 1) * (size_t)self_stride + (size_t)Nm * Nm) * sizeof(double2);
    const size_t a16 = 255;
    const size_t o_coef = (pos_b + a16) & ~a16, o_self = (o_coef + coef_b + a16) & ~a16;
    const size_t need = o_self + self_b;
    if (ctx->fin_bytes < need) {
      HARP_CUDA(cudaStreamSynchronize(ctx->fill_stream));
      if (ctx->fin) cudaFree(ctx->fin);
      ctx->fin = nullptr;
      ctx->fin_bytes = 0;
      if (cudaMalloc(&ctx->fin, need) != cudaSuccess) {
        cudaGetLastError();
        return HARP_E_NOMEM;
      }
      ctx->fin_bytes = need;
    }
    char* fb = static_cast<char*>(ctx->fin);
    HARP_CUDA(cudaStreamWaitEvent(st, ctx->ev_z64, 0));
    HARP_CUDA(cudaMemcpyAsync(fb, pos, pos_b, cudaMemcpyDeviceToDevice, st));
    HARP_CUDA(cudaMemcpyAsync(fb + o_coef, coef, coef_b, cudaMemcpyDeviceToDevice, st));
    HARP_CUDA(cudaMemcpyAsync(fb + o_self, self_blocks, self_b, cudaMemcpyDeviceToDevice, st));
    // The FP64-accurate Z64, which only the refinement reads, on the
    // context's fill stream beside the factorisation that follows, after the
    // caller's earlier work (a previous solve may still read Z64).
    HARP_CUDA(cudaEventRecord(ctx->ev_fill_fork, st));
    HARP_CUDA(cudaStreamWaitEvent(ctx->fill_stream, ctx->ev_fill_fork, 0));
    s = HARP_E_UNSUPPORTED;
    if (ctx->fill64_now)
      s = oz_fill_z64(ctx, Na, Nm, P, Q, reinterpret_cast<const double*>(fb),
                      2.0 * kPi * freq_hz / kC0, reinterpret_cast<const double2*>(fb + o_coef),
                      reinterpret_cast<const double2*>(fb + o_self), self_stride, ctx->z64,
                      ctx->ld64, ctx->dstatus + 3, ctx->fill_stream);
    if (s == HARP_E_UNSUPPORTED)
      s = fill_dispatch(ctx, Na, Nm, P, Q, reinterpret_cast<const double*>(fb), freq_hz,
                        reinterpret_cast<const double*>(fb + o_coef),
                        reinterpret_cast<const double*>(fb + o_self), self_stride, ctx->z64,
                        ctx->ld64, nullptr, 0, 1, ctx->fill_stream, ctx->dstatus + 3, true);
    if (s != HARP_OK) return s;
    // and, when the refinement uses the tensor-core residual, the digit
    // slices of Z64 for trans 'N' solves, on the same stream
    const long long ticket = ++ctx->z64_ticket;
    if (ctx->oz_a && ctx->residual_mode == HARP_RESIDUAL_SLICES &&
        oz_prepare(ctx, (int)N, ctx->z64, ctx->ld64, false, ctx->oz_znorm, ctx->fill_stream) ==
            HARP_OK)
      ctx->oz_ticket = ticket;
    HARP_CUDA(cudaEventRecord(ctx->ev_z64, ctx->fill_stream));
  }
  return HARP_OK;
}
