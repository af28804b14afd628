// panel_cluster.cu -- one-launch LU panel factorisation with partial pivoting
// on a thread-block cluster.
//
// The panel A[k0 : k0+M, k0 : k0+nb] is split into row blocks of Mb rows,
// one per CTA of a cluster (Mb >= nb, so the panel's own top rows all live
// in CTA 0). Each CTA keeps its block in shared memory, column-major, for
// the whole factorisation. Column j (one cluster barrier per column):
//   1. each CTA finds its local candidate (largest |z|^2 among its rows
//      >= j, first index on ties) and writes it -- value, row index and the
//      row's nb entries -- into every CTA's candidate table through
//      distributed shared memory; CTA 0 also writes its current row j;
//   2. cluster barrier;
//   3. every CTA reduces its copy of the table (same data, same order, same
//      pivot p) and has the pivot row and row j locally: CTA 0 writes the
//      pivot row into row j, the owner of p writes old row j into row p,
//      and every CTA scales its rows below j and applies the rank-1 update
//      to the panel's remaining columns.
// The tables are double-buffered by column parity: a CTA can only publish
// for column j+2 after every CTA has passed barrier j+1, that is after
// every CTA has finished reading the tables of column j. Every CTA executes
// the same sequence of barriers (all branches depend only on the shared
// tables), so they cannot deadlock. The row interchanges of the rest of the
// matrix, the triangular solve for U12 and the trailing update stay with
// the caller.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "dense.cuh"
#include "prof.cuh"

namespace cg = cooperative_groups;

namespace harp {

constexpr int kPcThreads = 512;
constexpr int kPcMaxNb = 64;
constexpr int kPcMaxCluster = 16;

// Bytes of dynamic shared memory for a panel of nb columns, Mb rows per CTA
// and a cluster of C CTAs.
__host__ __device__ inline size_t panel_smem_bytes(int nb, int Mb, int C) {
  return sizeof(float) * ((size_t)2 * nb * (Mb + 1)  // panel block (re, im), column stride Mb + 1

                          + (size_t)4 * C * nb     // candidate rows, 2 parities
                          + (size_t)4 * nb         // row j, 2 parities
                          + (size_t)2 * C)         // candidate values
         + sizeof(int) * (size_t)2 * C;            // candidate row indices
}

__global__ void __launch_bounds__(kPcThreads) panel_cluster_kernel(float* Are, float* Aim, long lda,
                                                                   int k0, int M, int nb, int Mb,
                                                                   int* ipiv, int* zero_col) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  extern __shared__ __align__(16) float pc_smem[];
  // Column stride Mb + 1: the row-wise accesses (a row's nb entries) then
  // fall in distinct banks.
  const int ldS = Mb + 1;
  float* sre = pc_smem;                        // [nb][ldS]
  float* sim = sre + (size_t)nb * ldS;
  float* tab_r = sim + (size_t)nb * ldS;       // [2][C][nb]
  float* tab_i = tab_r + (size_t)2 * C * nb;
  float* jrow_r = tab_i + (size_t)2 * C * nb;  // [2][nb]
  float* jrow_i = jrow_r + 2 * nb;
  float* cand_v = jrow_i + 2 * nb;             // [2][C]
  int* cand_i = reinterpret_cast<int*>(cand_v + 2 * C);
  __shared__ float red_v[kPcThreads / 32];
  __shared__ int red_i[kPcThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = crank * Mb;  // first panel row of this CTA
  const int rows = max(0, min(Mb, M - r0));
  float* gre = Are + (size_t)(k0 + r0) + (size_t)k0 * lda;
  float* gim = Aim + (size_t)(k0 + r0) + (size_t)k0 * lda;

  // load the row block (independent loads batched before the stores)
  for (int c = 0; c < nb; ++c)
    for (int rb = 0; rb < rows; rb += 4 * kPcThreads) {
      float vr[4], vi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = rb + tid + u * kPcThreads;
        vr[u] = (r < rows) ? gre[r + (size_t)c * lda] : 0.f;
        vi[u] = (r < rows) ? gim[r + (size_t)c * lda] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = rb + tid + u * kPcThreads;
        if (r < rows) {
          sre[(size_t)c * ldS + r] = vr[u];
          sim[(size_t)c * ldS + r] = vi[u];
        }
      }
    }
  __syncthreads();

  float inv_r = 0.f, inv_i = 0.f;  // 1 / pivot of the previous column
  bool scale_prev = false;
  for (int j = 0; j < nb; ++j) {
    const int par = j & 1;
    // 0. deferred scaling of column j-1 below its diagonal (L multipliers);
    // the update of step j-1 read it unscaled
    if (scale_prev) {
      for (int r = tid; r < rows; r += kPcThreads) {
        if (r0 + r <= j - 1) continue;
        float* xr = &sre[(size_t)(j - 1) * ldS + r];
        float* xi = &sim[(size_t)(j - 1) * ldS + r];
        const float ar = *xr, ai = *xi;
        *xr = ar * inv_r - ai * inv_i;
        *xi = ar * inv_i + ai * inv_r;
      }
      scale_prev = false;
    }
    // 1. local candidate
    float best = -1.f;
    int bi = INT_MAX;
    for (int r = tid; r < rows; r += kPcThreads) {
      const int g = r0 + r;
      if (g < j) continue;
      const float xr = sre[(size_t)j * ldS + r], xi = sim[(size_t)j * ldS + r];
      const float v = xr * xr + xi * xi;
      if (v > best) {
        best = v;
        bi = g;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ob = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      red_v[warp] = best;
      red_i[warp] = bi;
    }
    __syncthreads();
    // every warp reduces the kPcThreads/32 warp candidates with shuffles
    // (largest value, then smallest row), so all threads hold the result
    best = (lane < kPcThreads / 32) ? red_v[lane] : -2.f;
    bi = (lane < kPcThreads / 32) ? red_i[lane] : INT_MAX;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    // publish: value and index, the candidate row, and (CTA 0) row j
    if (tid < nb) {
      float vr = 0.f, vi = 0.f;
      if (best >= 0.f) {
        vr = sre[(size_t)tid * ldS + (bi - r0)];
        vi = sim[(size_t)tid * ldS + (bi - r0)];
      }
      float wr = 0.f, wi = 0.f;
      if (crank == 0) {
        wr = sre[(size_t)tid * ldS + j];
        wi = sim[(size_t)tid * ldS + j];
      }
      for (int q = 0; q < C; ++q) {
        float* tr = cluster.map_shared_rank(tab_r, q);
        float* ti = cluster.map_shared_rank(tab_i, q);
        tr[((size_t)par * C + crank) * nb + tid] = vr;
        ti[((size_t)par * C + crank) * nb + tid] = vi;
        if (crank == 0) {
          cluster.map_shared_rank(jrow_r, q)[par * nb + tid] = wr;
          cluster.map_shared_rank(jrow_i, q)[par * nb + tid] = wi;
        }
      }
    }
    if (tid < C) {
      cluster.map_shared_rank(cand_v, tid)[par * C + crank] = best;
      cluster.map_shared_rank(cand_i, tid)[par * C + crank] = bi;
    }
    cluster.sync();

    // 2. the pivot (same in every CTA), pivot row and row j from the tables
    // the C candidates reduced with shuffles in every warp (same order:
    // largest value, then smallest row; win = the owning CTA)
    int win = lane;
    best = (lane < C) ? cand_v[par * C + lane] : -2.f;
    bi = (lane < C) ? cand_i[par * C + lane] : INT_MAX;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      const int ow = __shfl_xor_sync(0xffffffffu, win, off);
      if (ob > best || (ob == best && oi < bi) || (ob == best && oi == bi && ow < win)) {
        best = ob;
        bi = oi;
        win = ow;
      }
    }
    const int p = bi;
    const bool zero = !(best > 0.f) || p >= M;
    if (crank == 0 && tid == 0) {
      if (zero) {
        ipiv[k0 + j] = k0 + j;
        atomicMin(zero_col, k0 + j + 1);
      } else {
        ipiv[k0 + j] = k0 + p;
      }
    }
    if (zero) continue;  // uniform across the cluster
    const float* prow_r = tab_r + ((size_t)par * C + win) * nb;
    const float* prow_i = tab_i + ((size_t)par * C + win) * nb;

    // 3. swap, scale, rank-1 update (local)
    if (tid < nb) {
      if (crank == 0) {
        sre[(size_t)tid * ldS + j] = prow_r[tid];
        sim[(size_t)tid * ldS + j] = prow_i[tid];
      }
      if (crank == win && p != j) {
        sre[(size_t)tid * ldS + (p - r0)] = jrow_r[par * nb + tid];
        sim[(size_t)tid * ldS + (p - r0)] = jrow_i[par * nb + tid];
      }
    }
    __syncthreads();
    const float pr = prow_r[j], pi = prow_i[j];
    const float den = pr * pr + pi * pi;
    inv_r = pr / den;
    inv_i = -pi / den;
    scale_prev = true;
    // rank-1 update of columns j+1.. below row j: warp w takes columns
    // j+1+w, j+1+w+16, ..., lanes take rows (conflict-free); the multiplier
    // of a row is formed from the unscaled column j in registers
    constexpr int kW = kPcThreads / 32;
    constexpr int kCpw = (kPcMaxNb + kW - 1) / kW;
    float ur[kCpw], ui[kCpw];
#pragma unroll
    for (int m = 0; m < kCpw; ++m) {
      const int cc = j + 1 + warp + kW * m;
      ur[m] = (cc < nb) ? prow_r[cc] : 0.f;
      ui[m] = (cc < nb) ? prow_i[cc] : 0.f;
    }
    if (j + 1 + warp < nb) {
      for (int r = lane; r < rows; r += 32) {
        if (r0 + r <= j) continue;
        const float ar = sre[(size_t)j * ldS + r], ai = sim[(size_t)j * ldS + r];
        const float lr = ar * inv_r - ai * inv_i, li = ar * inv_i + ai * inv_r;
#pragma unroll
        for (int m = 0; m < kCpw; ++m) {
          const int cc = j + 1 + warp + kW * m;
          if (cc < nb) {
            float* xr = &sre[(size_t)cc * ldS + r];
            float* xi = &sim[(size_t)cc * ldS + r];
            const float vr = *xr, vi = *xi;
            *xr = fmaf(-lr, ur[m], fmaf(li, ui[m], vr));
            *xi = fmaf(-lr, ui[m], fmaf(-li, ur[m], vi));
          }
        }
      }
    }
    __syncthreads();
  }
  // scaling of the last column
  if (scale_prev) {
    for (int r = tid; r < rows; r += kPcThreads) {
      if (r0 + r <= nb - 1) continue;
      float* xr = &sre[(size_t)(nb - 1) * ldS + r];
      float* xi = &sim[(size_t)(nb - 1) * ldS + r];
      const float ar = *xr, ai = *xi;
      *xr = ar * inv_r - ai * inv_i;
      *xi = ar * inv_i + ai * inv_r;
    }
  }
  __syncthreads();

  // store the row block
  for (int c = 0; c < nb; ++c)
    for (int r = tid; r < rows; r += kPcThreads) {
      gre[r + (size_t)c * lda] = sre[(size_t)c * ldS + r];
      gim[r + (size_t)c * lda] = sim[(size_t)c * ldS + r];
    }
  cluster.sync();  // no CTA leaves while a peer may still write its tables
}

// Plan a cluster panel for M rows: returns the panel width to use (0 when
// the cluster path does not apply) and the cluster size and rows per CTA.
bool panel_cluster_ok(int C, size_t smem);

// Residency of a cluster of C CTAs with this much shared memory, cached per
// C as the largest size known to fit and the smallest known not to.
static bool cluster_resident(int C, size_t smem) {
  static std::mutex mu;
  static size_t ok_max[kPcMaxCluster + 1] = {0};
  static size_t bad_min[kPcMaxCluster + 1] = {0};
  std::lock_guard<std::mutex> lock(mu);
  if (smem <= ok_max[C]) return true;
  if (bad_min[C] && smem >= bad_min[C]) return false;
  const bool ok = panel_cluster_ok(C, smem);
  if (ok) ok_max[C] = std::max(ok_max[C], smem);
  else bad_min[C] = bad_min[C] ? std::min(bad_min[C], smem) : smem;
  return ok;
}

int panel_cluster_plan(const harp_ctx* ctx, int M, int want_nb, int* csize, int* Mb) {
  // The per-column update is a pass over the CTA's rows, so more CTAs are
  // faster until a CTA holds ~192 rows (measured on the 3072 x 64 panel:
  // 5.2 us per column with 384 rows per CTA, 4.6 with 192); take the
  // smallest cluster that fits in shared memory and reaches that, else the
  // largest that fits.
  const size_t budget = std::min<size_t>(ctx->smem_optin, 220 * 1024) - 2048;
  constexpr int kRowsTarget = 192;
  for (int nb = std::min(want_nb, kPcMaxNb); nb >= 16; nb /= 2) {
    int best_c = 0, best_mb = 0;
    for (int C : {1, 2, 4, 8, 16}) {
      int mb = (M + C - 1) / C;
      if (mb < nb) mb = nb;
      if (C > 1 && (C - 1) * mb >= M) continue;  // every CTA owns rows
      if (panel_smem_bytes(nb, mb, C) > budget) continue;
      if (!cluster_resident(C, panel_smem_bytes(nb, mb, C))) continue;
      best_c = C;
      best_mb = mb;
      if (mb <= kRowsTarget) break;
    }
    if (best_c) {
      *csize = best_c;
      *Mb = best_mb;
      return nb;
    }
  }
  return 0;
}

int panel_cluster(const harp_ctx* ctx, float* re, float* im, long ld, int k0, int M, int nb,
                  int C, int Mb, int* ipiv, int* zero_col, cudaStream_t st) {
  const size_t smem = panel_smem_bytes(nb, Mb, C);
  static bool attr_set = false;
  if (!attr_set) {
    HARP_CUDA(cudaFuncSetAttribute(panel_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   220 * 1024));
    HARP_CUDA(cudaFuncSetAttribute(panel_cluster_kernel,
                                   cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kPcThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ProfScope ps(HARP_K_PANEL, 4.0 * M * nb * (double)(nb - 1), st);
  HARP_CUDA(cudaLaunchKernelEx(&cfg, panel_cluster_kernel, re, im, ld, k0, M, nb, Mb, ipiv,
                               zero_col));
  HARP_LAUNCHED();
  return HARP_OK;
}

// Whether a cluster of C CTAs with this much shared memory can be resident.
bool panel_cluster_ok(int C, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kPcThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaFuncSetAttribute(panel_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           220 * 1024) != cudaSuccess ||
      cudaFuncSetAttribute(panel_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                           1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, panel_cluster_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

}  // namespace harp
