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
  return sizeof(float) * ((size_t)2 * nb * Mb      // panel block (re, im)
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
  float* sre = pc_smem;                        // [nb][Mb]
  float* sim = sre + (size_t)nb * Mb;
  float* tab_r = sim + (size_t)nb * Mb;        // [2][C][nb]
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
          sre[(size_t)c * Mb + r] = vr[u];
          sim[(size_t)c * Mb + r] = vi[u];
        }
      }
    }
  __syncthreads();

  for (int j = 0; j < nb; ++j) {
    const int par = j & 1;
    // 1. local candidate
    float best = -1.f;
    int bi = INT_MAX;
    for (int r = tid; r < rows; r += kPcThreads) {
      const int g = r0 + r;
      if (g < j) continue;
      const float xr = sre[(size_t)j * Mb + r], xi = sim[(size_t)j * Mb + r];
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
    best = red_v[0];
    bi = red_i[0];
#pragma unroll
    for (int q = 1; q < kPcThreads / 32; ++q)
      if (red_v[q] > best || (red_v[q] == best && red_i[q] < bi)) {
        best = red_v[q];
        bi = red_i[q];
      }
    // publish: value and index, the candidate row, and (CTA 0) row j
    if (tid < nb) {
      float vr = 0.f, vi = 0.f;
      if (best >= 0.f) {
        vr = sre[(size_t)tid * Mb + (bi - r0)];
        vi = sim[(size_t)tid * Mb + (bi - r0)];
      }
      float wr = 0.f, wi = 0.f;
      if (crank == 0) {
        wr = sre[(size_t)tid * Mb + j];
        wi = sim[(size_t)tid * Mb + j];
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
    int win = 0;
    best = cand_v[par * C];
    bi = cand_i[par * C];
    for (int q = 1; q < C; ++q) {
      const float ob = cand_v[par * C + q];
      const int oi = cand_i[par * C + q];
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
        win = q;
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
        sre[(size_t)tid * Mb + j] = prow_r[tid];
        sim[(size_t)tid * Mb + j] = prow_i[tid];
      }
      if (crank == win && p != j) {
        sre[(size_t)tid * Mb + (p - r0)] = jrow_r[par * nb + tid];
        sim[(size_t)tid * Mb + (p - r0)] = jrow_i[par * nb + tid];
      }
    }
    __syncthreads();
    const float pr = prow_r[j], pi = prow_i[j];
    const float den = pr * pr + pi * pi;
    const float ir = pr / den, ii = -pi / den;
    for (int r = tid; r < rows; r += kPcThreads) {
      const int g = r0 + r;
      if (g <= j) continue;
      const float ar = sre[(size_t)j * Mb + r], ai = sim[(size_t)j * Mb + r];
      const float lr = ar * ir - ai * ii, li = ar * ii + ai * ir;
      sre[(size_t)j * Mb + r] = lr;
      sim[(size_t)j * Mb + r] = li;
      for (int cc = j + 1; cc < nb; ++cc) {
        const float ur = prow_r[cc], ui = prow_i[cc];
        float* xr = &sre[(size_t)cc * Mb + r];
        float* xi = &sim[(size_t)cc * Mb + r];
        *xr = fmaf(-lr, ur, fmaf(li, ui, *xr));
        *xi = fmaf(-lr, ui, fmaf(-li, ur, *xi));
      }
    }
    __syncthreads();
  }

  // store the row block
  for (int c = 0; c < nb; ++c)
    for (int r = tid; r < rows; r += kPcThreads) {
      gre[r + (size_t)c * lda] = sre[(size_t)c * Mb + r];
      gim[r + (size_t)c * lda] = sim[(size_t)c * Mb + r];
    }
  cluster.sync();  // no CTA leaves while a peer may still write its tables
}

// Plan a cluster panel for M rows: returns the panel width to use (0 when
// the cluster path does not apply) and the cluster size and rows per CTA.
int panel_cluster_plan(const harp_ctx* ctx, int M, int want_nb, int* csize, int* Mb) {
  const size_t budget = std::min<size_t>(ctx->smem_optin, 220 * 1024) - 2048;
  for (int nb = std::min(want_nb, kPcMaxNb); nb >= 16; nb /= 2) {
    for (int C : {1, 2, 4, 8, 16}) {
      int mb = (M + C - 1) / C;
      if (mb < nb) mb = nb;
      if (C > 1 && (C - 1) * mb >= M) continue;  // every CTA owns rows
      if (panel_smem_bytes(nb, mb, C) <= budget) {
        *csize = C;
        *Mb = mb;
        return nb;
      }
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
