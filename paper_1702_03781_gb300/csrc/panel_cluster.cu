// panel_cluster.cu -- one-launch LU panel factorisation with partial pivoting
// on a thread-block cluster, rows held in place.
//
// The panel A[k0 : k0+M, k0 : k0+nb] (nb <= 64, a multiple of 16, M >= nb)
// is split into row blocks of Mb rows, one per CTA of a cluster; each CTA
// keeps its block in shared memory for the whole factorisation. Rows never
// move: a pivot row is only marked as chosen, and the row interchanges
// (LAPACK's ipiv) are composed once at the end and applied when the block is
// written back (and, when asked, exported as a row map for the other
// columns' interchanges). Columns are taken in sub-blocks of 16; warp w of every CTA
// owns column 16 s + w of sub-block s and holds its rows of that column in
// registers while the sub-block is factored. Step t:
//   1. every warp applies the rank-1 term of pivot t-1 to its column (rows
//      not yet chosen; multiplier a[r][t-1] / pivot) in registers and stores
//      it to shared memory, and the warp owning column t also finds the
//      CTA's candidate (largest |a|^2, smallest row on ties: two warp
//      reductions) and writes it -- |a|^2, row, entry, one 16-byte entry --
//      into every CTA's table through distributed shared memory;
//   2. cluster barrier;
//   3. every warp loads column t (the next step's multipliers), reduces the
//      table (same data, same order: the same pivot in every CTA), marks the
//      pivot row as chosen and reads the pivot row's entry in its own column
//      from the owning CTA; chosen rows are never written again, so that
//      read needs no further barrier.
// At the end of a sub-block with columns to its right, U12 = L11^-1 A12 is
// formed from its 16 pivot rows (read from their owners) and every row not
// yet chosen gets -L21 U12 (a register-tiled rank-16 product); the owners
// write U12 into their pivot rows after the next cluster barrier, when no
// CTA reads the old values any more.
// Multipliers stay unscaled until the write-back (l = a / pivot). The tables
// are double-buffered by step parity: a CTA writes the tables of step t+2
// only after every CTA passed barrier t+1, that is after every CTA finished
// reading those of step t. Every CTA executes the same barriers. A zero
// pivot (all remaining |a| = 0) still chooses a row (the smallest), with a
// zero inverse, and reports its column through *zero_col.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "dense.cuh"
#include "panel_common.cuh"
#include "prof.cuh"

namespace cg = cooperative_groups;

namespace harp {

constexpr int kPcThreads = 512;
constexpr int kPcW = kPcThreads / 32;  // sub-block width: one column per warp
constexpr int kPcMaxNb = 64;
constexpr int kPcMaxCluster = 16;
constexpr int kPcMaxRpl = 12;                 // rows per lane (register arrays)
constexpr int kPcMaxRows = 32 * kPcMaxRpl;  // rows per CTA

// Bytes of dynamic shared memory for a panel of nb columns, Mb rows per CTA
// and a cluster of C CTAs (the layout of panel_cluster_kernel).
__host__ __device__ inline size_t panel_smem_bytes(int nb, int Mb, int C) {
  return sizeof(float) * ((size_t)2 * nb * (Mb + 1)     // panel block, column stride Mb + 1
                          + (size_t)2 * nb               // 1 / pivot per step
                          + (size_t)2 * kPcW * kPcW      // L11 of a sub-block
                          + (size_t)2 * kPcW * kPcMaxNb  // U12 of a sub-block
                          + (size_t)4 * 2 * C)           // candidate tables
         + sizeof(int) * ((size_t)nb                     // pivot row of each step
                          + (size_t)2 * Mb);             // step a row was chosen, its output row
}

// A22 -= L21 U12 for one sub-block on this CTA's rows not yet chosen. The
// multipliers stay unscaled in shared memory; each term forms l = a / pivot
// exactly as the write-back stores it, so that the update uses the L that
// is kept. Warp w takes columns c1 + w + 16 m (m < NM), lane l rows l + 32 k
// in chunks of kCh; the accumulators live in registers across the 16 terms,
// each term reading one multiplier per row and NM entries of U12 (the same
// for the whole warp).
template <int RPL, int NM>
__device__ __forceinline__ void panel_rank16(float* sre, float* sim, int ldS,
                                             const float* s_inv_r, const float* s_inv_i,
                                             const float* u12_r, const float* u12_i, int s0,
                                             int c1, int lane, int warp, unsigned inrows,
                                             unsigned live) {
  constexpr int kCh = RPL <= 6 ? RPL : (RPL % 6 == 0 ? 6 : 4);
  static_assert(RPL % kCh == 0, "row chunks");
#pragma unroll
  for (int k0 = 0; k0 < RPL; k0 += kCh) {
    float cr[kCh][NM], ci[kCh][NM];
#pragma unroll
    for (int kk = 0; kk < kCh; ++kk)
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const bool in = (inrows >> (k0 + kk)) & 1u;
        const size_t o = (size_t)(c1 + warp + kPcW * m) * ldS + lane + 32 * (k0 + kk);
        cr[kk][m] = in ? sre[o] : 0.f;
        ci[kk][m] = in ? sim[o] : 0.f;
      }
#pragma unroll 1
    for (int s = 0; s < kPcW; ++s) {
      const float ir = s_inv_r[s0 + s], ii = s_inv_i[s0 + s];
      float ur[NM], ui[NM];
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        ur[m] = u12_r[s * kPcMaxNb + c1 + warp + kPcW * m];
        ui[m] = u12_i[s * kPcMaxNb + c1 + warp + kPcW * m];
      }
#pragma unroll
      for (int kk = 0; kk < kCh; ++kk) {
        const bool in = (inrows >> (k0 + kk)) & 1u;
        const size_t o = (size_t)(s0 + s) * ldS + lane + 32 * (k0 + kk);
        const float a_r = in ? sre[o] : 0.f, a_i = in ? sim[o] : 0.f;
        const float lr = a_r * ir - a_i * ii, li = a_r * ii + a_i * ir;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          cr[kk][m] = fmaf(-lr, ur[m], fmaf(li, ui[m], cr[kk][m]));
          ci[kk][m] = fmaf(-lr, ui[m], fmaf(-li, ur[m], ci[kk][m]));
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < kCh; ++kk)
      if ((live >> (k0 + kk)) & 1u)
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          const size_t o = (size_t)(c1 + warp + kPcW * m) * ldS + lane + 32 * (k0 + kk);
          sre[o] = cr[kk][m];
          sim[o] = ci[kk][m];
        }
  }
}

// RPL: rows per lane (ceil(Mb / 32)), so that a lane's rows of a column are
// loaded into registers together and the step's arithmetic is unrolled.
template <int RPL>
__global__ void __launch_bounds__(kPcThreads, 1) panel_cluster_kernel(float* Are, float* Aim, long lda,
                                                                   int k0, int M, int nb, int Mb,
                                                                   int* ipiv, int* zero_col,
                                                                   int* rmap) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  extern __shared__ __align__(16) float pc_smem[];
  // Column stride Mb + 1: a row's entries fall in distinct banks.
  const int ldS = Mb + 1;
  // candidate tables by step parity: |a|^2 bits, row, re, im
  float4* tab = reinterpret_cast<float4*>(pc_smem);  // [2][C]
  float* sre = pc_smem + 8 * C;                      // [nb][ldS]
  float* sim = sre + (size_t)nb * ldS;
  float* s_inv_r = sim + (size_t)nb * ldS;           // [nb]
  float* s_inv_i = s_inv_r + nb;
  float* l11_r = s_inv_i + nb;                       // [kPcW][kPcW], by columns
  float* l11_i = l11_r + kPcW * kPcW;
  float* u12_r = l11_i + kPcW * kPcW;                // [kPcW][kPcMaxNb]
  float* u12_i = u12_r + kPcW * kPcMaxNb;
  int* piv_row = reinterpret_cast<int*>(u12_i + kPcW * kPcMaxNb);  // [nb] row chosen at each step
  int* step_of = piv_row + nb;                        // [Mb] step a local row was chosen (nb: not)
  int* dest = step_of + Mb;                           // [Mb] output panel row of a local row
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = crank * Mb;  // first panel row of this CTA
  const int rows = max(0, min(Mb, M - r0));
  float* gre = Are + (size_t)(k0 + r0) + (size_t)k0 * lda;
  float* gim = Aim + (size_t)(k0 + r0) + (size_t)k0 * lda;

  // load the row block: every element's asynchronous copy is issued before
  // any is waited for, so the block costs one memory round trip
  for (int e = tid; e < rows * nb; e += kPcThreads) {
    const int c = e / rows, r = e - c * rows;
    const unsigned dr = (unsigned)__cvta_generic_to_shared(sre + (size_t)c * ldS + r);
    const unsigned di = (unsigned)__cvta_generic_to_shared(sim + (size_t)c * ldS + r);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dr),
                 "l"(gre + r + (size_t)c * lda));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(di),
                 "l"(gim + r + (size_t)c * lda));
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  for (int r = tid; r < Mb; r += kPcThreads) {
    step_of[r] = nb;
    dest[r] = r0 + r;
  }
  __syncthreads();

  unsigned chosen = 0;  // bit k: local row lane + 32 k is chosen
  unsigned inrows = 0;  // bit k: local row lane + 32 k exists
#pragma unroll
  for (int k = 0; k < RPL; ++k)
    if (lane + 32 * k < rows) inrows |= 1u << k;
  float xr[RPL], xi[RPL];          // this warp's column of the current sub-block
  float ar[RPL], ai[RPL];          // the last pivot column (unscaled multipliers)
  float u_r = 0.f, u_i = 0.f;      // pivot row's entry in this warp's column
  float inv_r = 0.f, inv_i = 0.f;  // 1 / pivot of the last step
#pragma unroll
  for (int k = 0; k < RPL; ++k) xr[k] = xi[k] = ar[k] = ai[k] = 0.f;
  for (int t = 0; t < nb; ++t) {
    const int par = t & 1;
    const int sb = t / kPcW;
    const int c = sb * kPcW + warp;  // this warp's column
    const bool first = (t == sb * kPcW);
    if (first) {  // the sub-block's columns into registers
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        const bool in = (inrows >> k) & 1u;
        xr[k] = in ? sre[(size_t)c * ldS + lane + 32 * k] : 0.f;
        xi[k] = in ? sim[(size_t)c * ldS + lane + 32 * k] : 0.f;
      }
    }
    // 1. rank-1 term of pivot t-1 on the rows not yet chosen (registers,
    // then shared memory for the other warps and CTAs); the owner of column
    // t finds the candidate
    if (c >= t) {
      const unsigned live = inrows & ~chosen;
      if (!first) {
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
          const float lr = ar[k] * inv_r - ai[k] * inv_i, li = ar[k] * inv_i + ai[k] * inv_r;
          const float yr = fmaf(-lr, u_r, fmaf(li, u_i, xr[k]));
          const float yi = fmaf(-lr, u_i, fmaf(-li, u_r, xi[k]));
          if ((live >> k) & 1u) {
            xr[k] = yr;
            xi[k] = yi;
            sre[(size_t)c * ldS + lane + 32 * k] = yr;
            sim[(size_t)c * ldS + lane + 32 * k] = yi;
          }
        }
      }
      if (c == t) {
        float best = -1.f, bre = 0.f, bim = 0.f;
        int bi = INT_MAX;
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
          const float v = xr[k] * xr[k] + xi[k] * xi[k];
          if (((live >> k) & 1u) && v > best) {
            best = v;
            bi = r0 + lane + 32 * k;
            bre = xr[k];
            bim = xi[k];
          }
        }
        // warp argmax in two reductions: the largest |a|^2 (bit patterns of
        // non-negative floats order like their values), then the smallest
        // row among the lanes holding it; a lane without rows offers 0 and
        // row INT_MAX, which loses every tie
        const unsigned key = (best >= 0.f) ? __float_as_uint(best) : 0u;
        const unsigned row = (best >= 0.f) ? (unsigned)bi : (unsigned)INT_MAX;
        const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
        const unsigned rmin = __reduce_min_sync(0xffffffffu, key == kmax ? row : 0xffffffffu);
        const int src = __ffs(__ballot_sync(0xffffffffu, key == kmax && row == rmin)) - 1;
        bre = __shfl_sync(0xffffffffu, bre, src);
        bim = __shfl_sync(0xffffffffu, bim, src);
        if (lane < C)  // one 16-byte entry into every CTA's table
          cluster.map_shared_rank(tab, lane)[par * C + crank] =
              make_float4(__uint_as_float(kmax), __int_as_float((int)rmin), bre, bim);
      }
    }
    cluster.sync();

    // 3. the next step's multipliers (column t, complete since the barrier),
    // then the pivot (same in every CTA): the same two reductions over the C
    // table entries (lane q reads entry q; rows are distinct, so the winner
    // is unique unless no CTA had rows)
    if (c > t) {
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        const bool in = (inrows >> k) & 1u;
        ar[k] = in ? sre[(size_t)t * ldS + lane + 32 * k] : 0.f;
        ai[k] = in ? sim[(size_t)t * ldS + lane + 32 * k] : 0.f;
      }
    }
    const float4 te = (lane < C) ? tab[par * C + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const unsigned tkey = (lane < C) ? __float_as_uint(te.x) : 0u;
    const unsigned trow = (lane < C) ? (unsigned)__float_as_int(te.y) : 0xffffffffu;
    const unsigned tk = __reduce_max_sync(0xffffffffu, tkey);
    const unsigned tr = __reduce_min_sync(0xffffffffu, tkey == tk ? trow : 0xffffffffu);
    const int pw = __ffs(__ballot_sync(0xffffffffu, tkey == tk && trow == tr)) - 1;
    const float pvr = __shfl_sync(0xffffffffu, te.z, pw);
    const float pvi = __shfl_sync(0xffffffffu, te.w, pw);
    const float pm = __uint_as_float(tk);
    const int pr = (int)tr;
    const bool none = (tr >= (unsigned)M);  // no row left anywhere (M >= nb rules it out)
    const bool zero = !(pm > 0.f);
    // the pivot row's entry in this warp's column (chosen rows are not
    // written again)
    u_r = u_i = 0.f;
    if (!none && c > t) {
      const size_t o = (size_t)c * ldS + (pr - pw * Mb);
      u_r = cluster.map_shared_rank(sre, pw)[o];
      u_i = cluster.map_shared_rank(sim, pw)[o];
    }
    if (zero || none) {
      inv_r = inv_i = 0.f;
    } else {
      const float rd = __frcp_rn(pvr * pvr + pvi * pvi);
      inv_r = pvr * rd;
      inv_i = -pvi * rd;
    }
    if (tid == 0) {
      piv_row[t] = none ? -1 : pr;
      s_inv_r[t] = inv_r;
      s_inv_i[t] = inv_i;
      if (crank == 0 && zero) atomicMin(zero_col, k0 + t + 1);
    }
    if (!none && pw == crank && ((pr - r0) & 31) == lane) {
      chosen |= 1u << ((pr - r0) >> 5);
      if (warp == 0) step_of[pr - r0] = t;
    }
    // U12 of the previous sub-block into its pivot rows (their old values
    // were last read before the barrier above)
    if (first && sb > 0) {
      const int s0 = (sb - 1) * kPcW, c1 = sb * kPcW, nr = nb - c1;
      for (int e = tid; e < kPcW * nr; e += kPcThreads) {
        const int s = e / nr, cc = c1 + e % nr;
        const int row = piv_row[s0 + s];
        if (row >= r0 && row < r0 + rows) {
          sre[(size_t)cc * ldS + (row - r0)] = u12_r[s * kPcMaxNb + cc];
          sim[(size_t)cc * ldS + (row - r0)] = u12_i[s * kPcMaxNb + cc];
        }
      }
    }

    // end of a sub-block with columns to its right: U12 = L11^-1 A12 and
    // A22 -= L21 U12 on the rows not yet chosen
    if (t == (sb + 1) * kPcW - 1 && t + 1 < nb) {
      __syncthreads();  // this sub-block's pivot rows and inverses are in shared memory
      const int s0 = sb * kPcW, c1 = s0 + kPcW, nr = nb - c1;
      // the 16 x (16 + nr) <= 2 x 512 entries: both remote reads of a thread
      // issued before either is used
      {
        const int ne = kPcW * (kPcW + nr);
        float vr[2], vi[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int e = tid + h * kPcThreads;
          const int s = e / (kPcW + nr), j = e % (kPcW + nr);
          const int cc = (j < kPcW) ? s0 + j : c1 + (j - kPcW);
          const int row = (e < ne) ? piv_row[s0 + s] : -1;
          vr[h] = vi[h] = 0.f;
          if (row >= 0 && !(j < kPcW && j >= s)) {  // L11: strictly lower part only
            const int own = row / Mb;
            const size_t o = (size_t)cc * ldS + (row - own * Mb);
            vr[h] = cluster.map_shared_rank(sre, own)[o];
            vi[h] = cluster.map_shared_rank(sim, own)[o];
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int e = tid + h * kPcThreads;
          if (e >= ne) continue;
          const int s = e / (kPcW + nr), j = e % (kPcW + nr);
          const int cc = (j < kPcW) ? s0 + j : c1 + (j - kPcW);
          if (j < kPcW) {  // L11 by columns: entry (s, j) at j * 16 + s
            const float ir = s_inv_r[cc], ii = s_inv_i[cc];
            l11_r[j * kPcW + s] = vr[h] * ir - vi[h] * ii;
            l11_i[j * kPcW + s] = vr[h] * ii + vi[h] * ir;
          } else {
            u12_r[s * kPcMaxNb + cc] = vr[h];
            u12_i[s * kPcMaxNb + cc] = vi[h];
          }
        }
      }
      __syncthreads();
      // U12 = L11^-1 A12 by forward substitution: warp w takes columns
      // c1 + w + 16 m together, lane s holds row s; row q is final after
      // step q and reaches the other lanes by shuffle. This code and the
      // sub-block update run once per 16 columns; their loops stay rolled,
      // which keeps the kernel's code small.
      {
        constexpr int kCpw = (kPcMaxNb - kPcW + kPcW - 1) / kPcW;  // columns per warp
        float ur[kCpw], ui[kCpw];
#pragma unroll
        for (int m = 0; m < kCpw; ++m) {
          const int cc = c1 + warp + kPcW * m;
          ur[m] = (lane < kPcW && cc < nb) ? u12_r[lane * kPcMaxNb + cc] : 0.f;
          ui[m] = (lane < kPcW && cc < nb) ? u12_i[lane * kPcMaxNb + cc] : 0.f;
        }
#pragma unroll 1
        for (int q = 0; q < kPcW - 1; ++q) {
          const float lr = (lane < kPcW && q < lane) ? l11_r[q * kPcW + lane] : 0.f;
          const float li = (lane < kPcW && q < lane) ? l11_i[q * kPcW + lane] : 0.f;
#pragma unroll
          for (int m = 0; m < kCpw; ++m) {
            const float vr = __shfl_sync(0xffffffffu, ur[m], q);
            const float vi = __shfl_sync(0xffffffffu, ui[m], q);
            ur[m] = fmaf(-lr, vr, fmaf(li, vi, ur[m]));
            ui[m] = fmaf(-lr, vi, fmaf(-li, vr, ui[m]));
          }
        }
#pragma unroll
        for (int m = 0; m < kCpw; ++m) {
          const int cc = c1 + warp + kPcW * m;
          if (lane < kPcW && cc < nb) {
            u12_r[lane * kPcMaxNb + cc] = ur[m];
            u12_i[lane * kPcMaxNb + cc] = ui[m];
          }
        }
      }
      __syncthreads();
      {
        const unsigned live = inrows & ~chosen;
        const int nm = (nb - c1) / kPcW;  // columns per warp: 1, 2 or 3
        if (nm == 3)
          panel_rank16<RPL, 3>(sre, sim, ldS, s_inv_r, s_inv_i, u12_r, u12_i, s0, c1, lane, warp,
                               inrows, live);
        else if (nm == 2)
          panel_rank16<RPL, 2>(sre, sim, ldS, s_inv_r, s_inv_i, u12_r, u12_i, s0, c1, lane, warp,
                               inrows, live);
        else
          panel_rank16<RPL, 1>(sre, sim, ldS, s_inv_r, s_inv_i, u12_r, u12_i, s0, c1, lane, warp,
                               inrows, live);
      }
      __syncthreads();
    }
  }

  // Compose the interchanges (the same data in every CTA): ipiv and the row
  // map from CTA 0, the output position of this CTA's rows that move.
  __syncthreads();
  if (warp == 0) panel_compose(piv_row, nb, k0, r0, rows, crank, ipiv, rmap, dest, lane);
  __syncthreads();

  // write back: below a row's own step the scaled multipliers, from it on
  // the U entries
  float* ore = Are + (size_t)k0 + (size_t)k0 * lda;
  float* oim = Aim + (size_t)k0 + (size_t)k0 * lda;
#pragma unroll 4
  for (int e = tid; e < rows * nb; e += kPcThreads) {
    const int cc = e / rows, r = e - cc * rows;
    const float ir = s_inv_r[cc], ii = s_inv_i[cc];
    const float ar = sre[(size_t)cc * ldS + r], ai = sim[(size_t)cc * ldS + r];
    float vr = ar, vi = ai;
    if (cc < step_of[r]) {
      vr = ar * ir - ai * ii;
      vi = ar * ii + ai * ir;
    }
    const size_t o = (size_t)dest[r] + (size_t)cc * lda;
    ore[o] = vr;
    oim[o] = vi;
  }
  cluster.sync();  // no CTA leaves while a peer may still read its shared memory
}

// Plan a cluster panel for M rows: returns the panel width to use (0 when
// the cluster path does not apply) and the cluster size and rows per CTA.
bool panel_cluster_ok(int C, size_t smem, int Mb);

// Residency of a cluster of C CTAs (instantiation for Mb rows) with this
// much shared memory, cached per (C, instantiation) as the largest size
// known to fit and the smallest known not to.
static bool cluster_resident(int C, size_t smem, int Mb) {
  static std::mutex mu;
  static size_t ok_max[kPcMaxCluster + 1][5] = {};
  static size_t bad_min[kPcMaxCluster + 1][5] = {};
  const int rpl = (Mb + 31) / 32;
  const int i = rpl <= 2 ? 0 : rpl <= 4 ? 1 : rpl <= 6 ? 2 : rpl <= 8 ? 3 : 4;
  std::lock_guard<std::mutex> lock(mu);
  if (smem <= ok_max[C][i]) return true;
  if (bad_min[C][i] && smem >= bad_min[C][i]) return false;
  const bool ok = panel_cluster_ok(C, smem, Mb);
  if (ok) ok_max[C][i] = std::max(ok_max[C][i], smem);
  else bad_min[C][i] = bad_min[C][i] ? std::min(bad_min[C][i], smem) : smem;
  return ok;
}

int panel_cluster_plan(const harp_ctx* ctx, int M, int want_nb, int* csize, int* Mb) {
  // The per-column update is a pass over the CTA's rows, so more CTAs are
  // faster until a CTA holds ~192 rows (measured on the 3072 x 64 panel:
  // 5.2 us per column with 384 rows per CTA, 4.6 with 192); take the
  // smallest cluster that fits in shared memory and reaches that, else the
  // largest that fits.
  const size_t budget = std::min<size_t>(ctx->smem_optin, 220 * 1024) - 2048;
  const int kRowsTarget = ctx->panel_rows > 0 ? ctx->panel_rows : 192;
  for (int nb : {64, 32, 16}) {  // multiples of the sub-block width
    if (nb > want_nb || nb > kPcMaxNb) continue;
    int best_c = 0, best_mb = 0;
    for (int C : {1, 2, 4, 8, 16}) {
      int mb = (M + C - 1) / C;
      if (mb < nb) mb = nb;
      if (M < nb || mb > kPcMaxRows) continue;
      if (C > 1 && (C - 1) * mb >= M) continue;  // every CTA owns rows
      if (panel_smem_bytes(nb, mb, C) > budget) continue;
      if (!cluster_resident(C, panel_smem_bytes(nb, mb, C), mb)) continue;
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

using PanelKernel = void (*)(float*, float*, long, int, int, int, int, int*, int*, int*);

// The instantiation for Mb rows per CTA (rows per lane rounded up) and its
// index among them.
static PanelKernel panel_kernel_for(int Mb, int* idx) {
  const int rpl = (Mb + 31) / 32;
  static const PanelKernel ks[] = {panel_cluster_kernel<2>, panel_cluster_kernel<4>,
                                   panel_cluster_kernel<6>, panel_cluster_kernel<8>,
                                   panel_cluster_kernel<12>};
  const int i = rpl <= 2 ? 0 : rpl <= 4 ? 1 : rpl <= 6 ? 2 : rpl <= 8 ? 3 : 4;
  *idx = i;
  return ks[i];
}

static int panel_attrs(PanelKernel k, int idx) {
  static bool done[5] = {false, false, false, false, false};
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (done[idx]) return HARP_OK;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return cuda_status(cudaGetLastError());
  done[idx] = true;
  return HARP_OK;
}

int panel_cluster(const harp_ctx* ctx, float* re, float* im, long ld, int k0, int M, int nb,
                  int C, int Mb, int* ipiv, int* zero_col, cudaStream_t st, int* rmap) {
  if (Mb > kPcMaxRows || nb % kPcW != 0 || nb > kPcMaxNb || M < nb || C > kPcMaxCluster)
    return HARP_E_UNSUPPORTED;
  const size_t smem = panel_smem_bytes(nb, Mb, C);
  int idx = 0;
  PanelKernel kern = panel_kernel_for(Mb, &idx);
  HARP_TRY(panel_attrs(kern, idx));
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
  HARP_CUDA(cudaLaunchKernelEx(&cfg, kern, re, im, ld, k0, M, nb, Mb, ipiv, zero_col, rmap));
  HARP_LAUNCHED();
  return HARP_OK;
}

// Whether a cluster of C CTAs of the instantiation for Mb rows, with this
// much shared memory, can be resident.
bool panel_cluster_ok(int C, size_t smem, int Mb) {
  int idx = 0;
  PanelKernel kern = panel_kernel_for(Mb, &idx);
  if (panel_attrs(kern, idx) != HARP_OK) {
    cudaGetLastError();
    return false;
  }
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
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

}  // namespace harp
