// panel_calu.cu -- one-launch LU panel factorisation with tournament
// pivoting (communication-avoiding LU, Grigori, Demmel and Xiang 2011) on a
// thread-block cluster.
//
// The partial-pivoting cluster panel (panel_cluster.cu) needs one cluster
// barrier per column to agree on each pivot. Here the pivot rows of the
// whole panel are chosen by a tournament, so the CTAs synchronise a handful
// of times per panel instead of nb times:
//   1. every CTA factors its own row block (<= 256 rows of the panel A[k0:
//      k0+M, k0:k0+nb]) with partial pivoting, alone, and keeps the nb rows
//      it picked as its candidates;
//   2. the candidates meet in a tree of fan-in 4: at each level one CTA of
//      every group of four stacks the ORIGINAL rows of its group's
//      candidates (<= 256 rows, read from its peers' shared memory) and picks
//      nb of them by partial pivoting on that stack; the root's pick is the
//      pivot sequence of the panel, and its factorisation of the stack gives
//      the panel's L11 and U11 (the LU of the chosen rows in that order);
//   3. every CTA eliminates its other rows against the root's U11
//      (right-looking, pivots known): those rows become L21 = A21 U11^-1.
// The result has the output contract of the partial-pivoting panel: rows
// interchanged as LAPACK's ipiv describes (and the net row map, when asked),
// L below and U on and above the diagonal written back in place. The pivots
// may differ from partial pivoting's; the factorisation is of the same
// matrix with another row order, so the solve and its refinement are
// unchanged.
//
// Work layout (512 threads, 16 warps): warp w holds nb / 16 consecutive
// columns of the rows it factors in registers, lane l the rows l + 32 k. The
// steps of a factorisation come in groups, one group per warp: warp g picks
// the pivots of its own columns alone (largest |a|^2 among rows not yet
// chosen, smallest row on ties: two warp reductions), updating its later
// columns in registers, while the other warps apply the previous group's
// rank-1 updates, read from a two-group ring of multipliers in shared
// memory. One block barrier per group instead of one per step.
// A zero pivot of the root (all remaining |a| = 0) still chooses a row (the
// smallest), with a zero inverse, and reports its column through *zero_col.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "dense.cuh"
#include "panel_common.cuh"
#include "prof.cuh"

namespace cg = cooperative_groups;

namespace harp {

constexpr int kCaThreads = 512;
constexpr int kCaMaxNb = 64;
constexpr int kCaStack = 256;  // rows of a tree stack (fan-in 4 x 64) and of a CTA's block
constexpr int kCaLd = 260;     // column stride (floats) of the row buffer, a multiple of 4
constexpr int kCaLdU = 68;     // column stride (floats) of the root's nb x nb block
constexpr int kCaMaxCluster = 16;

// Shared memory of panel_calu_kernel (fixed layout, offsets in bytes).
struct CaLayout {
  static constexpr size_t buf = 0;                                    // 2 planes [64][kCaLd]
  static constexpr size_t u11 = buf + 2 * sizeof(float) * 64 * kCaLd;  // 2 planes [64][kCaLdU]
  static constexpr size_t mult = u11 + 2 * sizeof(float) * 64 * kCaLdU;  // 2 planes [8][kCaStack]
  static constexpr size_t inv = mult + 2 * sizeof(float) * 8 * kCaStack;  // 2 planes [64]
  static constexpr size_t ints = inv + 2 * sizeof(float) * 64;
  // int arrays: sel[64], cid[64], piv_id[64], sid[256], step_of[256], dest[256], misc[16]
  static constexpr size_t bytes = ints + sizeof(int) * (3 * 64 + 3 * kCaStack + 16);
};

struct CaSmem {
  float *bre, *bim;  // row buffer: column c at c * kCaLd, rows 0..255
  float *ure, *uim;  // the root's block: element (t, c) at c * kCaLdU + t
  float *mre, *mim;  // multipliers of two groups of steps: [(group parity * 4 + step) * kCaStack + row]
  float *inv_r, *inv_i;  // 1 / pivot of each step of the latest factorisation
  int* sel;      // stack row chosen at each step of the latest factorisation
  int* cid;      // panel rows of this CTA's current candidates (misc[2] of them)
  int* piv_id;   // panel rows of the final pivots
  int* sid;      // panel row of each stack row (-1: empty)
  int* step_of;  // step a stack row was chosen at (root), or a local row's pivot step
  int* dest;     // output position (panel row) of each local row
  int* misc;     // [2] candidate count, [3] first zero pivot
};

__device__ __forceinline__ CaSmem ca_smem(unsigned char* raw) {
  CaSmem S;
  S.bre = reinterpret_cast<float*>(raw + CaLayout::buf);
  S.bim = S.bre + 64 * kCaLd;
  S.ure = reinterpret_cast<float*>(raw + CaLayout::u11);
  S.uim = S.ure + 64 * kCaLdU;
  S.mre = reinterpret_cast<float*>(raw + CaLayout::mult);
  S.mim = S.mre + 8 * kCaStack;
  S.inv_r = reinterpret_cast<float*>(raw + CaLayout::inv);
  S.inv_i = S.inv_r + 64;
  int* ip = reinterpret_cast<int*>(raw + CaLayout::ints);
  S.sel = ip;
  S.cid = ip + 64;
  S.piv_id = ip + 128;
  S.sid = ip + 192;
  S.step_of = S.sid + kCaStack;
  S.dest = S.step_of + kCaStack;
  S.misc = S.dest + kCaStack;
  return S;
}

// The rows a warp holds: slot j = column warp * (nb / 16) + j, k = row lane + 32 k.
template <int RPL>
struct CaX {
  float r[4][RPL];
  float i[4][RPL];
};

template <int RPL>
__device__ __forceinline__ void ca_load(CaX<RPL>& X, const CaSmem& S, unsigned valid, int nb,
                                        int warp, int lane) {
  const int cpw = nb >> 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = warp * cpw + j;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const bool in = j < cpw && ((valid >> k) & 1u);
      X.r[j][k] = in ? S.bre[c * kCaLd + lane + 32 * k] : 0.f;
      X.i[j][k] = in ? S.bim[c * kCaLd + lane + 32 * k] : 0.f;
    }
  }
}

// Column ownership: warp w holds the columns w * cpw + j (slot j < cpw,
// cpw = nb / 16 consecutive columns), lane l the rows l + 32 k. A
// factorisation runs in groups of cpw steps: the steps of group g are the
// columns of warp g, which picks their pivots alone (no barrier between
// them); the other warps apply the group's rank-1 updates to their columns
// in the next group, reading the multipliers from a ring of two groups in
// shared memory. One block barrier per group.
__device__ __forceinline__ float* ca_lre(const CaSmem& S, int t, int cpw) {
  const int g = t / cpw, q = t - g * cpw;
  return S.mre + ((g & 1) * 4 + q) * kCaStack;
}
__device__ __forceinline__ float* ca_lim(const CaSmem& S, int t, int cpw) {
  const int g = t / cpw, q = t - g * cpw;
  return S.mim + ((g & 1) * 4 + q) * kCaStack;
}

// Pivot search of column t (slot J of the calling warp) among the live rows;
// the pivot row, 1 / pivot and the multipliers a / pivot (zero for rows not
// live, the pivot row included) go to shared memory and, for the caller's
// own later columns, to lr / li. Returns the pivot row.
template <int RPL>
__device__ __forceinline__ int ca_pick(const CaX<RPL>& X, int J, unsigned live, int t, int cpw,
                                       const CaSmem& S, int lane, bool report_zero,
                                       float (&lr)[RPL], float (&li)[RPL]) {
  float best = -1.f, br = 0.f, bi = 0.f;
  int brow = INT_MAX;
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const float xr = X.r[J][k], xi = X.i[J][k];
    const float a2 = xr * xr + xi * xi;
    const float v = (a2 == a2) ? a2 : 0.f;  // a NaN entry counts as zero
    if (((live >> k) & 1u) && v > best) {  // so every step picks a live row
      best = v;
      brow = lane + 32 * k;
      br = xr;
      bi = xi;
    }
  }
  // the largest |a|^2 (bit patterns of non-negative floats order like their
  // values), then the smallest row among the lanes holding it
  const unsigned key = (best >= 0.f) ? __float_as_uint(best) : 0u;
  const unsigned row = (best >= 0.f) ? (unsigned)brow : 0xffffffffu;
  const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
  const unsigned rmin = __reduce_min_sync(0xffffffffu, key == kmax ? row : 0xffffffffu);
  const int src = __ffs(__ballot_sync(0xffffffffu, key == kmax && row == rmin)) - 1;
  const float pvr = __shfl_sync(0xffffffffu, br, src);
  const float pvi = __shfl_sync(0xffffffffu, bi, src);
  const bool zero = !(__uint_as_float(kmax) > 0.f);
  float ir = 0.f, ii = 0.f;
  if (!zero) {
    const float rd = __frcp_rn(pvr * pvr + pvi * pvi);
    ir = pvr * rd;
    ii = -pvi * rd;
  }
  const int pr = (int)rmin;
  const unsigned now = live & ~((lane == (pr & 31)) ? (1u << (pr >> 5)) : 0u);
  float* Lr = ca_lre(S, t, cpw);
  float* Li = ca_lim(S, t, cpw);
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const float xr = X.r[J][k], xi = X.i[J][k];
    const bool on = (now >> k) & 1u;
    lr[k] = on ? xr * ir - xi * ii : 0.f;
    li[k] = on ? xr * ii + xi * ir : 0.f;
    Lr[lane + 32 * k] = lr[k];
    Li[lane + 32 * k] = li[k];
  }
  if (lane == 0) {
    S.sel[t] = pr;
    S.inv_r[t] = ir;
    S.inv_i[t] = ii;
    if (report_zero && zero && S.misc[3] > t) S.misc[3] = t;
  }
  return pr;
}

// Entry of the pivot row pr in slot J (all lanes get it).
template <int RPL>
__device__ __forceinline__ void ca_rowval(const CaX<RPL>& X, int J, int pr, float& ur, float& ui) {
  const int kp = pr >> 5;
  float vr = 0.f, vi = 0.f;
#pragma unroll
  for (int k = 0; k < RPL; ++k)
    if (k == kp) {
      vr = X.r[J][k];
      vi = X.i[J][k];
    }
  ur = __shfl_sync(0xffffffffu, vr, pr & 31);
  ui = __shfl_sync(0xffffffffu, vi, pr & 31);
}

// x -= l u on slot J (the multipliers of rows that must not change are 0).
template <int RPL>
__device__ __forceinline__ void ca_axpy(CaX<RPL>& X, int J, const float (&lr)[RPL],
                                        const float (&li)[RPL], float ur, float ui) {
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    X.r[J][k] = fmaf(-lr[k], ur, fmaf(li[k], ui, X.r[J][k]));
    X.i[J][k] = fmaf(-lr[k], ui, fmaf(-li[k], ur, X.i[J][k]));
  }
}

template <int RPL>
__device__ __forceinline__ void ca_load_mult(const CaSmem& S, int t, int cpw, int lane,
                                             float (&lr)[RPL], float (&li)[RPL]) {
  const float* Lr = ca_lre(S, t, cpw);
  const float* Li = ca_lim(S, t, cpw);
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    lr[k] = Lr[lane + 32 * k];
    li[k] = Li[lane + 32 * k];
  }
}

// Partial pivoting on the rows held in X (valid: this lane's rows that
// exist), nsel = min(rows, nb) steps. Leaves the stack row chosen at each
// step in S.sel[] and 1 / pivot in S.inv; with `root`, also the step of
// every chosen row in S.step_of[] and the first zero pivot in S.misc[3].
// Returns this lane's mask of chosen rows. A chosen row takes no update
// after its step, so it keeps U in the columns from its step on and its
// unscaled multipliers before it.
template <int RPL>
__device__ unsigned ca_gepp(CaX<RPL>& X, unsigned valid, int nb, int nsel, const CaSmem& S,
                            int warp, int lane, bool root) {
  const int cpw = nb >> 4;
  const int ngroups = (nsel + cpw - 1) / cpw;
  unsigned chosen = 0;
#pragma unroll 1
  for (int g = 0; g <= ngroups; ++g) {
    // the previous group's pivots, then its updates on the columns of the
    // warps still to pick (their columns all lie to its right)
    if (g > 0) {
      const int p0 = (g - 1) * cpw, p1 = min(nsel, p0 + cpw);
      for (int t = p0; t < p1; ++t) {
        const int pr = S.sel[t];
        if (lane == (pr & 31)) chosen |= 1u << (pr >> 5);
        if (root && warp == 0 && lane == 0) S.step_of[pr] = t;
        if (warp >= g) {
          float lr[RPL], li[RPL];
          ca_load_mult<RPL>(S, t, cpw, lane, lr, li);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (j >= cpw) continue;
            float ur, ui;
            ca_rowval<RPL>(X, j, pr, ur, ui);
            ca_axpy<RPL>(X, j, lr, li, ur, ui);
          }
        }
      }
    }
    if (g < ngroups && warp == g) {
      // the owner: pick its columns in order, each step applied at once to
      // its later columns (registers only)
      const int t0 = g * cpw, t1 = min(nsel, t0 + cpw);
      unsigned mine = chosen;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int t = t0 + j;
        if (j >= cpw || t >= t1) continue;
        float lr[RPL], li[RPL];
        const int pr = ca_pick<RPL>(X, j, valid & ~mine, t, cpw, S, lane, root, lr, li);
        if (lane == (pr & 31)) mine |= 1u << (pr >> 5);
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) {
          if (j2 <= j || j2 >= cpw) continue;
          float ur, ui;
          ca_rowval<RPL>(X, j2, pr, ur, ui);
          ca_axpy<RPL>(X, j2, lr, li, ur, ui);
        }
      }
    }
    __syncthreads();  // group g's pivots and multipliers are in shared memory
  }
  return chosen;
}

// Elimination with the pivots known (phase 3): the live rows in X against
// the root's block (U in S.ure/uim on and above the diagonal, 1 / pivot in
// S.inv), in the groups of ca_gepp. Afterwards x * inv[c] is the L entry of
// column c of every live row.
template <int RPL>
__device__ void ca_elim(CaX<RPL>& X, unsigned live, int nb, const CaSmem& S, int warp, int lane) {
  const int cpw = nb >> 4;
  const int ngroups = nb / cpw;
#pragma unroll 1
  for (int g = 0; g <= ngroups; ++g) {
    if (g > 0 && warp >= g) {
      const int p0 = (g - 1) * cpw;
      for (int t = p0; t < p0 + cpw; ++t) {
        float lr[RPL], li[RPL];
        ca_load_mult<RPL>(S, t, cpw, lane, lr, li);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (j >= cpw) continue;
          const int c = warp * cpw + j;
          ca_axpy<RPL>(X, j, lr, li, S.ure[c * kCaLdU + t], S.uim[c * kCaLdU + t]);
        }
      }
    }
    if (g < ngroups && warp == g) {
      const int t0 = g * cpw;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j >= cpw) continue;
        const int t = t0 + j;
        const float ir = S.inv_r[t], ii = S.inv_i[t];
        float lr[RPL], li[RPL];
        float* Lr = ca_lre(S, t, cpw);
        float* Li = ca_lim(S, t, cpw);
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
          const float xr = X.r[j][k], xi = X.i[j][k];
          const bool on = (live >> k) & 1u;
          lr[k] = on ? xr * ir - xi * ii : 0.f;
          li[k] = on ? xr * ii + xi * ir : 0.f;
          Lr[lane + 32 * k] = lr[k];
          Li[lane + 32 * k] = li[k];
        }
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) {
          if (j2 <= j || j2 >= cpw) continue;
          const int c = t0 + j2;
          ca_axpy<RPL>(X, j2, lr, li, S.ure[c * kCaLdU + t], S.uim[c * kCaLdU + t]);
        }
      }
    }
    __syncthreads();
  }
}

// The root keeps the final factorisation of its chosen rows: row t (its
// step) of the block gets the row's values (U from column t on, unscaled
// multipliers before it).
template <int RPL>
__device__ __forceinline__ void ca_keep(const CaX<RPL>& X, unsigned chosen, int nb,
                                        const CaSmem& S, int warp, int lane) {
  const int cpw = nb >> 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = warp * cpw + j;
    if (j >= cpw) continue;
#pragma unroll
    for (int k = 0; k < RPL; ++k)
      if ((chosen >> k) & 1u) {
        const int t = S.step_of[lane + 32 * k];
        S.ure[c * kCaLdU + t] = X.r[j][k];
        S.uim[c * kCaLdU + t] = X.i[j][k];
      }
  }
}

// Move this CTA's n candidates (stack rows S.sel[q]) to rows 0..n-1 of the
// buffer, in pick order, with their panel rows in S.cid (local rows of the
// CTA's block when `local`, else the stack's ids); n into S.misc[2].
__device__ __forceinline__ void ca_gather(const CaSmem& S, int n, int nb, int tid, bool local,
                                          int r0) {
  float vr[8], vi[8];
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    const int e = tid + kCaThreads * h, q = e & 63, c = e >> 6;
    const bool in = q < n && c < nb;
    const int src = in ? S.sel[q] : 0;
    vr[h] = in ? S.bre[c * kCaLd + src] : 0.f;
    vi[h] = in ? S.bim[c * kCaLd + src] : 0.f;
  }
  int id = -1;
  if (tid < n) id = local ? r0 + S.sel[tid] : S.sid[S.sel[tid]];
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    const int e = tid + kCaThreads * h, q = e & 63, c = e >> 6;
    if (q < n && c < nb) {
      S.bre[c * kCaLd + q] = vr[h];
      S.bim[c * kCaLd + q] = vi[h];
    }
  }
  if (tid < 64) S.cid[tid] = id;
  if (tid == 0) S.misc[2] = n;
  __syncthreads();
}

// RPL: rows per lane of the CTA's own block (ceil(Mb / 32) <= 8); the tree
// stacks use 8.
template <int RPL>
__global__ void __launch_bounds__(kCaThreads, 1) panel_calu_kernel(float* Are, float* Aim, long lda,
                                                                   int k0, int M, int nb, int Mb,
                                                                   int* ipiv, int* zero_col,
                                                                   int* rmap, int restricted) {
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int C = (int)cluster.num_blocks();
  extern __shared__ __align__(16) unsigned char ca_raw[];
  const CaSmem S = ca_smem(ca_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = crank * Mb;  // first panel row of this CTA
  const int rows = max(0, min(Mb, M - r0));
  const float* gre = Are + (size_t)(k0 + r0) + (size_t)k0 * lda;
  const float* gim = Aim + (size_t)(k0 + r0) + (size_t)k0 * lda;

  // ---- 1. the CTA's block: originals into the buffer (one round of
  // asynchronous copies), partial pivoting on it in registers. With
  // `restricted` only CTA 0 pivots, on the panel's first nb rows (the
  // diagonal block), and there is no tournament.
  const int lrows = restricted ? (crank == 0 ? min(rows, nb) : 0) : rows;
  for (int e = tid; e < lrows * nb; e += kCaThreads) {
    const int c = e / lrows, r = e - c * lrows;
    const unsigned dr = (unsigned)__cvta_generic_to_shared(S.bre + c * kCaLd + r);
    const unsigned di = (unsigned)__cvta_generic_to_shared(S.bim + c * kCaLd + r);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dr),
                 "l"(gre + r + (size_t)c * lda));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(di),
                 "l"(gim + r + (size_t)c * lda));
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  if (tid == 0) S.misc[3] = INT_MAX;
  for (int r = tid; r < kCaStack; r += kCaThreads) S.dest[r] = r0 + r;
  __syncthreads();
  unsigned valid = 0, lvalid = 0;
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    if (lane + 32 * k < rows) valid |= 1u << k;
    if (lane + 32 * k < lrows) lvalid |= 1u << k;
  }
  const bool single = (C == 1) || restricted;  // CTA 0's own pick is the panel's
  if (lrows > 0) {
    CaX<RPL> X;
    ca_load<RPL>(X, S, lvalid, nb, warp, lane);
    const unsigned chosen = ca_gepp<RPL>(X, lvalid, nb, min(lrows, nb), S, warp, lane, single);
    if (single) ca_keep<RPL>(X, chosen, nb, S, warp, lane);
  }

  // ---- 2. the tournament: levels of stride s = 1, 4, 16
  int ncand = min(rows, nb);
  bool local = true;  // S.sel indexes the CTA's own block (else the stack)
  for (int s = 1; !restricted && s < C; s *= 4) {
    const bool active = (crank % s) == 0;
    if (active) ca_gather(S, ncand, nb, tid, local, r0);
    cluster.sync();  // every active CTA's candidates are in rows 0..63
    if ((crank % (4 * s)) != 0) continue;  // not a leader at this level
    local = false;
    const bool root = (4 * s >= C);
    // stack: segment i (rows 64 i ..) holds the candidates of CTA
    // crank + i s; segment 0 (own) is in place
    if (tid < 64) S.sid[tid] = S.cid[tid];
    for (int i = 1; i < 4; ++i) {
      const int peer = crank + i * s;
      if (peer >= C) {
        if (tid < 64) S.sid[64 * i + tid] = -1;
        continue;
      }
      const float* pre = cluster.map_shared_rank(S.bre, peer);
      const float* pim = cluster.map_shared_rank(S.bim, peer);
      const int* pcid = cluster.map_shared_rank(S.cid, peer);
      const int* pmisc = cluster.map_shared_rank(S.misc, peer);
      if (tid < 64) {
        const int n = pmisc[2], id = pcid[tid];
        S.sid[64 * i + tid] = (tid < n) ? id : -1;
      }
      // rows 0..63 of every column, 16 float4 per column and plane
      for (int e = tid; e < nb * 32; e += kCaThreads) {
        const int c = e >> 5, h = e & 31, q = (h & 15) * 4;
        const float* src = (h < 16 ? pre : pim) + c * kCaLd + q;
        float* dst = (h < 16 ? S.bre : S.bim) + c * kCaLd + 64 * i + q;
        *reinterpret_cast<float4*>(dst) = *reinterpret_cast<const float4*>(src);
      }
    }
    __syncthreads();
    unsigned v8 = 0;
    int nvalid = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (S.sid[lane + 32 * k] >= 0) v8 |= 1u << k;
    for (int i = 0; i < 4; ++i)
      nvalid += __popc(__ballot_sync(0xffffffffu, S.sid[64 * i + lane] >= 0)) +
                __popc(__ballot_sync(0xffffffffu, S.sid[64 * i + 32 + lane] >= 0));
    CaX<8> Y;
    ca_load<8>(Y, S, v8, nb, warp, lane);
    const unsigned chosen = ca_gepp<8>(Y, v8, nb, min(nvalid, nb), S, warp, lane, root);
    if (root) ca_keep<8>(Y, chosen, nb, S, warp, lane);
    ncand = min(nvalid, nb);
  }

  // ---- the root publishes the pivot sequence
  if (crank == 0) {
    if (tid < nb) S.piv_id[tid] = single ? S.sel[tid] : S.sid[S.sel[tid]];
    if (tid == 0 && S.misc[3] < nb) atomicMin(zero_col, k0 + S.misc[3] + 1);
  }
  cluster.sync();  // the root's block, inverses and pivots are final

  // ---- 3. every CTA: the root's block, then its other rows' L entries
  if (crank != 0) {
    const float* pre = cluster.map_shared_rank(S.ure, 0);
    const float* pim = cluster.map_shared_rank(S.uim, 0);
    for (int e = tid; e < nb * 32; e += kCaThreads) {
      const int c = e >> 5, h = e & 31, q = (h & 15) * 4;
      const float* src = (h < 16 ? pre : pim) + c * kCaLdU + q;
      float* dst = (h < 16 ? S.ure : S.uim) + c * kCaLdU + q;
      *reinterpret_cast<float4*>(dst) = *reinterpret_cast<const float4*>(src);
    }
    if (tid < nb) {
      S.inv_r[tid] = cluster.map_shared_rank(S.inv_r, 0)[tid];
      S.inv_i[tid] = cluster.map_shared_rank(S.inv_i, 0)[tid];
      S.piv_id[tid] = cluster.map_shared_rank(S.piv_id, 0)[tid];
    }
  }
  for (int r = tid; r < kCaStack; r += kCaThreads) S.step_of[r] = nb;
  __syncthreads();
  if (tid < nb) {
    const int p = S.piv_id[tid];
    if (p >= r0 && p < r0 + rows) S.step_of[p - r0] = tid;
  }
  __syncthreads();
  unsigned piv = 0;
#pragma unroll
  for (int k = 0; k < RPL; ++k)
    if (((valid >> k) & 1u) && S.step_of[lane + 32 * k] < nb) piv |= 1u << k;
  const unsigned live = valid & ~piv;
  CaX<RPL> X;  // the originals, again from the panel (untouched until the write-back)
  const int cpw = nb >> 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = warp * cpw + j;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const bool in = j < cpw && ((live >> k) & 1u);
      X.r[j][k] = in ? gre[lane + 32 * k + (size_t)c * lda] : 0.f;
      X.i[j][k] = in ? gim[lane + 32 * k + (size_t)c * lda] : 0.f;
    }
  }
  ca_elim<RPL>(X, live, nb, S, warp, lane);
  if (warp == 0) panel_compose(S.piv_id, nb, k0, r0, rows, crank, ipiv, rmap, S.dest, lane);
  cluster.sync();  // every CTA has read its originals and no peer reads shared memory any more

  // ---- write back: the other rows' L entries at their output positions,
  // the root's block in positions 0..nb-1
  float* ore = Are + (size_t)k0 + (size_t)k0 * lda;
  float* oim = Aim + (size_t)k0 + (size_t)k0 * lda;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = warp * cpw + j;
    if (j >= cpw) continue;
    const float ir = S.inv_r[c], ii = S.inv_i[c];
#pragma unroll
    for (int k = 0; k < RPL; ++k)
      if ((live >> k) & 1u) {
        const float xr = X.r[j][k], xi = X.i[j][k];
        const size_t o = (size_t)S.dest[lane + 32 * k] + (size_t)c * lda;
        ore[o] = xr * ir - xi * ii;
        oim[o] = xr * ii + xi * ir;
      }
  }
  if (crank == 0) {
    for (int e = tid; e < nb * nb; e += kCaThreads) {
      const int t = e % nb, c = e / nb;
      float vr = S.ure[c * kCaLdU + t], vi = S.uim[c * kCaLdU + t];
      if (c < t) {
        const float ir = S.inv_r[c], ii = S.inv_i[c];
        const float wr = vr * ir - vi * ii, wi = vr * ii + vi * ir;
        vr = wr;
        vi = wi;
      }
      ore[t + (size_t)c * lda] = vr;
      oim[t + (size_t)c * lda] = vi;
    }
  }
}

using CaluKernel = void (*)(float*, float*, long, int, int, int, int, int*, int*, int*, int);

static CaluKernel calu_kernel_for(int Mb, int* idx) {
  const int rpl = (Mb + 31) / 32;
  static const CaluKernel ks[] = {panel_calu_kernel<2>, panel_calu_kernel<4>,
                                  panel_calu_kernel<6>, panel_calu_kernel<8>};
  const int i = rpl <= 2 ? 0 : rpl <= 4 ? 1 : rpl <= 6 ? 2 : 3;
  *idx = i;
  return ks[i];
}

static int calu_attrs(CaluKernel k, int idx) {
  static bool done[4] = {false, false, false, false};
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (done[idx]) return HARP_OK;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)CaLayout::bytes) != cudaSuccess ||
      cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return cuda_status(cudaGetLastError());
  done[idx] = true;
  return HARP_OK;
}

static bool calu_resident(int C, int Mb) {
  static std::mutex mu;
  static int known[kCaMaxCluster + 1][4] = {};  // 0 unknown, 1 yes, -1 no
  int idx = 0;
  CaluKernel kern = calu_kernel_for(Mb, &idx);
  std::lock_guard<std::mutex> lock(mu);
  if (known[C][idx]) return known[C][idx] > 0;
  bool ok = false;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)CaLayout::bytes) == cudaSuccess &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kCaThreads);
    cfg.dynamicSmemBytes = CaLayout::bytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    ok = cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1;
  }
  if (!ok) cudaGetLastError();
  known[C][idx] = ok ? 1 : -1;
  return ok;
}

// Estimated cycles of a tournament panel with C CTAs of Mb rows: three
// factorisations on the critical path per level structure (the block, the
// tree levels, the elimination), each bounded by its pivot-search chain
// (~300 cycles a step) or by its FP32 arithmetic, plus the cluster
// barriers.
static double calu_cost(int M, int nb, int C) {
  const int Mb = (M + C - 1) / C;
  int levels = 0;
  for (int s = 1; s < C; s *= 4) ++levels;
  const double work = (double)nb * (nb + 1) / 2 * 4 / 128 / 0.6;  // cycles per row
  const double chain = 300.0 * nb, chain3 = 170.0 * nb;
  return std::max(chain, Mb * work) + levels * std::max(chain, 256 * work) +
         std::max(chain3, Mb * work) + 600.0 * (levels + 2);
}

int panel_calu_plan(const harp_ctx* ctx, int M, int want_nb, int* csize, int* Mb) {
  if (ctx->smem_optin < CaLayout::bytes) return 0;
  for (int nb : {64, 32, 16}) {
    if (nb > want_nb || M < nb) continue;
    int best_c = 0;
    double best = 0.0;
    for (int C : {1, 2, 4, 8, 16}) {
      const int mb = (M + C - 1) / C;
      if (mb > kCaStack) continue;
      if (C > 1 && (C - 1) * mb >= M) continue;  // every CTA owns rows
      if (!calu_resident(C, mb)) continue;
      const double cost = calu_cost(M, nb, C);
      if (!best_c || cost < best) {
        best_c = C;
        best = cost;
      }
    }
    if (best_c) {
      *csize = best_c;
      *Mb = (M + best_c - 1) / best_c;
      return nb;
    }
  }
  return 0;
}

// Cluster size and rows per CTA for a panel pivoted within its diagonal
// block: only the elimination of the rows below is spread over the CTAs,
// so take the smallest cluster that brings a CTA to <= 192 rows (else the
// largest that fits). Returns false when no resident cluster holds the
// panel (at most 16 CTAs of 256 rows).
bool panel_block_plan(const harp_ctx* ctx, int M, int nb, int* csize, int* Mb) {
  if (ctx->smem_optin < CaLayout::bytes || M < nb || nb % 16 != 0 || nb > kCaMaxNb) return false;
  int best = 0;
  for (int C : {1, 2, 4, 8, 16}) {
    const int mb = (M + C - 1) / C;
    if (mb > kCaStack || mb < nb) continue;
    if (C > 1 && (C - 1) * mb >= M) continue;
    if (!calu_resident(C, mb)) continue;
    best = C;
    if (mb <= 192) break;
  }
  if (!best) return false;
  *csize = best;
  *Mb = (M + best - 1) / best;
  return true;
}

int panel_calu(const harp_ctx* ctx, float* re, float* im, long ld, int k0, int M, int nb, int C,
               int Mb, int* ipiv, int* zero_col, cudaStream_t st, int* rmap, int restricted) {
  (void)ctx;
  if (Mb > kCaStack || nb % 16 != 0 || nb > kCaMaxNb || M < nb || C > kCaMaxCluster || C < 1 ||
      (long)C * Mb < M)
    return HARP_E_UNSUPPORTED;
  int idx = 0;
  CaluKernel kern = calu_kernel_for(Mb, &idx);
  HARP_TRY(calu_attrs(kern, idx));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kCaThreads);
  cfg.dynamicSmemBytes = CaLayout::bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ProfScope ps(HARP_K_PANEL, 4.0 * M * nb * (double)(nb - 1), st);
  HARP_CUDA(cudaLaunchKernelEx(&cfg, kern, re, im, ld, k0, M, nb, Mb, ipiv, zero_col, rmap,
                               restricted));
  HARP_LAUNCHED();
  return HARP_OK;
}

}  // namespace harp
