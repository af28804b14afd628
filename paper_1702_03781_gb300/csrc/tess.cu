// tess.cu -- the tessellation approach for very large arrays (Section II-D,
// Fig. 3; Section IV-B): hexagonal subarrays analysed separately.
//
// The plane is tiled by flat-topped hexagons of circumradius R_in with
// centres x = 1.5 R_in i, y = sqrt(3) R_in (j + (i mod 2) / 2); an antenna
// belongs to the inner part of the tile of the nearest centre (smallest
// (i, j) on ties), and the subarray of a tile is every antenna inside the
// concentric hexagon of circumradius R_in + R_ext (its edge included). Each
// subarray is filled and solved on its own (many independent problems of
// uneven size: the batch scheduler), and only the currents for the
// excitation of the tile's inner antennas are kept: column m of the result
// holds the currents of port m on the subarray of m's tile, zero elsewhere.
//
// The membership decisions use plain IEEE FP64 arithmetic with every
// product and sum rounded separately (no fused multiply-add), so that they
// are reproducible bit for bit by any FP64 implementation of the same
// formulas.
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

extern "C" int harp_solve_batch(harp_ctx** ctxs, int n_ctx, harp_problem* probs, int n_probs,
                                int prec, double tol, int max_iter);

namespace harp {

constexpr double kSqrt3 = 1.7320508075688772;

__device__ __forceinline__ void hex_center(int i, int j, double R, double* cx, double* cy) {
  *cx = __dmul_rn(__dmul_rn(1.5, R), (double)i);
  *cy = __dmul_rn(__dmul_rn(kSqrt3, R), __dadd_rn((double)j, __dmul_rn(0.5, (double)(i & 1))));
}

__device__ __forceinline__ bool in_hexagon(double dx, double dy, double R) {
  const double ax = fabs(dx), ay = fabs(dy);
  return ay <= __dmul_rn(__dmul_rn(0.5, kSqrt3), R) &&
         __dadd_rn(__dmul_rn(kSqrt3, ax), ay) <= __dmul_rn(kSqrt3, R);
}

// (i, j) of the nearest lattice centre: the candidates around the point's
// column and row strips, the smallest squared distance, then (i, j).
__global__ void hex_tile_kernel(int Na, const double* __restrict__ pos, double R,
                                int* __restrict__ tij) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= Na) return;
  const double x = pos[2 * a], y = pos[2 * a + 1];
  const int i0 = (int)floor(__ddiv_rn(x, __dmul_rn(1.5, R)));
  double best = 0.0;
  int bi = 0, bj = 0;
  bool have = false;
  for (int i = i0 - 1; i <= i0 + 2; ++i) {
    const int j0 = (int)floor(
        __dsub_rn(__ddiv_rn(y, __dmul_rn(kSqrt3, R)), __dmul_rn(0.5, (double)(i & 1))));
    for (int j = j0 - 1; j <= j0 + 2; ++j) {
      double cx, cy;
      hex_center(i, j, R, &cx, &cy);
      const double dx = __dsub_rn(x, cx), dy = __dsub_rn(y, cy);
      const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      if (!have || d2 < best || (d2 == best && (i < bi || (i == bi && j < bj)))) {
        best = d2;
        bi = i;
        bj = j;
        have = true;
      }
    }
  }
  tij[2 * a] = bi;
  tij[2 * a + 1] = bj;
}

// Per tile (one thread each), in antenna order: the inner members (same
// tile) and the subarray (inside the extended hexagon). count: only the
// sizes into in_cnt / out_cnt; else the indices at in_ptr / out_ptr.
__global__ void tile_lists_kernel(int T, const int* __restrict__ tiles, int Na,
                                  const double* __restrict__ pos, const int* __restrict__ tij,
                                  double R_in, double R_out, int count, int* in_cnt, int* out_cnt,
                                  const int* __restrict__ in_ptr, const int* __restrict__ out_ptr,
                                  int* in_idx, int* out_idx) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int ti = tiles[2 * t], tj = tiles[2 * t + 1];
  double cx, cy;
  hex_center(ti, tj, R_in, &cx, &cy);
  int ni = 0, no = 0;
  for (int a = 0; a < Na; ++a) {
    if (tij[2 * a] == ti && tij[2 * a + 1] == tj) {
      if (!count) in_idx[in_ptr[t] + ni] = a;
      ++ni;
    }
    if (in_hexagon(__dsub_rn(pos[2 * a], cx), __dsub_rn(pos[2 * a + 1], cy), R_out)) {
      if (!count) out_idx[out_ptr[t] + no] = a;
      ++no;
    }
  }
  if (count) {
    in_cnt[t] = ni;
    out_cnt[t] = no;
  }
}

// A subarray's positions and self blocks gathered from the array's.
__global__ void tile_gather_kernel(int Nt, const int* __restrict__ members,
                                   const double* __restrict__ pos, const double2* __restrict__ sb,
                                   long stride, int nm2, double* __restrict__ pos_t,
                                   double2* __restrict__ sb_t) {
  const int la = blockIdx.x;
  if (la >= Nt) return;
  const int a = members[la];
  if (threadIdx.x == 0) {
    pos_t[2 * la] = pos[2 * a];
    pos_t[2 * la + 1] = pos[2 * a + 1];
  }
  if (stride > 0)
    for (int e = threadIdx.x; e < nm2; e += blockDim.x)
      sb_t[(size_t)la * nm2 + e] = sb[(size_t)a * stride + e];
}

// Column m (an inner antenna of the tile, local column lcol[q]) of the
// array's currents from the tile's solution: rows of the subarray's
// antennas, the others were zeroed.
__global__ void tile_scatter_kernel(int Nt, int Nm, const int* __restrict__ members,
                                    const int* __restrict__ inner, const int* __restrict__ lcol,
                                    const double2* __restrict__ Xt, long ldt, double2* X,
                                    long ldx) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (r >= Nt * Nm) return;
  const int la = r / Nm, T = r - la * Nm;
  const int m = inner[q];
  X[(size_t)members[la] * Nm + T + (size_t)m * ldx] = Xt[r + (size_t)lcol[q] * ldt];
}

__global__ void zero_c128_kernel(int M, int N, double2* X, long ldx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) X[i + (size_t)blockIdx.y * ldx] = make_double2(0.0, 0.0);
}

}  // namespace harp

using namespace harp;

extern "C" int harp_tessellate(int Na, const double* pos, double R_in, double R_ext,
                               int max_tiles, int* tiles, int* inner_ptr, int* inner_idx,
                               int* outer_ptr, int* outer_idx, long outer_cap, int* n_tiles,
                               long* outer_total, void* stream) {
  if (Na < 1) return -1;
  if (!pos) return -2;
  if (!(R_in > 0.0) || !std::isfinite(R_in)) return -3;
  if (!(R_ext >= 0.0)) return -4;
  if (max_tiles < 1) return -5;
  if (!tiles) return -6;
  if (!inner_ptr) return -7;
  if (!inner_idx) return -8;
  if (!outer_ptr) return -9;
  if (!outer_idx) return -10;
  if (outer_cap < 0) return -11;
  if (!n_tiles) return -12;
  if (!outer_total) return -13;
  cudaStream_t st = (cudaStream_t)stream;
  const double R_out = R_in + R_ext;
  int* tij = nullptr;
  int* cnt = nullptr;
  HARP_CUDA(cudaMallocAsync(&tij, sizeof(int) * 2 * (size_t)Na, st));
  struct Free {
    int** p;
    cudaStream_t s;
    ~Free() {
      if (*p) cudaFreeAsync(*p, s);
    }
  } f1{&tij, st}, f2{&cnt, st};
  hex_tile_kernel<<<(Na + 255) / 256, 256, 0, st>>>(Na, pos, R_in, tij);
  HARP_LAUNCHED();
  std::vector<int> h(2 * (size_t)Na);
  HARP_CUDA(cudaMemcpyAsync(h.data(), tij, sizeof(int) * 2 * (size_t)Na, cudaMemcpyDeviceToHost, st));
  HARP_CUDA(cudaStreamSynchronize(st));
  std::vector<std::pair<int, int>> u;
  u.reserve(Na);
  for (int a = 0; a < Na; ++a) u.emplace_back(h[2 * a], h[2 * a + 1]);
  std::sort(u.begin(), u.end());
  u.erase(std::unique(u.begin(), u.end()), u.end());
  const int T = (int)u.size();
  *n_tiles = T;
  if (T > max_tiles) return HARP_E_UNSUPPORTED;
  std::vector<int> ht(2 * (size_t)T);
  for (int t = 0; t < T; ++t) {
    ht[2 * t] = u[t].first;
    ht[2 * t + 1] = u[t].second;
  }
  HARP_CUDA(cudaMemcpyAsync(tiles, ht.data(), sizeof(int) * 2 * (size_t)T, cudaMemcpyHostToDevice,
                            st));
  HARP_CUDA(cudaMallocAsync(&cnt, sizeof(int) * 2 * (size_t)T, st));
  tile_lists_kernel<<<(T + 127) / 128, 128, 0, st>>>(T, tiles, Na, pos, tij, R_in, R_out, 1, cnt,
                                                     cnt + T, nullptr, nullptr, nullptr, nullptr);
  HARP_LAUNCHED();
  std::vector<int> hc(2 * (size_t)T);
  HARP_CUDA(cudaMemcpyAsync(hc.data(), cnt, sizeof(int) * 2 * (size_t)T, cudaMemcpyDeviceToHost, st));
  HARP_CUDA(cudaStreamSynchronize(st));
  std::vector<int> ip(T + 1, 0), op(T + 1, 0);
  long tot = 0;
  for (int t = 0; t < T; ++t) {
    ip[t + 1] = ip[t] + hc[t];
    tot += hc[T + t];
    if (tot > 2147483647L) return HARP_E_UNSUPPORTED;
    op[t + 1] = (int)tot;
  }
  *outer_total = tot;
  if (tot > outer_cap) return HARP_E_UNSUPPORTED;
  HARP_CUDA(cudaMemcpyAsync(inner_ptr, ip.data(), sizeof(int) * (T + 1), cudaMemcpyHostToDevice, st));
  HARP_CUDA(cudaMemcpyAsync(outer_ptr, op.data(), sizeof(int) * (T + 1), cudaMemcpyHostToDevice, st));
  tile_lists_kernel<<<(T + 127) / 128, 128, 0, st>>>(T, tiles, Na, pos, tij, R_in, R_out, 0,
                                                     nullptr, nullptr, inner_ptr, outer_ptr,
                                                     inner_idx, outer_idx);
  HARP_LAUNCHED();
  HARP_CUDA(cudaStreamSynchronize(st));
  return HARP_OK;
}

extern "C" int harp_solve_tessellated(harp_ctx** ctxs, int n_ctx, int Na, int Nm, int P, int Q,
                                      const double* pos, double freq_hz, const double* coef,
                                      const double* self_blocks, long self_stride, int n_tiles,
                                      const int* inner_ptr, const int* inner_idx,
                                      const int* outer_ptr, const int* outer_idx, double* X,
                                      int ldx, int prec, double tol, int max_iter) {
  if (!ctxs || n_ctx < 1) return -1;
  if (n_ctx > 64) return -2;
  if (Na < 1) return -3;
  if (Nm < 1) return -4;
  if (P < 0) return -5;
  if (Q < 0) return -6;
  if (!pos) return -7;
  if (!(freq_hz > 0.0)) return -8;
  if (!coef) return -9;
  if (!self_blocks) return -10;
  if (self_stride < 0) return -11;
  if (n_tiles < 1) return -12;
  if (!inner_ptr) return -13;
  if (!inner_idx) return -14;
  if (!outer_ptr) return -15;
  if (!outer_idx) return -16;
  if (!X) return -17;
  if ((long)ldx < (long)Na * Nm) return -18;
  for (int c = 0; c < n_ctx; ++c)
    if (!ctxs[c]) return -1;
  DeviceGuard g(ctxs[0]->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t st = ctxs[0]->stream;
  // the lists on the host
  std::vector<int> ip(n_tiles + 1), op(n_tiles + 1);
  HARP_CUDA(cudaMemcpy(ip.data(), inner_ptr, sizeof(int) * (n_tiles + 1), cudaMemcpyDeviceToHost));
  HARP_CUDA(cudaMemcpy(op.data(), outer_ptr, sizeof(int) * (n_tiles + 1), cudaMemcpyDeviceToHost));
  std::vector<int> hin(ip[n_tiles]), hout(op[n_tiles]);
  HARP_CUDA(cudaMemcpy(hin.data(), inner_idx, sizeof(int) * hin.size(), cudaMemcpyDeviceToHost));
  HARP_CUDA(cudaMemcpy(hout.data(), outer_idx, sizeof(int) * hout.size(), cudaMemcpyDeviceToHost));
  // each inner antenna's column in its subarray's solution (lists sorted)
  std::vector<int> lcol(hin.size());
  size_t pool = 0;
  const size_t nm2 = (size_t)Nm * Nm;
  std::vector<size_t> off(n_tiles);
  for (int t = 0; t < n_tiles; ++t) {
    const int nt = op[t + 1] - op[t];
    if (nt < 1 || ip[t + 1] - ip[t] < 1) return HARP_E_STATE;
    for (int q = ip[t]; q < ip[t + 1]; ++q) {
      const int* b = hout.data() + op[t];
      const int* e = b + nt;
      const int* it = std::lower_bound(b, e, hin[q]);
      if (it == e || *it != hin[q]) return HARP_E_STATE;  // inner not in its subarray
      lcol[q] = (int)(it - b);
    }
    off[t] = pool;
    const size_t Nt = (size_t)nt * Nm;
    pool += (2 * (size_t)nt * sizeof(double) + 255) / 256 * 256;           // positions
    if (self_stride > 0) pool += ((size_t)nt * nm2 * 16 + 255) / 256 * 256;  // self blocks
    pool += (Nt * nt * 16 + 255) / 256 * 256;                               // X_t
  }
  pool += ((size_t)hin.size() * sizeof(int) + 255) / 256 * 256;            // lcol
  char* base = nullptr;
  HARP_CUDA(cudaMalloc(&base, pool));
  struct FreePool {
    char* p;
    ~FreePool() { cudaFree(p); }
  } fp{base};
  int* d_lcol = reinterpret_cast<int*>(base + pool - (hin.size() * sizeof(int) + 255) / 256 * 256);
  HARP_CUDA(cudaMemcpyAsync(d_lcol, lcol.data(), sizeof(int) * lcol.size(), cudaMemcpyHostToDevice,
                            st));
  std::vector<harp_problem> probs(n_tiles);
  for (int t = 0; t < n_tiles; ++t) {
    const int nt = op[t + 1] - op[t];
    char* p = base + off[t];
    double* pos_t = reinterpret_cast<double*>(p);
    p += (2 * (size_t)nt * sizeof(double) + 255) / 256 * 256;
    double2* sb_t = nullptr;
    if (self_stride > 0) {
      sb_t = reinterpret_cast<double2*>(p);
      p += ((size_t)nt * nm2 * 16 + 255) / 256 * 256;
    }
    double* X_t = reinterpret_cast<double*>(p);
    tile_gather_kernel<<<nt, 128, 0, st>>>(nt, outer_idx + op[t], pos,
                                           reinterpret_cast<const double2*>(self_blocks),
                                           self_stride, (int)nm2, pos_t, sb_t);
    HARP_LAUNCHED();
    harp_problem& pr = probs[t];
    pr.Na = nt;
    pr.Nm = Nm;
    pr.P = P;
    pr.Q = Q;
    pr.pos = pos_t;
    pr.freq_hz = freq_hz;
    pr.coef = coef;
    pr.self_blocks = self_stride > 0 ? reinterpret_cast<const double*>(sb_t) : self_blocks;
    pr.self_stride = self_stride > 0 ? (long)nm2 : 0;
    pr.X = X_t;
    pr.ldx = nt * Nm;
  }
  HARP_CUDA(cudaStreamSynchronize(st));
  // the subarrays, largest first, on the contexts' workers
  std::vector<int> order(n_tiles);
  for (int t = 0; t < n_tiles; ++t) order[t] = t;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return probs[a].Na > probs[b].Na; });
  std::vector<harp_problem> sorted(n_tiles);
  for (int t = 0; t < n_tiles; ++t) sorted[t] = probs[order[t]];
  const int s = harp_solve_batch(ctxs, n_ctx, sorted.data(), n_tiles, prec, tol, max_iter);
  if (s != HARP_OK) return s;
  // the kept columns into the array's currents
  const int N = Na * Nm;
  zero_c128_kernel<<<dim3((N + 255) / 256, Na), 256, 0, st>>>(N, Na, reinterpret_cast<double2*>(X),
                                                               ldx);
  HARP_LAUNCHED();
  for (int t = 0; t < n_tiles; ++t) {
    const int nt = op[t + 1] - op[t], ni = ip[t + 1] - ip[t];
    tile_scatter_kernel<<<dim3((nt * Nm + 255) / 256, ni), 256, 0, st>>>(
        nt, Nm, outer_idx + op[t], inner_idx + ip[t], d_lcol + ip[t],
        reinterpret_cast<const double2*>(probs[t].X), probs[t].ldx, reinterpret_cast<double2*>(X),
        ldx);
    HARP_LAUNCHED();
  }
  HARP_CUDA(cudaStreamSynchronize(st));
  return HARP_OK;
}
