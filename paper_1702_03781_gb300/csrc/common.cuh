// common.cuh -- shared definitions of the GB300 HARP/MBF library.
//
// Complex helpers, status plumbing and the context structure. Everything
// here is internal to the shared library; the public surface is
// include/harp_gb300.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/harp_gb300.h"

namespace harp {

// ---------------------------------------------------------------------------
// Complex types: interleaved storage (float2 / double2) at the ABI, split
// real/imaginary planes inside the dense kernels.
template <typename R> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename R> using cplx_t = typename cplx_of<R>::type;

template <typename R> __host__ __device__ __forceinline__ cplx_t<R> mk(R re, R im) {
  cplx_t<R> z;
  z.x = re;
  z.y = im;
  return z;
}
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C z;
  z.x = a.x * b.x - a.y * b.y;
  z.y = a.x * b.y + a.y * b.x;
  return z;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) {
  a.y = -a.y;
  return a;
}
// acc += a * b
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// A complex matrix view with arbitrary element strides: element (i, j) has
// its real part at re[i*rs + j*cs] and its imaginary part at im[i*rs + j*cs].
// Split planes use rs = 1, cs = ld; interleaved storage uses re = base,
// im = base + 1, rs = 2, cs = 2*ld. A transposed view swaps rs and cs.
template <typename R> struct CView {
  R* re;
  R* im;
  long rs, cs;
  __host__ __device__ R& r(long i, long j) const { return re[i * rs + j * cs]; }
  __host__ __device__ R& m(long i, long j) const { return im[i * rs + j * cs]; }
  __host__ __device__ CView sub(long i, long j) const {
    return CView{re + i * rs + j * cs, im + i * rs + j * cs, rs, cs};
  }
  __host__ __device__ CView t() const { return CView{re, im, cs, rs}; }
};
template <typename R> inline CView<R> planes(R* re, R* im, long ld) { return CView<R>{re, im, 1, ld}; }
template <typename R> inline CView<R> interleaved(R* base, long ld) {
  return CView<R>{base, base + 1, 2, 2 * ld};
}

// ---------------------------------------------------------------------------
// Status plumbing.
extern int g_last_cuda_error;
extern std::atomic<unsigned long long> g_kernel_launches;  // host-side count of launches

inline int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HARP_OK;
  g_last_cuda_error = (int)e;
  return HARP_E_CUDA;
}
#define HARP_CUDA(...)                             \
  do {                                             \
    int _s = ::harp::cuda_status((__VA_ARGS__));   \
    if (_s != HARP_OK) return _s;                  \
  } while (0)
#define HARP_LAUNCHED()                            \
  do {                                             \
    ++::harp::g_kernel_launches;                   \
    HARP_CUDA(cudaGetLastError());                 \
  } while (0)
#define HARP_TRY(...)                              \
  do {                                             \
    int _s = (__VA_ARGS__);                        \
    if (_s != HARP_OK) return _s;                  \
  } while (0)

// Device status word bits (ctx->dstatus[0]); dstatus[1] holds the smallest
// 1-based column with an exactly zero pivot (INT32_MAX when none).
enum : int { ST_COINCIDENT = 1, ST_NONFINITE = 2 };

// Switch to the context's device for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace harp

// ---------------------------------------------------------------------------
// The context: device workspace sized at creation.
constexpr int kPmapInts = 1 + 2 * 128;  // count, then up to 128 row pairs

struct harp_ctx {
  int device;
  int max_N, max_nrhs;
  int num_sms;
  size_t smem_optin;  // max dynamic shared memory per block (bytes)

  // FP64 reduced matrix for the refinement residual (c128, ld = max_N).
  double2* z64;
  int ld64;

  // LU factors in split planes (room for doubles), pivots, state.
  void* lu_re;
  void* lu_im;
  int ld_lu;
  int* ipiv;
  int* perm;  // net row permutation of the cached factorisation
  // inverses of the 64 x 64 diagonal blocks of L then U (room for doubles),
  // real and imaginary planes, 2 * ceil(max_N / 64) * 4096 entries each
  void* dinv_re;
  void* dinv_im;
  int lu_N;
  int lu_prec;  // -1 = none
  int lu_valid;
  int lu_pivot;  // HARP_PIVOT_* the cached factorisation was made with

  // Solve buffers (room for doubles), N x nrhs planes, ld = max_N.
  void* w_re;
  void* w_im;
  double* x_re;
  double* x_im;
  double* r_re;
  double* r_im;
  double* v_re;
  double* v_im;
  void* t_re;  // scratch for the row permutation of the triangular solves
  void* t_im;

  // Float-float (hi/lo) splits for the refinement residual: Z64 as four
  // float planes (re hi, im hi, re lo, im lo; max_N x max_N, ld max_N) and
  // the iterate X likewise (max_N x max_nrhs); row-sum scratch.
  float* zff;
  float* xff;
  float* rowsum;
  double* rpart;  // split-K partials: kResidMaxSplit x 2 x max_N x max_nrhs doubles

  // K-major hi/lo operand planes of the tensor-core GEMM (lu_tc.cu).
  float* tc_a;
  size_t tc_a_floats;
  float* tc_b;
  size_t tc_b_floats;

  // Adjoint per-pair partial gradients, Na x Na x 2 doubles (lazily sized).
  double* gpair;
  size_t gpair_bytes;
  // columns of G = Lambda X^T for the digit-product adjoint (allocated on
  // first use)
  void* gbuf;
  size_t gbuf_bytes;

  // Stream and c64 matrix buffer used by the batch scheduler (batch.cu).
  cudaStream_t stream;
  float2* zbuf;

  // Explicit inverses of the FP32 factors (L^-1, U^-1 planes, ld max_N) and
  // scratch for building them; valid for the cached factorisation.
  float* finv;  // 4 planes: Linv re, im, Uinv re, im
  float* finv_tmp;  // 2 planes
  int finv_valid;
  // L^-1 and U^-1 as tensor-core operand planes (K-major hi/lo TF32, split
  // once per factorisation for the forward solves), finv_split_floats each;
  // finv_split_mode: the GEMM mode they were split for, -1 when not valid.
  float* finv_split;
  size_t finv_split_floats;
  int finv_split_mode;

  // Captured graphs of the FP32 triangular solves of the refinement, keyed
  // by (N, nrhs, mode, finv_incremental) for trans 'N' [0] and 'T' [1];
  // replayed on the caller's stream.
  cudaGraphExec_t solve_graph[2];
  int solve_key[2][4];
  // the refinement's two per-correction segments as graphs: the correction
  // (by trans) and the residual update (by digit-group count, or by the
  // float-float accumulator), with their keys; seen: run once uncaptured
  cudaGraphExec_t ref_graph[18];
  int ref_key[18][6];
  int ref_seen[18];

  // Look-ahead LU: side stream for the trailing updates and event pools
  // (panel factored / trailing update done), n_events each.
  cudaStream_t side;
  // the FP32 factorisation's critical chain (highest priority; forked from
  // and joined to the caller's stream), and its fork/join events
  cudaStream_t lu_stream;
  cudaEvent_t ev_lu_fork, ev_lu_join;
  int lu_fork;  // run the chain on lu_stream (0 inside a batch of several contexts)
  // Stream of the FP64-accurate fill of Z64 in the mixed modes, which runs
  // beside the factorisation (it needs only the FP32 matrix); ev_fill_fork
  // orders it after the caller's earlier work, ev_z64 marks Z64 complete.
  cudaStream_t fill_stream;
  cudaEvent_t ev_fill_fork, ev_z64;
  // Copies of the last mixed fill's inputs (positions, coefficients, self
  // blocks) that the background fill reads, fin_bytes long (grown on demand).
  void* fin;
  size_t fin_bytes;
  // Workspace of harp_eep (the currents by MBF, a chunk of the phase matrix
  // and of the array factors), eep_bytes long (grown on demand).
  void* eep_ws;
  size_t eep_bytes;
  // U11^-1 of the latest block-local panel (2 planes of 64 x 64 floats).
  float* blk_uinv;
  // Factorisations whose pivoting restricted to the diagonal blocks did not
  // give factors the refinement could use, redone with partial pivoting.
  long long pivot_fallbacks;
  // Streams on which the FP32 look-ahead LU builds the factor inverses
  // panel by panel beside the factorisation ([0] (L^-1)^T, [1] U^-1);
  // ev_inv marks them complete. finv_incremental: the last FP32
  // factorisation left U^-1 in the U slot of finv with its tensor-core
  // split, and (L^-1)^T = (L^T)^-1 in the L slot (its split still to be
  // made, transposed, by the solve).
  cudaStream_t inv_stream[2];
  cudaEvent_t ev_inv[2];
  int finv_incremental;
  // Whether the FP32 factorisation may build the inverses beside itself (1),
  // or builds them after it (0: the batch scheduler, whose concurrent
  // factorisations leave no idle SMs for them).
  int inv_beside;
  // HARP_OPT_INVERSES: 0 after, 1 beside, 2 beside unless in a batch of
  // several contexts (default)
  int inv_policy;
  // HARP_OPT_FILL_CLUSTERS: GPC-sized clusters of the background FP64 fill
  // (0: about half of those a GPU holds)
  int fill_clusters;
  // HARP_OPT_FILL64: 0 float-float background fill, 1 exact digit products,
  // 2 digit products inside a batch of several contexts (default);
  // fill64_now: what the next fill uses (the batch sets it for its run)
  int fill64;
  int fill64_now;
  // HARP_OPT_ADJOINT_G: the mixed adjoint's G = Lambda X^T by 1 digit
  // products on the tensor cores (default), 0 double-float on the CUDA cores
  int adj_g;
  cudaEvent_t* ev_fac;
  cudaEvent_t* ev_big;
  int n_events;
  // Row maps of the cluster-factored panels (n_events x kPmapInts ints): the
  // net interchange of panel i as (destination, source) row pairs.
  int* pmap;

  // Tensor-core refinement residual (ozaki.cu), allocated when memory
  // allows (oz_a == nullptr: the float-float residual is used): bf16 digit
  // planes of op(Z) (2 * oz_max_slices planes of Np x Kp) and of the FP32
  // right-hand side (2 * oz_max_slices planes of roundup(max_nrhs, 64) x Kp),
  // integer pair results (oz_slot_pairs x 2 x max_N x max_nrhs), FP64 Horner
  // accumulators (2 x max_N x max_nrhs), row / column exponents, row-sum
  // partials; then the state of the last oz_prepare.
  void* oz_a;
  void* oz_y;
  int* oz_slots;
  int oz_slot_pairs;
  int oz_max_slices;
  double* oz_acc;
  int* oz_rexp;
  int* oz_cexp;
  double* oz_part;
  int oz_N, oz_bits, oz_slices, oz_Kp, oz_Np;
  // Ticket of the mixed fill whose Z64 the current slices (trans 'N') were
  // made from, on the fill stream with ||Z64||_inf in oz_znorm; -1 after any
  // other preparation or after harp_ctx_z64 handed Z64 out for writing.
  long long z64_ticket, oz_ticket;
  double* oz_znorm;
  int residual_mode;  // HARP_RESIDUAL_*
  int pivot_mode;     // HARP_PIVOT_* of the FP32 factorisation's panels
  // Tile-shape knobs (HARP_OPT_PANEL_ROWS, HARP_OPT_FILL_CHUNK,
  // HARP_OPT_SPLITK_MAX): target rows per CTA of the cluster panel, the
  // largest source-MBF chunk of the fill (0: the largest that fits), the cap
  // on the K splits of the tensor-core products.
  int panel_rows;
  int fill_chunk;
  int splitk_max;
  // Device time of the last harp_solve_batch that used this context as its
  // first, microseconds (first start to last end over the workers' streams).
  double batch_device_us;

  // Reductions and status.
  double* red;      // device scratch, 16 + 2*max_nrhs doubles
  double* red_host; // pinned host mirror, same size
  int* dstatus;     // device status words [0] bits, [1] zero-pivot column, [2] timeout,
                    // [3] bits of the background Z64 fill (not read)
  int* hstatus;     // pinned host mirror
};
