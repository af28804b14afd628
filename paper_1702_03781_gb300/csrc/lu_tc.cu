// lu_tc.cu -- tensor-core (tcgen05) complex GEMM for the FP32 LU trailing
// updates and the triangular-solve updates of the mixed-precision solve:
//   C = beta*C + alpha * A B,   A: M x K, B: K x N, complex, split planes.
//
// The complex product is four real products accumulated in two TMEM
// accumulators, Dr = Ar Br - Ai Bi and Di = Ar Bi + Ai Br (the minus sign is
// the instruction descriptor's negate-A bit). In the three-term TF32 mode
// each FP32 operand x is split as x = hi + lo with hi = x rounded to TF32 and
// lo = x - hi rounded to TF32 (both to nearest), and a*b ~ ah bh + ah bl +
// al bh (12 MMAs per k8 step), which keeps the product accurate to about
// 3 x 2^-24 relative; the one-term
// mode uses ah bh only (4 MMAs per k8 step).
//
// Operands are first copied into "K-major" hi/lo planes (row r of the MMA
// operand holds its K values contiguously, K padded to a multiple of 32,
// planes [re_hi, im_hi, re_lo, im_lo]); the kernel loads 16-wide K tiles of
// them with TMA (64-byte swizzle, one 3-D tensor map per operand with the
// plane as third coordinate) into a two-stage shared-memory ring of 48 KB
// stages, so that two CTAs share an SM and one's epilogue (the C
// read-modify-write) overlaps the other's loads and MMAs.
// Warp roles: warp 0 lane 0 issues TMA, warp 1 lane 0 issues tcgen05.mma
// (single thread, accumulators in TMEM) and commits each stage back to the
// producer; then all four warps read the accumulators with tcgen05.ld
// (warp w owns TMEM lanes 32w..32w+31 = rows of the tile) and update C.
// Every mbarrier wait is bounded by a clock budget; on expiry the kernel
// records HARP timeout status, drains what it issued and frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "dense.cuh"
#include "prof.cuh"

namespace harp {

constexpr int TC_BM = 128;  // rows of C per CTA (TMEM lanes)
constexpr int TC_BN = 64;   // columns of C per CTA
constexpr int TC_BK = 16;   // K per stage: one 64-byte swizzle atom of fp32
constexpr int TC_KPAD = 32; // K padding of the split planes (a multiple of TC_BK)
constexpr int TC_STAGES = 2;
constexpr int TC_THREADS = 128;
constexpr int TC_A_PLANE = TC_BM * TC_BK * 4;  // 8 KB
constexpr int TC_B_PLANE = TC_BN * TC_BK * 4;  // 4 KB
constexpr long long TC_WAIT_CYCLES = 1LL << 30;  // ~0.5 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the error bit set) when the clock budget runs out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > TC_WAIT_CYCLES) {
      atomicOr(err, 1);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups
// 512 bytes apart (the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_64B).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;           // leading byte offset (unused for this layout)
  d |= (uint64_t)(512 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;           // descriptor version
  d |= (uint64_t)4 << 61;           // 64-byte swizzle
  return d;
}

// Instruction descriptor: kind::tf32, FP32 accumulate, K-major A and B.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N, bool negA) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((negA ? 1u : 0u) << 13) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

#define TC_LD16(taddr, v)                                                                         \
  asm volatile(                                                                                   \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14," \
      "%15}, [%16];"                                                                              \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),      \
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),  \
        "=r"(v[14]), "=r"(v[15])                                                                  \
      : "r"(taddr))

struct TcArgs {
  int M, N, nk;
  float alpha, beta;
  float* cre;
  float* cim;
  long crs, ccs;
  long cstride;  // element offset of product z's C (grid z)
  int* err;
  int ksplit;    // 1: grid z splits K (one product, nk k-tiles each) instead of
                 // batching; 2: grid y runs over chunks of the row tiles' k ranges
  int tri;       // A triangular: 1 upper (row i zero below k = i), 2 lower (zero above)
  // ksplit 2: row tile t owns chunks [slot_base[t], slot_base[t + 1]) of ck
  // k-tiles each over its nonzero k range; chunk s writes its partial tile
  // (128 x N, column-major, ld 128) at cre/cim + s * cstride
  int ck, ntiles;
  int slot_base[129];
};

template <bool THREE, int BN>
__global__ void __launch_bounds__(TC_THREADS, BN == 64 ? 2 : 1)
    tc_cgemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    TcArgs a) {
  constexpr int NP = THREE ? 4 : 2;  // planes per operand
  constexpr int B_PLANE = BN * TC_BK * 4;
  constexpr int STAGE = NP * (TC_A_PLANE + B_PLANE);
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[TC_STAGES], bar_empty[TC_STAGES], bar_done;
  __shared__ uint32_t tmem_slot;

  // A CTA of a call that already timed out does no work (the caller reports
  // HARP_E_TIMEOUT); the flag is uniform across the CTA.
  if (*reinterpret_cast<volatile int*>(a.err)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;  // 1024-byte aligned tiles
  // chunked split: this CTA's row tile (the chunks are few, a linear scan)
  int ty = blockIdx.y, chunk = 0;
  if (a.ksplit == 2) {
    ty = 0;
    while (ty + 1 < a.ntiles && a.slot_base[ty + 1] <= (int)blockIdx.y) ++ty;
    chunk = (int)blockIdx.y - a.slot_base[ty];
  }
  const int i0 = ty * TC_BM, j0 = blockIdx.x * BN;
  // batched: grid z is the product (its planes in the split operands);
  // split K: grid z is the K range, all of one product
  const int pz = a.ksplit ? 0 : blockIdx.z * NP;
  const int kt0 = (a.ksplit == 1) ? blockIdx.z * a.nk : 0;
  // k-tiles [kb, ke) of this CTA's range (relative to kt0): with a
  // triangular A the tiles that are zero for all of its rows are skipped
  int kb = 0, ke = a.nk;
  if (a.tri == 1) kb = max(0, i0 / TC_BK - kt0);
  if (a.tri == 2) ke = min(a.nk, (i0 + TC_BM + TC_BK - 1) / TC_BK - kt0);
  if (a.ksplit == 2) {
    kb += chunk * a.ck;
    ke = min(ke, kb + a.ck);
  }
  const bool empty = (kb >= ke);
  const long zoff = (a.ksplit == 2) ? (long)blockIdx.y : (long)blockIdx.z;
  float* cre = a.cre + zoff * a.cstride;
  float* cim = a.cim + zoff * a.cstride;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(su32(&bar_full[s]), 1);
      mbar_init(su32(&bar_empty[s]), 1);
    }
    mbar_init(su32(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_slot)),
                 "r"(2 * BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t d_re = tmem, d_im = tmem + BN;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      int issued = 0;
      for (int kt = kb; kt < ke; ++kt) {
        const int j = kt - kb;  // ring iteration
        const int s = j % TC_STAGES, use = j / TC_STAGES;
        if (use > 0 && !mbar_wait(su32(&bar_empty[s]), (use - 1) & 1, a.err)) break;
        const uint32_t st = base + s * STAGE;
        const uint32_t fb = su32(&bar_full[s]);
        mbar_expect_tx(fb, STAGE);
        for (int q = 0; q < NP; ++q) {
          tma_load_3d(st + q * TC_A_PLANE, &tmA, fb, (kt0 + kt) * TC_BK, i0, pz + q);
          tma_load_3d(st + NP * TC_A_PLANE + q * B_PLANE, &tmB, fb, (kt0 + kt) * TC_BK, j0,
                      pz + q);
        }
        issued = j + 1;
      }
      // make sure every issued copy has landed before the CTA can exit
      for (int q = (issued > TC_STAGES ? issued - TC_STAGES : 0); q < issued; ++q)
        mbar_wait(su32(&bar_full[q % TC_STAGES]), (q / TC_STAGES) & 1, a.err);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer (single thread)
      constexpr uint32_t ID = tf32_idesc(TC_BM, BN, false);
      constexpr uint32_t IDN = tf32_idesc(TC_BM, BN, true);
      bool first = true;
      for (int kt = kb; kt < ke; ++kt) {
        const int it = kt - kb;  // ring iteration, as the producer counts them
        const int s = it % TC_STAGES, use = it / TC_STAGES;
        if (!mbar_wait(su32(&bar_full[s]), use & 1, a.err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = base + s * STAGE;
        const uint32_t Ab = st, Bb = st + NP * TC_A_PLANE;
#pragma unroll
        for (int j = 0; j < TC_BK / 8; ++j) {
          const uint32_t ko = 32u * j;  // 8 tf32 = 32 bytes along K inside the 64-byte atom
          const uint64_t arh = sw64_desc(Ab + 0 * TC_A_PLANE + ko);
          const uint64_t aih = sw64_desc(Ab + 1 * TC_A_PLANE + ko);
          const uint64_t brh = sw64_desc(Bb + 0 * B_PLANE + ko);
          const uint64_t bih = sw64_desc(Bb + 1 * B_PLANE + ko);
          const uint32_t acc = first ? 0u : 1u;
          mma_tf32(d_re, arh, brh, ID, acc);
          mma_tf32(d_im, arh, bih, ID, acc);
          mma_tf32(d_re, aih, bih, IDN, 1u);
          mma_tf32(d_im, aih, brh, ID, 1u);
          if (THREE) {
            const uint64_t arl = sw64_desc(Ab + 2 * TC_A_PLANE + ko);
            const uint64_t ail = sw64_desc(Ab + 3 * TC_A_PLANE + ko);
            const uint64_t brl = sw64_desc(Bb + 2 * B_PLANE + ko);
            const uint64_t bil = sw64_desc(Bb + 3 * B_PLANE + ko);
            mma_tf32(d_re, arh, brl, ID, 1u);
            mma_tf32(d_re, arl, brh, ID, 1u);
            mma_tf32(d_re, aih, bil, IDN, 1u);
            mma_tf32(d_re, ail, bih, IDN, 1u);
            mma_tf32(d_im, arh, bil, ID, 1u);
            mma_tf32(d_im, arl, bih, ID, 1u);
            mma_tf32(d_im, aih, brl, ID, 1u);
            mma_tf32(d_im, ail, brh, ID, 1u);
          }
          first = false;
        }
        mma_commit(su32(&bar_empty[s]));  // stage s free once these MMAs are done
      }
      mma_commit(su32(&bar_done));  // always: tracks completion of every issued MMA
    }
    __syncwarp();
  }

  // ---- epilogue: TMEM -> registers -> C
  const bool ok = mbar_wait(su32(&bar_done), 0, a.err);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int r = warp * 32 + lane;
  const int gi = i0 + r;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 16) {
    uint32_t vr[16], vi[16];
    TC_LD16(d_re + lane_off + c0, vr);
    TC_LD16(d_im + lane_off + c0, vi);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (ok && gi < a.M) {
      // All loads of the chunk are issued before any store, so the 32 L2
      // round trips overlap instead of serialising behind possible aliasing.
      // (A chunk's partial tile is indexed by the row within the tile.)
      const long o0 = (long)(a.ksplit == 2 ? r : gi) * a.crs + (long)(j0 + c0) * a.ccs;
      const int nj = min(16, a.N - (j0 + c0));
      float cr[16], ci[16];
      if (a.beta != 0.f) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          cr[j] = (j < nj) ? cre[o0 + (long)j * a.ccs] : 0.f;
          ci[j] = (j < nj) ? cim[o0 + (long)j * a.ccs] : 0.f;
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        // no k-tile in range: the accumulator was never written, the product is 0
        float xr = empty ? 0.f : a.alpha * __uint_as_float(vr[j]);
        float xi = empty ? 0.f : a.alpha * __uint_as_float(vi[j]);
        if (a.beta != 0.f) {
          xr = fmaf(a.beta, cr[j], xr);
          xi = fmaf(a.beta, ci[j], xi);
        }
        cr[j] = xr;
        ci[j] = xi;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j < nj) {
          cre[o0 + (long)j * a.ccs] = cr[j];
          cim[o0 + (long)j * a.ccs] = ci[j];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * BN)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Operand preparation: a view V (R x Kc) -> K-major planes out[q][r*Kp + c]
// (zero padded to Kp columns), q = re_hi, im_hi, re_lo, im_lo; hi is V
// rounded to TF32 (10 explicit mantissa bits), lo = V - hi exactly. A 32 x 32
// tile goes through shared memory so both the view reads and the plane
// writes are coalesced whichever of the view's strides is contiguous.
__global__ void split_kmajor_kernel(int R, int Kc, int Kp, CView<float> V, float* out,
                                    size_t plane, int three, long sV) {
  __shared__ float tr[32][33], ti[32][33];  // [k_local][r_local]
  // product z: view moved by z*sV, planes of product z after those of z-1
  V.re += blockIdx.z * sV;
  V.im += blockIdx.z * sV;
  out += (size_t)blockIdx.z * (three ? 4 : 2) * plane;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const bool rows_contig = (V.rs == 1);
  for (int l = ty; l < 32; l += 8) {
    const int rl = rows_contig ? tx : l, kl = rows_contig ? l : tx;
    const int r = r0 + rl, k = k0 + kl;
    const bool in = (r < R) && (k < Kc);
    tr[kl][rl] = in ? V.r(r, k) : 0.f;
    ti[kl][rl] = in ? V.m(r, k) : 0.f;
  }
  __syncthreads();
  for (int l = ty; l < 32; l += 8) {
    const int r = r0 + l, k = k0 + tx;
    if (r >= R || k >= Kp) continue;
    const float xr = tr[tx][l], xi = ti[tx][l];
    const float hr = __uint_as_float((__float_as_uint(xr) + 0x1000u) & 0xffffe000u);
    const float hi = __uint_as_float((__float_as_uint(xi) + 0x1000u) & 0xffffe000u);
    const size_t o = (size_t)r * Kp + k;
    out[o] = hr;
    out[plane + o] = hi;
    if (three) {
      // lo = x - hi (exact), itself rounded to nearest TF32: the MMA would
      // otherwise drop its low mantissa bits by truncation
      const float lr = xr - hr, li = xi - hi;
      out[2 * plane + o] = __uint_as_float((__float_as_uint(lr) + 0x1000u) & 0xffffe000u);
      out[3 * plane + o] = __uint_as_float((__float_as_uint(li) + 0x1000u) & 0xffffe000u);
    }
  }
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// 3-D map over planes [NP][rows][Kp] fp32, box (16, box_rows, 1), 64B swizzle.
static bool make_map_ld(CUtensorMap* m, float* base, int rows, int Kp, long ld, size_t plane,
                        int NP, int box_rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)NP};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)plane * 4};
  cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};  // 64 bytes of K
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static bool make_map(CUtensorMap* m, float* base, int rows, int Kp, int NP, int box_rows) {
  return make_map_ld(m, base, rows, Kp, Kp, (size_t)Kp * rows, NP, box_rows);
}

// Workspace for the split operands and the timeout flag (set per solve).
struct TcWorkspace {
  float* a = nullptr;
  size_t a_floats = 0;
  float* b = nullptr;
  size_t b_floats = 0;
  int* err = nullptr;
};
static thread_local TcWorkspace g_tc;
static thread_local int g_splitk_max = 8;  // the calling solve's cap on K splits

void tc_set_splitk_max(int s) { g_splitk_max = (s >= 1 && s <= 8) ? s : 8; }

void tc_set_workspace(float* a, size_t a_floats, float* b, size_t b_floats, int* err) {
  g_tc.a = a;
  g_tc.a_floats = a_floats;
  g_tc.b = b;
  g_tc.b_floats = b_floats;
  g_tc.err = err;
}

void tc_get_workspace(float** a, size_t* a_floats, float** b, size_t* b_floats, int** err) {
  *a = g_tc.a;
  *a_floats = g_tc.a_floats;
  *b = g_tc.b;
  *b_floats = g_tc.b_floats;
  *err = g_tc.err;
}

// Kernel attributes of one instantiation, set once per process (which also
// keeps the call out of captured graphs): the dynamic shared memory of its
// stages and the largest carveout (two CTAs per SM for the 64-wide tile).
template <bool THREE, int BN>
static int tc_kernel_attrs(void (**kern)(const CUtensorMap, const CUtensorMap, TcArgs),
                           size_t* smem) {
  constexpr int NP = THREE ? 4 : 2;
  *kern = tc_cgemm_kernel<THREE, BN>;
  *smem = (size_t)TC_STAGES * NP * (TC_A_PLANE + BN * TC_BK * 4) + 1024;
  static bool done = false;
  if (!done) {
    HARP_CUDA(cudaFuncSetAttribute(*kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)*smem));
    HARP_CUDA(cudaFuncSetAttribute(*kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    done = true;
  }
  return HARP_OK;
}

int cgemm_tc_f32(int M, int N, int K, float alpha, CView<float> A, CView<float> B, float beta,
                 CView<float> C, int mode, cudaStream_t st, long sA, long sB, long sC,
                 int batch) {
  // Narrow products (the in-panel updates) stay on the CUDA cores.
  if (M < 64 || N < 64 || K < 32 || !g_tc.a || !g_tc.b) return HARP_E_UNSUPPORTED;
  if (batch < 1 || batch > 65535) return HARP_E_UNSUPPORTED;
  const bool three = (mode == GEMM_TC_3XTF32);
  const int NP = three ? 4 : 2;
  const int Kp = (K + TC_KPAD - 1) / TC_KPAD * TC_KPAD;
  const size_t pa = (size_t)M * Kp, pb = (size_t)N * Kp;
  if ((size_t)batch * NP * pa > g_tc.a_floats || (size_t)batch * NP * pb > g_tc.b_floats)
    return HARP_E_UNSUPPORTED;
  {
    ProfScope ps(HARP_K_OTHER, 0.0, st);
    dim3 blk(32, 8);
    split_kmajor_kernel<<<dim3(Kp / 32, (M + 31) / 32, batch), blk, 0, st>>>(M, K, Kp, A, g_tc.a,
                                                                              pa, three, sA);
    HARP_LAUNCHED();
    split_kmajor_kernel<<<dim3(Kp / 32, (N + 31) / 32, batch), blk, 0, st>>>(N, K, Kp, B.t(),
                                                                              g_tc.b, pb, three, sB);
    HARP_LAUNCHED();
  }
  CUtensorMap ma, mb;
  if (!make_map(&ma, g_tc.a, M, Kp, NP * batch, TC_BM) ||
      !make_map(&mb, g_tc.b, N, Kp, NP * batch, TC_BN))
    return HARP_E_UNSUPPORTED;
  TcArgs args;
  args.M = M;
  args.N = N;
  args.nk = Kp / TC_BK;
  args.alpha = alpha;
  args.beta = beta;
  args.cre = C.re;
  args.cim = C.im;
  args.crs = C.rs;
  args.ccs = C.cs;
  args.cstride = sC;
  args.err = g_tc.err;
  args.ksplit = 0;
  args.tri = 0;
  args.ck = 0;
  args.ntiles = 0;
  void (*kern)(const CUtensorMap, const CUtensorMap, TcArgs) = nullptr;
  size_t smem = 0;
  HARP_TRY(three ? tc_kernel_attrs<true, TC_BN>(&kern, &smem)
                 : tc_kernel_attrs<false, TC_BN>(&kern, &smem));
  dim3 grid((N + TC_BN - 1) / TC_BN, (M + TC_BM - 1) / TC_BM, batch);
  ProfScope ps(HARP_K_GEMM, 8.0 * M * (double)N * K * batch, st);
  kern<<<grid, TC_THREADS, smem, st>>>(ma, mb, args);
  HARP_LAUNCHED();
  return HARP_OK;
}

// C = alpha * (sum of the S split-K partials) + beta * C; the partials are
// column-major M x N planes, re at ws + z M N, im at ws + (S + z) M N.
__global__ void splitk_reduce_kernel(int M, int N, int S, const float* __restrict__ ws,
                                     float alpha, float beta, CView<float> C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= M) return;
  const size_t mn = (size_t)M * N, o = i + (size_t)j * M;
  float sr = 0.f, si = 0.f;
  for (int z = 0; z < S; ++z) {
    sr += ws[o + z * mn];
    si += ws[o + (S + z) * mn];
  }
  const size_t c = (size_t)i * C.rs + (size_t)j * C.cs;
  float cr = alpha * sr, ci = alpha * si;
  if (beta != 0.f) {
    cr = fmaf(beta, C.re[c], cr);
    ci = fmaf(beta, C.im[c], ci);
  }
  C.re[c] = cr;
  C.im[c] = ci;
}

// C = alpha * (sum of the chunk partials of each row's tile) + beta * C:
// row i belongs to tile t = i / 128, whose chunks s in [slot_base[t],
// slot_base[t + 1]) hold 128 x N partial tiles (column-major, ld 128) at
// re + s 128 N and im + s 128 N; a tile without chunks contributes 0.
struct TcChunkSum {
  int ntiles;
  int slot_base[129];
};

__global__ void chunk_reduce_kernel(int M, int N, TcChunkSum cs, const float* __restrict__ re,
                                    const float* __restrict__ im, float alpha, float beta,
                                    CView<float> C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= M) return;
  const int t = i / TC_BM, r = i - t * TC_BM;
  float sr = 0.f, si = 0.f;
  for (int s = cs.slot_base[t]; s < cs.slot_base[t + 1]; ++s) {
    const size_t o = (size_t)s * TC_BM * N + r + (size_t)j * TC_BM;
    sr += re[o];
    si += im[o];
  }
  const size_t c = (size_t)i * C.rs + (size_t)j * C.cs;
  float cr = alpha * sr, ci = alpha * si;
  if (beta != 0.f) {
    cr = fmaf(beta, C.re[c], cr);
    ci = fmaf(beta, C.im[c], ci);
  }
  C.re[c] = cr;
  C.im[c] = ci;
}

// K splits for a product of `tiles` output tiles and nk k-tiles: the count
// (at most the solve's cap, 8 by default; at least 16 k-tiles, K = 256,
// each) that minimises the waves of two-CTAs-per-SM work,
// ceil(tiles S / (2 SMs)) / S.
static int splitk_count(int tiles, int nk) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 1;
  }
  int best = 1;
  double best_t = 1.0;
  for (int S = 2; S <= g_splitk_max && nk / S >= 16; ++S) {
    if (nk % S) continue;
    const double t = (double)((tiles * S + 2 * sms - 1) / (2 * sms)) / S;
    if (t < best_t - 1e-9) {
      best_t = t;
      best = S;
    }
  }
  return best;
}

// The TF32 planes of V (R x Kc) written into a sub-block of larger split
// planes: element (r, k) at out[p * plane + r * ldo + k]; nothing outside
// the R x Kc block is touched.
__global__ void split_block_kernel(int R, int Kc, CView<float> V, float* out, long ldo,
                                   size_t plane, int three) {
  __shared__ float tr[32][33], ti[32][33];  // [k_local][r_local]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const bool rows_contig = (V.rs == 1);
  for (int l = ty; l < 32; l += 8) {
    const int rl = rows_contig ? tx : l, kl = rows_contig ? l : tx;
    const int r = r0 + rl, k = k0 + kl;
    const bool in = (r < R) && (k < Kc);
    tr[kl][rl] = in ? V.r(r, k) : 0.f;
    ti[kl][rl] = in ? V.m(r, k) : 0.f;
  }
  __syncthreads();
  for (int l = ty; l < 32; l += 8) {
    const int r = r0 + l, k = k0 + tx;
    if (r >= R || k >= Kc) continue;
    const float xr = tr[tx][l], xi = ti[tx][l];
    const float hr = __uint_as_float((__float_as_uint(xr) + 0x1000u) & 0xffffe000u);
    const float hi = __uint_as_float((__float_as_uint(xi) + 0x1000u) & 0xffffe000u);
    const size_t o = (size_t)r * ldo + k;
    out[o] = hr;
    out[plane + o] = hi;
    if (three) {
      const float lr = xr - hr, li = xi - hi;
      out[2 * plane + o] = __uint_as_float((__float_as_uint(lr) + 0x1000u) & 0xffffe000u);
      out[3 * plane + o] = __uint_as_float((__float_as_uint(li) + 0x1000u) & 0xffffe000u);
    }
  }
}

int tc_split_block(int R, int Kc, CView<float> V, float* out, long ldo, size_t plane, int mode,
                   cudaStream_t st) {
  if (R <= 0 || Kc <= 0) return HARP_OK;
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  split_block_kernel<<<dim3((Kc + 31) / 32, (R + 31) / 32), dim3(32, 8), 0, st>>>(
      R, Kc, V, out, ldo, plane, mode == GEMM_TC_3XTF32 ? 1 : 0);
  HARP_LAUNCHED();
  return HARP_OK;
}

// K-major TF32 planes of an operand V (R x K) into out, as the GEMM's own
// split makes them (NP planes of R x Kp), for an operand used by many products.
int tc_split_operand(int R, int K, CView<float> V, float* out, size_t out_floats, int mode,
                     cudaStream_t st) {
  const bool three = (mode == GEMM_TC_3XTF32);
  const int Kp = (K + TC_KPAD - 1) / TC_KPAD * TC_KPAD;
  const size_t pl = (size_t)R * Kp;
  if ((size_t)(three ? 4 : 2) * pl > out_floats) return HARP_E_UNSUPPORTED;
  ProfScope ps(HARP_K_OTHER, 0.0, st);
  split_kmajor_kernel<<<dim3(Kp / 32, (R + 31) / 32, 1), dim3(32, 8), 0, st>>>(R, K, Kp, V, out, pl,
                                                                              three, 0);
  HARP_LAUNCHED();
  return HARP_OK;
}

// C = beta*C + alpha * A B with A given as planes from tc_split_operand
// (M x K, same mode): only B is split here. A grid that would leave SMs
// idle splits K, the partials going to the (here unused) A workspace and a
// reduction forming C.
int cgemm_tc_f32_asplit(int M, int N, int K, float alpha, const float* a_split, CView<float> B,
                        float beta, CView<float> C, int mode, cudaStream_t st, long a_ld,
                        size_t a_plane, bool split_k, int a_tri) {
  if (M < 64 || N < 64 || K < 32 || !g_tc.b || !a_split) return HARP_E_UNSUPPORTED;
  const bool three = (mode == GEMM_TC_3XTF32);
  const int NP = three ? 4 : 2;
  const int Kp = (K + TC_KPAD - 1) / TC_KPAD * TC_KPAD;
  const size_t pb = (size_t)N * Kp;
  if ((size_t)NP * pb > g_tc.b_floats) return HARP_E_UNSUPPORTED;
  {
    ProfScope ps(HARP_K_OTHER, 0.0, st);
    split_kmajor_kernel<<<dim3(Kp / 32, (N + 31) / 32, 1), dim3(32, 8), 0, st>>>(N, K, Kp, B.t(),
                                                                                g_tc.b, pb, three, 0);
    HARP_LAUNCHED();
  }
  // A's planes: row stride a_ld and plane stride a_plane when it is a block
  // of larger split planes (K extent Kp, a multiple of the k-tile)
  if (a_ld > 0 && (K % TC_KPAD != 0 || a_ld < Kp || a_ld % 4 != 0)) return HARP_E_UNSUPPORTED;
  // The refinement's solve products (a triangular A times many right-hand
  // sides) take 128 x 256 output tiles, one CTA per SM, with each row
  // tile's nonzero k range cut into equal chunks, so that the SMs get equal
  // work whatever the triangle leaves each row tile; the other products
  // 128 x 64 tiles, two CTAs per SM, K split evenly when the grid is small.
  const int gy = (M + TC_BM - 1) / TC_BM;
  const int nk = Kp / TC_BK;
  const bool wide = split_k && a_tri != 0 && N >= 256 && gy <= 128 && g_tc.a;
  const int BN = wide ? 256 : TC_BN;
  CUtensorMap ma, mb;
  if (!make_map_ld(&ma, const_cast<float*>(a_split), M, Kp, a_ld > 0 ? a_ld : Kp,
                   a_ld > 0 ? a_plane : (size_t)M * Kp, NP, TC_BM) ||
      !make_map(&mb, g_tc.b, N, Kp, NP, BN))
    return HARP_E_UNSUPPORTED;
  TcArgs args;
  args.M = M;
  args.N = N;
  args.nk = nk;
  args.alpha = alpha;
  args.beta = beta;
  args.cre = C.re;
  args.cim = C.im;
  args.crs = C.rs;
  args.ccs = C.cs;
  args.cstride = 0;
  args.err = g_tc.err;
  args.ksplit = 0;
  args.tri = a_tri;
  args.ck = 0;
  args.ntiles = 0;
  const int gx = (N + BN - 1) / BN;
  int S = 1, nslots = 0;
  if (wide) {
    // chunk length: the triangle's k-tiles over about one CTA per SM, at
    // least 16 k-tiles (K = 256) per chunk
    static int sms = 0;
    if (!sms) {
      int dev = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          sms < 1)
        sms = 1;
    }
    long total = 0;
    for (int t = 0; t < gy; ++t) {
      const int i0 = t * TC_BM;
      const int kb = (a_tri == 1) ? std::min(nk, i0 / TC_BK) : 0;
      const int ke = (a_tri == 2) ? std::min(nk, (i0 + TC_BM + TC_BK - 1) / TC_BK) : nk;
      total += std::max(0, ke - kb);
    }
    const int ck = std::max<int>(16, (int)((total * gx + sms - 1) / sms));
    for (int t = 0; t < gy; ++t) {
      const int i0 = t * TC_BM;
      const int kb = (a_tri == 1) ? std::min(nk, i0 / TC_BK) : 0;
      const int ke = (a_tri == 2) ? std::min(nk, (i0 + TC_BM + TC_BK - 1) / TC_BK) : nk;
      args.slot_base[t] = nslots;
      nslots += (std::max(0, ke - kb) + ck - 1) / ck;
    }
    args.slot_base[gy] = nslots;
    if (nslots < 1 || (size_t)2 * nslots * TC_BM * N > g_tc.a_floats) return HARP_E_UNSUPPORTED;
    args.ksplit = 2;
    args.ck = ck;
    args.ntiles = gy;
    args.alpha = 1.f;
    args.beta = 0.f;
    args.cre = g_tc.a;
    args.cim = g_tc.a + (size_t)nslots * TC_BM * N;
    args.crs = 1;
    args.ccs = TC_BM;
    args.cstride = (long)TC_BM * N;
  } else {
    S = split_k ? splitk_count(gx * gy, nk) : 1;
    if ((size_t)2 * S * M * N > g_tc.a_floats || !g_tc.a) S = 1;
    if (S > 1) {
      args.nk = nk / S;
      args.ksplit = 1;
      args.alpha = 1.f;
      args.beta = 0.f;
      args.cre = g_tc.a;
      args.cim = g_tc.a + (size_t)S * M * N;
      args.crs = 1;
      args.ccs = M;
      args.cstride = (long)M * N;
    }
  }
  void (*kern)(const CUtensorMap, const CUtensorMap, TcArgs) = nullptr;
  size_t smem = 0;
  if (wide)
    HARP_TRY(three ? tc_kernel_attrs<true, 256>(&kern, &smem)
                   : tc_kernel_attrs<false, 256>(&kern, &smem));
  else
    HARP_TRY(three ? tc_kernel_attrs<true, TC_BN>(&kern, &smem)
                   : tc_kernel_attrs<false, TC_BN>(&kern, &smem));
  const dim3 grid(gx, wide ? nslots : gy, S);
  // a triangular A: the algorithmic work is half the full product's
  ProfScope ps(HARP_K_GEMM, (a_tri ? 4.0 : 8.0) * M * (double)N * K, st);
  kern<<<grid, TC_THREADS, smem, st>>>(ma, mb, args);
  HARP_LAUNCHED();
  if (wide) {
    TcChunkSum cs;
    cs.ntiles = gy;
    for (int t = 0; t <= gy; ++t) cs.slot_base[t] = args.slot_base[t];
    chunk_reduce_kernel<<<dim3((M + 255) / 256, N), 256, 0, st>>>(M, N, cs, g_tc.a,
                                                                  g_tc.a + (size_t)nslots * TC_BM * N,
                                                                  alpha, beta, C);
    HARP_LAUNCHED();
  } else if (S > 1) {
    splitk_reduce_kernel<<<dim3((M + 255) / 256, N), 256, 0, st>>>(M, N, S, g_tc.a, alpha, beta, C);
    HARP_LAUNCHED();
  }
  return HARP_OK;
}

// One thread waits, with the tensor-core kernels' bounded wait, on a fresh
// mbarrier of arrival count 1. With release != 0 the thread arrives first and
// the wait ends at once; with release == 0 nothing arrives, the wait runs out
// its clock budget and sets *err.
__global__ void wait_check_kernel(int release, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = su32(&bar);
  mbar_init(b, 1);
  if (release) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
  mbar_wait(b, 0, err);
}

}  // namespace harp

extern "C" int harp_wait_check(harp_ctx* ctx, int release, void* stream) {
  using namespace harp;
  if (!ctx) return -1;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t st = (cudaStream_t)stream;
  HARP_CUDA(cudaMemsetAsync(ctx->dstatus + 2, 0, sizeof(int), st));
  wait_check_kernel<<<1, 32, 0, st>>>(release, ctx->dstatus + 2);
  HARP_LAUNCHED();
  HARP_CUDA(cudaMemcpyAsync(ctx->hstatus + 2, ctx->dstatus + 2, sizeof(int),
                            cudaMemcpyDeviceToHost, st));
  HARP_CUDA(cudaStreamSynchronize(st));
  const int timed_out = ctx->hstatus[2];
  HARP_CUDA(cudaMemsetAsync(ctx->dstatus + 2, 0, sizeof(int), st));
  return timed_out ? HARP_E_TIMEOUT : HARP_OK;
}
