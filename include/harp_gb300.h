/*
 * harp_gb300.h -- C ABI of the GB300 (sm_103a) HARP fill and MBF solve.
 *
 * The library computes the data-parallel hot path of the Macro Basis
 * Function (MBF) analysis of a large irregular array (Bui-Van et al.,
 * "Fast and Accurate Simulation Technique for Large Irregular Arrays",
 * Section II):
 *
 *   1. harp_fill: the reduced MBF impedance matrix Z, one Nm x Nm block per
 *      ordered antenna pair, from the harmonic-polynomial (HARP) model
 *        Z_TS = e^{-jkr} sum_{p=-P..P} e^{j p alpha} sum_{q=0..Q} c_pq^{TS} d^q,
 *      d = 1/r (Eq. 3 with the improved change of variables of Section
 *      II-B, inserted in Eq. 4). The far-field term of Eq. 1 with d = 1/r is
 *      a q = 1 term and is passed folded into c_p1 by the caller.
 *      Diagonal blocks are the caller's self blocks, copied.
 *   2. mbf_solve: Z X = V for every port excitation (the O((Na Nm)^3) direct
 *      solve of Section II-B), LU with partial pivoting.
 *   3. harp_fill_adjoint: the gradient of a real objective with respect to
 *      the antenna positions (array synthesis, Section V), from the adjoint
 *      Lambda and the forward solution X, with the fill recomputed.
 *
 * Conventions shared by every entry point:
 *  - Pointers are DEVICE pointers owned by the caller unless stated. The
 *    library never frees caller memory.
 *  - Complex numbers are interleaved (re, im). "c128" = two doubles, "c64" =
 *    two floats.
 *  - Matrices are column-major with a leading dimension in elements.
 *  - Row i = m*Nm + T carries testing MBF T of antenna m; column
 *    j = n*Nm + S carries source MBF S of antenna n. alpha is the direction
 *    from source antenna n to testing antenna m, anticlockwise from +x.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream). Calls that must read a device result (the zero-pivot check of
 *    a factorisation, the stopping test of the mixed-precision refinement)
 *    synchronise that stream before returning; harp_fill does not.
 *  - Statuses found on the device by a call that does not synchronise
 *    (coincident antennas or non-finite entries in harp_fill, non-finite
 *    right-hand sides of an FP64 solve) stay pending in the context and
 *    are returned by the next call that synchronises (mbf_solve) or by
 *    harp_ctx_sync, which then clears them.
 *  - Return value: HARP_OK (0) on success; -i when argument i (1-based) is
 *    invalid (LAPACK convention); +i (1 <= i <= N) when the LU met an
 *    exactly zero pivot in column i (X is not written); or one of the
 *    HARP_E_* codes below. No C++ exception crosses this boundary.
 */
#ifndef HARP_GB300_H
#define HARP_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct harp_ctx harp_ctx;

/* Arithmetic of a call.
 * HARP_FP64:          everything in FP64 (the plain double-precision path).
 * HARP_MIXED_3XTF32:  FP32 storage, LU trailing updates and triangular
 *                     solves on the tensor cores with a three-term TF32
 *                     split (FP32-level accuracy), FP64-accurate residual
 *                     and iterative refinement.
 * HARP_MIXED_TF32:    as above with single-term TF32 products (faster,
 *                     10-bit mantissa; refinement may not converge when
 *                     cond(Z) * 2^-11 is not small).
 * HARP_FP32:          FP32 fill (c64 only) and FP32-accurate solve
 *                     (three-term TF32 tensor-core LU), no refinement. */
typedef enum {
  HARP_FP64 = 0,
  HARP_MIXED_3XTF32 = 1,
  HARP_MIXED_TF32 = 2,
  HARP_FP32 = 3
} harp_prec;

#define HARP_OK 0
#define HARP_E_COINCIDENT 0x40000001 /* two antennas at the same position (r == 0)          */
#define HARP_E_NOCONV 0x40000002     /* refinement missed tol within max_iter               */
#define HARP_E_TIMEOUT 0x40000003    /* a bounded device wait gave up                       */
#define HARP_E_CUDA 0x40000004       /* a CUDA runtime error (see harp_last_cuda_error)     */
#define HARP_E_NOMEM 0x40000005      /* device allocation failed in harp_ctx_create         */
#define HARP_E_UNSUPPORTED 0x40000006 /* sizes beyond what this build supports              */
#define HARP_E_STATE 0x40000007      /* call order violated (e.g. 'T' solve before 'N')     */
#define HARP_E_NONFINITE 0x40000008  /* NaN or Inf met in the inputs or the factorisation   */

/* Human-readable text for a status code (static storage). */
const char* harp_status_string(int status);

/* Last CUDA error code seen by the library in this process (0 if none). */
int harp_last_cuda_error(void);

/* Number of CUDA kernels this library has launched in this process (an
 * atomic host counter, for instrumentation; launches from every thread and
 * context are counted). */
unsigned long long harp_kernel_launches(void);

/* Create a context on CUDA device `device` with workspace for systems up to
 * max_N unknowns and max_nrhs right-hand sides. The context owns its device
 * workspace, about 144 max_N^2 + 224 max_N max_nrhs bytes: the FP64 copy of
 * the reduced matrix used by the refinement, the LU factors, pivots and
 * factor inverses of the last factorisation, tensor-core operand planes,
 * solve buffers, and a stream and c64 matrix buffer for harp_solve_batch.
 * The exact-slice residual's buffers come on top when they fit (0.57 GB at
 * max_N = 3072, max_nrhs = 256, 2.1 GB in all at that size); the mixed
 * harp_fill_adjoint grows one more buffer on first use (G's columns and the
 * coefficient contraction's operands, ~0.21 GB at the station). Returns
 * HARP_E_NOMEM when the allocation fails. One
 * context serves one stream at a time. A process may hold several contexts,
 * all on one device: the library's one-time setup (kernel shared-memory
 * attributes, the SM count behind its split-K choice) is made for the first
 * device it runs on. Use one process per GPU. */
int harp_ctx_create(harp_ctx** ctx, int device, int max_N, int max_nrhs);

/* Release the context and its workspace (synchronises the device). */
int harp_ctx_destroy(harp_ctx* ctx);

/* Wait until the work enqueued on `stream` (and the context's background
 * Z64 fill) is done, then return the context's pending device status and
 * clear it: HARP_E_TIMEOUT (a bounded device wait gave up), else
 * HARP_E_COINCIDENT or HARP_E_NONFINITE left by harp_fill or by an FP64
 * solve's right-hand-side check, else HARP_OK. This is how the statuses of
 * calls that do not synchronise are collected (Section II's fill has no
 * such check; the status words are this library's). Errors: -1 null ctx,
 * HARP_E_CUDA. */
int harp_ctx_sync(harp_ctx* ctx, void* stream);

/* Device pointer and leading dimension of the context's FP64 reduced
 * matrix (c128, max_N x max_N). harp_fill writes it in the mixed modes (this
 * call first waits, on the host, until that write is complete); a caller may
 * also write its own FP64 matrix there before a mixed solve. */
int harp_ctx_z64(harp_ctx* ctx, void** z64, int* ld);

/* Fill the reduced MBF matrix (Eq. 3 and 4 for every ordered pair m != n,
 * self blocks on the diagonal). The inputs are read in the order of
 * `stream`: in the mixed modes the call copies pos, coef and the self blocks
 * into the context (the first mixed fill of a larger model may allocate
 * room for them), so the background fill never reads the caller's buffers
 * after work queued later on `stream`.
 *   ctx          context (workspace for the mixed modes)          [1]
 *   Na, Nm       antennas, MBFs per antenna; N = Na*Nm <= max_N   [2, 3]
 *   P, Q         harmonic order and polynomial degree (>= 0)      [4, 5]
 *   pos          double [Na][2], metres                           [6]
 *   freq_hz      frequency (> 0); k = 2 pi f / c0                 [7]
 *   coef         c128 [Nm][Nm][2P+1][Q+1], index (T, S, p+P, q)   [8]
 *   self_blocks  c128, element (T, S) of antenna a at
 *                self_blocks[a*self_stride + T + S*Nm]            [9]
 *   self_stride  complex elements between antennas; 0 = one block
 *                shared by all antennas                           [10]
 *   Z            output, N x N column-major: c128 for HARP_FP64, c64 for
 *                HARP_FP32 and the mixed modes (FP32 evaluation)   [11]
 *   ldz          leading dimension of Z (>= N)                    [12]
 *   prec         harp_prec                                        [13]
 * In the mixed modes the call also starts the FP64-accurate evaluation of the
 * context's matrix Z64 on the context's own fill stream, after the work
 * already queued on `stream`; it runs beside whatever follows (the
 * factorisation needs only Z). mbf_solve waits for it before its first use
 * of Z64, and harp_ctx_z64 waits for it on the host.
 * Coincident antennas (r == 0) are detected on the device: the entries of
 * that pair are written as zero and HARP_E_COINCIDENT becomes the context's
 * pending status. An entry that comes out NaN or infinite (non-finite
 * positions, coefficients or self blocks) makes HARP_E_NONFINITE pending.
 * The call does not synchronise: the next mbf_solve on this context (or
 * harp_ctx_sync) returns the pending status, coincidence first. */
int harp_fill(harp_ctx* ctx, int Na, int Nm, int P, int Q, const double* pos, double freq_hz,
              const double* coef, const double* self_blocks, long self_stride, void* Z, int ldz,
              int prec, void* stream);

/* Solve Z X = V (trans 'N') or Z^T X = V (trans 'T', plain transpose).
 *   N            system size (<= max_N)                          [2]
 *   Z, ldz       the matrix for trans 'N': c128 (HARP_FP64) or c64 (mixed)
 *                N x N; it is copied, factorised (PZ = LU) and the factors
 *                are kept in the context. For trans 'T' Z is ignored (may
 *                be NULL) and the cached factors of the last 'N' call of
 *                the same N and prec are reused.                  [3, 4]
 *   V, ldv       c128 N x nrhs right-hand sides; NULL = the port
 *                excitations E (unit entry at row m*Nm of column m, with
 *                Nm = N / nrhs)                                    [5, 6]
 *   nrhs         right-hand sides (<= max_nrhs)                   [7]
 *   X, ldx       c128 N x nrhs output                             [8, 9]
 *   trans        'N' or 'T'                                       [10]
 *   prec         harp_prec                                        [11]
 *   tol          mixed modes: stop when every column j has
 *                max_i |R_ij| <= tol ||Z64||_inf max_i |X_ij|, with
 *                R = V - Z64 X and |z| = |re| + |im| (the test of
 *                LAPACK's zcgesv); <= 0 selects sqrt(N) * 2^-53     [12]
 *   max_iter     mixed modes: at most this many refinement steps  [13]
 *   iters_out    host int, refinement steps taken (may be NULL)   [14]
 *   resid_out    host double, the largest per-column ratio of that test
 *                at exit (may be NULL; -1 for HARP_FP64, HARP_FP32) [15]
 * The mixed modes refine against the context's FP64 matrix (written by the
 * last mixed harp_fill, or by the caller through harp_ctx_z64) and
 * synchronise the stream once per step. For trans 'N' the call reads the
 * pending status after the factorisation: HARP_E_COINCIDENT or
 * HARP_E_NONFINITE left by the fill, or HARP_E_NONFINITE when Z or V holds a
 * NaN or an infinity (checked as they are copied in); X is then not
 * written. The FP32 factorisation runs on streams of the context: its panel
 * chain on the highest-priority one, its trailing updates on a middle
 * priority, the factor inverses built panel by panel beside it (and the
 * background FP64 fill) on the lowest, so that the critical chain gets the
 * SMs first; all of it is ordered after the caller's earlier work on
 * `stream` and before anything the call later enqueues there. Returns +i on an exactly zero pivot
 * in column i, HARP_E_NOCONV when tol was not met within max_iter steps: X
 * then holds the iterate with the smallest backward error seen and
 * resid_out that error. */
int mbf_solve(harp_ctx* ctx, int N, const void* Z, int ldz, const double* V, int ldv, int nrhs,
              double* X, int ldx, char trans, int prec, double tol, int max_iter, int* iters_out,
              double* resid_out, void* stream);

/* ---- Refinement residual ---------------------------------------------------
 * A building block of the mixed solve, exported so that it can be checked on
 * its own (the paper has no counterpart: it solves in one precision).
 *
 * How the mixed modes form R = V - Z64 X (option HARP_OPT_RESIDUAL):
 *   HARP_RESIDUAL_SLICES  tensor cores: Z64 and the FP32 right-hand side are
 *                         cut into exact bf16 integer digits after a
 *                         power-of-two scaling per row (column); every
 *                         digit product is exact in the FP32 accumulator and
 *                         the products are combined in FP64 (the default
 *                         where the context could allocate its buffers)
 *   HARP_RESIDUAL_FF      FP32 pipe: float-float products with a three-float
 *                         accumulator (FP64-accurate)
 * harp_ctx_set_option returns HARP_E_UNSUPPORTED for SLICES when the context
 * has no buffers for it; harp_ctx_get_option reports the method in use.
 * Errors of both: -1 null ctx, -2 unknown option, -3 unknown value (set) or
 * null value pointer (get). */
#define HARP_OPT_RESIDUAL 1
#define HARP_RESIDUAL_SLICES 0
#define HARP_RESIDUAL_FF 1
/* How the FP32 factorisation of the mixed modes (and of HARP_FP32) picks
 * its pivots within each 64-column panel (option HARP_OPT_PIVOT):
 *   HARP_PIVOT_PARTIAL     partial pivoting (the largest |z| of the column,
 *                          as LAPACK's getrf), one cluster barrier per column
 *   HARP_PIVOT_TOURNAMENT  tournament pivoting (communication-avoiding LU):
 *                          each CTA of the panel's cluster pivots its own
 *                          row block, the candidates meet in a tree of
 *                          fan-in 4, and the root's pick pivots the panel;
 *                          a few cluster barriers per panel
 *   HARP_PIVOT_BLOCK       pivoting restricted to each panel's 64 x 64
 *                          diagonal block (one CTA), the rows below solved
 *                          against its U (no pivot search across the panel).
 *                          Its factors are only used where the refinement
 *                          checks them: HARP_FP32 uses partial pivoting
 *                          instead, and a factorisation that meets a zero
 *                          pivot, or whose refinement stops contracting (a
 *                          correction that does not halve the backward
 *                          error), is redone with partial pivoting and
 *                          counted in HARP_OPT_PIVOT_FALLBACKS
 * All factor the same matrix (rows in another order); the refinement then
 * converges to the same FP64-accurate solution. The FP64 mode always uses
 * partial pivoting. HARP_OPT_PIVOT_FALLBACKS (get only) reads the number of
 * such redone factorisations of the context. */
#define HARP_OPT_PIVOT 2
#define HARP_PIVOT_PARTIAL 0
#define HARP_PIVOT_TOURNAMENT 1
#define HARP_PIVOT_BLOCK 2
#define HARP_OPT_PIVOT_FALLBACKS 3
/* Tile-shape knobs (the autotuner's search space; results are the same up
 * to rounding whatever their values):
 *   HARP_OPT_PANEL_ROWS   target rows per CTA of the partial-pivoting
 *                         cluster panel (32..384, default 192): the planner
 *                         takes the smallest cluster that reaches it
 *   HARP_OPT_FILL_CHUNK   the largest number of source MBFs a fill CTA
 *                         stages at once (0: the largest that fits shared
 *                         memory, the default)
 *   HARP_OPT_SPLITK_MAX   the cap (1..8, default 8) on the K splits of the
 *                         tensor-core products of mbf_solve
 * HARP_OPT_BATCH_DEVICE_US (get only): device time of the last
 * harp_solve_batch whose first context this is, in microseconds, from the
 * first worker's start to the last worker's end (CUDA events on the
 * workers' streams).
 * HARP_OPT_INVERSES: where the FP32 factorisation builds the explicit
 * inverses of its triangular factors (used by every solve of the
 * refinement): 0 after the factorisation, 1 beside it (block column by
 * block column on two more streams, as each panel is done), 2 beside it
 * except in a harp_solve_batch of several contexts (default).
 * HARP_OPT_FILL_CLUSTERS: how many GPC-sized (16-CTA) clusters the
 * background FP64 fill of the mixed modes runs on beside the factorisation
 * (0..64; 0, the default: about half of those the GPU holds; more than it
 * holds means all of them).
 * HARP_OPT_FILL64: how the background fill of the mixed modes forms the
 * FP64-accurate Z (Eq. 3 in Eq. 4): 0 float-float products on the CUDA
 * cores (the GPC-sized clusters above), 1 exact digit products on the bf16
 * tensor cores, combined in integers (needs the tensor-core residual's
 * buffers, K <= 128 and P, Q < 32; otherwise it falls back to 0), 2 (the
 * default) digit products inside a harp_solve_batch of several contexts,
 * float-float otherwise. The digit products take a quarter of the time on
 * the whole GPU; the float-float kernel, confined to half of the GPCs,
 * overlaps a single factorisation better.
 * HARP_OPT_ADJOINT_G: how harp_fill_adjoint forms G = Lambda X^T in the
 * mixed modes: 1 (the default) exact digit products on the bf16 tensor
 * cores, rounded once to FP64, in chunks of source antennas (needs the
 * tensor-core residual's buffers, whose Z64 slices it replaces: the next
 * solve slices Z64 again; it first waits for the context's pending
 * background fill); 0 double-float products on the CUDA cores.
 * HARP_OPT_TC_FALLBACKS (get only, process-wide): FP32 products in a
 * tensor-core mode whose shapes the tensor cores take (M, N >= 64,
 * K >= 32) but which ran on the CUDA cores because the tensor-core path
 * refused them (workspace too small, a tensor map the driver would not
 * encode). A health counter: it stays 0 in a well-sized context. */
#define HARP_OPT_PANEL_ROWS 4
#define HARP_OPT_FILL_CHUNK 5
#define HARP_OPT_SPLITK_MAX 6
#define HARP_OPT_BATCH_DEVICE_US 7
#define HARP_OPT_TC_FALLBACKS 8
#define HARP_OPT_INVERSES 9
#define HARP_OPT_FILL_CLUSTERS 10
#define HARP_OPT_FILL64 11
#define HARP_OPT_ADJOINT_G 12
int harp_ctx_set_option(harp_ctx* ctx, int option, int value);
int harp_ctx_get_option(harp_ctx* ctx, int option, int* value);

/* R = V - op(Z) X with the context's residual method.
 *   Z, ldz       c128 N x N (device, column-major), N <= max_N   [2, 3, 4]
 *   X, ldx       c64 N x nrhs: the FP32 right-hand side           [5, 6]
 *   V, ldv       c128 N x nrhs                                    [7, 8]
 *   nrhs         <= max_nrhs                                      [9]
 *   R, ldr       c128 N x nrhs output (may not alias Z, X, V)     [10, 11]
 *   trans        'N' (op(Z) = Z) or 'T' (op(Z) = Z^T)             [12]
 * Device pointers; work runs on `stream` and uses the context's solve
 * buffers (not concurrently with a solve on the same context). */
int harp_residual(harp_ctx* ctx, int N, const double* Z, int ldz, const float* X, int ldx,
                  const double* V, int ldv, int nrhs, double* R, int ldr, char trans,
                  void* stream);

/* Check of the bounded device wait that every mbarrier wait of the
 * tensor-core kernels uses (a budget of 2^30 SM clock cycles, about 0.5 s at
 * 2 GHz). One thread waits on a fresh mbarrier of arrival count 1:
 *   release != 0  the thread arrives first; the wait ends at once -> HARP_OK
 *   release == 0  nothing arrives; the wait runs out its budget, sets the
 *                 context's timeout word and the call returns HARP_E_TIMEOUT
 * The status is read back exactly as mbf_solve reads it, and the word is
 * cleared afterwards, so the context stays usable. Synchronises `stream`;
 * not concurrently with a solve on the same context (they share the word).
 * Errors: -1 null ctx; HARP_E_CUDA. */
int harp_wait_check(harp_ctx* ctx, int release, void* stream);

/* Position gradient of a real objective J(X) of the solution of Z X = V:
 *   grad[m] = -2 Re sum over pairs (m, n) and (n, m) of
 *             sum_TS G_TS dZ_TS/dx_m,       G = Lambda X^T,
 * where Lambda solves Z^T Lambda = (dJ/dX)^* (for the port objective
 * J = sum |E^T X|^2, Lambda = Z^{-T} E conj(E^T X)). The derivative of each
 * block (Eq. 3, 4 differentiated in r and alpha) is recomputed, not stored.
 *   Na, Nm, P, Q, pos, freq_hz, coef  as in harp_fill         [2..8]
 *   Lambda, X    c128 N x nrhs, same leading dimension ld     [9, 10, 11]
 *   nrhs                                                       [12]
 *   grad_pos     double [Na][2], overwritten                   [13]
 *   prec         how G = Lambda X^T is contracted: HARP_FP64 in FP64;
 *                a mixed mode as exact digit products on the bf16 tensor
 *                cores rounded once to FP64 (HARP_OPT_ADJOINT_G = 1, the
 *                default, where the context holds the tensor-core residual's
 *                buffers; it waits for the context's pending background fill
 *                and replaces the residual's slices of Z64, which the next
 *                solve makes again), else in double-float on the FP32 pipe
 *                (operands split into float pairs, error-free products,
 *                Dot2 accumulation: FP64-accurate) using the context's
 *                float-float scratch when N <= max_N, nrhs <= max_nrhs and
 *                N nrhs <= max_N^2, else in FP64; HARP_FP32 in FP32. The
 *                contraction with the coefficients is double-float (mixed)
 *                or FP64, and the per-pair derivative sums are FP64   [14] */
int harp_fill_adjoint(harp_ctx* ctx, int Na, int Nm, int P, int Q, const double* pos,
                      double freq_hz, const double* coef, const double* Lambda, const double* X,
                      int ld, int nrhs, double* grad_pos, int prec, void* stream);

/* One problem of a batch: one frequency (or layout) of the fill + solve for
 * the port excitations. Inputs as for harp_fill; X (c128 N x Na, ld ldx,
 * device memory) receives the solution; status, iters and resid are
 * written by harp_solve_batch (status as returned by harp_fill/mbf_solve). */
typedef struct {
  int Na, Nm, P, Q;
  const double* pos;
  double freq_hz;
  const double* coef;
  const double* self_blocks;
  long self_stride;
  double* X;
  int ldx;
  int status;
  int iters;
  double resid;
} harp_problem;

/* Fill and solve many independent problems (the wideband case of the paper's
 * analysis over frequency, Section III: one reduced system per frequency,
 * with an MBF count that grows with frequency). Each of the n_ctx contexts
 * is a worker with its own host thread and stream; problems are taken in
 * array order (put the largest first), and workers overlap on the GPU.
 *   ctxs, n_ctx       contexts (each sized for the largest problem it may
 *                     take; all on one device, see harp_ctx_create) [1, 2]
 *   probs, n_probs    problems (host array)                          [3, 4]
 *   prec              HARP_FP64 or a mixed mode                      [5]
 *   tol, max_iter     as for mbf_solve                               [6, 7]
 * Blocks until every problem is done. Returns HARP_OK, or the first
 * non-zero per-problem status. */
int harp_solve_batch(harp_ctx** ctxs, int n_ctx, harp_problem* probs, int n_probs, int prec,
                     double tol, int max_iter);

/* ---- Tessellation (Section II-D, Fig. 3; Section IV-B) -------------------
 * Reading of the paper's hexagons: flat-topped, circumradius R. The inner
 * hexagons of circumradius R_in tile the plane with centres x = 1.5 R_in i,
 * y = sqrt(3) R_in (j + (i mod 2) / 2); an antenna belongs to the inner part
 * of the tile of the nearest centre (smallest (i, j) on ties); a tile's
 * subarray is every antenna inside the concentric hexagon of circumradius
 * R_in + R_ext, edge included. The membership decisions are plain IEEE FP64
 * with every product and sum rounded separately (no fused multiply-add).
 *
 * harp_tessellate: the tiles that hold antennas, sorted by (i, j), and per
 * tile its inner members and its subarray, each in increasing antenna
 * order, as CSR lists.
 *   Na, pos          antennas, double [Na][2] metres (device)       [1, 2]
 *   R_in, R_ext      metres (R_in > 0, R_ext >= 0)                   [3, 4]
 *   max_tiles        room in the tile arrays                         [5]
 *   tiles            output int [max_tiles][2]: (i, j)               [6]
 *   inner_ptr/_idx   output int [max_tiles + 1] / [Na]               [7, 8]
 *   outer_ptr/_idx   output int [max_tiles + 1] / [outer_cap]        [9, 10]
 *   outer_cap        room in outer_idx                               [11]
 *   n_tiles          host int: the number of tiles                   [12]
 *   outer_total      host long: the total subarray membership        [13]
 * Device outputs; synchronises `stream` (allocates stream-ordered scratch).
 * Returns HARP_E_UNSUPPORTED, with the sizes needed in *n_tiles and
 * *outer_total, when max_tiles or outer_cap is too small. */
int harp_tessellate(int Na, const double* pos, double R_in, double R_ext, int max_tiles,
                    int* tiles, int* inner_ptr, int* inner_idx, int* outer_ptr, int* outer_idx,
                    long outer_cap, int* n_tiles, long* outer_total, void* stream);

/* The currents of every port by the tessellation approach: each tile's
 * subarray is filled (Eq. 3-4) and solved for its port excitations with the
 * batch scheduler (the subarrays are independent problems of uneven size,
 * largest first), and column m of X keeps the currents of port m on the
 * subarray of m's tile, zero on the other antennas' rows (the paper keeps
 * the EEPs of the inner elements only).
 *   ctxs, n_ctx        contexts, each sized for the largest subarray  [1, 2]
 *   Na, Nm, P, Q, pos, freq_hz, coef, self_blocks, self_stride
 *                      the array, as for harp_fill                    [3..11]
 *   n_tiles, inner_ptr, inner_idx, outer_ptr, outer_idx
 *                      harp_tessellate's lists (device)               [12..16]
 *   X, ldx             output c128 (Na Nm) x Na                       [17, 18]
 *   prec, tol, max_iter   as for harp_solve_batch                     [19, 20, 21]
 * Device pointers; blocks until done; allocates the subarrays' inputs and
 * solutions for the call. Returns HARP_OK or the first non-zero status of
 * a subarray's fill or solve. */
int harp_solve_tessellated(harp_ctx** ctxs, int n_ctx, int Na, int Nm, int P, int Q,
                           const double* pos, double freq_hz, const double* coef,
                           const double* self_blocks, long self_stride, int n_tiles,
                           const int* inner_ptr, const int* inner_idx, const int* outer_ptr,
                           const int* outer_idx, double* X, int ldx, int prec, double tol,
                           int max_iter);

/* ---- Radius of influence (Section II-D, Section IV-A) ---------------------
 * Interactions kept only between antennas closer than RI: block (m, n) of
 * the reduced matrix is kept when m == n or r^2 < RI^2 (plain IEEE FP64,
 * each product and sum rounded separately), and the matrix is block sparse.
 *
 * harp_ri_pairs: the block-CSR structure: row_ptr (long [Na + 1], device)
 * and col_idx (int [cap], device), each block row's columns in increasing
 * order, the diagonal included; *nnzb (host) the number of kept blocks.
 * Synchronises `stream`. Returns HARP_E_UNSUPPORTED with *nnzb set when
 * cap is too small. Arguments: Na [1], pos (device double [Na][2]) [2],
 * RI (metres, >= 0) [3], cap [4], row_ptr [5], col_idx [6], nnzb [7]. */
int harp_ri_pairs(int Na, const double* pos, double RI, long cap, long* row_ptr, int* col_idx,
                  long* nnzb, void* stream);

/* harp_ri_fill: the kept blocks' values, Eq. 3 in Eq. 4 for m != n and the
 * self blocks on the diagonal, in the block-CSR order: block b at
 * values[b * Nm * Nm], column-major Nm x Nm, c128 for HARP_FP64, c64 (FP32
 * evaluation) for the other modes. Arguments 1..9 as for harp_fill (without
 * the context), then row_ptr, col_idx, nnzb from harp_ri_pairs [10, 11, 12],
 * values [13], prec [14], flag (device int: ST bits or-ed in, 1 coincident
 * antennas, 2 non-finite entries) [15]. Asynchronous on `stream`. */
int harp_ri_fill(int Na, int Nm, int P, int Q, const double* pos, double freq_hz,
                 const double* coef, const double* self_blocks, long self_stride,
                 const long* row_ptr, const int* col_idx, long nnzb, void* values, int prec,
                 int* flag, void* stream);

/* harp_bsr_to_dense: the block-sparse matrix in dense column-major storage
 * (zeros outside the kept blocks), c128 or c64 by prec as in harp_ri_fill,
 * for the dense solve (mbf_solve; in the mixed modes the FP64 copy goes to
 * the context's Z64 through harp_ctx_z64). N = Na Nm <= 65535. Arguments:
 * Na, Nm [1, 2], row_ptr, col_idx, nnzb [3, 4, 5], values [6], prec [7],
 * Z, ldz [8, 9]. Asynchronous on `stream`. */
int harp_bsr_to_dense(int Na, int Nm, const long* row_ptr, const int* col_idx, long nnzb,
                      const void* values, int prec, void* Z, int ldz, void* stream);

/* Port objective of the synthesis workload (the array-synthesis use the
 * paper's conclusion names; reading: the port response of the solution for
 * the port excitations V = E):
 *   P = E^T X   (Na x Na, c128, column-major; row m*Nm of each column of X),
 *   J = sum_mn |P_mn|^2   (one double, device memory),
 *   W = E conj(P)  (N x Na, c128, ld ldw; the right-hand side of the
 *                   adjoint solve Z^T Lambda = W for dJ/dZ).
 *   X, ldx  c128 N x Na solution of Z X = E, N = Na*Nm     [3, 4]
 *   P       output or NULL                                  [5]
 *   J       output (device double)                          [6]
 *   W, ldw  output or NULL                                  [7, 8]
 * Asynchronous on `stream`; J is reduced in a fixed order. */
int harp_port_objective(int Na, int Nm, const double* X, int ldx, double* P, double* J,
                        double* W, int ldw, void* stream);

/* Impedance reading of the synthesis objective (the same passage; the port
 * impedance is the inverse of the port response P = E^T X):
 *   Y = P^-1  (Na x Na, c128; the FP64 solve of P Y = I on ctx),
 *   J = sum_mn |Y_mn|^2   (one double, device memory),
 *   G = -Y^H Y Y^H        (Na x Na, c128; dJ = 2 Re tr(G^H dP)),
 *   W = E conj(G)         (N x Na, c128; the right-hand side of the adjoint
 *                          solve Z^T Lambda = W, as for harp_port_objective).
 *   ctx     a context with max_N >= Na and max_nrhs >= Na; its factorisation
 *           is replaced by P's (use a context other than the one holding
 *           Z's factors)                                    [1]
 *   Na, Nm  antennas, MBFs per antenna                      [2, 3]
 *   P, ldp  c128 Na x Na port response (harp_port_objective) [4, 5]
 *   Y, ldy  output                                          [6, 7]
 *   J       output (device double)                          [8]
 *   G, ldg  output                                          [9, 10]
 *   W, ldw  output, ldw >= Na Nm; also the scratch of Y^H Y [11, 12]
 * Returns mbf_solve's status for P (+i on an exactly zero pivot); the rest
 * is asynchronous on `stream`. */
int harp_port_impedance(harp_ctx* ctx, int Na, int Nm, const double* P, int ldp, double* Y,
                        int ldy, double* J, double* G, int ldg, double* W, int ldw, void* stream);

/* ---- Patterns (Section II-C) ---------------------------------------------
 * Embedded element patterns of the ports from the solution of the port
 * excitations: Eq. 5 with the sums swapped as in Eq. 6,
 *   E_m(u) = sum_j F_j(u) sum_i X[i*Nm + j, m] e^{jk (u_x x_i + u_y y_i)},
 * for the D directions u of the caller's grid (direction cosines ux, uy)
 * and both field components. The array factors of all MBFs and ports are
 * one product of the phase matrix e^{jk u.x_i} (made on the device, a
 * chunk of directions at a time) and the currents, on the tensor cores
 * with three-term TF32 products and FP32 accumulation; the result carries
 * FP32-level error (relative ~1e-6 of the pattern's scale).
 *   ctx          context (its tensor-core workspace; the call grows the
 *                context's pattern workspace on first use)        [1]
 *   Na, Nm       antennas, MBFs per antenna                       [2, 3]
 *   pos          double [Na][2], metres                           [4]
 *   freq_hz      frequency (> 0); k = 2 pi f / c0                 [5]
 *   X, ldx       c128 (Na Nm) x nports, column-major: the MBF
 *                coefficients for excitation at each port (the
 *                solution of mbf_solve)                           [6, 7]
 *   nports       ports (columns of X)                             [8]
 *   D            directions                                       [9]
 *   ux, uy       double [D]: direction cosines sin(theta) cos(phi),
 *                sin(theta) sin(phi)                              [10, 11]
 *   F            c128 [2][D][Nm]: the MBF patterns, theta then phi
 *                component, per direction and MBF                 [12]
 *   E            output c64 [2][nports][D]: the patterns, theta then
 *                phi component, per port and direction            [13]
 * Device pointers; asynchronous on `stream` (a bounded wait that gives up
 * is reported by harp_ctx_sync). The array pattern of an excitation law w
 * over the ports is the call with X w as its single column. Errors: -i
 * argument i; HARP_E_UNSUPPORTED when Na, Nm * nports or nports exceed
 * 65535; HARP_E_NOMEM; HARP_E_CUDA. */
int harp_eep(harp_ctx* ctx, int Na, int Nm, const double* pos, double freq_hz, const double* X,
             int ldx, int nports, int D, const double* ux, const double* uy, const double* F,
             float* E, void* stream);

/* The error between two patterns in each of n directions (Eq. 8, Section
 * III-A): eps[q] = sqrt(|E_theta - Eref_theta|^2 + |E_phi - Eref_phi|^2)
 * / norm, with norm the maximum of the isolated antenna's pattern.
 *   n       directions (times ports)                    [1]
 *   E, Eref c64 [2][n]: theta then phi components       [2, 3]
 *   norm    > 0                                         [4]
 *   eps     output float [n]                            [5]
 * Device pointers; asynchronous on `stream`; no context. */
int harp_pattern_error(long n, const float* E, const float* Eref, double norm, float* eps,
                       void* stream);

/* ---- HARP model construction (Section II-A, Eq. 2-3; Section II-B) ------
 * The coefficients c_pq^{TS} of Eq. 3 from samples of the complementary
 * interaction B_TS (Eq. 2) on a polar grid: angles alpha_a = 2 pi a /
 * Nalpha (regular), radii given as d_l = 1/r_l (the paper samples them
 * regularly in 1/r). Per MBF pair: the DFT over alpha (the improved model's
 * DFT estimate of the harmonics), then a least-squares polynomial in d for
 * each harmonic (thin QR of the Vandermonde matrix), all in FP64. Exact
 * for a model band-limited to |p| <= P when Nalpha >= 2P + 1 and
 * Nd >= Q + 1.
 *   Nm, P, Q     model sizes (Q + 1 <= 16)                        [1, 2, 3]
 *   Nd, Nalpha   grid sizes (Nd >= Q + 1, Nalpha >= 2P + 1)       [4, 5]
 *   d            double [Nd]: the sampled d = 1/r                 [6]
 *   B            c128 [Nm][Nm][Nd][Nalpha]: samples B_TS(d_l, alpha_a) [7]
 *   coef         output c128 [Nm][Nm][2P+1][Q+1], the layout harp_fill
 *                reads                                            [8]
 *   rms          output double [Nm][Nm] (or NULL): root-mean-square
 *                residual of the fitted model on the samples      [9]
 * Device pointers; asynchronous on `stream`; no context. Errors: -i
 * argument i; HARP_E_UNSUPPORTED when Q + 1 > 16 or one pair's samples
 * exceed the shared memory of a CTA. */
int harp_model_fit(int Nm, int P, int Q, int Nd, int Nalpha, const double* d, const double* B,
                   double* coef, double* rms, void* stream);

/* Allocation-free variant of harp_fill_adjoint (no counterpart in the paper:
 * it exists for callers that cannot allocate device memory, for instance an
 * application whose allocator owns all device memory or that runs under a
 * fixed memory budget). It takes no context and calls no allocating routine:
 * its per-pair scratch is a fixed device array inside this library, sized
 * for at most HARP_NOALLOC_MAX_NA antennas (HARP_NOALLOC_MAX_NA^2 * 2
 * doubles, 4 MiB, held on every GPU that loads the library until the
 * process exits). Its 14 arguments are arguments 2..15 of harp_fill_adjoint
 * (everything but the context, stream included); it works on the current
 * CUDA device, which must hold every pointer and the stream. A negative
 * status -i names the 1-based position i of the bad argument in THIS call
 * (one less than the same argument's position in harp_fill_adjoint, e.g.
 * Na < 1 gives -1). Returns HARP_E_UNSUPPORTED when Na > HARP_NOALLOC_MAX_NA.
 * While profiling is on, its pair kernel is recorded in HARP_K_ADJOINT like
 * harp_fill_adjoint's.
 * The first call on a device looks up that device's address of the array
 * (a runtime query, with the device current); make that first call before
 * any stream capture. All calls share the one array: each call clears what
 * it uses, and calls whose work overlaps on the GPU (different streams)
 * race on it, so serialise them. Precision: HARP_FP64 contracts G = Lambda
 * X^T in FP64 as harp_fill_adjoint does; every other mode contracts it in
 * FP32 (harp_fill_adjoint's HARP_FP32 kernel): the double-float contraction
 * of harp_fill_adjoint's mixed modes needs a context's scratch. */
#define HARP_NOALLOC_MAX_NA 512
int harp_fill_adjoint_noalloc(int Na, int Nm, int P, int Q, const double* pos, double freq_hz,
                              const double* coef, const double* Lambda, const double* X, int ld,
                              int nrhs, double* grad_pos, int prec, void* stream);

/* ---- Instrumentation: device time per kernel class -------------------------
 * Not part of the method; used to report each kernel's share of the time and
 * its achieved fraction of the hardware's peak. While recording, each launch
 * of a selected class is bracketed by a CUDA event pair on its own stream,
 * and the class accumulates the launch's algorithmic flop count
 * (8 real flops per complex multiply-add). */
#define HARP_PROF_KINDS 10
#define HARP_K_FILL 0     /* harp_fill kernels (FP64 and FP32 evaluation)        */
#define HARP_K_GEMM 1     /* tensor-core products: LU trailing updates, the
                             factor inverses' products, the solves' products    */
#define HARP_K_RESIDUAL 2 /* FP64-accurate residual R = V - Z X of the refinement */
#define HARP_K_PANEL 3    /* in-panel LU leaves (pivot search)                  */
#define HARP_K_TRSM 4     /* triangular-solve leaves, triangle-block inverses and
                             the narrow look-ahead products (64 wide)          */
#define HARP_K_SWAP 5     /* row interchanges                                   */
#define HARP_K_ADJOINT 6  /* harp_fill_adjoint kernels                          */
#define HARP_K_OTHER 7    /* conversions, norms, permutations                   */
#define HARP_K_RESID_UPDATE 8 /* residual updates R - Z D (small D)              */
#define HARP_K_FILL_FF 9  /* the mixed fill's FP64-accurate Z64 (float-float or
                             digit products)                                    */

/* Start recording the classes whose bit (1 << HARP_K_*) is set in mask.
 * Process-wide; discards earlier records. */
int harp_profile_begin(harp_ctx* ctx, unsigned mask);

/* Synchronise the recorded events and return, per class, the summed device
 * milliseconds, algorithmic flops and launch count (arrays of
 * HARP_PROF_KINDS entries, host memory). Stops recording. */
int harp_profile_end(harp_ctx* ctx, double* ms, double* flops, long long* launches);

#ifdef __cplusplus
}
#endif

#endif /* HARP_GB300_H */
