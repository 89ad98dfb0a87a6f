/*
 * trals.h -- C ABI of libtrals: tensor-ring alternating least squares on one GB300 GPU.
 *
 * Method: Yu & Li, "Practical Alternating Least Squares for Tensor Ring
 * Decomposition" (arXiv 2210.11362).  The library fits TR({G_n}) to a dense
 * tensor X (problem eq. trmin, Sec. 1) by ALS sweeps over n = 1..N (Alg. 1),
 * computing each core update the TR-ALS-NE way (Alg. 2, lines 6-10):
 *   S_n  = structured coefficient matrix from per-core Gram matrices
 *          (Prop. subchain_gram, Alg. 2 lines 2, 6, 10),
 *   M_n  = X_[n] G^{!=n}_[2]   (MTTSP, Alg. 2 lines 7-8),
 *   G_n  : G_{n(2)} S_n = M_n  (normal equation, Alg. 2 line 9),
 * or with the QR-stabilised solve of Sec. 3.2 (Alg. 3).
 *
 * Conventions (all entry points)
 *  - Mode indices n are 0-based (the paper's mode n is n-1 here).
 *  - Dense tensors are column-major: linear index sum_n i_n prod_{j<n} I_j,
 *    first index fastest (Sec. 2).
 *  - Core n is R_n x I_n x R_{n+1}, column-major (r_n fastest, then i_n, then
 *    r_{n+1}), with R_N wrapping to R_0 (Sec. 1).
 *  - Matrices are column-major.  G_{n(2)} (classical mode-2 unfolding) is
 *    I_n x R_n R_{n+1} with column r_n + R_n r_{n+1}; S_n is r x r and M_n is
 *    I_n x r with r = R_n R_{n+1} in the same column order.
 *  - Gamma_k = sum_i G_k(i) (x) G_k(i) is R_k^2 x R_{k+1}^2 with Kronecker row
 *    index p R_k + q and column index s R_{k+1} + t.
 *  - "dev" pointers are device memory of the context's device; "host" pointers
 *    are host memory.  The caller owns every buffer it passes in; the library
 *    never frees or retains caller pointers after a call returns.
 *  - Every call is ordered on the context's stream.  Calls that return results
 *    to host memory synchronize that stream before returning; the others only
 *    enqueue work.
 *  - Errors are returned, never thrown, and no call traps the GPU.  Device-side
 *    failures (a non-positive Cholesky pivot, a non-finite value) set a device
 *    status word that the next synchronizing call reports.  trals_last_error()
 *    returns a human-readable message for the last failing call on a context.
 *  - No entry point is thread-safe on the same context.
 */
#ifndef TRALS_H
#define TRALS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TRALS_MAX_ORDER 8

typedef enum {
  TRALS_OK = 0,
  TRALS_E_ARG = 1,        /* invalid argument (shape, rank, null pointer, unsupported combination) */
  TRALS_E_OOM = 2,        /* device memory allocation failed */
  TRALS_E_CUDA = 3,       /* a CUDA runtime call failed */
  TRALS_E_NOT_SPD = 4,    /* Cholesky met a non-positive pivot: S_n is not numerically SPD */
  TRALS_E_NONFINITE = 5,  /* a NaN or Inf reached a solve */
  TRALS_E_TIMEOUT = 6,    /* a bounded device wait gave up */
  TRALS_E_REJECTED = 7,   /* serving: request does not fit the admission budget */
  TRALS_E_PENDING = 8     /* serving: result not ready yet */
} trals_status;

/* Element type of the caller's X.  TRALS_X_BF16PAIR: 2 prod(I) BF16 values, the hi plane of every
 * element (column-major) followed by the lo plane, value hi + lo (the split trals_quantize_bf16 writes);
 * accepted by trals_mttsp in the BF16 modes (BF16 and BF16X2 read the hi plane). */
typedef enum { TRALS_X_F64 = 0, TRALS_X_F32 = 1, TRALS_X_BF16 = 2, TRALS_X_BF16PAIR = 3 } trals_xtype;

/* Storage of X and arithmetic of the RHS contraction M_n (the Gram chain, S_n and the solve are
 * FP64 in every mode).
 *  FP64  : X read as FP64, MTTSP in FP64 on the CUDA cores.
 *  FP32  : X read as FP32 (converted once from FP64 if needed); MTTSP on the CUDA cores in FP32
 *          arithmetic, per-block sums reduced in FP64 (a plan takes the two-stage GEMM MTTSP instead
 *          where trals_plan_mttsp_path reports code 5).
 *  BF16  : X quantised once to BF16 (round to nearest even); MTTSP on BF16 tensor cores
 *          (tcgen05) with FP32 accumulation where trals_mttsp_path reports a tensor-core
 *          geometry, else on the CUDA cores in FP32 arithmetic (or, in a plan, the two-stage GEMM
 *          MTTSP, code 5 of trals_plan_mttsp_path).
 *  BF16X3: X split once into hi/lo BF16 pairs (hi = bf16(x), lo = bf16(x - hi)), the subchain
 *          table likewise; on the tensor cores every K step is three BF16 products
 *          (X_hi T_hi + X_hi T_lo + X_lo T_hi) into one FP32 accumulator (the CUDA-core path reads
 *          hi + lo in FP32 arithmetic).
 *  BF16X2: X quantised once to BF16 as in BF16, the subchain table split into hi/lo BF16 pairs;
 *          two products per K step (X T_hi + X T_lo): only the rounding of X remains.  Off the
 *          tensor-core geometries as BF16. */
typedef enum {
  TRALS_MODE_FP64 = 0,
  TRALS_MODE_FP32 = 1,
  TRALS_MODE_BF16 = 2,
  TRALS_MODE_BF16X3 = 3,
  TRALS_MODE_BF16X2 = 4
} trals_mode;

/* Solver for the R_n R_{n+1} subproblem:
 *  CHOL          Cholesky on the normal equations (Alg. 2 line 9);
 *  QR            the QR-stabilised solve (Sec. 3.2): R factor of G^{!=n}_[2] by structured recursive QR and
 *                corrected semi-normal steps, for any shape;
 *  QRNE          TR-ALS-QRNE (Alg. 4, Sec. 3.3): the normal equations of the problem compressed by the mode-2
 *                QR of every core (CholeskyQR2), with the Multi-TTM Y = X x_{j!=n} Q_j^T;
 *  QR_COMPRESSED the literal TR-ALS-QR (Alg. 3) for the compressible regime (I_j > R_j R_{j+1}): Householder
 *                mode-2 QRs of the cores, the Multi-TTM, the explicit subchain V_n of the R factors and its
 *                Householder QR V_n[2] = Q_0 R, W_n = Y_[n] Q_0 and the triangular solve with R; needs
 *                R_n R_{n+1} <= prod_{j!=n} min(I_j, R_j R_{j+1}) <= 2^22.
 * QRNE and QR_COMPRESSED run in the FP64 mode through trals_decompose only. */
typedef enum {
  TRALS_SOLVE_CHOL = 0,
  TRALS_SOLVE_QR = 1,
  TRALS_SOLVE_QRNE = 2,
  TRALS_SOLVE_QR_COMPRESSED = 3
} trals_solver;

/* How S_n is formed: structured Gamma chain (Prop. subchain_gram) or the explicit
 * subchain matrix's Gram (G^{!=n}_[2])^T G^{!=n}_[2] (regular TR-ALS, Alg. 1). */
typedef enum { TRALS_GRAM_STRUCTURED = 0, TRALS_GRAM_EXPLICIT = 1 } trals_gram;

typedef struct {
  int mode;              /* trals_mode */
  int solver;            /* trals_solver */
  int gram;              /* trals_gram */
  int explicit_residual; /* 1: per-sweep residual by a full reconstruction pass against X (Sec. 4 formula;
                               FP64 reconstruction in the FP64 mode, FP32 in the others);
                            0: the cheap identity of Sec. 4 in the FP64 mode.  The reduced-precision
                               modes then record NaN per sweep: with BF16 rounding in M_N the
                               identity's cancellation leaves no accurate digits at small residuals
                               (trals_decompose still fills the last entry by one explicit pass). */
} trals_opts;

typedef struct trals_ctx trals_ctx;
typedef struct trals_plan trals_plan;

/* ------------------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, ordering all work on `cuda_stream`
 * (a cudaStream_t; NULL = a stream the context creates, which synchronizes with the
 * legacy default stream).  Errors: TRALS_E_ARG for a bad device, TRALS_E_CUDA. */
trals_status trals_create(trals_ctx** out, int device, void* cuda_stream);
/* Destroy a context (synchronizes its stream first).  NULL is ignored. */
void trals_destroy(trals_ctx* ctx);
/* Message for the last failing call on ctx (never NULL; "" if none). */
const char* trals_last_error(const trals_ctx* ctx);
/* Library version string. */
const char* trals_version(void);

/* ------------------------------------------------------------------------- whole decomposition */

/* Fit TR cores to X by `sweeps` ALS sweeps (problem eq. trmin; Alg. 1 sweep order
 * n = 1..N with the core update of Alg. 2, or Alg. 3's QR-stabilised solve).
 *   N          order, 3 <= N <= TRALS_MAX_ORDER
 *   I[N]       mode sizes (>= 1); R[N] TR ranks (>= 1), R_{N} wraps to R_0
 *   X          the tensor, column-major, element type xt; device memory if
 *              x_on_host == 0, else host memory (copied in by this call)
 *   cores[N]   host pointers; in: initial cores, out: fitted cores (FP64, layout above)
 *   opts       NULL = {FP64, CHOL, STRUCTURED, explicit_residual 0}
 *   rel_res    host array of `sweeps` doubles, out: relative residual |X - X_hat|_F/|X|_F
 *              after each sweep (may be NULL); see trals_opts.explicit_residual for the
 *              reduced-precision modes, whose last entry is always the explicit residual
 * Requires J_n = prod_{j != n} I_j >= R_n R_{n+1} for every n (else the
 * subproblem is underdetermined): TRALS_E_ARG.  Synchronous. */
trals_status trals_decompose(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                             const void* X, int xt, int x_on_host,
                             double* const* cores, int sweeps, const trals_opts* opts,
                             double* rel_res);

/* ------------------------------------------------------------------------- resident plan */

/* A plan keeps X (device, caller-owned, must outlive the plan), the cores, the
 * Gamma_k caches and all workspace resident, so sweeps can be replayed (as one
 * captured CUDA graph per sweep) without host work.  Arguments as in
 * trals_decompose; X_dev is device memory.  The workspace is allocated stream-ordered
 * (cudaMallocAsync on the context's stream) and freed the same way by trals_plan_destroy,
 * so plans can come and go while other streams keep the device busy. */
trals_status trals_plan_create(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                               const void* X_dev, int xt, const trals_opts* opts, trals_plan** out);
/* Bytes of device workspace trals_plan_create would allocate for these arguments (X itself not
 * included), computed on the host without allocating or launching anything: the admission
 * figure of the serving loop.  X_dev is only inspected for alignment. */
trals_status trals_plan_footprint(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                                  const void* X_dev, int xt, const trals_opts* opts, size_t* bytes);
/* Bytes of device workspace a plan holds (equals trals_plan_footprint for its arguments). */
size_t trals_plan_bytes(const trals_plan* plan);
void trals_plan_destroy(trals_plan* plan);
/* Upload cores (host pointers, FP64) and recompute every Gamma_k (Alg. 2 line 2).
 * Resets the sweep counter.  Synchronous. */
trals_status trals_plan_set_cores(trals_plan* plan, double* const* cores_host);
/* Download cores (host pointers, FP64).  Synchronous; reports device status. */
trals_status trals_plan_get_cores(trals_plan* plan, double* const* cores_host);
/* Enqueue `sweeps` ALS sweeps.  Enqueue only (no host sync, graph replays when
 * use_graph != 0). */
trals_status trals_plan_run(trals_plan* plan, int sweeps, int use_graph);
/* Copy the residual history (count = sweeps run since set_cores, at most `cap`)
 * to host; synchronous; reports device status. */
trals_status trals_plan_residuals(trals_plan* plan, double* rel_res_host, int cap, int* count);
/* Enqueue only the MTTSP of mode n (Alg. 2 lines 7-8) with the plan's current cores and
 * workspace, writing M_n (I_n x R_n R_{n+1}, FP64) to M_dev (NULL: the plan's internal buffer).
 * Allocates nothing; used to time and test the RHS contraction in isolation. */
trals_status trals_plan_mttsp(trals_plan* plan, int n, double* M_dev);
/* Relative residual |X - TR(cores)|_F / |X|_F of the plan's current cores against the caller's X
 * (the explicit error of Sec. 4), by one pass over X that regenerates X_hat: in FP64 in the FP64
 * mode, in FP32 (differences and sums in FP64) in the reduced-precision modes, where the
 * regeneration error (~1e-7 relative) is far below the residuals being compared.  Synchronous. */
trals_status trals_plan_explicit_residual(trals_plan* plan, double* rel_res_host);
/* Measurement hook (the paper has no counterpart): enqueue the MTTSP of mode n once, exactly as a
 * sweep does, with CUDA events around the part of the step a sweep has on its critical path (for the
 * tensor-core kernel: the link of the subchain tables through the core updated just before, the
 * contraction and the reduction of its per-CTA partials; the other table builds, which a sweep runs
 * during the previous mode on a side stream, are enqueued before the first event) and around the
 * main contraction kernel alone; waits for it and returns both durations in milliseconds.  The caller
 * may evict L2 on the context's stream beforehand.  Not for use while the stream is being captured. */
trals_status trals_plan_time_mttsp(trals_plan* plan, int n, float* kernel_ms, float* total_ms);
/* Device pointer of core n (FP64, layout above), valid until the plan is destroyed. */
const double* trals_plan_core_dev(const trals_plan* plan, int n);
/* Which kernel the plan uses for the MTTSP of mode n (codes of trals_mttsp_path, plus 5: the two-stage
 * GEMM MTTSP, taken in the FP32, BF16 and BF16X2 modes by modes without a tensor-core geometry whose
 * stage-1 table is 64 to 256 columns wide, for tensors of at least 2^21 entries: X is first contracted
 * with the subchain table of the modes that lead it in memory, a plain GEMM through cuBLAS (FP32, or
 * BF16 operands with FP32 accumulation), then with the other table in this library's kernels).  This
 * can also differ from trals_mttsp_path when the TMA descriptor encoder rejects a tensor-core geometry
 * or X is not 16-byte aligned: the plan then falls back to the CUDA cores. */
int trals_plan_mttsp_path(const trals_plan* plan, int n);
/* Number of kernel launches one sweep issues (for launch accounting). */
int trals_plan_launches_per_sweep(const trals_plan* plan);

/* ------------------------------------------------------------------------- per-step kernels
 * Each computes one step of the core update on device buffers, for testing and
 * composition.  These allocate their own temporaries and are synchronous. */

/* Gamma = sum_i G(i) (x) G(i) (Alg. 2 lines 2 and 10; Prop. subchain_gram), FP64.
 * G_dev: Rn x In x Rn1 core; Gamma_dev: Rn^2 x Rn1^2 (column-major). */
trals_status trals_gamma(trals_ctx* ctx, const double* G_dev, int Rn, int64_t In, int Rn1, double* Gamma_dev);

/* Structured coefficient matrix of mode n (Alg. 2 line 6): Pi_n = Gamma_{n+1} ...
 * Gamma_N Gamma_1 ... Gamma_{n-1} (products in FP64), regrouped to
 * S_n[(a + R_n b), (a' + R_n b')] = Pi_n[(b R_{n+1} + b'), (a R_n + a')].
 * gammas_dev[k] for k != n are used.  S_dev: r x r, r = R_n R_{n+1}. */
trals_status trals_coef_matrix(trals_ctx* ctx, int N, const int32_t* R, const double* const* gammas_dev,
                               int n, double* S_dev);

/* R factor of the subchain matrix G^{!=n}_[2] (Sec. 3.2: the QR factorisation TR-ALS-QR solves
 * with), computed without forming S_n: recursive structured QR along the subchain (the mode-2 QR of
 * G_{n+1}, then at each further core the QR of (R_t [x]_2 G_c)_[2], which Prop. slice_kron shows
 * has the same R factor as the running product), each step by a Householder TSQR tree, all FP64.
 * R_dev: r x r upper triangular with a positive diagonal (column-major, columns a + R_n b as in
 * G_{n(2)}), so R^T R = S_n.  TRALS_E_NOT_SPD when a diagonal entry is zero (rank deficient).
 * cores_dev[N] device FP64 cores.  Synchronous. */
trals_status trals_qr_r_factor(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                               const double* const* cores_dev, int n, double* R_dev);

/* Explicit-subchain coefficient matrix of mode n (regular TR-ALS, Alg. 1): the subchain matrix
 * G^{!=n}_[2] (J_n x R_n R_{n+1}, Def. subchain tensor) is formed explicitly on the device in row
 * blocks and S_dev (r x r, full symmetric, column-major) = (G^{!=n}_[2])^T G^{!=n}_[2] is accumulated by
 * a blocked SYRK: in FP64 when fp64 != 0, else with FP32 rows and FP32 tile sums reduced in FP64.
 * The comparison variant of trals_coef_matrix.  cores_dev[N] device FP64 cores.  Synchronous. */
trals_status trals_coef_matrix_explicit(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                                        const double* const* cores_dev, int n, int fp64, double* S_dev);

/* MTTSP of mode n (Alg. 2 lines 7-8): M_dev (I_n x r, FP64) = X_[n] G^{!=n}_[2], with the
 * subchain rows generated on the fly from cores_dev (FP64) in the arithmetic of `mode`
 * (X element type must match the mode: F64 for FP64, F32 for FP32, BF16 or BF16PAIR for BF16 and
 * BF16X2 (the hi plane is read), BF16PAIR -- or BF16 laid out the same way -- for BF16X3: the hi
 * plane followed by the lo plane, 2 * prod(I) elements).  trals_last_mttsp_path tells which kernel
 * ran. */
trals_status trals_mttsp(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                         const void* X_dev, int xt, int mode, const double* const* cores_dev, int n,
                         double* M_dev);

/* Solve Z S = M for Z (I_n x r) by Cholesky S = L L^T and two triangular solves
 * (Alg. 2 line 9, FP64), writing Z folded into core layout: G[a + Rn (i + In b)] =
 * Z[i, a + Rn b].  S_dev r x r SPD (only the lower triangle is read), M_dev In x r.
 * Synchronous: returns TRALS_E_NOT_SPD / TRALS_E_NONFINITE from the device status. */
trals_status trals_solve_chol(trals_ctx* ctx, int Rn, int64_t In, int Rn1, const double* S_dev,
                              const double* M_dev, double* G_dev);

/* Verification hook for the Cholesky pivots; not a step of the method.  For n positive finite doubles
 * d_dev (device), out_dev[i] = the reciprocal square root the Cholesky kernel of trals_solve_chol uses for
 * its pivots and ref_dev[i] = CUDA's rsqrt(d_dev[i]), both device arrays of n doubles.  Other inputs give
 * unspecified values.  n = 0 is a no-op.  Synchronous. */
trals_status trals_check_pivot_rsqrt(trals_ctx* ctx, const double* d_dev, int64_t n, double* out_dev,
                                     double* ref_dev);

/* trals_mttsp in FP64 mode (X FP64) without any device allocation, for callers that cannot allocate:
 * an allocator hook that must not re-enter the CUDA allocator, a fixed-budget real-time loop whose
 * device memory may not grow, or a runtime that owns all device memory and hands the library only
 * its inputs and outputs.  The paper has no counterpart; it is an interface convenience.  Its
 * subchain tables, offsets and per-block partial sums live in one static 32 MiB device array that
 * every GPU loading the library holds until process exit; shapes whose tables plus one block's
 * partial sums do not fit return TRALS_E_ARG with a message, as do the shapes trals_mttsp rejects.
 * The array's device address is looked up on the first call made on each device.  The call is
 * synchronous (it copies index offsets from host memory and waits for its stream), so it must not be
 * made from a stream callback (cudaLaunchHostFunc, where CUDA calls are not allowed) nor while any
 * stream is being captured.  All calls share the array, so calls that overlap on the GPU race:
 * serialise them.  Arguments and result layout as trals_mttsp. */
trals_status trals_mttsp_noalloc(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R, const void* X_dev,
                                 const double* const* cores_dev, int n, double* M_dev);

/* Which kernel the last successful trals_mttsp call on ctx actually ran (codes of trals_mttsp_path;
 * -1 before any call or after a failed one).  trals_mttsp takes the tensor-core kernel where
 * trals_mttsp_path reports a geometry and the TMA descriptor encoder and X's 16-byte alignment
 * allow it, else the CUDA cores; this query tells which happened.  Host only. */
int trals_last_mttsp_path(const trals_ctx* ctx);

/* Which kernel computes the MTTSP of mode n in `mode` (host-only query, needs no GPU):
 * 0 = CUDA cores (the FP64 path, and shapes the tensor-core kernel does not take);
 * 1 = tensor cores, X K-major with the stage-2 factor on the left;
 * 2 = tensor cores, X K-major with the stage-2 factor on the right;
 * 3 = tensor cores, X MN-major with the stage-2 factor on the right;
 * 4 = tensor cores, X MN-major with the stage-2 factor on the left (mode 0: a tile's rows are consecutive
 *     elements of X).  Negative on invalid arguments. */
int trals_mttsp_path(int N, const int64_t* I, const int32_t* R, int n, int mode);

/* X_hat = TR(cores) written to out_dev (column-major, element type xt) (Sec. 1 element formula). */
trals_status trals_reconstruct(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                               const double* const* cores_dev, void* out_dev, int xt);

/* Explicit squared residual |X - TR(cores)|_F^2 and |X|_F^2 in FP64 by one fused
 * reconstruction pass (Sec. 4 error formula).  Synchronous; results to host. */
trals_status trals_residual_explicit(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                                     const void* X_dev, int xt, const double* const* cores_dev,
                                     double* res2_host, double* normx2_host);

/* Quantise count elements of src (type src_t, F64 or F32) to BF16 (round to nearest
 * even).  If dst_lo_dev != NULL also write lo = bf16(x - float(hi)). */
trals_status trals_quantize_bf16(trals_ctx* ctx, const void* src_dev, int src_t, int64_t count,
                                 void* dst_hi_dev, void* dst_lo_dev);

/* ------------------------------------------------------------------------- serving
 * A request loop that runs many TR decompositions at once on one GPU (continuous batching; the
 * paper has no counterpart -- it runs one decomposition at a time).  Requests of any order, sizes
 * and ranks are submitted from any host thread and queue in arrival order.  A worker thread admits
 * the head of the queue as soon as a slot is free and the request's device footprint (the plan
 * workspace of trals_plan_footprint, plus a device copy of X when X is on the host) fits in what
 * is left of the HBM budget.  Each admitted request runs as a resident plan on its slot's own
 * stream, all its sweeps enqueued as replays of the plan's captured per-sweep CUDA graph, so the
 * work of every active request overlaps on the device.  A request computes exactly what
 * trals_decompose computes for it alone: kernels are deterministic and slots share no device
 * state, so results do not depend on what else is in flight. */
typedef struct trals_server trals_server;

typedef struct {
  int N;                            /* order, 3 <= N <= TRALS_MAX_ORDER */
  const int64_t* I;                 /* [N] mode sizes (copied at submit) */
  const int32_t* R;                 /* [N] TR ranks (copied at submit) */
  const void* X;                    /* column-major tensor of element type xt: device memory of the
                                       server's device, or host memory when x_on_host != 0 (pinned
                                       memory copies fastest).  Caller-owned; must stay valid and
                                       unchanged until the result is ready. */
  int xt;                           /* trals_xtype */
  int x_on_host;
  const double* const* init_cores;  /* [N] host pointers, initial cores (copied at submit) */
  int sweeps;                       /* ALS sweeps to run */
  trals_opts opts;                  /* as for trals_decompose */
} trals_request;

typedef struct {
  trals_status status;     /* outcome of the decomposition (TRALS_OK, or its error) */
  int sweeps;
  double submit_s;         /* host clock, seconds since the server was created */
  double admit_s;          /* when the request got a slot and its memory */
  double done_s;           /* when its results were back on the host */
  size_t footprint_bytes;  /* device memory it held while active */
} trals_result;

typedef struct {
  int queued;              /* submitted, not yet admitted */
  int active;              /* holding a slot */
  uint64_t completed;
  size_t used_bytes;       /* footprint of the active requests */
  size_t peak_used_bytes;
  int peak_active;
  double host_start_s;     /* host time the worker spent starting requests (plan set-up, graph capture,
                              launches; grouped admissions) */
  uint64_t grouped_completed; /* requests served by the grouped step engine */
  uint64_t grouped_steps;  /* steps the grouped engine has launched */
} trals_server_info;

/* Start a server on `device` with at most max_slots plan requests in flight, plus up to 64 small
 * requests in the grouped step engine, whose footprints sum to at most hbm_budget_bytes.  Starts one
 * worker thread.
 *
 * Small requests -- order 3 to 5, every R_k <= 8, at most 2^18 entries (see
 * trals_server_set_group_limit), FP32 X, mode TRALS_MODE_FP32 or TRALS_MODE_BF16, the Cholesky solve
 * of the structured Gram chain, no per-sweep explicit residual, sweeps >= 1 -- join the grouped step
 * engine: each step advances every such request by one core update of Alg. 2 (its own mode n), the
 * Gamma-chain products, the MTTSP (X_[n] times the subchain in FP32, from the BF16 copy of X in the
 * BF16 mode), the FP64 Cholesky solve and the Gamma update, as one graph of grouped kernels over a
 * device table of the active requests.  Results follow the reduced-precision plans' conventions: FP64
 * cores, no per-sweep residual (NaN), the explicit relative residual against the FP32 X after the last
 * sweep.  Other requests run as plans (what trals_decompose runs). */
trals_status trals_server_create(trals_server** out, int device, size_t hbm_budget_bytes, int max_slots);
/* Stop the server: requests still queued are dropped, active ones finish; results not yet taken
 * are freed.  Joins the worker thread. */
void trals_server_destroy(trals_server* server);
/* Queue a request (non-blocking).  TRALS_E_ARG for invalid shapes or arguments (see
 * trals_decompose), TRALS_E_REJECTED when its footprint alone exceeds the budget. */
trals_status trals_server_submit(trals_server* server, const trals_request* request, uint64_t* ticket);
/* TRALS_E_PENDING while the request runs; TRALS_OK once it is done, after filling *result and
 * copying the fitted cores (host pointers [N], core layout, may be NULL) and the per-sweep
 * residuals (host array of `sweeps`, may be NULL; same semantics as trals_decompose).  The ticket
 * is then released (a further poll returns TRALS_E_ARG). */
trals_status trals_server_poll(trals_server* server, uint64_t ticket, trals_result* result,
                               double* const* cores_out, double* rel_res_out);
/* As trals_server_poll, but blocks up to timeout_s seconds (negative: no limit). */
trals_status trals_server_wait(trals_server* server, uint64_t ticket, double timeout_s, trals_result* result,
                               double* const* cores_out, double* rel_res_out);
trals_status trals_server_stats(trals_server* server, trals_server_info* out);
/* Requests submitted from now on with at most max_elems entries (and otherwise small, see
 * trals_server_create) join the grouped step engine; 0 sends every request to a plan.  TRALS_E_ARG for a
 * negative limit. */
trals_status trals_server_set_group_limit(trals_server* server, int64_t max_elems);
/* Message for the last rejected submit or failed request taken by poll/wait. */
const char* trals_server_last_error(const trals_server* server);

#ifdef __cplusplus
}
#endif
#endif /* TRALS_H */
