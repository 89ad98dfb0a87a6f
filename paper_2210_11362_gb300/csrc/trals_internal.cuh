// Internal declarations shared by the libtrals translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/trals.h"

namespace trals {

constexpr int kMaxOrder = TRALS_MAX_ORDER;

// Device status word: first failure wins (atomicCAS on code).
struct DevStatus {
  int code;    // trals_status
  int sweep;   // sweep index (plan runs) or -1
  int mode;    // core index n or -1
  int index;   // pivot / element index
  double value;
};

// Record the first failure (later ones are dropped).
__device__ __forceinline__ void set_status(DevStatus* st, int code, int sweep, int mode, int index, double v) {
  if (st == nullptr) return;
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->sweep = sweep;
    st->mode = mode;
    st->index = index;
    st->value = v;
  }
}

// Validate a shape for every entry point: 3 <= N <= TRALS_MAX_ORDER, I_n >= 1, 1 <= R_n <= 64,
// prod I_n <= 2^46, R_n R_{n+1} <= 256 and J_n >= R_n R_{n+1}.  Sets ctx->last_error on failure.
trals_status check_shape(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R);

// ---------------------------------------------------------------- per-mode MTTSP layout
// The other modes of mode n in subchain order c_1..c_{N-1} = n+1..N,1..n-1 (eq. subchain_new)
// are split into Left = c_1..c_m and Right = c_{m+1}..c_{N-1}.  G^{!=n}(k) = L(l) U(u) with
// k = l + |L| u.  Ltab[l] is R_{n+1} x R_s, Utab[u] is R_s x R_n (s = c_{m+1}), column-major.
// offL[l] + offU[u] is the memory offset of X(i) with i_n = 0; i_n adds i_n * strideN.
struct ModeLayout {
  int N;
  int n;
  int chain[kMaxOrder];
  int m;                 // number of Left modes
  int64_t nL, nU;        // table entries
  int Rn, Rn1, Rs;       // R_n, R_{n+1}, R at the split
  int64_t In, strideN;   // I_n, memory stride of i_n (prod_{j<n} of the stored extents)
  int64_t J;             // prod_{j != n} I_j
  int64_t Kpre;          // prod_{j<n} I_j (a count; equals strideN unless mode 0 is stored padded)
};

// Build the layout for mode n choosing the split that minimises nL + nU.  With Istore given, X is
// stored with those extents (Istore[j] >= I[j], the extra entries zero) and strides follow them.
ModeLayout make_mode_layout(int N, const int64_t* I, const int32_t* R, int n, const int64_t* Istore = nullptr);
// Host-side offsets for the layout (sizes nL and nU), strides from Istore when given.
void mode_offsets(int N, const int64_t* I, const ModeLayout& L, std::vector<int64_t>& offL,
                  std::vector<int64_t>& offU, const int64_t* Istore = nullptr);

// ---------------------------------------------------------------- kernel launchers (stream-ordered)
// Gamma_k (K1).
void launch_gamma(const double* G, int Rn, int64_t In, int Rn1, double* Gamma, cudaStream_t s);
// C (m x n) = A (m x k) * B (k x n), column-major FP64.
void launch_gemm_f64(int m, int n, int k, const double* A, const double* B, double* C, cudaStream_t s);
// Pi = A B (R_{n+1}^2 x R_n^2, inner dimension k) stored directly as the regrouped S_n (r x r).
void launch_gemm_f64_regroup(int k, const double* A, const double* B, int Rn, int Rn1, double* S, cudaStream_t s);
// S_n regroup of Pi (R_{n+1}^2 x R_n^2) -> S (r x r).
void launch_regroup_S(const double* Pi, int Rn, int Rn1, double* S, cudaStream_t s);
// Chain table: out[l + nPrev * i][x + Ra * y] = sum_c prev[l][x + Ra c] * G[c + Rc (i + I y)]
// (prev == nullptr: out = core slices, Ra = Rc).
void launch_chain_level(const double* prev, int64_t nPrev, int Ra, int Rc, const double* G, int64_t Ii,
                        int Rb, double* out, cudaStream_t s);
// Tables for one mode layout into ltab/utab.
void build_tables(const ModeLayout& L, const double* const* cores, const int64_t* I, const int32_t* R,
                  double* ltab, double* utab, double* scratch, cudaStream_t s);
// Largest level of either table (elements); ltab, utab and scratch each need this many doubles.
int64_t table_level_max_elems(const ModeLayout& L, const int64_t* I, const int32_t* R);

// MTTSP on CUDA cores (any X type): partial sums per block then a fixed-order reduction.
struct MttspSimtArgs {
  const void* X;
  const void* Xlo = nullptr;   // BF16 X only: the lo half of a split-BF16 pair (NULL: none)
  int xt;               // trals_xtype (F64, F32, BF16)
  const double* ltab;
  const double* utab;
  const int64_t* offL;
  const int64_t* offU;
  ModeLayout L;
  double* partials;     // [gridX][I_n * r]
  double* M;            // I_n x r
  int gridX;
  cudaEvent_t ev0 = nullptr;   // optional: recorded directly before / after the contraction kernel
  cudaEvent_t ev1 = nullptr;
};
size_t mttsp_simt_partials_elems(const ModeLayout& L, int gridX);
// FP32-arithmetic CUDA-core MTTSP for the reduced-precision modes: reads FP32 copies of the two
// subchain tables (fl: nL*Rn1*Rs floats, fu: nU*Rs*Rn floats; see launch_tables_to_f32), visits X in
// memory order.  Usable when mttsp_simt_f32_fits(L); grid from mttsp_simt_f32_grid(L).
bool mttsp_simt_f32_fits(const ModeLayout& L);
int mttsp_simt_f32_grid(const ModeLayout& L);
void launch_mttsp_simt_f32(const MttspSimtArgs& a, const float* fl, const float* fu, cudaStream_t s);
void launch_tables_to_f32(const double* a, int64_t na, float* fa, const double* b, int64_t nb, float* fb,
                          cudaStream_t s);
int mttsp_simt_default_grid(const ModeLayout& L);
void launch_mttsp_simt(const MttspSimtArgs& a, cudaStream_t s);

// Reconstruction / explicit residual (same layout as the MTTSP): for each column k,
// xhat(i_n, k) = sum_r Z[i_n, r] G^{!=n}(k)[b, a] with Z the unfolding of core n.
void launch_reconstruct(const ModeLayout& L, const double* ltab, const double* utab, const int64_t* offL,
                        const int64_t* offU, const double* coreN, void* out, int out_t, const void* X, int xt,
                        double* partials, int gridX, cudaStream_t s, bool out_diff = false);
// Sum of `count` partials into out[0] (and out[1] if two interleaved series), fixed order.
void launch_reduce_pairs(const double* partials, int count, double* out, cudaStream_t s);
// Explicit residual with X_hat regenerated in FP32 (reduced-precision modes): converts the two FP64
// subchain tables into `ftab` (ltab_elems + utab_elems floats), then writes per-block
// (|X - X_hat|^2, |X|^2) pairs to partials[2 * gridX].  Shared memory: residual_f32_smem(L) bytes.
size_t residual_f32_smem(const ModeLayout& L);
int residual_f32_grid(const ModeLayout& L);
void launch_residual_f32(const ModeLayout& L, const double* ltab, const double* utab, float* ftab, int64_t ltab_elems,
                         int64_t utab_elems, const int64_t* offL, const int64_t* offU, const double* coreN,
                         const void* X, int xt, double* partials, int gridX, cudaStream_t s, float* Eout = nullptr);

// Layout of a factor buffer `Lmat` (FP64): L (r x r, column-major, lower triangle; zeros above), then
// the r reciprocal diagonal entries 1/L_jj, then the inverses of the 32 x 32 diagonal blocks of L
// (block q covers rows and columns [32q, 32q + 32), identity-padded past r; each column-major, 1024
// doubles), then 1024 doubles of scratch for the blocked factorization.  Every producer of a factor
// (Cholesky, the QR path) fills the first three parts.
constexpr int kSolveBlock = 32;
__host__ __device__ inline size_t lmat_scratch_offset(int r) {
  return (size_t)r * r + r + (size_t)((r + kSolveBlock - 1) / kSolveBlock) * kSolveBlock * kSolveBlock;
}
inline size_t lmat_elems(int r) { return lmat_scratch_offset(r) + (size_t)kSolveBlock * kSolveBlock; }
// Cholesky (K4): factor S (r x r, lower triangle) into Lmat; status on failure.
// Returns the number of kernel launches.
int launch_cholesky(const double* S, double* Lmat, int r, DevStatus* st, const int* sweep_ctr, int mode,
                    cudaStream_t s);
// Whether launch_cholesky takes the blocked, many-SM path for order r (else one CTA on one SM).
bool cholesky_is_blocked(int r);
// The same factor by the blocked, many-SM path (any r).
int launch_cholesky_blocked(const double* S, double* Lmat, int r, DevStatus* st, const int* sweep_ctr, int mode,
                            cudaStream_t s);
// Inverses of the diagonal blocks of L into the third part of Lmat (from L and its reciprocal diagonal).
void launch_chol_block_inverse(double* Lmat, int r, cudaStream_t s);
// Triangular solves with In right-hand sides; writes core layout.
// out[i] = the Cholesky kernel's pivot reciprocal square root of d[i], ref[i] = CUDA's rsqrt(d[i])
void launch_pivot_rsqrt_check(const double* d, int64_t n, double* out, double* ref, cudaStream_t s);
// With G32 set, the core is also stored in FP32 there (R_n x Ist x R_{n+1}, Ist >= In slices; the
// slices past In are left as they are).  part selects the solves: 0 both (Z = M L^{-T} L^{-1}),
// 1 the forward one alone (Z = M L^{-T}), 2 the backward one alone (Z = M L^{-1}).
constexpr int kSolveBoth = 0, kSolveForward = 1, kSolveBackward = 2;
void launch_chol_solve(const double* Lmat, const double* M, int Rn, int64_t In, int Rn1, double* G,
                       DevStatus* st, cudaStream_t s, float* G32 = nullptr, int64_t Ist = 0, int part = kSolveBoth);
// FP32 copy of one core (R_n x In x R_{n+1}) into G32 laid out with Ist >= In slices.
void launch_core_to_f32(const double* G, int Rn, int64_t In, int64_t Ist, int Rn1, float* G32, cudaStream_t s);

// Residual identity (K6): res2 = normX2 - 2<M, Z> + <S, Z^T Z>; Gamma holds the regrouped Z^T Z.
void launch_residual_identity(const double* normX2, const double* M, const double* coreN, const double* S,
                              const double* gammaN, int Rn, int64_t In, int Rn1, double* res_hist,
                              int* sweep_ctr, cudaStream_t s);
// sum of squares of X in FP64 -> partials then reduce
void launch_sumsq(const void* X, int xt, int64_t count, double* partials, int gridX, double* out, cudaStream_t s);
// BF16 quantisation (K7).
// X (element type src_t, extent I0 along mode 0, `rest` = prod of the other extents) to BF16 with
// mode 0 padded to I0p >= I0 with zeros (and, with lo != NULL, the lo halves likewise).
void launch_quantize_padded(const void* src, int src_t, int64_t I0, int64_t I0p, int64_t rest, __nv_bfloat16* hi,
                            __nv_bfloat16* lo, cudaStream_t s);
void launch_quantize(const void* src, int src_t, int64_t count, __nv_bfloat16* hi, __nv_bfloat16* lo,
                     cudaStream_t s);
// FP64 -> FP32 copy (FP32 mode fed with an FP64 X).
void launch_convert_f32(const void* src_f64, int64_t count, float* dst, cudaStream_t s);
void launch_zero_status(DevStatus* st, cudaStream_t s);

// ---------------------------------------------------------------- explicit-subchain Gram (Alg. 1)
struct ExplicitGramSizes {
  int64_t block_rows = 0;   // subchain rows formed per block
  int groups = 0;           // CTAs along the rows (partial Gram matrices)
  size_t A_bytes = 0;       // row-block buffer
  size_t part_elems = 0;    // partial Gram matrices (doubles)
};
ExplicitGramSizes explicit_gram_sizes(const ModeLayout& L, bool fp64);
// S (r x r, full symmetric, column-major) = (G^{!=n}_[2])^T G^{!=n}_[2] with the subchain matrix formed
// explicitly from the two FP64 partial-chain tables (build_tables).  Returns the launch count.
int launch_explicit_gram(const ModeLayout& L, const double* ltab, const double* utab, bool fp64, void* Ablk,
                         double* part, double* S, cudaStream_t s);

// ---------------------------------------------------------------- QR-stabilised solve (Sec. 3.2)
struct QrSizes {
  int64_t B_elems = 0;   // largest chain-step matrix
  int64_t R_elems = 0;   // TSQR leaf factors (each of the two ping-pong buffers)
  int64_t W_elems = 0;   // TSQR merge workspace
};
QrSizes qr_sizes(int N, const int64_t* I, const int32_t* R, int n);
// R factor of G^{!=n}_[2] by recursive structured QR (FP64), delivered as Lmat = R^T (r x r) followed by
// its reciprocal diagonal: the layout launch_chol_solve reads.  Returns the launch count.
int launch_qr_factor(int N, const int64_t* I, const int32_t* R, int n, const double* const* cores, double* B,
                     double* R0, double* R1, double* Wk, double* Lmat, DevStatus* st, const int* sweep_ctr,
                     cudaStream_t s);
void launch_llt(const double* Lmat, int r, double* S, cudaStream_t s);
void launch_transpose(const double* A, int r, double* B, cudaStream_t s);
void launch_axpy(int64_t n, const double* x, double* y, cudaStream_t s);
cudaError_t init_qr_attributes();

// ---------------------------------------------------------------- TR-ALS-QRNE (Alg. 4)
// The whole decomposition by TR-ALS-QRNE (literal = false) or by the literal TR-ALS-QR of Alg. 3 with its
// Multi-TTM (literal = true), in FP64 (X_dev FP64 on the device, cores on the host as in
// trals_decompose).  Synchronous.
trals_status qrne_decompose(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R, const double* X_dev,
                            double* const* cores_host, int sweeps, double* rel_res, bool literal = false);

// ---------------------------------------------------------------- asynchronous plan steps (serving)
// As trals_plan_create / trals_plan_set_cores but without waiting on the stream (host sources may
// be pageable: they are staged before the calls return).
trals_status plan_create_async(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R, const void* X_dev, int xt,
                               const trals_opts* opts, trals_plan** out);
trals_status plan_set_cores_async(trals_plan* p, const double* const* cores_host);
size_t plan_core_elems(const trals_plan* p);
// Enqueue, after the sweeps: (optionally) the explicit residual of the final cores into the last
// history entry, then copies of `sweeps` residuals, all cores (concatenated, core layout) and the
// device status word (sizeof(DevStatus) bytes) to host buffers (pinned, for the copies to be
// asynchronous), and a reset of the status word.
trals_status plan_enqueue_results(trals_plan* p, int sweeps, bool final_explicit, double* res_host,
                                  double* cores_host, void* status_host);
std::string status_message(const void* status_host);
int status_code(const void* status_host);
// One-time kernel attribute setup (dynamic shared memory opt-in); called at context creation.
cudaError_t init_small_attributes();
cudaError_t init_simt_attributes();
cudaError_t init_kernel_attributes();

}  // namespace trals

// ---------------------------------------------------------------- context
struct trals_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  std::string last_error;
  trals::DevStatus* d_status = nullptr;   // per-context device status word
  int* d_zero_ctr = nullptr;              // a device int holding 0 (sweep counter for one-off calls)
  int last_mttsp_path = -1;               // kernel the last trals_mttsp call ran (trals_mttsp_path codes)
  void* cublas = nullptr;                 // cuBLAS handle of the two-stage GEMM MTTSP (created on demand)
};

#define TRALS_CUDA_TRY(ctx, call)                                                        \
  do {                                                                                   \
    cudaError_t e__ = (call);                                                            \
    if (e__ != cudaSuccess) {                                                            \
      if (ctx) (ctx)->last_error = std::string(#call) + ": " + cudaGetErrorString(e__); \
      return e__ == cudaErrorMemoryAllocation ? TRALS_E_OOM : TRALS_E_CUDA;              \
    }                                                                                    \
  } while (0)
