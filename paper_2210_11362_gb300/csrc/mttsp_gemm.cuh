// Two-stage MTTSP through a plain GEMM, for the reduced-precision modes of shapes the tensor-core
// kernel does not take (wide subchain tables: R = 16 makes the stage-1 table 256 columns wide).
#pragma once

#include <vector>

#include "trals_internal.cuh"

namespace trals {

// Stage-1 operand types.
enum { kGemmF32 = 0, kGemmBF16 = 1, kGemmBF16Split = 2 };
// Workspace buffers: the two FP64 subchain tables and their scratch, the GEMM's table (and its lo plane),
// the stage-2 table, T, the stage-2 partial sums, the cuBLAS workspace.
constexpr int kGemmBufs = 9;

// Per-mode plan.  The subchain G^{!=n}(k) = L(l) U(u) (eq. subchain_new) is split so that one of the two
// tables runs over a block of modes that leads X in memory; that block is the GEMM's inner dimension:
//   form 1 (1 <= n <= N-2: the block is modes 0..n-1; n = 0: the block is the trailing modes):
//     T[(i + I l), s + R_s a] = sum_u X(i, l, u) U(u)[s, a],
//     M_n(i)[a + R_n b] = sum_l sum_s L(l)[b, s] T[(i + I l), s + R_s a];
//   form 2 (n = N-1: the block is modes 0..m-1):
//     T[(u + nU i), b + R_{n+1} s] = sum_l X(l, u, i) L(l)[b, s],
//     M_n(i)[a + R_n b] = sum_u sum_s T[(u + nU i), b + R_{n+1} s] U(u)[s, a].
// Stage 1 is one cuBLAS GEMM (FP32, or BF16 operands with FP32 accumulation; the split mode adds the
// product with the table's lo plane), stage 2 a kernel of this library with FP32 partial sums per chunk
// reduced in FP64.
struct GemmMttsp {
  bool valid = false;
  int n = 0, form = 0, xmode = 0;
  ModeLayout L{};
  int64_t K = 0;         // GEMM inner dimension as stored (a padded leading mode 0 included)
  int64_t rowsT = 0;     // rows of T
  int W1 = 0;            // columns of T
  int64_t Irows = 0;     // form 1: stride of l in the rows of T (I_n, or the padded I_0 when n = 0)
  int64_t nOther = 0;    // entries of the stage-2 table
  bool padK = false;     // the GEMM's table runs over a padded mode 0: I0 real, I0st stored
  int64_t I0 = 0, I0st = 0;
  int nchunk = 0;
  int64_t In = 0;
  size_t need[kGemmBufs] = {};   // bytes of each workspace buffer this mode needs
  // workspace, shared by all the modes of a plan (they run one after another on one stream)
  double *ltab64 = nullptr, *utab64 = nullptr, *scr64 = nullptr;
  void *tabK = nullptr, *tabK_lo = nullptr;   // the GEMM's table, converted (entries x W1 as stored)
  float* tabO = nullptr;                       // the stage-2 table in FP32
  float* T = nullptr;
  float* part = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
};

// Whether cuBLAS could be opened (the library itself never links it).
bool gemm_available();
// Geometry of mode n (Ist: X's stored extents; I the real ones) and the workspace it needs (g.need).
// Returns 1 when the shape takes this path: numel >= 2^21 and a stage-1 table 64 to 256 columns wide.
int gemm_mttsp_plan(GemmMttsp& g, int N, const int64_t* I, const int64_t* Ist, const int32_t* R, int n, int xmode);
// Point a planned mode at workspace buffers bufs[kGemmBufs] (each at least the largest need of the
// modes sharing them).
void gemm_mttsp_bind(GemmMttsp& g, void* const* bufs);
// Enqueue M_n (I_n x r, FP64) on s from X (as stored) and the FP64 cores.  Returns the launches of this
// library's kernels, or -1 with ctx->last_error set when cuBLAS fails.
// ev0 / ev1 (optional) are recorded on s directly before the GEMM and after the FP64 reduction.  With
// tables_ready the subchain tables of the current cores are taken as left by gemm_residual_enqueue.
int gemm_mttsp_enqueue(GemmMttsp& g, trals_ctx* ctx, const void* X, double* const* cores, const int64_t* I,
                       const int32_t* R, double* M, cudaStream_t s, cudaEvent_t ev0 = nullptr,
                       cudaEvent_t ev1 = nullptr, bool tables_ready = false);
// The residual tensor E = X - X_hat (FP32, X's layout, unpadded) of the cores, by the same split: with
// P the product of core n and the stage-2 table (P[(i + I l), s + R_s a] = sum_b G_n(i)[a, b] L(l)[b, s]
// in form 1; P[(u + nU i), b + R_{n+1} s] = sum_a U(u)[s, a] G_n(i)[a, b] in form 2), X_hat is the GEMM
// of the GEMM-side table with P, taken with coefficient -1 onto E = X.  FP32 modes only (g.xmode F32,
// no padding); X is FP32 or FP64 (xt).  Returns launches, or -1 with ctx->last_error set.
int gemm_residual_enqueue(GemmMttsp& g, trals_ctx* ctx, const void* X, int xt, double* const* cores, const int64_t* I,
                          const int32_t* R, float* E, cudaStream_t s);
// Create the context's cuBLAS handle ahead of any stream capture; false when cuBLAS is unavailable.
bool gemm_prepare(trals_ctx* ctx);
// Release the context's cuBLAS handle (trals_destroy).
void gemm_release(trals_ctx* ctx);

}  // namespace trals
