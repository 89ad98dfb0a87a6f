// libtrals C ABI: contexts, resident plans and the ALS sweep driver (Alg. 1 sweep order with the
// TR-ALS-NE core update of Alg. 2, lines 6-10), plus the per-step entry points.
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "trals_internal.cuh"
#include "mttsp_tc.cuh"
#include "mttsp_gemm.cuh"
#include "../../include/trals_testing.h"

using namespace trals;

namespace {

constexpr int kResCap = 1 << 14;
// Corrected semi-normal steps after the QR solve.  Each multiplies the solution error by about
// cond(G^{!=n}_[2])^2 u; two steps bring it to the Householder least-squares level for condition
// numbers up to about 1e7 (one step leaves (cond^2 u)^2, e.g. 2e-6 at cond = 3.5e6).
constexpr int kQrRefineSteps = 2;

__global__ void finalize_explicit_residual(const double* red2, double* res_hist, int* sweep_ctr) {
  const int s = *sweep_ctr;
  res_hist[s] = sqrt(fmax(red2[0], 0.0) / red2[1]);
  *sweep_ctr = s + 1;
}

__global__ void set_int_kernel(int* p, int v) { *p = v; }

// Reduced-precision modes without the explicit pass: the residual identity cannot be evaluated to
// the needed accuracy from a BF16 M_N (the subchain table is rounded too), so the sweep records NaN.
__global__ void skip_residual_kernel(double* res_hist, int* sweep_ctr) {
  const int s = *sweep_ctr;
  res_hist[s] = __longlong_as_double(0x7ff8000000000000LL);
  *sweep_ctr = s + 1;
}

// sqrt(|X - X_hat|^2 / |X|^2) into the history entry of the last sweep run
__global__ void finalize_last_residual_kernel(const double* red2, double* res_hist, const int* sweep_ctr) {
  const int s = *sweep_ctr;
  if (s > 0) res_hist[s - 1] = sqrt(fmax(red2[0], 0.0) / red2[1]);
}

// sqrt(|X - X_hat|^2 / |X|^2) of the current cores into *out
__global__ void finalize_ratio_kernel(const double* red2, double* out) { *out = sqrt(fmax(red2[0], 0.0) / red2[1]); }

std::string fmt(const char* f, long long a = 0, long long b = 0, long long c = 0) {
  char buf[256];
  snprintf(buf, sizeof buf, f, a, b, c);
  return buf;
}

trals_status read_status(trals_ctx* ctx) {
  DevStatus st{};
  cudaError_t e = cudaMemcpyAsync(&st, ctx->d_status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    ctx->last_error = std::string("stream error: ") + cudaGetErrorString(e);
    return TRALS_E_CUDA;
  }
  if (st.code != 0) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s at sweep %d, core %d, index %d (value %.6g)",
             st.code == TRALS_E_NOT_SPD ? "non-positive Cholesky pivot"
             : st.code == TRALS_E_NONFINITE ? "non-finite value in a solve"
             : st.code == TRALS_E_TIMEOUT   ? "a bounded wait of the tensor-core kernel gave up"
                                            : "device error",
             st.sweep, st.mode, st.index, st.value);
    ctx->last_error = buf;
    launch_zero_status(ctx->d_status, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    return (trals_status)st.code;
  }
  return TRALS_OK;
}

}  // namespace

// ------------------------------------------------------------------ plan
namespace trals {
trals_status check_shape(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R) {
  if (N < 3 || N > TRALS_MAX_ORDER) {
    ctx->last_error = fmt("order N=%lld outside [3, %lld]", N, TRALS_MAX_ORDER);
    return TRALS_E_ARG;
  }
  if (!I || !R) {
    ctx->last_error = "null shape or rank array";
    return TRALS_E_ARG;
  }
  for (int n = 0; n < N; ++n) {
    if (I[n] < 1 || R[n] < 1 || R[n] > 64) {
      ctx->last_error = fmt("mode %lld: I=%lld R=%lld (need I>=1, 1<=R<=64)", n, I[n], R[n]);
      return TRALS_E_ARG;
    }
  }
  {
    // every size computed from the shape (element counts, table and workspace bytes) stays far from
    // int64 overflow: prod I_n is capped at 2^46 elements, beyond any device memory
    int64_t numel = 1;
    for (int n = 0; n < N; ++n) {
      if (I[n] > ((int64_t)1 << 46) / numel) {
        ctx->last_error = "prod I_n exceeds 2^46 elements";
        return TRALS_E_ARG;
      }
      numel *= I[n];
    }
  }
  for (int n = 0; n < N; ++n) {
    int64_t J = 1;
    for (int j = 0; j < N; ++j)
      if (j != n) J *= I[j];
    const int64_t r = (int64_t)R[n] * R[(n + 1) % N];
    if (r > 256) {
      ctx->last_error = fmt("mode %lld: R_n R_{n+1} = %lld exceeds 256", n, r);
      return TRALS_E_ARG;
    }
    if (J < r) {
      ctx->last_error = fmt("mode %lld: J_n=%lld < R_n R_{n+1}=%lld (underdetermined subproblem)", n, J, r);
      return TRALS_E_ARG;
    }
  }
  return TRALS_OK;
}

cudaError_t init_kernel_attributes() {
  cudaError_t e = init_small_attributes();
  if (e == cudaSuccess) e = init_simt_attributes();
  if (e == cudaSuccess) e = init_tc_attributes();
  if (e == cudaSuccess) e = init_qr_attributes();
  return e;
}
}  // namespace trals

struct trals_plan {
  trals_ctx* ctx = nullptr;
  int N = 0;
  int64_t I[TRALS_MAX_ORDER] = {};
  int32_t R[TRALS_MAX_ORDER] = {};
  const void* X = nullptr;        // caller's X (full precision source)
  int xt = 0;
  const void* Xk = nullptr;       // X as read by the MTTSP (caller's or an owned converted copy)
  const void* Xk_lo = nullptr;    // BF16X3: lo half of the split pair
  int xk_t = 0;
  trals_opts opts{};
  int64_t numel = 0;
  std::vector<void*> allocs;
  double* cores[TRALS_MAX_ORDER] = {};
  double* gam[TRALS_MAX_ORDER] = {};
  double *S = nullptr, *Lmat = nullptr, *M = nullptr, *chainA = nullptr, *chainB = nullptr;
  double *ltab = nullptr, *utab = nullptr, *tscratch = nullptr;
  int64_t* offL[TRALS_MAX_ORDER] = {};
  int64_t* offU[TRALS_MAX_ORDER] = {};
  ModeLayout lay[TRALS_MAX_ORDER];
  // Layout of Xk, the copy the MTTSP reads: in the BF16 mode mode 0 is stored zero-padded to a
  // multiple of 8 (Ist[0]) so every tensor-core geometry meets the 16-byte stride rule of TMA.
  int64_t Ist[TRALS_MAX_ORDER] = {};
  int64_t numel_st = 0;
  ModeLayout layk[TRALS_MAX_ORDER];
  int64_t* offLk[TRALS_MAX_ORDER] = {};
  int64_t* offUk[TRALS_MAX_ORDER] = {};
  int gridX[TRALS_MAX_ORDER] = {};
  double* partials = nullptr;
  double *qrB = nullptr, *qrR0 = nullptr, *qrR1 = nullptr, *qrW = nullptr;   // QR solve workspace
  void* E = nullptr;              // QR solve: residual tensor X - X_hat for the refinement step
  double *dM = nullptr, *dG = nullptr;
  void* Ablk = nullptr;           // explicit-Gram variant: subchain row block
  double* gpart = nullptr;        // explicit-Gram variant: partial Gram matrices
  double* red2 = nullptr;         // [2] explicit residual reduction
  double* normX2 = nullptr;
  double* res_hist = nullptr;
  int* sweep_ctr = nullptr;
  int host_sweeps = 0;
  cudaGraphExec_t gexec = nullptr;
  // The coefficient-matrix branch (Gamma chain or explicit Gram or QR factor, then the Cholesky)
  // depends only on the other cores, so it runs on `side`, concurrently with the MTTSP of the same
  // mode, and joins before the solve.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork[TRALS_MAX_ORDER] = {}, ev_join[TRALS_MAX_ORDER] = {};
  // Gamma-chain prefixes for the next mode, formed on `side2` while the current mode is updated
  cudaStream_t side2 = nullptr;
  cudaEvent_t ev_pre[TRALS_MAX_ORDER] = {};
  cudaEvent_t ev_gam[TRALS_MAX_ORDER] = {};   // Gamma_{n-1} formed on the side stream during mode n
  // the parts of the next mode's tensor-core subchain tables that do not read the core being updated,
  // built on `side3` during the current mode
  cudaStream_t side3 = nullptr;
  cudaEvent_t ev_tcpre[TRALS_MAX_ORDER] = {};
  // S_n formed (structured Gram): the tensor-core MTTSP kernel waits for it, so that the FP64 Gamma and
  // GEMM steps run on the whole GPU instead of the one SM that kernel leaves free
  cudaEvent_t ev_coef[TRALS_MAX_ORDER] = {};
  double *pre[2] = {}, *preA = nullptr, *preB = nullptr;
  // mode 0's prefix Gamma_1 ... Gamma_{N-2}: formed during mode N-1 for the next sweep (and by every run's
  // prologue), in a buffer of its own since mode N-1 may be reading pre[(N-1) % 2] = pre[0] meanwhile
  double* pre0 = nullptr;
  double *ltab2 = nullptr, *utab2 = nullptr, *tscratch2 = nullptr;   // explicit Gram on the side branch
  int launches = 0;
  TcPlan tc[TRALS_MAX_ORDER];
  bool use_tc[TRALS_MAX_ORDER] = {};
  // two-stage GEMM MTTSP for modes without a tensor-core geometry (reduced modes): of Xk, and of the
  // FP32 residual tensor E of the QR solve's refinement
  GemmMttsp gemm[TRALS_MAX_ORDER];
  GemmMttsp gemmE[TRALS_MAX_ORDER];
  // FP32 copies of the cores for the tensor-core subchain tables (core 0 with Ist[0] slices, the padded
  // ones zero): refreshed at the start of every run and by each core update inside the sweep
  float* c32buf = nullptr;
  float* c32[TRALS_MAX_ORDER] = {};
  // set when the cores may have changed outside a run (set from the host, or their device pointer
  // handed out): the next run refreshes the FP32 copies and mode 0's prepared inputs first
  bool prep_stale = true;
  // Workspace is allocated stream-ordered (cudaMallocAsync / cudaFreeAsync on the context's
  // stream), so creating and destroying plans never synchronises the whole device: plans of other
  // streams keep running.  In the counting pass nothing is allocated and `bytes` sums the sizes.
  bool counting = false;
  size_t bytes = 0;

  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    const size_t b = (std::max<size_t>(count, 1) * sizeof(T) + 255) & ~(size_t)255;
    if (counting) {
      *p = reinterpret_cast<T*>((uintptr_t(1) << 40) + bytes);   // never dereferenced
      bytes += b;
      return cudaSuccess;
    }
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, b, ctx->stream);
    if (e == cudaSuccess) {
      allocs.push_back(q);
      *p = static_cast<T*>(q);
      bytes += b;
    }
    return e;
  }
};

namespace {

// Structured coefficient matrix S_n (Alg. 2 line 6): Pi_n = Gamma_{n+1} ... Gamma_{n-1}, regrouped.  With
// `pre` set, it holds Gamma_{n+1} ... Gamma_{n-2} (formed while mode n-1 was being updated, from cores
// that update did not touch), so only the product with the freshly updated Gamma_{n-1} remains.
int enqueue_coef(const int N, const int32_t* R, double* const* gam, int n, double* chainA, double* chainB, double* S,
                 cudaStream_t s, const double* pre = nullptr) {
  if (pre) {
    const int c = (n - 1 + N) % N;
    launch_gemm_f64_regroup(R[c] * R[c], pre, gam[c], R[n], R[(n + 1) % N], S, s);
    return 1;
  }
  int launches = 0;
  const int c0 = (n + 1) % N;
  const double* cur = gam[c0];
  int rows = R[c0] * R[c0];
  double* bufs[2] = {chainA, chainB};
  for (int t = 2; t < N; ++t) {
    const int c = (n + t) % N;
    const int k = R[c] * R[c];
    const int cols = R[(c + 1) % N] * R[(c + 1) % N];
    double* out = bufs[t % 2];
    launch_gemm_f64(rows, cols, k, cur, gam[c], out, s);
    ++launches;
    cur = out;
  }
  launch_regroup_S(cur, R[n], R[(n + 1) % N], S, s);
  return launches + 1;
}

// P_n = Gamma_{n+1} ... Gamma_{n-2} (N - 2 factors, N >= 4) into `out`.
int enqueue_prefix(const int N, const int32_t* R, double* const* gam, int n, double* tmpA, double* tmpB, double* out,
                   cudaStream_t s) {
  const int c0 = (n + 1) % N;
  const double* cur = gam[c0];
  const int rows = R[c0] * R[c0];
  double* bufs[2] = {tmpA, tmpB};
  int launches = 0;
  for (int t = 2; t <= N - 2; ++t) {
    const int c = (n + t) % N;
    double* dst = (t == N - 2) ? out : bufs[t % 2];
    launch_gemm_f64(rows, R[(c + 1) % N] * R[(c + 1) % N], R[c] * R[c], cur, gam[c], dst, s);
    cur = dst;
    ++launches;
  }
  return launches;
}

// tc_pre_done: the tensor-core tables' first part was enqueued already (tc_enqueue_pre on side3)
int enqueue_mttsp(trals_plan* p, int n, cudaStream_t s, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr,
                  bool tc_pre_done = false, cudaEvent_t before_kernel = nullptr) {
  const ModeLayout& L = p->layk[n];
  int launches = 0;
  if (p->use_tc[n]) {
    if (tc_pre_done)
      launches += tc_enqueue_main(p->tc[n], p->cores, p->M, s, ev0, ev1, p->c32, before_kernel);
    else
      launches += tc_enqueue(p->tc[n], p->Xk, p->cores, p->M, s, ev0, ev1);
    return launches;
  }
  if (p->gemm[n].valid) {
    const int l = gemm_mttsp_enqueue(p->gemm[n], p->ctx, p->Xk, p->cores, p->I, p->R, p->M, s, ev0, ev1);
    if (l >= 0) return launches + l;
    p->gemm[n].valid = false;   // cuBLAS failed (reported in last_error): the CUDA-core kernel below
  }
  build_tables(L, p->cores, p->I, p->R, p->ltab, p->utab, p->tscratch, s);
  launches += L.N - 1;
  if (p->opts.mode != TRALS_MODE_FP64 && mttsp_simt_f32_fits(L)) {
    // reduced-precision modes: FP32 arithmetic (the tables' FP32 copies go to the scratch buffer)
    const int64_t nl = L.nL * L.Rn1 * L.Rs, nu = L.nU * L.Rs * L.Rn;
    float* fl = reinterpret_cast<float*>(p->tscratch);
    launch_tables_to_f32(p->ltab, nl, fl, p->utab, nu, fl + nl, s);
    MttspSimtArgs a;
    a.X = p->Xk;
    a.Xlo = p->Xk_lo;
    a.xt = p->xk_t;
    a.offL = p->offLk[n];
    a.offU = p->offUk[n];
    a.L = L;
    a.partials = p->partials;
    a.M = p->M;
    a.gridX = mttsp_simt_f32_grid(L);
    a.ev0 = ev0;
    a.ev1 = ev1;
    launch_mttsp_simt_f32(a, fl, fl + nl, s);
    return launches + 3;
  }
  MttspSimtArgs a;
  a.X = p->Xk;
  a.Xlo = p->Xk_lo;
  a.xt = p->xk_t;
  a.ltab = p->ltab;
  a.utab = p->utab;
  a.offL = p->offLk[n];
  a.offU = p->offUk[n];
  a.L = L;
  a.partials = p->partials;
  a.M = p->M;
  a.gridX = p->gridX[n];
  a.ev0 = ev0;
  a.ev1 = ev1;
  launch_mttsp_simt(a, s);
  return launches + 2;
}

// Explicit residual pass of the current cores against the caller's full-precision X (Sec. 4): FP64
// reconstruction in the FP64 mode, FP32 reconstruction in the reduced-precision modes.  Leaves
// (|X - X_hat|^2, |X|^2) in p->red2.  Returns the number of launches.
int enqueue_explicit_residual(trals_plan* p, cudaStream_t s) {
  const int N = p->N;
  const int n = N - 1;
  const ModeLayout& L = p->lay[n];
  build_tables(L, p->cores, p->I, p->R, p->ltab, p->utab, p->tscratch, s);
  int gridX;
  if (p->opts.mode == TRALS_MODE_FP64) {
    gridX = p->gridX[n];
    launch_reconstruct(L, p->ltab, p->utab, p->offL[n], p->offU[n], p->cores[n], nullptr, TRALS_X_F64, p->X, p->xt,
                       p->partials, gridX, s);
  } else {
    gridX = residual_f32_grid(L);
    launch_residual_f32(L, p->ltab, p->utab, reinterpret_cast<float*>(p->tscratch), L.nL * L.Rn1 * L.Rs,
                        L.nU * L.Rs * L.Rn, p->offL[n], p->offU[n], p->cores[n], p->X, p->xt, p->partials, gridX,
                        s);
  }
  launch_reduce_pairs(p->partials, gridX, p->red2, s);
  return (N - 1) + (p->opts.mode == TRALS_MODE_FP64 ? 1 : 2) + 1;
}

// One corrected semi-normal step after the QR solve (Bjorck, CSNE): with the residual tensor
// E = X - TR(cores) taken against the caller's full-precision X, dM = E_[n] G^{!=n}_[2] (an MTTSP of
// E) and G_{n(2)} += dM R^{-1} R^{-T}.  In the reduced-precision modes this also lifts the BF16 or
// FP32 right-hand side to the accuracy of the source X.
int enqueue_qr_refinement(trals_plan* p, int n, cudaStream_t s) {
  const ModeLayout& L = p->lay[n];
  const int N = p->N;
  int launches = 0;
  bool done = false;
  if (p->opts.mode != TRALS_MODE_FP64 && p->gemmE[n].valid) {
    // the residual tensor and its MTTSP by the two-stage GEMM route (the subchain tables built once)
    const int r1 = gemm_residual_enqueue(p->gemmE[n], p->ctx, p->X, p->xt, p->cores, p->I, p->R,
                                         static_cast<float*>(p->E), s);
    const int r2 = r1 >= 0 ? gemm_mttsp_enqueue(p->gemmE[n], p->ctx, p->E, p->cores, p->I, p->R, p->dM, s, nullptr,
                                                nullptr, true)
                           : -1;
    if (r1 >= 0 && r2 >= 0) {
      launches += r1 + r2;
      done = true;
    } else {
      p->gemmE[n].valid = false;   // cuBLAS failed (reported in last_error): the CUDA-core kernels below
    }
  }
  if (!done) {
    launches += N - 1;
    build_tables(L, p->cores, p->I, p->R, p->ltab, p->utab, p->tscratch, s);
    MttspSimtArgs a;
    a.X = p->E;
    a.ltab = p->ltab;
    a.utab = p->utab;
    a.offL = p->offL[n];
    a.offU = p->offU[n];
    a.L = L;
    a.partials = p->partials;
    a.M = p->dM;
    if (p->opts.mode == TRALS_MODE_FP64) {
      launch_reconstruct(L, p->ltab, p->utab, p->offL[n], p->offU[n], p->cores[n], p->E, TRALS_X_F64, p->X, p->xt,
                         nullptr, p->gridX[n], s, true);
      a.xt = TRALS_X_F64;
      a.gridX = p->gridX[n];
      launch_mttsp_simt(a, s);
      launches += 3;
    } else {
      const int64_t nl = L.nL * L.Rn1 * L.Rs, nu = L.nU * L.Rs * L.Rn;
      float* fl = reinterpret_cast<float*>(p->tscratch);
      launch_residual_f32(L, p->ltab, p->utab, fl, nl, nu, p->offL[n], p->offU[n], p->cores[n], p->X, p->xt,
                          p->partials, residual_f32_grid(L), s, static_cast<float*>(p->E));
      a.xt = TRALS_X_F32;
      if (mttsp_simt_f32_fits(L)) {
        a.gridX = mttsp_simt_f32_grid(L);
        launch_mttsp_simt_f32(a, fl, fl + nl, s);   // the tables' FP32 copies are still in the scratch
      } else {
        a.gridX = p->gridX[n];
        launch_mttsp_simt(a, s);
      }
      launches += 4;
    }
  }
  launch_chol_solve(p->Lmat, p->dM, L.Rn, L.In, L.Rn1, p->dG, p->ctx->d_status, s);
  launch_axpy((int64_t)L.Rn * L.In * L.Rn1, p->dG, p->cores[n], s);
  return launches + 2;
}

int enqueue_sweep(trals_plan* p) {
  cudaStream_t s = p->ctx->stream;
  int launches = 0;
  const int N = p->N;
  const bool qr = p->opts.solver == TRALS_SOLVE_QR;
  const bool gam_last_deferred = p->opts.mode != TRALS_MODE_FP64;
  for (int n = 0; n < N; ++n) {
    const int Rn = p->R[n], Rn1 = p->R[(n + 1) % N];
    // fork: the coefficient-matrix branch on the side stream
    cudaStream_t b = p->side;
    cudaEventRecord(p->ev_fork[n], s);
    cudaStreamWaitEvent(b, p->ev_fork[n], 0);
    // Gamma of the core the previous mode updated, on the side stream: only the coefficient branches
    // read it, so the MTTSP of this mode does not wait for it.  Mode 0 forms the last core's, left by
    // the previous sweep, except in the FP64 mode, whose residual identity needs it at the end of
    // the sweep itself.
    if (n >= 1 || gam_last_deferred) {
      const int c = (n + N - 1) % N;
      launch_gamma(p->cores[c], p->R[c], p->I[c], Rn, p->gam[c], b);
      ++launches;
    }
    cudaEventRecord(p->ev_gam[n], b);
    cudaEvent_t coef_ev = nullptr;
    // the next mode's tensor-core tables, all but the link through core n (updated below); after the
    // last mode, mode 0's for the next sweep (cores 1 .. N-2 do not change before it)
    const int nx = (n + 1) % N;
    if (p->use_tc[nx]) {
      cudaStreamWaitEvent(p->side3, p->ev_fork[n], 0);
      launches += tc_enqueue_pre(p->tc[nx], p->cores, p->side3, p->c32);
      cudaEventRecord(p->ev_tcpre[nx], p->side3);
    }
    if (qr) {
      // R factor of G^{!=n}_[2] by structured QR; L = R^T replaces the Cholesky factor of S_n
      launches += launch_qr_factor(N, p->I, p->R, n, p->cores, p->qrB, p->qrR0, p->qrR1, p->qrW, p->Lmat,
                                   p->ctx->d_status, p->sweep_ctr, b);
    } else {
      if (p->opts.gram == TRALS_GRAM_EXPLICIT) {
        // regular TR-ALS normal equations: S_n from the explicitly formed subchain matrix
        build_tables(p->lay[n], p->cores, p->I, p->R, p->ltab2, p->utab2, p->tscratch2, b);
        launches += (N - 1) + launch_explicit_gram(p->lay[n], p->ltab2, p->utab2, p->opts.mode == TRALS_MODE_FP64,
                                                   p->Ablk, p->gpart, p->S, b);
      } else if (p->pre[0]) {
        // prefix formed during mode n-1 (mode 0's: during the previous sweep's last mode, or the prologue)
        if (n >= 1) cudaStreamWaitEvent(b, p->ev_pre[n], 0);
        launches += enqueue_coef(N, p->R, p->gam, n, p->chainA, p->chainB, p->S, b, n == 0 ? p->pre0 : p->pre[n % 2]);
        coef_ev = p->ev_coef[n];
      } else {
        launches += enqueue_coef(N, p->R, p->gam, n, p->chainA, p->chainB, p->S, b);
        coef_ev = p->ev_coef[n];
      }
      if (coef_ev) cudaEventRecord(coef_ev, b);
      launches += launch_cholesky(p->S, p->Lmat, Rn * Rn1, p->ctx->d_status, p->sweep_ctr, n, b);
    }
    cudaEventRecord(p->ev_join[n], b);
    if (p->pre[0]) {
      // prefix of the next mode: Gamma_{n+2} ... Gamma_{n-1}, none of which this update changes (after the
      // last mode: mode 0's prefix Gamma_1 ... Gamma_{N-2} for the next sweep)
      cudaStream_t c = p->side2;
      cudaStreamWaitEvent(c, p->ev_gam[n], 0);   // reads Gamma_{n-1}
      launches += enqueue_prefix(N, p->R, p->gam, nx, p->preA, p->preB, nx == 0 ? p->pre0 : p->pre[nx % 2], c);
      cudaEventRecord(p->ev_pre[nx], c);
    }
    // the MTTSP on the main stream, then join
    const bool tc_pre = p->use_tc[n];
    if (tc_pre && n >= 1) cudaStreamWaitEvent(s, p->ev_tcpre[n], 0);   // mode 0's came before this sweep
    launches += enqueue_mttsp(p, n, s, nullptr, nullptr, tc_pre, tc_pre ? coef_ev : nullptr);
    cudaStreamWaitEvent(s, p->ev_join[n], 0);
    launch_chol_solve(p->Lmat, p->M, Rn, p->I[n], Rn1, p->cores[n], p->ctx->d_status, s,
                      qr ? nullptr : p->c32[n], p->Ist[n]);
    ++launches;
    if (qr) {
      for (int step = 0; step < kQrRefineSteps; ++step) launches += enqueue_qr_refinement(p, n, s);
      if (p->c32buf) {
        launch_core_to_f32(p->cores[n], Rn, p->I[n], p->Ist[n], Rn1, p->c32[n], s);
        ++launches;
      }
    }
  }
  // Gamma of the last core on the main stream when the residual identity below reads it (else the next
  // sweep's mode 0 forms it)
  if (!gam_last_deferred) {
    launch_gamma(p->cores[N - 1], p->R[N - 1], p->I[N - 1], p->R[0], p->gam[N - 1], s);
    ++launches;
  }
  // join what was prepared for the next sweep's mode 0
  if (p->pre[0]) cudaStreamWaitEvent(s, p->ev_pre[0], 0);
  if (p->use_tc[0]) cudaStreamWaitEvent(s, p->ev_tcpre[0], 0);
  if (qr) {
    // the residual identity needs S_N = L L^T
    launch_llt(p->Lmat, p->R[N - 1] * p->R[0], p->S, s);
    ++launches;
  }
  const int n = N - 1;
  if (p->opts.explicit_residual) {
    launches += enqueue_explicit_residual(p, s);
    finalize_explicit_residual<<<1, 1, 0, s>>>(p->red2, p->res_hist, p->sweep_ctr);
    launches += 1;
  } else if (p->opts.mode == TRALS_MODE_FP64) {
    launch_residual_identity(p->normX2, p->M, p->cores[n], p->S, p->gam[n], p->R[n], p->I[n], p->R[0], p->res_hist,
                             p->sweep_ctr, s);
    launches += 1;
  } else {
    skip_residual_kernel<<<1, 1, 0, s>>>(p->res_hist, p->sweep_ctr);
    launches += 1;
  }
  return launches;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* trals_version(void) { return "libtrals 0.1 (sm_103a)"; }

trals_status trals_create(trals_ctx** out, int device, void* cuda_stream) {
  if (!out) return TRALS_E_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return TRALS_E_ARG;
  trals_ctx* ctx = new trals_ctx();
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      e = cudaStreamCreate(&ctx->stream);
      ctx->owns_stream = true;
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, sizeof(DevStatus), ctx->stream);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_zero_ctr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_zero_ctr, 0, sizeof(int), ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = init_kernel_attributes();
  if (e != cudaSuccess) {
    trals_destroy(ctx);
    return TRALS_E_CUDA;
  }
  *out = ctx;
  return TRALS_OK;
}

void trals_destroy(trals_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_zero_ctr) cudaFree(ctx->d_zero_ctr);
  gemm_release(ctx);
  if (ctx->owns_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* trals_last_error(const trals_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

void trals_plan_destroy(trals_plan* p) {
  if (!p) return;
  if (!p->counting) {
    if (p->ctx && p->ctx->stream) cudaStreamSynchronize(p->ctx->stream);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    for (int n = 0; n < p->N; ++n) tc_destroy(p->tc[n]);
    for (void* q : p->allocs) cudaFreeAsync(q, p->ctx->stream);
    for (int n = 0; n < TRALS_MAX_ORDER; ++n) {
      if (p->ev_fork[n]) cudaEventDestroy(p->ev_fork[n]);
      if (p->ev_join[n]) cudaEventDestroy(p->ev_join[n]);
      if (p->ev_pre[n]) cudaEventDestroy(p->ev_pre[n]);
      if (p->ev_gam[n]) cudaEventDestroy(p->ev_gam[n]);
      if (p->ev_tcpre[n]) cudaEventDestroy(p->ev_tcpre[n]);
      if (p->ev_coef[n]) cudaEventDestroy(p->ev_coef[n]);
    }
    if (p->side) {
      cudaStreamSynchronize(p->side);
      cudaStreamDestroy(p->side);
    }
    if (p->side2) {
      cudaStreamSynchronize(p->side2);
      cudaStreamDestroy(p->side2);
    }
    if (p->side3) {
      cudaStreamSynchronize(p->side3);
      cudaStreamDestroy(p->side3);
    }
  }
  delete p;
}

}  // extern "C"

namespace {

// Builds a plan, or with `counting` only sums the bytes its workspace needs (*count_out) without
// allocating, copying or launching anything.
trals_status plan_build(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R, const void* X_dev, int xt,
                        const trals_opts* opts, bool counting, size_t* count_out, trals_plan** out,
                        bool sync = true) {
  if (!ctx || (!out && !counting)) return TRALS_E_ARG;
  if (out) *out = nullptr;
  trals_status st = check_shape(ctx, N, I, R);
  if (st != TRALS_OK) return st;
  if (!X_dev) {
    ctx->last_error = "null X";
    return TRALS_E_ARG;
  }
  trals_opts o = opts ? *opts : trals_opts{TRALS_MODE_FP64, TRALS_SOLVE_CHOL, TRALS_GRAM_STRUCTURED, 0};
  if (o.mode < TRALS_MODE_FP64 || o.mode > TRALS_MODE_BF16X2 || xt < TRALS_X_F64 || xt > TRALS_X_BF16) {
    ctx->last_error = "unknown mode or X type";
    return TRALS_E_ARG;
  }
  if ((o.solver != TRALS_SOLVE_CHOL && o.solver != TRALS_SOLVE_QR) ||
      (o.gram != TRALS_GRAM_STRUCTURED && o.gram != TRALS_GRAM_EXPLICIT)) {
    ctx->last_error = "unknown solver or gram option";
    return TRALS_E_ARG;
  }
  if (o.mode == TRALS_MODE_FP64 && xt != TRALS_X_F64) {
    ctx->last_error = "FP64 mode needs an FP64 X";
    return TRALS_E_ARG;
  }
  if (o.mode == TRALS_MODE_FP32 && xt == TRALS_X_BF16) {
    ctx->last_error = "FP32 mode needs an FP32 or FP64 X";
    return TRALS_E_ARG;
  }
  if (o.mode == TRALS_MODE_BF16X3 && xt == TRALS_X_BF16) {
    ctx->last_error = "BF16X3 mode needs an FP32 or FP64 X (to split into hi/lo)";
    return TRALS_E_ARG;
  }
  cudaSetDevice(ctx->device);
  trals_plan* p = new trals_plan();
  p->ctx = ctx;
  p->counting = counting;
  p->N = N;
  for (int n = 0; n < N; ++n) {
    p->I[n] = I[n];
    p->R[n] = R[n];
  }
  p->X = X_dev;
  p->xt = xt;
  p->opts = o;
  p->numel = 1;
  for (int n = 0; n < N; ++n) p->numel *= I[n];
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaSuccess;
#define PLAN_TRY(call)                                                      \
  do {                                                                      \
    e = (call);                                                             \
    if (e != cudaSuccess) {                                                 \
      ctx->last_error = std::string(#call) + ": " + cudaGetErrorString(e);  \
      trals_plan_destroy(p);                                                \
      return e == cudaErrorMemoryAllocation ? TRALS_E_OOM : TRALS_E_CUDA;   \
    }                                                                       \
  } while (0)

  for (int n = 0; n < N; ++n) p->Ist[n] = I[n];
  if (o.mode != TRALS_MODE_FP64 && o.mode != TRALS_MODE_FP32 && I[0] % 8 != 0) p->Ist[0] = (I[0] + 7) / 8 * 8;
  p->numel_st = p->numel / I[0] * p->Ist[0];
  const bool padded = p->Ist[0] != I[0];
  int maxR2 = 0, maxr = 0;
  int64_t maxMr = 0, maxTab = 0;
  size_t maxPart = 0;
  for (int n = 0; n < N; ++n) {
    const int Rn = R[n], Rn1 = R[(n + 1) % N];
    PLAN_TRY(p->alloc(&p->cores[n], (size_t)Rn * I[n] * Rn1));
    PLAN_TRY(p->alloc(&p->gam[n], (size_t)Rn * Rn * Rn1 * Rn1));
    maxR2 = std::max(maxR2, Rn * Rn);
    maxr = std::max(maxr, Rn * Rn1);
    maxMr = std::max<int64_t>(maxMr, I[n] * Rn * Rn1);
    p->lay[n] = make_mode_layout(N, I, R, n);
    maxTab = std::max<int64_t>(maxTab, table_level_max_elems(p->lay[n], I, R));
    p->gridX[n] = mttsp_simt_default_grid(p->lay[n]);
    maxPart = std::max(maxPart, mttsp_simt_partials_elems(p->lay[n], p->gridX[n]));
    maxPart = std::max(maxPart, (size_t)2 * p->gridX[n]);
    if (o.mode != TRALS_MODE_FP64)
      maxPart = std::max(maxPart, mttsp_simt_partials_elems(p->lay[n], mttsp_simt_f32_grid(p->lay[n])));
    std::vector<int64_t> offL, offU;
    mode_offsets(N, I, p->lay[n], offL, offU);
    PLAN_TRY(p->alloc(&p->offL[n], offL.size()));
    PLAN_TRY(p->alloc(&p->offU[n], offU.size()));
    if (!counting) {
      // pageable sources: staged before the call returns
      PLAN_TRY(cudaMemcpyAsync(p->offL[n], offL.data(), offL.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
      PLAN_TRY(cudaMemcpyAsync(p->offU[n], offU.data(), offU.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }
    p->layk[n] = make_mode_layout(N, I, R, n, p->Ist);
    if (padded) {
      std::vector<int64_t> kL, kU;
      mode_offsets(N, I, p->layk[n], kL, kU, p->Ist);
      PLAN_TRY(p->alloc(&p->offLk[n], kL.size()));
      PLAN_TRY(p->alloc(&p->offUk[n], kU.size()));
      if (!counting) {
        PLAN_TRY(cudaMemcpyAsync(p->offLk[n], kL.data(), kL.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        PLAN_TRY(cudaMemcpyAsync(p->offUk[n], kU.data(), kU.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
      }
    } else {
      p->offLk[n] = p->offL[n];
      p->offUk[n] = p->offU[n];
    }
  }
  PLAN_TRY(p->alloc(&p->S, (size_t)maxr * maxr));
  PLAN_TRY(p->alloc(&p->Lmat, lmat_elems(maxr)));   // L, its reciprocal diagonal, diagonal-block inverses
  PLAN_TRY(p->alloc(&p->chainA, (size_t)maxR2 * maxR2));
  PLAN_TRY(p->alloc(&p->chainB, (size_t)maxR2 * maxR2));
  if (N >= 4 && o.solver == TRALS_SOLVE_CHOL && o.gram == TRALS_GRAM_STRUCTURED) {
    PLAN_TRY(p->alloc(&p->pre[0], (size_t)maxR2 * maxR2));
    PLAN_TRY(p->alloc(&p->pre[1], (size_t)maxR2 * maxR2));
    PLAN_TRY(p->alloc(&p->pre0, (size_t)maxR2 * maxR2));
    PLAN_TRY(p->alloc(&p->preA, (size_t)maxR2 * maxR2));
    PLAN_TRY(p->alloc(&p->preB, (size_t)maxR2 * maxR2));
  }
  PLAN_TRY(p->alloc(&p->M, (size_t)maxMr));
  PLAN_TRY(p->alloc(&p->ltab, (size_t)maxTab));
  PLAN_TRY(p->alloc(&p->utab, (size_t)maxTab));
  PLAN_TRY(p->alloc(&p->tscratch, (size_t)maxTab));
  PLAN_TRY(p->alloc(&p->partials, std::max<size_t>(maxPart, 2 * 1024)));
  if (o.solver == TRALS_SOLVE_QR) {
    QrSizes qz;
    for (int n = 0; n < N; ++n) {
      const QrSizes z = qr_sizes(N, I, R, n);
      qz.B_elems = std::max(qz.B_elems, z.B_elems);
      qz.R_elems = std::max(qz.R_elems, z.R_elems);
      qz.W_elems = std::max(qz.W_elems, z.W_elems);
    }
    PLAN_TRY(p->alloc(&p->qrB, (size_t)qz.B_elems));
    PLAN_TRY(p->alloc(&p->qrR0, (size_t)qz.R_elems));
    PLAN_TRY(p->alloc(&p->qrR1, (size_t)qz.R_elems));
    PLAN_TRY(p->alloc(&p->qrW, (size_t)std::max<int64_t>(qz.W_elems, 1)));
    unsigned char* e8 = nullptr;
    PLAN_TRY(p->alloc(&e8, (size_t)p->numel * (o.mode == TRALS_MODE_FP64 ? 8 : 4)));
    p->E = e8;
    PLAN_TRY(p->alloc(&p->dM, (size_t)maxMr));
    int64_t maxCore = 0;
    for (int n = 0; n < N; ++n) maxCore = std::max<int64_t>(maxCore, (int64_t)R[n] * I[n] * R[(n + 1) % N]);
    PLAN_TRY(p->alloc(&p->dG, (size_t)maxCore));
  }
  if (o.gram == TRALS_GRAM_EXPLICIT) {
    size_t ab = 0, pe = 0;
    for (int n = 0; n < N; ++n) {
      const ExplicitGramSizes z = explicit_gram_sizes(p->lay[n], o.mode == TRALS_MODE_FP64);
      ab = std::max(ab, z.A_bytes);
      pe = std::max(pe, z.part_elems);
    }
    unsigned char* a = nullptr;
    PLAN_TRY(p->alloc(&a, ab));
    p->Ablk = a;
    PLAN_TRY(p->alloc(&p->gpart, pe));
    PLAN_TRY(p->alloc(&p->ltab2, (size_t)maxTab));
    PLAN_TRY(p->alloc(&p->utab2, (size_t)maxTab));
    PLAN_TRY(p->alloc(&p->tscratch2, (size_t)maxTab));
  }
  PLAN_TRY(p->alloc(&p->red2, 2));
  PLAN_TRY(p->alloc(&p->normX2, 1));
  PLAN_TRY(p->alloc(&p->res_hist, kResCap));
  PLAN_TRY(p->alloc(&p->sweep_ctr, 1));
  if (!counting) PLAN_TRY(cudaMemsetAsync(p->sweep_ctr, 0, sizeof(int), s));

  // X as the MTTSP reads it (quantised once, K7), and |X|^2 from the full-precision source.
  p->Xk = X_dev;
  p->xk_t = xt;
  if ((o.mode == TRALS_MODE_BF16 || o.mode == TRALS_MODE_BF16X2) && (xt != TRALS_X_BF16 || padded)) {
    __nv_bfloat16* q = nullptr;
    PLAN_TRY(p->alloc(&q, (size_t)p->numel_st));
    if (!counting) {
      if (padded)
        launch_quantize_padded(X_dev, xt, I[0], p->Ist[0], p->numel / I[0], q, nullptr, s);
      else
        launch_quantize(X_dev, xt, p->numel, q, nullptr, s);
    }
    p->Xk = q;
    p->xk_t = TRALS_X_BF16;
  } else if (o.mode == TRALS_MODE_BF16X3) {
    // hi and lo planes, each in the (padded) layout the MTTSP reads
    __nv_bfloat16* q = nullptr;
    PLAN_TRY(p->alloc(&q, (size_t)p->numel_st * 2));
    if (!counting) launch_quantize_padded(X_dev, xt, I[0], p->Ist[0], p->numel / I[0], q, q + p->numel_st, s);
    p->Xk = q;
    p->Xk_lo = q + p->numel_st;
    p->xk_t = TRALS_X_BF16;
  } else if (o.mode == TRALS_MODE_FP32 && xt == TRALS_X_F64) {
    float* q = nullptr;
    PLAN_TRY(p->alloc(&q, (size_t)p->numel));
    if (!counting) launch_convert_f32(X_dev, p->numel, q, s);
    p->Xk = q;
    p->xk_t = TRALS_X_F32;
  }
  if (!counting) {
    const int g = 152 * 4;
    launch_sumsq(X_dev, xt, p->numel, p->partials, g, p->normX2, s);
  }
  // tensor-core MTTSP plans for the reduced-precision modes
  for (int n = 0; n < N; ++n) {
    p->use_tc[n] = false;
    if (o.mode != TRALS_MODE_FP64) {
      // the blocked Cholesky's panel kernels run beside this MTTSP: leave them SMs (its factor kernels
      // use up to 16 CTAs); the one-CTA Cholesky needs one
      const bool blocked = o.solver == TRALS_SOLVE_CHOL && cholesky_is_blocked(R[n] * R[(n + 1) % N]);
      const int ok = tc_plan(p->tc[n], N, p->Ist, R, n, o.mode, p->Xk, p->numel_st, &e, s,
                             counting ? &p->bytes : nullptr, I[0], p->Xk_lo, blocked ? 17 : 1);
      if (e != cudaSuccess) PLAN_TRY(e);
      p->use_tc[n] = ok != 0;
      if (ok && !counting) {
        tc_set_status(p->tc[n], ctx->d_status);
        p->bytes += p->tc[n].bytes;
      }
    }
  }
  // the two-stage GEMM MTTSP where no tensor-core geometry applies (FP32, BF16 and BF16X2 modes; the QR
  // solve's refinement reads the FP32 residual tensor), all its modes on one shared workspace
  if (o.mode == TRALS_MODE_FP32 || o.mode == TRALS_MODE_BF16 || o.mode == TRALS_MODE_BF16X2) {
    const int xm = o.mode == TRALS_MODE_FP32 ? kGemmF32 : o.mode == TRALS_MODE_BF16 ? kGemmBF16 : kGemmBF16Split;
    bool any = false;
    for (int n = 0; n < N; ++n) {
      if (!p->use_tc[n]) any |= gemm_mttsp_plan(p->gemm[n], N, I, p->Ist, R, n, xm) != 0;
      if (o.solver == TRALS_SOLVE_QR) any |= gemm_mttsp_plan(p->gemmE[n], N, I, I, R, n, kGemmF32) != 0;
    }
    if (any && !counting && !gemm_prepare(ctx)) {
      for (int n = 0; n < N; ++n) p->gemm[n].valid = p->gemmE[n].valid = false;
      any = false;
    }
    if (any) {
      size_t need[kGemmBufs] = {};
      for (int n = 0; n < N; ++n)
        for (const GemmMttsp* g : {&p->gemm[n], &p->gemmE[n]})
          if (g->valid)
            for (int k = 0; k < kGemmBufs; ++k) need[k] = std::max(need[k], g->need[k]);
      void* bufs[kGemmBufs] = {};
      for (int k = 0; k < kGemmBufs; ++k) {
        unsigned char* b = nullptr;
        if (need[k]) PLAN_TRY(p->alloc(&b, need[k]));
        bufs[k] = b;
      }
      for (int n = 0; n < N; ++n) {
        if (p->gemm[n].valid) gemm_mttsp_bind(p->gemm[n], bufs);
        if (p->gemmE[n].valid) gemm_mttsp_bind(p->gemmE[n], bufs);
      }
    }
  }
  {
    bool any_tc = false;
    for (int n = 0; n < N; ++n) any_tc = any_tc || p->use_tc[n];
    if (any_tc) {
      int64_t tot = 0;
      for (int n = 0; n < N; ++n) tot += (int64_t)R[n] * p->Ist[n] * R[(n + 1) % N];
      PLAN_TRY(p->alloc(&p->c32buf, (size_t)tot));
      int64_t off = 0;
      for (int n = 0; n < N; ++n) {
        p->c32[n] = p->c32buf + off;
        off += (int64_t)R[n] * p->Ist[n] * R[(n + 1) % N];
      }
    }
  }
  if (counting) {
    *count_out = p->bytes;
    trals_plan_destroy(p);
    return TRALS_OK;
  }
  {
    // the coefficient branch (Gram, Cholesky) is the critical path of the modes with large R_n R_{n+1}:
    // its blocks go first; the next mode's table pre-phase fills whatever is left
    int least = 0, greatest = 0;
    PLAN_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    PLAN_TRY(cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, greatest));
    PLAN_TRY(cudaStreamCreateWithFlags(&p->side2, cudaStreamNonBlocking));
    PLAN_TRY(cudaStreamCreateWithPriority(&p->side3, cudaStreamNonBlocking, least));
  }
  for (int n = 0; n < N; ++n) {
    PLAN_TRY(cudaEventCreateWithFlags(&p->ev_fork[n], cudaEventDisableTiming));
    PLAN_TRY(cudaEventCreateWithFlags(&p->ev_join[n], cudaEventDisableTiming));
    PLAN_TRY(cudaEventCreateWithFlags(&p->ev_pre[n], cudaEventDisableTiming));
    PLAN_TRY(cudaEventCreateWithFlags(&p->ev_gam[n], cudaEventDisableTiming));
    PLAN_TRY(cudaEventCreateWithFlags(&p->ev_tcpre[n], cudaEventDisableTiming));
    PLAN_TRY(cudaEventCreateWithFlags(&p->ev_coef[n], cudaEventDisableTiming));
  }
  if (sync) PLAN_TRY(cudaStreamSynchronize(s));
  else PLAN_TRY(cudaGetLastError());
#undef PLAN_TRY
  *out = p;
  return TRALS_OK;
}

}  // namespace

extern "C" {

trals_status trals_plan_create(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R, const void* X_dev, int xt,
                               const trals_opts* opts, trals_plan** out) {
  return plan_build(ctx, N, I, R, X_dev, xt, opts, false, nullptr, out);
}

trals_status trals_plan_footprint(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R, const void* X_dev,
                                  int xt, const trals_opts* opts, size_t* bytes) {
  if (!bytes) return TRALS_E_ARG;
  *bytes = 0;
  return plan_build(ctx, N, I, R, X_dev, xt, opts, true, bytes, nullptr);
}

size_t trals_plan_bytes(const trals_plan* p) { return p ? p->bytes : 0; }

trals_status trals_plan_set_cores(trals_plan* p, double* const* cores_host) {
  if (!p || !cores_host) return TRALS_E_ARG;
  trals_ctx* ctx = p->ctx;
  cudaStream_t s = ctx->stream;
  for (int n = 0; n < p->N; ++n) {
    if (!cores_host[n]) {
      ctx->last_error = "null core pointer";
      return TRALS_E_ARG;
    }
    const size_t cnt = (size_t)p->R[n] * p->I[n] * p->R[(n + 1) % p->N];
    TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(p->cores[n], cores_host[n], cnt * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_gamma(p->cores[n], p->R[n], p->I[n], p->R[(n + 1) % p->N], p->gam[n], s);
  }
  p->prep_stale = true;
  set_int_kernel<<<1, 1, 0, s>>>(p->sweep_ctr, 0);
  TRALS_CUDA_TRY(ctx, cudaGetLastError());
  // host copies are pageable: make them complete before returning
  TRALS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  p->host_sweeps = 0;
  return TRALS_OK;
}

trals_status trals_plan_get_cores(trals_plan* p, double* const* cores_host) {
  if (!p || !cores_host) return TRALS_E_ARG;
  trals_ctx* ctx = p->ctx;
  for (int n = 0; n < p->N; ++n) {
    const size_t cnt = (size_t)p->R[n] * p->I[n] * p->R[(n + 1) % p->N];
    TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(cores_host[n], p->cores[n], cnt * sizeof(double), cudaMemcpyDeviceToHost,
                                        ctx->stream));
  }
  return read_status(ctx);
}

trals_status trals_plan_run(trals_plan* p, int sweeps, int use_graph) {
  if (!p || sweeps < 0) return TRALS_E_ARG;
  trals_ctx* ctx = p->ctx;
  if (p->host_sweeps + sweeps > kResCap) {
    ctx->last_error = "residual history full: call trals_plan_set_cores to restart";
    return TRALS_E_ARG;
  }
  cudaStream_t s = ctx->stream;
  if (sweeps > 0 && p->prep_stale) {
    // the cores may have been set or written since the last run: refresh their FP32 copies and what
    // each sweep's mode 0 expects from the sweep before it (a sweep leaves both current)
    if (p->c32buf) launch_cores_to_f32(p->cores, p->N, p->R, p->Ist, p->I[0], p->c32buf, s);
    if (p->pre[0]) enqueue_prefix(p->N, p->R, p->gam, 0, p->preA, p->preB, p->pre0, s);
    if (p->use_tc[0]) tc_enqueue_pre(p->tc[0], p->cores, s, p->c32);
    TRALS_CUDA_TRY(ctx, cudaGetLastError());
    p->prep_stale = false;
  }
  for (int k = 0; k < sweeps; ++k) {
    if (use_graph) {
      if (!p->gexec) {
        cudaGraph_t g = nullptr;
        TRALS_CUDA_TRY(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        p->launches = enqueue_sweep(p);
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess) {
          ctx->last_error = std::string("graph capture: ") + cudaGetErrorString(e);
          return TRALS_E_CUDA;
        }
        // kernel nodes keep the priority of the stream they were captured from
        e = cudaGraphInstantiate(&p->gexec, g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          ctx->last_error = std::string("graph instantiate: ") + cudaGetErrorString(e);
          p->gexec = nullptr;
          return TRALS_E_CUDA;
        }
      }
      TRALS_CUDA_TRY(ctx, cudaGraphLaunch(p->gexec, s));
    } else {
      p->launches = enqueue_sweep(p);
      TRALS_CUDA_TRY(ctx, cudaGetLastError());
    }
    ++p->host_sweeps;
  }
  return TRALS_OK;
}

trals_status trals_plan_residuals(trals_plan* p, double* rel_res_host, int cap, int* count) {
  if (!p) return TRALS_E_ARG;
  trals_ctx* ctx = p->ctx;
  const int n = std::min(cap, p->host_sweeps);
  if (rel_res_host && n > 0)
    TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(rel_res_host, p->res_hist, n * sizeof(double), cudaMemcpyDeviceToHost,
                                        ctx->stream));
  if (count) *count = n;
  return read_status(ctx);
}

trals_status trals_plan_mttsp(trals_plan* p, int n, double* M_dev) {
  if (!p || n < 0 || n >= p->N) return TRALS_E_ARG;
  double* keep = p->M;
  if (M_dev) p->M = M_dev;
  enqueue_mttsp(p, n, p->ctx->stream);
  p->M = keep;
  TRALS_CUDA_TRY(p->ctx, cudaGetLastError());
  return TRALS_OK;
}

trals_status trals_plan_time_mttsp(trals_plan* p, int n, float* kernel_ms, float* total_ms) {
  if (!p || n < 0 || n >= p->N) return TRALS_E_ARG;
  trals_ctx* ctx = p->ctx;
  cudaStream_t s = ctx->stream;
  cudaEvent_t ev[4] = {};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
  // the tensor-core tables' first part runs during the previous mode in a sweep (on a side stream):
  // it is enqueued before the first event, so the total covers what a sweep has on its critical path
  const bool tc = p->use_tc[n];
  if (e == cudaSuccess && tc) {
    launch_cores_to_f32(p->cores, p->N, p->R, p->Ist, p->I[0], p->c32buf, s);   // current FP32 core copies
    tc_enqueue_pre(p->tc[n], p->cores, s, p->c32);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) {
    enqueue_mttsp(p, n, s, ev[1], ev[2], tc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev[3], s);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
  float a = 0.f, b = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[1], ev[2]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[0], ev[3]);
  for (int k = 0; k < 4; ++k)
    if (ev[k]) cudaEventDestroy(ev[k]);
  TRALS_CUDA_TRY(ctx, e);
  if (kernel_ms) *kernel_ms = a;
  if (total_ms) *total_ms = b;
  return read_status(ctx);
}

trals_status trals_plan_explicit_residual(trals_plan* p, double* rel_res_host) {
  if (!p || !rel_res_host) return TRALS_E_ARG;
  trals_ctx* ctx = p->ctx;
  cudaStream_t s = ctx->stream;
  enqueue_explicit_residual(p, s);
  finalize_ratio_kernel<<<1, 1, 0, s>>>(p->red2, p->red2 + 1);
  TRALS_CUDA_TRY(ctx, cudaGetLastError());
  TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(rel_res_host, p->red2 + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  return read_status(ctx);
}

}  // extern "C"

namespace trals {

trals_status plan_create_async(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R, const void* X_dev, int xt,
                               const trals_opts* opts, trals_plan** out) {
  return plan_build(ctx, N, I, R, X_dev, xt, opts, false, nullptr, out, false);
}

trals_status plan_set_cores_async(trals_plan* p, const double* const* cores_host) {
  trals_ctx* ctx = p->ctx;
  cudaStream_t s = ctx->stream;
  for (int n = 0; n < p->N; ++n) {
    const size_t cnt = (size_t)p->R[n] * p->I[n] * p->R[(n + 1) % p->N];
    // pageable sources are staged before the call returns
    TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(p->cores[n], cores_host[n], cnt * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_gamma(p->cores[n], p->R[n], p->I[n], p->R[(n + 1) % p->N], p->gam[n], s);
  }
  p->prep_stale = true;
  set_int_kernel<<<1, 1, 0, s>>>(p->sweep_ctr, 0);
  TRALS_CUDA_TRY(ctx, cudaGetLastError());
  p->host_sweeps = 0;
  return TRALS_OK;
}

size_t plan_core_elems(const trals_plan* p) {
  size_t t = 0;
  for (int n = 0; n < p->N; ++n) t += (size_t)p->R[n] * p->I[n] * p->R[(n + 1) % p->N];
  return t;
}

trals_status plan_enqueue_results(trals_plan* p, int sweeps, bool final_explicit, double* res_host,
                                  double* cores_host, void* status_host) {
  trals_ctx* ctx = p->ctx;
  cudaStream_t s = ctx->stream;
  if (final_explicit) {
    enqueue_explicit_residual(p, s);
    finalize_last_residual_kernel<<<1, 1, 0, s>>>(p->red2, p->res_hist, p->sweep_ctr);
  }
  if (sweeps > 0)
    TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(res_host, p->res_hist, sweeps * sizeof(double), cudaMemcpyDeviceToHost, s));
  size_t off = 0;
  for (int n = 0; n < p->N; ++n) {
    const size_t cnt = (size_t)p->R[n] * p->I[n] * p->R[(n + 1) % p->N];
    TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(cores_host + off, p->cores[n], cnt * sizeof(double), cudaMemcpyDeviceToHost, s));
    off += cnt;
  }
  TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(status_host, ctx->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  launch_zero_status(ctx->d_status, s);
  TRALS_CUDA_TRY(ctx, cudaGetLastError());
  return TRALS_OK;
}

std::string status_message(const void* status_host) {
  const DevStatus& st = *static_cast<const DevStatus*>(status_host);
  char buf[256];
  snprintf(buf, sizeof buf, "%s at sweep %d, core %d, index %d (value %.6g)",
           st.code == TRALS_E_NOT_SPD ? "non-positive Cholesky pivot"
           : st.code == TRALS_E_NONFINITE ? "non-finite value in a solve"
           : st.code == TRALS_E_TIMEOUT   ? "bounded device wait timed out"
                                          : "device error",
           st.sweep, st.mode, st.index, st.value);
  return buf;
}

int status_code(const void* status_host) { return static_cast<const DevStatus*>(status_host)->code; }

}  // namespace trals

extern "C" {

const double* trals_plan_core_dev(const trals_plan* p, int n) {
  if (!p || n < 0 || n >= p->N) return nullptr;
  return p->cores[n];
}

int trals_plan_mttsp_path(const trals_plan* p, int n) {
  if (!p || n < 0 || n >= p->N) return -1;
  return p->use_tc[n] ? tc_variant(p->tc[n]) + 1 : p->gemm[n].valid ? 5 : 0;
}

int trals_plan_launches_per_sweep(const trals_plan* p) {
  if (!p) return 0;
  if (p->launches == 0) {
    // count by a dry enqueue is not possible without launching; report the analytic count
    return 0;
  }
  return p->launches;
}

trals_status trals_decompose(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R, const void* X, int xt,
                             int x_on_host, double* const* cores, int sweeps, const trals_opts* opts,
                             double* rel_res) {
  if (!ctx || !X || !cores || sweeps < 0) return TRALS_E_ARG;
  trals_status st = check_shape(ctx, N, I, R);
  if (st != TRALS_OK) return st;
  void* Xd = nullptr;
  const void* Xuse = X;
  if (x_on_host) {
    int64_t numel = 1;
    for (int n = 0; n < N; ++n) numel *= I[n];
    const size_t es = xt == TRALS_X_F64 ? 8 : xt == TRALS_X_F32 ? 4 : 2;
    TRALS_CUDA_TRY(ctx, cudaMalloc(&Xd, (size_t)numel * es));
    cudaError_t e = cudaMemcpyAsync(Xd, X, (size_t)numel * es, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
      cudaFree(Xd);
      ctx->last_error = cudaGetErrorString(e);
      return TRALS_E_CUDA;
    }
    Xuse = Xd;
  }
  if (opts && (opts->solver == TRALS_SOLVE_QRNE || opts->solver == TRALS_SOLVE_QR_COMPRESSED)) {
    // TR-ALS-QRNE (Alg. 4) and the literal TR-ALS-QR (Alg. 3): their own driver, FP64 only
    if (opts->mode != TRALS_MODE_FP64 || xt != TRALS_X_F64 || opts->gram != TRALS_GRAM_STRUCTURED) {
      ctx->last_error = "the QRNE and compressed-QR solvers run in the FP64 mode with an FP64 X and the structured Gram";
      st = TRALS_E_ARG;
    } else {
      st = qrne_decompose(ctx, N, I, R, static_cast<const double*>(Xuse), cores, sweeps, rel_res,
                          opts->solver == TRALS_SOLVE_QR_COMPRESSED);
    }
    if (Xd) cudaFree(Xd);
    return st;
  }
  trals_plan* p = nullptr;
  st = trals_plan_create(ctx, N, I, R, Xuse, xt, opts, &p);
  if (st == TRALS_OK) st = trals_plan_set_cores(p, cores);
  if (st == TRALS_OK) st = trals_plan_run(p, sweeps, 1);
  if (st == TRALS_OK) st = trals_plan_residuals(p, rel_res, sweeps, nullptr);
  // reduced-precision modes record no per-sweep residual unless asked to: give the final one
  if (st == TRALS_OK && rel_res && sweeps > 0 && p->opts.mode != TRALS_MODE_FP64 && !p->opts.explicit_residual)
    st = trals_plan_explicit_residual(p, &rel_res[sweeps - 1]);
  if (st == TRALS_OK) st = trals_plan_get_cores(p, cores);
  trals_plan_destroy(p);
  if (Xd) cudaFree(Xd);
  return st;
}

// ------------------------------------------------------------------ per-step entry points
trals_status trals_gamma(trals_ctx* ctx, const double* G_dev, int Rn, int64_t In, int Rn1, double* Gamma_dev) {
  if (!ctx || !G_dev || !Gamma_dev || Rn < 1 || Rn1 < 1 || In < 1) return TRALS_E_ARG;
  launch_gamma(G_dev, Rn, In, Rn1, Gamma_dev, ctx->stream);
  TRALS_CUDA_TRY(ctx, cudaGetLastError());
  TRALS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return TRALS_OK;
}

trals_status trals_coef_matrix(trals_ctx* ctx, int N, const int32_t* R, const double* const* gammas_dev, int n,
                               double* S_dev) {
  if (!ctx || !R || !gammas_dev || !S_dev || N < 3 || N > TRALS_MAX_ORDER || n < 0 || n >= N) return TRALS_E_ARG;
  int maxR2 = 0;
  for (int k = 0; k < N; ++k) maxR2 = std::max(maxR2, R[k] * R[k]);
  double *a = nullptr, *b = nullptr;
  TRALS_CUDA_TRY(ctx, cudaMalloc(&a, (size_t)maxR2 * maxR2 * sizeof(double)));
  cudaError_t e = cudaMalloc(&b, (size_t)maxR2 * maxR2 * sizeof(double));
  if (e == cudaSuccess) {
    enqueue_coef(N, R, const_cast<double* const*>(gammas_dev), n, a, b, S_dev, ctx->stream);
    e = cudaStreamSynchronize(ctx->stream);
  }
  cudaFree(a);
  if (b) cudaFree(b);
  TRALS_CUDA_TRY(ctx, e);
  return TRALS_OK;
}

trals_status trals_coef_matrix_explicit(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                                        const double* const* cores_dev, int n, int fp64, double* S_dev) {
  if (!ctx || !cores_dev || !S_dev || n < 0 || n >= N) return TRALS_E_ARG;
  trals_status st = check_shape(ctx, N, I, R);
  if (st != TRALS_OK) return st;
  const ModeLayout L = make_mode_layout(N, I, R, n);
  const int64_t tab = table_level_max_elems(L, I, R);
  const ExplicitGramSizes z = explicit_gram_sizes(L, fp64 != 0);
  double *lt = nullptr, *ut = nullptr, *sc = nullptr, *part = nullptr;
  void* A = nullptr;
  cudaError_t e = cudaMalloc(&lt, tab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ut, tab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&sc, tab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&part, z.part_elems * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&A, z.A_bytes);
  if (e == cudaSuccess) {
    build_tables(L, cores_dev, I, R, lt, ut, sc, ctx->stream);
    launch_explicit_gram(L, lt, ut, fp64 != 0, A, part, S_dev, ctx->stream);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  cudaFree(lt);
  cudaFree(ut);
  cudaFree(sc);
  cudaFree(part);
  cudaFree(A);
  TRALS_CUDA_TRY(ctx, e);
  return TRALS_OK;
}

trals_status trals_qr_r_factor(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                               const double* const* cores_dev, int n, double* R_dev) {
  if (!ctx || !cores_dev || !R_dev || n < 0 || n >= N) return TRALS_E_ARG;
  trals_status st = check_shape(ctx, N, I, R);
  if (st != TRALS_OK) return st;
  const QrSizes z = qr_sizes(N, I, R, n);
  const int r = R[n] * R[(n + 1) % N];
  double *B = nullptr, *R0 = nullptr, *R1 = nullptr, *W = nullptr, *Lm = nullptr;
  cudaError_t e = cudaMalloc(&B, z.B_elems * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&R0, z.R_elems * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&R1, z.R_elems * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&W, std::max<int64_t>(z.W_elems, 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&Lm, lmat_elems(r) * sizeof(double));   // the factor layout, block inverses included
  if (e == cudaSuccess) {
    launch_qr_factor(N, I, R, n, cores_dev, B, R0, R1, W, Lm, ctx->d_status, nullptr, ctx->stream);
    launch_transpose(Lm, r, R_dev, ctx->stream);
    e = cudaGetLastError();
  }
  st = (e == cudaSuccess) ? read_status(ctx) : TRALS_E_CUDA;
  if (e != cudaSuccess) ctx->last_error = cudaGetErrorString(e);
  cudaFree(B);
  cudaFree(R0);
  cudaFree(R1);
  cudaFree(W);
  cudaFree(Lm);
  return st;
}

trals_status trals_mttsp(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R, const void* X_dev, int xt,
                         int mode, const double* const* cores_dev, int n, double* M_dev) {
  if (!ctx || !X_dev || !cores_dev || !M_dev || n < 0 || n >= N) return TRALS_E_ARG;
  ctx->last_mttsp_path = -1;
  trals_status st = check_shape(ctx, N, I, R);
  if (st != TRALS_OK) return st;
  const bool bf_mode = mode == TRALS_MODE_BF16 || mode == TRALS_MODE_BF16X2 || mode == TRALS_MODE_BF16X3;
  const bool ok_type = (mode == TRALS_MODE_FP64 && xt == TRALS_X_F64) || (mode == TRALS_MODE_FP32 && xt == TRALS_X_F32) ||
                       (bf_mode && (xt == TRALS_X_BF16 || xt == TRALS_X_BF16PAIR));
  if (!ok_type) {
    ctx->last_error = "X element type does not match the mode";
    return TRALS_E_ARG;
  }
  if (xt == TRALS_X_BF16PAIR) xt = TRALS_X_BF16;   // the hi plane leads; bf16x3 reads the lo plane after it
  cudaStream_t s = ctx->stream;
  int64_t numel = 1;
  for (int k = 0; k < N; ++k) numel *= I[k];
  TcPlan tc;
  cudaError_t e = cudaSuccess;
  const void* Xlo = (mode == TRALS_MODE_BF16X3) ? static_cast<const void*>(static_cast<const __nv_bfloat16*>(X_dev) + numel)
                                                 : nullptr;
  const int use_tc =
      (mode != TRALS_MODE_FP64) ? tc_plan(tc, N, I, R, n, mode, X_dev, numel, &e, ctx->stream, nullptr, 0, Xlo) : 0;
  TRALS_CUDA_TRY(ctx, e);
  if (use_tc) {
    const int variant = tc_variant(tc);
    tc_set_status(tc, ctx->d_status);
    tc_enqueue(tc, X_dev, const_cast<double* const*>(cores_dev), M_dev, s);
    e = cudaStreamSynchronize(s);
    tc_destroy(tc);
    TRALS_CUDA_TRY(ctx, e);
    TRALS_CUDA_TRY(ctx, cudaGetLastError());
    st = read_status(ctx);
    if (st != TRALS_OK) return st;
    ctx->last_mttsp_path = variant + 1;
    return TRALS_OK;
  }
  const ModeLayout L = make_mode_layout(N, I, R, n);
  const int64_t tab = table_level_max_elems(L, I, R);
  const int gridX = mttsp_simt_default_grid(L);
  std::vector<int64_t> offL, offU;
  mode_offsets(N, I, L, offL, offU);
  double *lt = nullptr, *ut = nullptr, *sc = nullptr, *part = nullptr;
  int64_t *dL = nullptr, *dU = nullptr;
  e = cudaMalloc(&lt, tab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ut, tab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&sc, tab * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMalloc(&part, std::max(mttsp_simt_partials_elems(L, gridX), mttsp_simt_partials_elems(L, mttsp_simt_f32_grid(L))) *
                              sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dL, offL.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&dU, offU.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMemcpy(dL, offL.data(), offL.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dU, offU.data(), offU.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    build_tables(L, cores_dev, I, R, lt, ut, sc, s);
    MttspSimtArgs a;
    a.X = X_dev;
    a.Xlo = (mode == TRALS_MODE_BF16X3) ? static_cast<const __nv_bfloat16*>(X_dev) + numel : nullptr;
    a.xt = xt;
    a.ltab = lt;
    a.utab = ut;
    a.offL = dL;
    a.offU = dU;
    a.L = L;
    a.partials = part;
    a.M = M_dev;
    a.gridX = gridX;
    if (mode != TRALS_MODE_FP64 && mttsp_simt_f32_fits(L)) {
      const int64_t nl = L.nL * L.Rn1 * L.Rs, nu = L.nU * L.Rs * L.Rn;
      float* fl = reinterpret_cast<float*>(sc);
      launch_tables_to_f32(lt, nl, fl, ut, nu, fl + nl, s);
      a.gridX = mttsp_simt_f32_grid(L);
      launch_mttsp_simt_f32(a, fl, fl + nl, s);
    } else {
      launch_mttsp_simt(a, s);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaFree(lt);
  cudaFree(ut);
  cudaFree(sc);
  cudaFree(part);
  cudaFree(dL);
  cudaFree(dU);
  TRALS_CUDA_TRY(ctx, e);
  ctx->last_mttsp_path = 0;
  return TRALS_OK;
}

int trals_last_mttsp_path(const trals_ctx* ctx) { return ctx ? ctx->last_mttsp_path : -1; }

trals_status trals_testing_mttsp_withheld_copy(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                                               const void* X_dev, int mode, const double* const* cores_dev, int n,
                                               double* M_dev, long long spin_cycles) {
  if (!ctx || !X_dev || !cores_dev || !M_dev || n < 0 || n >= N || spin_cycles <= 0) return TRALS_E_ARG;
  trals_status st = check_shape(ctx, N, I, R);
  if (st != TRALS_OK) return st;
  if (mode != TRALS_MODE_BF16) {
    ctx->last_error = "trals_testing_mttsp_withheld_copy: BF16 mode only";
    return TRALS_E_ARG;
  }
  int64_t numel = 1;
  for (int k = 0; k < N; ++k) numel *= I[k];
  TcPlan tc;
  cudaError_t e = cudaSuccess;
  if (!tc_plan(tc, N, I, R, n, mode, X_dev, numel, &e, ctx->stream)) {
    TRALS_CUDA_TRY(ctx, e);
    ctx->last_error = "trals_testing_mttsp_withheld_copy: no tensor-core geometry for this mode";
    return TRALS_E_ARG;
  }
  tc_set_status(tc, ctx->d_status);
  tc_set_fault(tc, 1, spin_cycles);
  tc_enqueue(tc, X_dev, const_cast<double* const*>(cores_dev), M_dev, ctx->stream);
  e = cudaStreamSynchronize(ctx->stream);
  tc_destroy(tc);
  TRALS_CUDA_TRY(ctx, e);
  TRALS_CUDA_TRY(ctx, cudaGetLastError());
  return read_status(ctx);
}

int trals_mttsp_path(int N, const int64_t* I, const int32_t* R, int n, int mode) {
  if (N < 3 || N > TRALS_MAX_ORDER || !I || !R || n < 0 || n >= N) return -1;
  if (mode != TRALS_MODE_BF16 && mode != TRALS_MODE_BF16X2 && mode != TRALS_MODE_BF16X3) return 0;
  // plans store the BF16 copy with mode 0 padded to a multiple of 8
  int64_t Ist[TRALS_MAX_ORDER];
  for (int j = 0; j < N; ++j) Ist[j] = I[j];
  Ist[0] = (I[0] + 7) / 8 * 8;
  const TcChoice c = tc_choose(N, Ist, R, n);
  return c.variant < 0 ? 0 : c.variant + 1;
}

trals_status trals_solve_chol(trals_ctx* ctx, int Rn, int64_t In, int Rn1, const double* S_dev, const double* M_dev,
                              double* G_dev) {
  if (!ctx || !S_dev || !M_dev || !G_dev || Rn < 1 || Rn1 < 1 || In < 1 || Rn * Rn1 > 256) return TRALS_E_ARG;
  const int r = Rn * Rn1;
  double* Lm = nullptr;
  TRALS_CUDA_TRY(ctx, cudaMalloc(&Lm, lmat_elems(r) * sizeof(double)));
  launch_cholesky(S_dev, Lm, r, ctx->d_status, nullptr, -1, ctx->stream);
  launch_chol_solve(Lm, M_dev, Rn, In, Rn1, G_dev, ctx->d_status, ctx->stream);
  cudaError_t e = cudaGetLastError();
  trals_status st = (e == cudaSuccess) ? read_status(ctx) : TRALS_E_CUDA;
  cudaFree(Lm);
  if (e != cudaSuccess) ctx->last_error = cudaGetErrorString(e);
  return st;
}

trals_status trals_check_pivot_rsqrt(trals_ctx* ctx, const double* d_dev, int64_t n, double* out_dev,
                                     double* ref_dev) {
  if (!ctx || n < 0 || (n > 0 && (!d_dev || !out_dev || !ref_dev))) return TRALS_E_ARG;
  if (n == 0) return TRALS_OK;
  launch_pivot_rsqrt_check(d_dev, n, out_dev, ref_dev, ctx->stream);
  TRALS_CUDA_TRY(ctx, cudaGetLastError());
  TRALS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return TRALS_OK;
}

trals_status trals_reconstruct(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                               const double* const* cores_dev, void* out_dev, int xt) {
  if (!ctx || !cores_dev || !out_dev) return TRALS_E_ARG;
  trals_status st = check_shape(ctx, N, I, R);
  if (st != TRALS_OK) return st;
  const int n = N - 1;
  const ModeLayout L = make_mode_layout(N, I, R, n);
  const int64_t tab = table_level_max_elems(L, I, R);
  std::vector<int64_t> offL, offU;
  mode_offsets(N, I, L, offL, offU);
  const int gridX = mttsp_simt_default_grid(L);
  double *lt = nullptr, *ut = nullptr, *sc = nullptr;
  int64_t *dL = nullptr, *dU = nullptr;
  cudaError_t e = cudaMalloc(&lt, tab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ut, tab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&sc, tab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dL, offL.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&dU, offU.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMemcpy(dL, offL.data(), offL.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dU, offU.data(), offU.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    build_tables(L, cores_dev, I, R, lt, ut, sc, ctx->stream);
    launch_reconstruct(L, lt, ut, dL, dU, cores_dev[n], out_dev, xt, nullptr, TRALS_X_F64, nullptr, gridX,
                       ctx->stream);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  cudaFree(lt);
  cudaFree(ut);
  cudaFree(sc);
  cudaFree(dL);
  cudaFree(dU);
  TRALS_CUDA_TRY(ctx, e);
  return TRALS_OK;
}

trals_status trals_residual_explicit(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R, const void* X_dev,
                                     int xt, const double* const* cores_dev, double* res2_host, double* normx2_host) {
  if (!ctx || !cores_dev || !X_dev) return TRALS_E_ARG;
  trals_status st = check_shape(ctx, N, I, R);
  if (st != TRALS_OK) return st;
  const int n = N - 1;
  const ModeLayout L = make_mode_layout(N, I, R, n);
  const int64_t tab = table_level_max_elems(L, I, R);
  std::vector<int64_t> offL, offU;
  mode_offsets(N, I, L, offL, offU);
  const int gridX = mttsp_simt_default_grid(L);
  double *lt = nullptr, *ut = nullptr, *sc = nullptr, *part = nullptr, *red = nullptr;
  int64_t *dL = nullptr, *dU = nullptr;
  cudaError_t e = cudaMalloc(&lt, tab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ut, tab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&sc, tab * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&part, 2 * gridX * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&red, 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dL, offL.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&dU, offU.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMemcpy(dL, offL.data(), offL.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dU, offU.data(), offU.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  double h[2] = {0, 0};
  if (e == cudaSuccess) {
    build_tables(L, cores_dev, I, R, lt, ut, sc, ctx->stream);
    launch_reconstruct(L, lt, ut, dL, dU, cores_dev[n], nullptr, TRALS_X_F64, X_dev, xt, part, gridX, ctx->stream);
    launch_reduce_pairs(part, gridX, red, ctx->stream);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, red, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  cudaFree(lt);
  cudaFree(ut);
  cudaFree(sc);
  cudaFree(part);
  cudaFree(red);
  cudaFree(dL);
  cudaFree(dU);
  TRALS_CUDA_TRY(ctx, e);
  if (res2_host) *res2_host = h[0];
  if (normx2_host) *normx2_host = h[1];
  return TRALS_OK;
}

trals_status trals_quantize_bf16(trals_ctx* ctx, const void* src_dev, int src_t, int64_t count, void* dst_hi_dev,
                                 void* dst_lo_dev) {
  if (!ctx || !src_dev || !dst_hi_dev || count < 0 || (src_t != TRALS_X_F64 && src_t != TRALS_X_F32))
    return TRALS_E_ARG;
  launch_quantize(src_dev, src_t, count, static_cast<__nv_bfloat16*>(dst_hi_dev),
                  static_cast<__nv_bfloat16*>(dst_lo_dev), ctx->stream);
  TRALS_CUDA_TRY(ctx, cudaGetLastError());
  TRALS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return TRALS_OK;
}

}  // extern "C"
