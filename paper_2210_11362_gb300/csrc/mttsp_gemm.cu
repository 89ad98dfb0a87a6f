// Two-stage MTTSP through a plain GEMM (interface and the two forms in mttsp_gemm.cuh).
//
// For a wide subchain table the generic CUDA-core MTTSP regenerates a 256-entry subchain row for every
// column of X_[n]; with I_n = 3 that is 4096 multiply-adds for 768 useful ones.  Here the contraction is
// reassociated (eq. subchain_new: G^{!=n}(k) = L(l) U(u)): X is contracted first with the table of the
// modes that lead it in memory, a plain GEMM, and the result with the other table.  cuBLAS is opened at
// run time for that GEMM only, so the library loads without it; every other step runs in this file's
// kernels.
#include <dlfcn.h>

#include <algorithm>
#include <mutex>

#include <cublas_v2.h>

#include "mttsp_gemm.cuh"

namespace trals {
namespace {

constexpr int64_t kMinElems = (int64_t)1 << 21;
constexpr int kMinWidth = 64;
constexpr size_t kWorkspace = (size_t)32 << 20;

// The few cuBLAS entry points used, resolved from the shared library at run time.
struct CublasApi {
  bool ok = false;
  decltype(&cublasCreate_v2) create = nullptr;
  decltype(&cublasDestroy_v2) destroy = nullptr;
  decltype(&cublasSetStream_v2) set_stream = nullptr;
  decltype(&cublasSetWorkspace_v2) set_workspace = nullptr;
  decltype(&cublasSetMathMode) set_math = nullptr;
  cublasStatus_t (*gemm)(cublasHandle_t, cublasOperation_t, cublasOperation_t, int, int, int, const void*,
                         const void*, cudaDataType, int, const void*, cudaDataType, int, const void*, void*,
                         cudaDataType, int, cublasComputeType_t, cublasGemmAlgo_t) = nullptr;
};

const CublasApi& api() {
  static const CublasApi a = []() {
    CublasApi r;
    void* h = dlopen("libcublas.so.13", RTLD_NOW | RTLD_LOCAL);
    if (!h) h = dlopen("libcublas.so", RTLD_NOW | RTLD_LOCAL);
    if (!h) return r;
    r.create = reinterpret_cast<decltype(r.create)>(dlsym(h, "cublasCreate_v2"));
    r.destroy = reinterpret_cast<decltype(r.destroy)>(dlsym(h, "cublasDestroy_v2"));
    r.set_stream = reinterpret_cast<decltype(r.set_stream)>(dlsym(h, "cublasSetStream_v2"));
    r.set_workspace = reinterpret_cast<decltype(r.set_workspace)>(dlsym(h, "cublasSetWorkspace_v2"));
    r.set_math = reinterpret_cast<decltype(r.set_math)>(dlsym(h, "cublasSetMathMode"));
    r.gemm = reinterpret_cast<decltype(r.gemm)>(dlsym(h, "cublasGemmEx"));
    r.ok = r.create && r.destroy && r.set_stream && r.set_workspace && r.set_math && r.gemm;
    return r;
  }();
  return a;
}

// dst[e_st * W + w] = src[e * W + w] (entries of a subchain table, W values each) converted to FP32 or to
// BF16 (and its lo plane); with pad set the entries run over a mode 0 stored with I0st >= I0 slices,
// e_st = i0 + I0st rest <- e = i0 + I0 rest, zero for i0 >= I0.
__global__ void table_convert_kernel(const double* __restrict__ src, int64_t Kst, int W, int pad, int64_t I0,
                                     int64_t I0st, int xmode, void* __restrict__ dst, void* __restrict__ dst_lo) {
  const int64_t total = Kst * W;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t est = x / W;
    const int w = (int)(x - est * W);
    double v = 0.0;
    if (pad) {
      const int64_t i0 = est % I0st, rest = est / I0st;
      if (i0 < I0) v = src[(i0 + I0 * rest) * W + w];
    } else {
      v = src[est * W + w];
    }
    const float f = (float)v;
    if (xmode == kGemmF32) {
      static_cast<float*>(dst)[x] = f;
    } else {
      const __nv_bfloat16 hi = __float2bfloat16_rn(f);
      static_cast<__nv_bfloat16*>(dst)[x] = hi;
      if (dst_lo) static_cast<__nv_bfloat16*>(dst_lo)[x] = __float2bfloat16_rn(f - __bfloat162float(hi));
    }
  }
}

constexpr int kBatch = 16;
constexpr int kMaxW = 256;

// Stage 2, one CTA per (i_n, chunk of the other table's entries); thread t owns output column
// t = a + R_n b.  T is stored row-contiguous: T[w + W1 row].
template <int FORM>
__global__ void __launch_bounds__(256) gemm_stage2_kernel(const float* __restrict__ T, int W1,
                                                          const float* __restrict__ tabO, int WO, int64_t nO,
                                                          int64_t Irows, int Rn, int Rn1, int Rs, int64_t In,
                                                          int nchunk, float* __restrict__ part) {
  __shared__ float Ts[kBatch][kMaxW + 1];
  __shared__ float Os[kBatch][kMaxW + 1];
  const int64_t i = blockIdx.x;
  const int c = blockIdx.y;
  const int r = Rn * Rn1;
  const int col = threadIdx.x;
  const int a = col % Rn, b = col / Rn;
  const int64_t e0 = nO * c / nchunk, e1 = nO * (c + 1) / nchunk;
  float acc = 0.0f;
  for (int64_t eb = e0; eb < e1; eb += kBatch) {
    const int ne = (int)min((int64_t)kBatch, e1 - eb);
    for (int x = threadIdx.x; x < kBatch * W1; x += blockDim.x) {
      const int q = x / W1, w = x - q * W1;
      float v = 0.0f;
      if (q < ne) {
        const int64_t row = FORM == 1 ? i + Irows * (eb + q) : (eb + q) + nO * i;
        v = T[w + (int64_t)W1 * row];
      }
      Ts[q][w] = v;
    }
    for (int x = threadIdx.x; x < kBatch * WO; x += blockDim.x) {
      const int q = x / WO, w = x - q * WO;
      Os[q][w] = q < ne ? tabO[(eb + q) * WO + w] : 0.0f;
    }
    __syncthreads();
    if (col < r) {
      for (int q = 0; q < ne; ++q)
        for (int s = 0; s < Rs; ++s)
          acc = FORM == 1 ? fmaf(Os[q][b + Rn1 * s], Ts[q][s + Rs * a], acc)
                          : fmaf(Ts[q][b + Rn1 * s], Os[q][s + Rs * a], acc);
    }
    __syncthreads();
  }
  if (col < r) part[(int64_t)c * In * r + i + In * col] = acc;
}

// P of gemm_residual_enqueue, stored row-contiguous: P[w + W1 row].
template <int FORM>
__global__ void residual_p_kernel(const double* __restrict__ G, const float* __restrict__ tabO, int64_t rowsT, int W1,
                                  int WO, int64_t nO, int64_t In, int Rn, int Rn1, int Rs, float* __restrict__ P) {
  const int64_t total = rowsT * W1;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = x / W1;
    const int w = (int)(x - row * W1);
    float acc = 0.0f;
    if (FORM == 1) {   // row = i + In l, w = s + Rs a
      const int64_t i = row % In, l = row / In;
      const int s = w % Rs, a = w / Rs;
      const float* Lr = tabO + l * WO + Rn1 * s;   // L(l)[b, s] at b + Rn1 s
      for (int b = 0; b < Rn1; ++b) acc = fmaf((float)G[a + (int64_t)Rn * (i + In * b)], Lr[b], acc);
    } else {           // row = u + nO i, w = b + Rn1 s
      const int64_t u = row % nO, i = row / nO;
      const int b = w % Rn1, s = w / Rn1;
      const float* Ur = tabO + u * WO + s;         // U(u)[s, a] at s + Rs a
      for (int a = 0; a < Rn; ++a) acc = fmaf(Ur[(int64_t)Rs * a], (float)G[a + (int64_t)Rn * (i + In * b)], acc);
    }
    P[x] = acc;
  }
}

__global__ void f64_to_f32_kernel(const double* __restrict__ src, int64_t n, float* __restrict__ dst) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    dst[x] = (float)src[x];
}

// M[e] = sum over chunks of part[c E + e] in FP64, chunks in order.
__global__ void gemm_reduce_kernel(const float* __restrict__ part, int nchunk, int64_t E, double* __restrict__ M) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += (double)part[c * E + e];
    M[e] = s;
  }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

std::mutex handle_mu;

cublasHandle_t handle_of(trals_ctx* ctx) {
  std::lock_guard<std::mutex> lk(handle_mu);
  if (!ctx->cublas && api().ok) {
    cublasHandle_t h = nullptr;
    if (api().create(&h) == CUBLAS_STATUS_SUCCESS) {
      api().set_math(h, CUBLAS_DEFAULT_MATH);   // FP32 products in FP32 (no TF32)
      ctx->cublas = h;
    }
  }
  return static_cast<cublasHandle_t>(ctx->cublas);
}

}  // namespace

bool gemm_available() { return api().ok; }

void gemm_release(trals_ctx* ctx) {
  if (ctx && ctx->cublas && api().ok) api().destroy(static_cast<cublasHandle_t>(ctx->cublas));
  if (ctx) ctx->cublas = nullptr;
}

int gemm_mttsp_plan(GemmMttsp& g, int N, const int64_t* I, const int64_t* Ist, const int32_t* R, int n, int xmode) {
  g = GemmMttsp();
  if (!gemm_available()) return 0;
  int64_t numel = 1;
  for (int j = 0; j < N; ++j) numel *= I[j];
  if (numel < kMinElems) return 0;
  ModeLayout L = make_mode_layout(N, I, R, n);
  if (n >= 1 && n <= N - 2) {
    // the GEMM runs over the modes before n, which lead X: force the split there
    L.m = N - 1 - n;
    L.nL = 1;
    L.nU = 1;
    for (int t = 0; t < L.m; ++t) L.nL *= I[L.chain[t]];
    for (int t = L.m; t < N - 1; ++t) L.nU *= I[L.chain[t]];
    L.Rs = R[L.chain[L.m]];
  }
  const int Rn = R[n], Rn1 = R[(n + 1) % N], Rs = L.Rs;
  g.n = n;
  g.form = n == N - 1 ? 2 : 1;
  g.xmode = xmode;
  g.L = L;
  g.In = I[n];
  g.I0 = I[0];
  g.I0st = Ist[0];
  const bool padded = Ist[0] != I[0];
  if (n >= 1 && n <= N - 2) {          // K = modes 0..n-1 (U table), T rows (i + I_n l)
    g.K = L.nU / I[0] * Ist[0];
    g.padK = padded;
    g.rowsT = I[n] * L.nL;
    g.Irows = I[n];
    g.W1 = Rs * Rn;
    g.nOther = L.nL;
  } else if (n == N - 1) {             // K = modes 0..m-1 (L table), T rows (u + nU i)
    g.K = L.nL / I[0] * Ist[0];
    g.padK = padded;
    g.rowsT = L.nU * I[n];
    g.W1 = Rn1 * Rs;
    g.nOther = L.nU;
  } else {                             // n = 0: K = modes m+1..N-1 (U table), T rows (i + I0st l)
    g.K = L.nU;
    g.padK = false;
    g.rowsT = Ist[0] * L.nL;
    g.Irows = Ist[0];
    g.W1 = Rs * Rn;
    g.nOther = L.nL;
  }
  const int WO = g.form == 1 ? Rn1 * Rs : Rs * Rn;
  if (g.W1 < kMinWidth || g.W1 > kMaxW || WO > kMaxW || Rn * Rn1 > 256) return 0;
  if (g.K > INT32_MAX || g.rowsT > INT32_MAX) return 0;
  g.nchunk = (int)std::max<int64_t>(1, std::min<int64_t>((g.nOther + kBatch - 1) / kBatch, (2048 + g.In - 1) / g.In));
  const int64_t tab = table_level_max_elems(L, I, R);
  const size_t ebytes = xmode == kGemmF32 ? 4 : 2;
  const size_t need[kGemmBufs] = {(size_t)tab * 8,
                                  (size_t)tab * 8,
                                  (size_t)tab * 8,
                                  (size_t)g.K * g.W1 * ebytes,
                                  xmode == kGemmBF16Split ? (size_t)g.K * g.W1 * 2 : 0,
                                  (size_t)g.nOther * WO * 4,
                                  (size_t)g.rowsT * g.W1 * 4,
                                  (size_t)g.nchunk * g.In * Rn * Rn1 * 4,
                                  kWorkspace};
  for (int k = 0; k < kGemmBufs; ++k) g.need[k] = need[k];
  g.valid = true;
  return 1;
}

void gemm_mttsp_bind(GemmMttsp& g, void* const* q) {
  g.ltab64 = static_cast<double*>(q[0]);
  g.utab64 = static_cast<double*>(q[1]);
  g.scr64 = static_cast<double*>(q[2]);
  g.tabK = q[3];
  g.tabK_lo = q[4];
  g.tabO = static_cast<float*>(q[5]);
  g.T = static_cast<float*>(q[6]);
  g.part = static_cast<float*>(q[7]);
  g.ws = q[8];
  g.ws_bytes = kWorkspace;
}

bool gemm_prepare(trals_ctx* ctx) { return handle_of(ctx) != nullptr; }

namespace {
// The subchain tables of the current cores: FP64, then the GEMM's table and the stage-2 table converted.
int prepare_tables(GemmMttsp& g, double* const* cores, const int64_t* I, const int32_t* R, cudaStream_t s) {
  const ModeLayout& L = g.L;
  const int N = L.N, n = g.n;
  const int Rn = R[n], Rn1 = R[(n + 1) % N], Rs = L.Rs;
  const int WO = g.form == 1 ? Rn1 * Rs : Rs * Rn;
  build_tables(L, cores, I, R, g.ltab64, g.utab64, g.scr64, s);
  // the GEMM's table: U for n < N-1, L for n = N-1; the other one for stage 2
  const double* tk = (n == N - 1) ? g.ltab64 : g.utab64;
  const double* to = (n == N - 1) ? g.utab64 : g.ltab64;
  table_convert_kernel<<<grid_for(g.K * g.W1), 256, 0, s>>>(tk, g.K, g.W1, g.padK ? 1 : 0, g.I0, g.I0st, g.xmode, g.tabK,
                                                           g.tabK_lo);
  table_convert_kernel<<<grid_for(g.nOther * WO), 256, 0, s>>>(to, g.nOther, WO, 0, 0, 1, kGemmF32, g.tabO, nullptr);
  return N - 1 + 2;
}
}  // namespace

int gemm_residual_enqueue(GemmMttsp& g, trals_ctx* ctx, const void* X, int xt, double* const* cores, const int64_t* I,
                          const int32_t* R, float* E, cudaStream_t s) {
  if (g.xmode != kGemmF32 || g.padK || g.I0st != g.I0 || (xt != TRALS_X_F32 && xt != TRALS_X_F64)) {
    ctx->last_error = "two-stage residual: FP32 operands of an unpadded X only";
    return -1;
  }
  const ModeLayout& L = g.L;
  const int N = L.N, n = g.n;
  const int Rn = R[n], Rn1 = R[(n + 1) % N], Rs = L.Rs;
  const int WO = g.form == 1 ? Rn1 * Rs : Rs * Rn;
  int launches = prepare_tables(g, cores, I, R, s);
  const int64_t numel = g.K * g.rowsT;
  if (xt == TRALS_X_F32) {
    if (cudaMemcpyAsync(E, X, (size_t)numel * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      ctx->last_error = "two-stage residual: copy of X";
      return -1;
    }
  } else {
    f64_to_f32_kernel<<<grid_for(numel), 256, 0, s>>>(static_cast<const double*>(X), numel, E);
    ++launches;
  }
  if (g.form == 1)
    residual_p_kernel<1><<<grid_for(g.rowsT * g.W1), 256, 0, s>>>(cores[n], g.tabO, g.rowsT, g.W1, WO, g.nOther, g.In,
                                                                  Rn, Rn1, Rs, g.T);
  else
    residual_p_kernel<2><<<grid_for(g.rowsT * g.W1), 256, 0, s>>>(cores[n], g.tabO, g.rowsT, g.W1, WO, g.nOther, g.In,
                                                                  Rn, Rn1, Rs, g.T);
  ++launches;
  cublasHandle_t h = handle_of(ctx);
  if (!h) {
    ctx->last_error = "cuBLAS handle unavailable";
    return -1;
  }
  const CublasApi& c = api();
  const float minus_one = -1.0f, one = 1.0f;
  cublasStatus_t st = c.set_stream(h, s);
  if (st == CUBLAS_STATUS_SUCCESS) st = c.set_workspace(h, g.ws, g.ws_bytes);
  if (st == CUBLAS_STATUS_SUCCESS) {
    if (n == 0)   // E (rowsT x K) -= P^T (rowsT x W1) tab (W1 x K)
      st = c.gemm(h, CUBLAS_OP_T, CUBLAS_OP_N, (int)g.rowsT, (int)g.K, g.W1, &minus_one, g.T, CUDA_R_32F, g.W1,
                  g.tabK, CUDA_R_32F, g.W1, &one, E, CUDA_R_32F, (int)g.rowsT, CUBLAS_COMPUTE_32F,
                  CUBLAS_GEMM_DEFAULT);
    else          // E (K x rowsT) -= tab^T (K x W1) P (W1 x rowsT)
      st = c.gemm(h, CUBLAS_OP_T, CUBLAS_OP_N, (int)g.K, (int)g.rowsT, g.W1, &minus_one, g.tabK, CUDA_R_32F, g.W1,
                  g.T, CUDA_R_32F, g.W1, &one, E, CUDA_R_32F, (int)g.K, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
  }
  if (st != CUBLAS_STATUS_SUCCESS) {
    ctx->last_error = "cuBLAS GEMM of the two-stage residual failed (status " + std::to_string((int)st) + ")";
    return -1;
  }
  return launches;
}

int gemm_mttsp_enqueue(GemmMttsp& g, trals_ctx* ctx, const void* X, double* const* cores, const int64_t* I,
                       const int32_t* R, double* M, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                       bool tables_ready) {
  const ModeLayout& L = g.L;
  const int N = L.N, n = g.n;
  const int Rn = R[n], Rn1 = R[(n + 1) % N], Rs = L.Rs;
  const int WO = g.form == 1 ? Rn1 * Rs : Rs * Rn;
  int launches = tables_ready ? 0 : prepare_tables(g, cores, I, R, s);
  // stage 1: T^T (W1 x rowsT, so that each row of T is contiguous) = table (W1 x K) times X
  cublasHandle_t h = handle_of(ctx);
  if (!h) {
    ctx->last_error = "cuBLAS handle unavailable";
    return -1;
  }
  const CublasApi& c = api();
  const cudaDataType ty = g.xmode == kGemmF32 ? CUDA_R_32F : CUDA_R_16BF;
  const float one = 1.0f, zero = 0.0f;
  cublasStatus_t st = c.set_stream(h, s);
  if (st == CUBLAS_STATUS_SUCCESS) st = c.set_workspace(h, g.ws, g.ws_bytes);
  const cublasOperation_t opX = (n == 0) ? CUBLAS_OP_T : CUBLAS_OP_N;
  const int ldX = (n == 0) ? (int)g.rowsT : (int)g.K;
  if (ev0) cudaEventRecord(ev0, s);
  if (st == CUBLAS_STATUS_SUCCESS)
    st = c.gemm(h, CUBLAS_OP_N, opX, g.W1, (int)g.rowsT, (int)g.K, &one, g.tabK, ty, g.W1, X, ty, ldX, &zero, g.T,
                CUDA_R_32F, g.W1, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
  if (st == CUBLAS_STATUS_SUCCESS && g.xmode == kGemmBF16Split)
    st = c.gemm(h, CUBLAS_OP_N, opX, g.W1, (int)g.rowsT, (int)g.K, &one, g.tabK_lo, ty, g.W1, X, ty, ldX, &one, g.T,
                CUDA_R_32F, g.W1, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
  if (st != CUBLAS_STATUS_SUCCESS) {
    ctx->last_error = "cuBLAS GEMM of the two-stage MTTSP failed (status " + std::to_string((int)st) + ")";
    return -1;
  }
  // stage 2 and the FP64 reduction
  const dim3 grid((unsigned)g.In, (unsigned)g.nchunk);
  if (g.form == 1)
    gemm_stage2_kernel<1><<<grid, 256, 0, s>>>(g.T, g.W1, g.tabO, WO, g.nOther, g.Irows, Rn, Rn1, Rs, g.In, g.nchunk,
                                               g.part);
  else
    gemm_stage2_kernel<2><<<grid, 256, 0, s>>>(g.T, g.W1, g.tabO, WO, g.nOther, 0, Rn, Rn1, Rs, g.In, g.nchunk,
                                               g.part);
  const int64_t E = g.In * Rn * Rn1;
  gemm_reduce_kernel<<<grid_for(E), 256, 0, s>>>(g.part, g.nchunk, E, M);
  if (ev1) cudaEventRecord(ev1, s);
  return launches + 2;
}

}  // namespace trals
