// Small, latency-bound steps of one TR-ALS-NE core update (Alg. 2 lines 2, 6, 9, 10) and the
// per-sweep residual (Sec. 4), all in FP64.
#include <math.h>

#include <algorithm>

#include "trals_internal.cuh"

namespace trals {

namespace {

__device__ __forceinline__ void set_status(DevStatus* st, int code, int sweep, int mode, int index, double v) {
  if (st == nullptr) return;
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->sweep = sweep;
    st->mode = mode;
    st->index = index;
    st->value = v;
  }
}

template <typename T>
__device__ __forceinline__ double load_as_double(const void* p, int64_t i);
template <>
__device__ __forceinline__ double load_as_double<double>(const void* p, int64_t i) {
  return static_cast<const double*>(p)[i];
}
template <>
__device__ __forceinline__ double load_as_double<float>(const void* p, int64_t i) {
  return (double)static_cast<const float*>(p)[i];
}
template <>
__device__ __forceinline__ double load_as_double<__nv_bfloat16>(const void* p, int64_t i) {
  return (double)__bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
}

// ------------------------------------------------------------------ K1: Gamma_k
// Gamma[(p Rn + q) + Rn^2 (s Rn1 + t)] = sum_i G[p,i,s] G[q,i,t]  (Alg. 2 lines 2/10, as the
// Kronecker sum G(i) (x) G(i)).  Symmetric under (p,s) <-> (q,t): each thread computes one entry
// with (p,s) <= (q,t) in column-major pair order and mirrors it.
__global__ void gamma_kernel(const double* __restrict__ G, int Rn, int64_t In, int Rn1,
                             double* __restrict__ Gamma) {
  const int64_t r = (int64_t)Rn * Rn1;
  const int64_t total = r * r;
  const int64_t rows = (int64_t)Rn * Rn;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = e % r;   // (p, s) flattened p + Rn s
    const int64_t v = e / r;   // (q, t)
    if (u > v) continue;
    const int p = (int)(u % Rn), s = (int)(u / Rn);
    const int q = (int)(v % Rn), t = (int)(v / Rn);
    const double* gu = G + p + (int64_t)Rn * In * s;
    const double* gv = G + q + (int64_t)Rn * In * t;
    double acc = 0.0;
    for (int64_t i = 0; i < In; ++i) acc = fma(gu[Rn * i], gv[Rn * i], acc);
    Gamma[(p * Rn + q) + rows * (int64_t)(s * Rn1 + t)] = acc;
    Gamma[(q * Rn + p) + rows * (int64_t)(t * Rn1 + s)] = acc;
  }
}

// ------------------------------------------------------------------ FP64 GEMM (Gamma chain, K2)
constexpr int GT = 16;
__global__ void gemm_f64_kernel(int m, int n, int k, const double* __restrict__ A, const double* __restrict__ B,
                                double* __restrict__ C) {
  __shared__ double As[GT][GT + 1];
  __shared__ double Bs[GT][GT + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.x * GT + tx;
  const int col = blockIdx.y * GT + ty;
  double acc = 0.0;
  for (int k0 = 0; k0 < k; k0 += GT) {
    // As[tx][ty] = A[row, k0+ty]; Bs[tx][ty] = B[k0+tx, col]
    As[tx][ty] = (row < m && k0 + ty < k) ? A[row + (int64_t)m * (k0 + ty)] : 0.0;
    Bs[tx][ty] = (k0 + tx < k && col < n) ? B[(k0 + tx) + (int64_t)k * col] : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GT; ++kk) acc = fma(As[tx][kk], Bs[kk][ty], acc);
    __syncthreads();
  }
  if (row < m && col < n) C[row + (int64_t)m * col] = acc;
}

// S[(a + Rn b) + r (a' + Rn b')] = Pi[(b Rn1 + b') + Rn1^2 (a Rn + a')]   (Prop. subchain_gram regrouping)
__global__ void regroup_S_kernel(const double* __restrict__ Pi, int Rn, int Rn1, double* __restrict__ S) {
  const int r = Rn * Rn1;
  const int total = r * r;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int row = e % r, col = e / r;
    const int a = row % Rn, b = row / Rn;
    const int a2 = col % Rn, b2 = col / Rn;
    S[e] = Pi[(b * Rn1 + b2) + (int64_t)Rn1 * Rn1 * (a * Rn + a2)];
  }
}

// ------------------------------------------------------------------ subchain tables (eq. subchain_new)
__global__ void chain_level_kernel(const double* __restrict__ prev, int64_t nPrev, int Ra, int Rc,
                                   const double* __restrict__ G, int64_t Ii, int Rb, double* __restrict__ out) {
  const int64_t per = (int64_t)Ra * Rb;
  const int64_t total = nPrev * Ii * per;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ent = e / per;
    const int xy = (int)(e % per);
    const int x = xy % Ra, y = xy / Ra;
    const int64_t l = ent % nPrev, i = ent / nPrev;
    double acc;
    if (prev == nullptr) {
      acc = G[x + (int64_t)Rc * (i + Ii * y)];
    } else {
      const double* P = prev + l * (int64_t)Ra * Rc;
      acc = 0.0;
      for (int c = 0; c < Rc; ++c) acc = fma(P[x + (int64_t)Ra * c], G[c + (int64_t)Rc * (i + Ii * y)], acc);
    }
    out[e] = acc;
  }
}

// ------------------------------------------------------------------ K4: Cholesky (single CTA)
// Right-looking column Cholesky of the lower triangle of S (r x r), Golub & Van Loan Sec. 5.3.2
// method cited for Alg. 2 line 9.  Works in shared memory when r <= kCholSmemMax, else in Lmat.
constexpr int kCholSmemMax = 128;
constexpr int kCholThreads = 1024;

__global__ void __launch_bounds__(kCholThreads) cholesky_kernel(const double* __restrict__ S, double* __restrict__ Lmat,
                                                                 int r, DevStatus* st, const int* sweep_ctr, int mode) {
  extern __shared__ double sm[];
  __shared__ int fail;
  const bool in_smem = r <= kCholSmemMax;
  double* A = in_smem ? sm : Lmat;
  const int lda = r;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < r * r; e += nt) {
    const int i = e % r, j = e / r;
    A[e] = (i >= j) ? S[e] : 0.0;
  }
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (tid == 0) {
      const double d = A[j + lda * j];
      if (!(d > 0.0) || !isfinite(d)) {
        fail = 1;
        set_status(st, isfinite(d) ? TRALS_E_NOT_SPD : TRALS_E_NONFINITE, sweep_ctr ? *sweep_ctr : -1, mode, j, d);
      } else {
        A[j + lda * j] = sqrt(d);
      }
    }
    __syncthreads();
    if (fail) return;
    const double djj = A[j + lda * j];
    for (int i = j + 1 + tid; i < r; i += nt) A[i + lda * j] = A[i + lda * j] / djj;
    __syncthreads();
    const int m = r - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int i = j + 1 + e % m, k = j + 1 + e / m;
      if (i >= k) A[i + lda * k] = fma(-A[i + lda * j], A[k + lda * j], A[i + lda * k]);
    }
    __syncthreads();
  }
  if (in_smem)
    for (int e = tid; e < r * r; e += nt) Lmat[e] = A[e];
}

// Two triangular solves per right-hand side (one warp per row i of M):  L y = M[i,:]^T,
// L^T z = y, then G[a + Rn (i + In b)] = z[a + Rn b] (classical mode-2 folding).
__global__ void chol_solve_kernel(const double* __restrict__ Lmat, const double* __restrict__ M, int Rn, int64_t In,
                                  int Rn1, double* __restrict__ G, DevStatus* st) {
  extern __shared__ double y[];
  const int r = Rn * Rn1;
  const int lane = threadIdx.x;
  const int64_t i = blockIdx.x;
  for (int j = lane; j < r; j += 32) y[j] = M[i + In * (int64_t)j];
  __syncwarp();
  for (int j = 0; j < r; ++j) {
    const double yj = y[j] / Lmat[j + (int64_t)r * j];
    __syncwarp();
    if (lane == 0) y[j] = yj;
    for (int k = j + 1 + lane; k < r; k += 32) y[k] = fma(-Lmat[k + (int64_t)r * j], yj, y[k]);
    __syncwarp();
  }
  for (int j = r - 1; j >= 0; --j) {
    double part = 0.0;
    for (int k = j + 1 + lane; k < r; k += 32) part = fma(Lmat[k + (int64_t)r * j], y[k], part);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const double zj = (y[j] - part) / Lmat[j + (int64_t)r * j];
    __syncwarp();
    if (lane == 0) y[j] = zj;
    __syncwarp();
  }
  for (int c = lane; c < r; c += 32) {
    const double z = y[c];
    if (!isfinite(z)) set_status(st, TRALS_E_NONFINITE, -1, -1, (int)i, z);
    const int a = c % Rn, b = c / Rn;
    G[a + (int64_t)Rn * (i + In * b)] = z;
  }
}

// ------------------------------------------------------------------ K6: residual identity (Sec. 4)
// res2 = |X|^2 - 2 <M, Z> + <S, Z^T Z>,  Z = G_{n(2)};  (Z^T Z)[(a + Rn b), (a' + Rn b')] =
// Gamma[(a Rn + a') + Rn^2 (b Rn1 + b')].
__global__ void residual_identity_kernel(const double* __restrict__ normX2, const double* __restrict__ M,
                                         const double* __restrict__ G, const double* __restrict__ S,
                                         const double* __restrict__ Gam, int Rn, int64_t In, int Rn1,
                                         double* __restrict__ res_hist, int* sweep_ctr) {
  __shared__ double red[2][32];
  const int r = Rn * Rn1;
  double cross = 0.0, quad = 0.0;
  for (int64_t e = threadIdx.x; e < In * r; e += blockDim.x) {
    const int64_t i = e % In;
    const int c = (int)(e / In);
    const int a = c % Rn, b = c / Rn;
    cross = fma(M[e], G[a + (int64_t)Rn * (i + In * b)], cross);
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int row = e % r, col = e / r;
    const int a = row % Rn, b = row / Rn, a2 = col % Rn, b2 = col / Rn;
    quad = fma(S[e], Gam[(a * Rn + a2) + (int64_t)Rn * Rn * (b * Rn1 + b2)], quad);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cross += __shfl_xor_sync(0xffffffffu, cross, o);
    quad += __shfl_xor_sync(0xffffffffu, quad, o);
  }
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) {
    red[0][w] = cross;
    red[1][w] = quad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double c = 0.0, q = 0.0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) {
      c += red[0][k];
      q += red[1][k];
    }
    const double nx = *normX2;
    const double res2 = nx - 2.0 * c + q;
    const int s = *sweep_ctr;
    res_hist[s] = sqrt(fmax(res2, 0.0) / nx);
    *sweep_ctr = s + 1;
  }
}

// ------------------------------------------------------------------ reductions and conversions
template <typename XT>
__global__ void sumsq_kernel(const void* __restrict__ X, int64_t count, double* __restrict__ partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = load_as_double<XT>(X, e);
    acc = fma(v, v, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) s += red[k];
    partials[blockIdx.x] = s;
  }
}

// out[j] = sum_b partials[j + stride * b] for j < width, fixed order (one block, deterministic)
__global__ void reduce_fixed_kernel(const double* __restrict__ partials, int count, int width, double* __restrict__ out) {
  __shared__ double red[1024];
  for (int j = 0; j < width; ++j) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < count; b += blockDim.x) acc += partials[j + (int64_t)width * b];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = red[0];
    __syncthreads();
  }
}

template <typename XT>
__global__ void quantize_kernel(const void* __restrict__ src, int64_t count, __nv_bfloat16* __restrict__ hi,
                                __nv_bfloat16* __restrict__ lo) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = load_as_double<XT>(src, e);
    const float vf = (float)v;
    const __nv_bfloat16 h = __float2bfloat16_rn(vf);
    hi[e] = h;
    if (lo != nullptr) lo[e] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
  }
}

__global__ void convert_f32_kernel(const double* __restrict__ src, int64_t count, float* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}

__global__ void zero_status_kernel(DevStatus* st) {
  st->code = 0;
  st->sweep = -1;
  st->mode = -1;
  st->index = -1;
  st->value = 0.0;
}

inline int grid_for(int64_t total, int block, int cap = 152 * 16) {
  int64_t g = (total + block - 1) / block;
  if (g < 1) g = 1;
  return (int)std::min<int64_t>(g, cap);
}

}  // namespace

// ------------------------------------------------------------------ launchers
void launch_gamma(const double* G, int Rn, int64_t In, int Rn1, double* Gamma, cudaStream_t s) {
  const int64_t total = (int64_t)Rn * Rn1 * Rn * Rn1;
  gamma_kernel<<<grid_for(total, 256), 256, 0, s>>>(G, Rn, In, Rn1, Gamma);
}

void launch_gemm_f64(int m, int n, int k, const double* A, const double* B, double* C, cudaStream_t s) {
  dim3 grid((m + GT - 1) / GT, (n + GT - 1) / GT);
  gemm_f64_kernel<<<grid, dim3(GT, GT), 0, s>>>(m, n, k, A, B, C);
}

void launch_regroup_S(const double* Pi, int Rn, int Rn1, double* S, cudaStream_t s) {
  const int r = Rn * Rn1;
  regroup_S_kernel<<<grid_for((int64_t)r * r, 256), 256, 0, s>>>(Pi, Rn, Rn1, S);
}

void launch_chain_level(const double* prev, int64_t nPrev, int Ra, int Rc, const double* G, int64_t Ii, int Rb,
                        double* out, cudaStream_t s) {
  const int64_t total = nPrev * Ii * Ra * Rb;
  chain_level_kernel<<<grid_for(total, 256, 152 * 64), 256, 0, s>>>(prev, nPrev, Ra, Rc, G, Ii, Rb, out);
}

void build_tables(const ModeLayout& L, const double* const* cores, const int64_t* I, const int32_t* R,
                  double* ltab, double* utab, double* scratch, cudaStream_t s) {
  // Left table over chain positions [0, m), Right table over [m, N-1); each level multiplies the
  // running product by the next core's slice (subchain product, eq. subchain_new), ping-ponging
  // between the destination and the scratch buffer so the last level lands in the destination.
  auto build = [&](int t0, int t1, double* dst) {
    const int levels = t1 - t0;
    double* buf0 = (levels % 2 == 1) ? dst : scratch;
    double* buf1 = (levels % 2 == 1) ? scratch : dst;
    const double* prev = nullptr;
    int64_t nPrev = 1;
    const int Ra = R[L.chain[t0]];
    for (int t = t0; t < t1; ++t) {
      const int mode = L.chain[t];
      const int Rc = R[mode];
      const int Rb = R[(mode + 1) % L.N];
      double* out = ((t - t0) % 2 == 0) ? buf0 : buf1;
      launch_chain_level(prev, nPrev, Ra, Rc, cores[mode], I[mode], Rb, out, s);
      prev = out;
      nPrev *= I[mode];
    }
  };
  build(0, L.m, ltab);
  build(L.m, L.N - 1, utab);
}

int64_t table_level_max_elems(const ModeLayout& L, const int64_t* I, const int32_t* R) {
  int64_t mx = 0;
  auto scan = [&](int t0, int t1) {
    int64_t n = 1;
    const int Ra = R[L.chain[t0]];
    for (int t = t0; t < t1; ++t) {
      const int mode = L.chain[t];
      n *= I[mode];
      mx = std::max<int64_t>(mx, n * Ra * R[(mode + 1) % L.N]);
    }
  };
  scan(0, L.m);
  scan(L.m, L.N - 1);
  return mx;
}

void launch_cholesky(const double* S, double* Lmat, int r, DevStatus* st, const int* sweep_ctr, int mode,
                     cudaStream_t s) {
  const size_t smem = (r <= kCholSmemMax) ? (size_t)r * r * sizeof(double) : 0;
  cholesky_kernel<<<1, kCholThreads, smem, s>>>(S, Lmat, r, st, sweep_ctr, mode);
}

void launch_chol_solve(const double* Lmat, const double* M, int Rn, int64_t In, int Rn1, double* G, DevStatus* st,
                       cudaStream_t s) {
  const int r = Rn * Rn1;
  chol_solve_kernel<<<(unsigned)In, 32, (size_t)r * sizeof(double), s>>>(Lmat, M, Rn, In, Rn1, G, st);
}

void launch_residual_identity(const double* normX2, const double* M, const double* coreN, const double* S,
                              const double* gammaN, int Rn, int64_t In, int Rn1, double* res_hist, int* sweep_ctr,
                              cudaStream_t s) {
  residual_identity_kernel<<<1, 1024, 0, s>>>(normX2, M, coreN, S, gammaN, Rn, In, Rn1, res_hist, sweep_ctr);
}

void launch_sumsq(const void* X, int xt, int64_t count, double* partials, int gridX, double* out, cudaStream_t s) {
  if (xt == TRALS_X_F64)
    sumsq_kernel<double><<<gridX, 256, 0, s>>>(X, count, partials);
  else if (xt == TRALS_X_F32)
    sumsq_kernel<float><<<gridX, 256, 0, s>>>(X, count, partials);
  else
    sumsq_kernel<__nv_bfloat16><<<gridX, 256, 0, s>>>(X, count, partials);
  reduce_fixed_kernel<<<1, 1024, 0, s>>>(partials, gridX, 1, out);
}

void launch_reduce_pairs(const double* partials, int count, double* out, cudaStream_t s) {
  reduce_fixed_kernel<<<1, 1024, 0, s>>>(partials, count, 2, out);
}

void launch_quantize(const void* src, int src_t, int64_t count, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t s) {
  const int g = grid_for(count, 256, 152 * 32);
  if (src_t == TRALS_X_F64)
    quantize_kernel<double><<<g, 256, 0, s>>>(src, count, hi, lo);
  else
    quantize_kernel<float><<<g, 256, 0, s>>>(src, count, hi, lo);
}

void launch_zero_status(DevStatus* st, cudaStream_t s) { zero_status_kernel<<<1, 1, 0, s>>>(st); }

void launch_convert_f32(const void* src_f64, int64_t count, float* dst, cudaStream_t s) {
  convert_f32_kernel<<<grid_for(count, 256, 152 * 32), 256, 0, s>>>(static_cast<const double*>(src_f64), count, dst);
}

cudaError_t init_small_attributes() {
  return cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kCholSmemMax * kCholSmemMax * (int)sizeof(double));
}

}  // namespace trals
