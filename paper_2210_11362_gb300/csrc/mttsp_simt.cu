// MTTSP on CUDA cores (Alg. 2 lines 7-8): M_n = X_[n] G^{!=n}_[2], subchain rows generated on the
// fly from two partial-chain tables, never materialising G^{!=n}.  This is the FP64 path (and the
// generic fallback for the other element types on shapes the tensor-core kernel does not take).
// Also: the fused reconstruction / explicit residual pass over X (Sec. 4 error formula).
#include <algorithm>

#include "trals_internal.cuh"

namespace trals {

// ------------------------------------------------------------------ host: mode layout
ModeLayout make_mode_layout(int N, const int64_t* I, const int32_t* R, int n) {
  ModeLayout L{};
  L.N = N;
  L.n = n;
  for (int t = 1; t < N; ++t) L.chain[t - 1] = (n + t) % N;
  L.Rn = R[n];
  L.Rn1 = R[(n + 1) % N];
  L.In = I[n];
  L.strideN = 1;
  for (int j = 0; j < n; ++j) L.strideN *= I[j];
  L.J = 1;
  for (int j = 0; j < N; ++j)
    if (j != n) L.J *= I[j];
  int64_t best = -1;
  for (int m = 1; m <= N - 2; ++m) {
    int64_t nL = 1, nU = 1;
    for (int t = 0; t < m; ++t) nL *= I[L.chain[t]];
    for (int t = m; t < N - 1; ++t) nU *= I[L.chain[t]];
    const int Rs = R[L.chain[m]];
    const int64_t cost = nL * L.Rn1 * Rs + nU * Rs * L.Rn;
    if (best < 0 || cost < best) {
      best = cost;
      L.m = m;
      L.nL = nL;
      L.nU = nU;
      L.Rs = Rs;
    }
  }
  return L;
}

void mode_offsets(int N, const int64_t* I, const ModeLayout& L, std::vector<int64_t>& offL,
                  std::vector<int64_t>& offU) {
  int64_t stride[kMaxOrder];
  stride[0] = 1;
  for (int j = 1; j < N; ++j) stride[j] = stride[j - 1] * I[j - 1];
  auto fill = [&](int t0, int t1, int64_t count, std::vector<int64_t>& out) {
    out.assign((size_t)count, 0);
    for (int64_t e = 0; e < count; ++e) {
      int64_t rem = e, off = 0;
      for (int t = t0; t < t1; ++t) {
        const int mode = L.chain[t];
        off += (rem % I[mode]) * stride[mode];
        rem /= I[mode];
      }
      out[(size_t)e] = off;
    }
  };
  fill(0, L.m, L.nL, offL);
  fill(L.m, N - 1, L.nU, offU);
}

namespace {

constexpr int KT = 16;          // columns of X_[n] per tile
constexpr int THREADS = 256;
constexpr int NACC = 16;        // accumulators per thread
constexpr int OUTC = THREADS * NACC;

template <typename T>
__device__ __forceinline__ double ld(const void* p, int64_t i);
template <>
__device__ __forceinline__ double ld<double>(const void* p, int64_t i) {
  return static_cast<const double*>(p)[i];
}
template <>
__device__ __forceinline__ double ld<float>(const void* p, int64_t i) {
  return (double)static_cast<const float*>(p)[i];
}
template <>
__device__ __forceinline__ double ld<__nv_bfloat16>(const void* p, int64_t i) {
  return (double)__bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
}

// Subchain rows of one tile: Gs[kk * r + (a + Rn b)] = sum_c Ltab[l][b + Rn1 c] Utab[u][c + Rs a]
__device__ __forceinline__ void gen_tile(const ModeLayout& L, const double* __restrict__ ltab,
                                         const double* __restrict__ utab, const int64_t* __restrict__ offL,
                                         const int64_t* __restrict__ offU, int64_t kbase, int64_t kend, double* Gs,
                                         int64_t* base) {
  const int r = L.Rn * L.Rn1;
  for (int e = threadIdx.x; e < KT * r; e += blockDim.x) {
    const int kk = e / r, rr = e % r;
    const int64_t k = kbase + kk;
    double acc = 0.0;
    if (k < kend) {
      const int64_t l = k % L.nL, u = k / L.nL;
      const int a = rr % L.Rn, b = rr / L.Rn;
      const double* Lp = ltab + l * (int64_t)L.Rn1 * L.Rs;
      const double* Up = utab + u * (int64_t)L.Rs * L.Rn;
      for (int c = 0; c < L.Rs; ++c) acc = fma(Lp[b + L.Rn1 * c], Up[c + L.Rs * a], acc);
    }
    Gs[e] = acc;
  }
  for (int kk = threadIdx.x; kk < KT; kk += blockDim.x) {
    const int64_t k = kbase + kk;
    base[kk] = (k < kend) ? offL[k % L.nL] + offU[k / L.nL] : -1;
  }
}

template <typename XT>
__global__ void __launch_bounds__(THREADS) mttsp_simt_kernel(const void* __restrict__ X, const void* __restrict__ Xlo,
                                                             const double* __restrict__ ltab,
                                                             const double* __restrict__ utab,
                                                             const int64_t* __restrict__ offL,
                                                             const int64_t* __restrict__ offU, ModeLayout L,
                                                             double* __restrict__ partials) {
  extern __shared__ double smem[];
  const int r = L.Rn * L.Rn1;
  const int64_t In = L.In;
  double* Gs = smem;                       // KT * r
  double* Xs = Gs + KT * r;                // In * KT
  int64_t* base = reinterpret_cast<int64_t*>(Xs + In * KT);
  const int64_t outN = In * r;
  const int64_t e0 = (int64_t)blockIdx.y * OUTC;
  const int64_t chunk = (L.J + gridDim.x - 1) / gridDim.x;
  const int64_t k0 = (int64_t)blockIdx.x * chunk;
  const int64_t k1 = min(L.J, k0 + chunk);
  double acc[NACC];
#pragma unroll
  for (int j = 0; j < NACC; ++j) acc[j] = 0.0;
  for (int64_t kb = k0; kb < k1; kb += KT) {
    gen_tile(L, ltab, utab, offL, offU, kb, k1, Gs, base);
    __syncthreads();
    for (int64_t e = threadIdx.x; e < In * KT; e += blockDim.x) {
      const int64_t i = e % In;
      const int kk = (int)(e / In);
      const int64_t bo = base[kk];
      double v = 0.0;
      if (bo >= 0) {
        v = ld<XT>(X, bo + i * L.strideN);
        if (Xlo != nullptr) v += ld<XT>(Xlo, bo + i * L.strideN);   // split-BF16 pair: hi + lo
      }
      Xs[i * KT + kk] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NACC; ++j) {
      const int64_t e = e0 + threadIdx.x + (int64_t)THREADS * j;
      if (e < outN) {
        const int64_t i = e % In;
        const int rr = (int)(e / In);
        double s = acc[j];
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) s = fma(Xs[i * KT + kk], Gs[kk * r + rr], s);
        acc[j] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < NACC; ++j) {
    const int64_t e = e0 + threadIdx.x + (int64_t)THREADS * j;
    if (e < outN) partials[(int64_t)blockIdx.x * outN + e] = acc[j];
  }
}

// M[e] = sum_b partials[b * outN + e], fixed order over b
__global__ void reduce_partials_kernel(const double* __restrict__ partials, int gridX, int64_t outN,
                                       double* __restrict__ M) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < outN; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < gridX; ++b) s += partials[(int64_t)b * outN + e];
    M[e] = s;
  }
}

// Reconstruction (Sec. 1 element formula in the unfolded form X_[n] = G_{n(2)} (G^{!=n}_[2])^T):
// writes X_hat to `out` (typed) and/or accumulates |X - X_hat|^2 and |X|^2 per block.
template <typename XT, typename OT>
__global__ void __launch_bounds__(THREADS) reconstruct_kernel(const double* __restrict__ ltab,
                                                              const double* __restrict__ utab,
                                                              const int64_t* __restrict__ offL,
                                                              const int64_t* __restrict__ offU, ModeLayout L,
                                                              const double* __restrict__ coreN, OT* __restrict__ out,
                                                              const void* __restrict__ X, double* __restrict__ partials) {
  extern __shared__ double smem[];
  __shared__ double red[2][THREADS / 32];
  const int r = L.Rn * L.Rn1;
  const int64_t In = L.In;
  double* Gs = smem;
  int64_t* base = reinterpret_cast<int64_t*>(Gs + KT * r);
  const int64_t chunk = (L.J + gridDim.x - 1) / gridDim.x;
  const int64_t k0 = (int64_t)blockIdx.x * chunk;
  const int64_t k1 = min(L.J, k0 + chunk);
  double d2 = 0.0, x2 = 0.0;
  for (int64_t kb = k0; kb < k1; kb += KT) {
    gen_tile(L, ltab, utab, offL, offU, kb, k1, Gs, base);
    __syncthreads();
    for (int64_t e = threadIdx.x; e < In * KT; e += blockDim.x) {
      const int64_t i = e % In;
      const int kk = (int)(e / In);
      const int64_t bo = base[kk];
      if (bo < 0) continue;
      double xh = 0.0;
      for (int c = 0; c < r; ++c) {
        const int a = c % L.Rn, b = c / L.Rn;
        xh = fma(coreN[a + (int64_t)L.Rn * (i + In * b)], Gs[kk * r + c], xh);
      }
      const int64_t off = bo + i * L.strideN;
      if (out != nullptr) out[off] = (OT)xh;
      if (X != nullptr) {
        const double xv = ld<XT>(X, off);
        const double d = xv - xh;
        d2 = fma(d, d, d2);
        x2 = fma(xv, xv, x2);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    x2 += __shfl_xor_sync(0xffffffffu, x2, o);
  }
  if (threadIdx.x % 32 == 0) {
    red[0][threadIdx.x / 32] = d2;
    red[1][threadIdx.x / 32] = x2;
  }
  __syncthreads();
  if (threadIdx.x == 0 && partials != nullptr) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < THREADS / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

}  // namespace

size_t mttsp_simt_partials_elems(const ModeLayout& L, int gridX) {
  return (size_t)gridX * (size_t)(L.In * L.Rn * L.Rn1);
}

int mttsp_simt_default_grid(const ModeLayout& L) {
  const int64_t tiles = (L.J + KT - 1) / KT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 152 * 2));
}

static size_t simt_smem(const ModeLayout& L) {
  const int r = L.Rn * L.Rn1;
  return (size_t)KT * r * sizeof(double) + (size_t)L.In * KT * sizeof(double) + KT * sizeof(int64_t);
}

void launch_mttsp_simt(const MttspSimtArgs& a, cudaStream_t s) {
  const ModeLayout& L = a.L;
  const int64_t outN = L.In * L.Rn * L.Rn1;
  dim3 grid(a.gridX, (unsigned)((outN + OUTC - 1) / OUTC));
  const size_t smem = simt_smem(L);
  if (a.xt == TRALS_X_F64)
    mttsp_simt_kernel<double><<<grid, THREADS, smem, s>>>(a.X, nullptr, a.ltab, a.utab, a.offL, a.offU, L, a.partials);
  else if (a.xt == TRALS_X_F32)
    mttsp_simt_kernel<float><<<grid, THREADS, smem, s>>>(a.X, nullptr, a.ltab, a.utab, a.offL, a.offU, L, a.partials);
  else
    mttsp_simt_kernel<__nv_bfloat16><<<grid, THREADS, smem, s>>>(a.X, a.Xlo, a.ltab, a.utab, a.offL, a.offU, L,
                                                                   a.partials);
  const int rg = (int)std::min<int64_t>((outN + 255) / 256, 152 * 8);
  reduce_partials_kernel<<<rg, 256, 0, s>>>(a.partials, a.gridX, outN, a.M);
}

cudaError_t init_simt_attributes() {
  cudaError_t e = cudaFuncSetAttribute(mttsp_simt_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mttsp_simt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mttsp_simt_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return e;
}

void launch_reconstruct(const ModeLayout& L, const double* ltab, const double* utab, const int64_t* offL,
                        const int64_t* offU, const double* coreN, void* out, int out_t, const void* X, int xt,
                        double* partials, int gridX, cudaStream_t s) {
  const int r = L.Rn * L.Rn1;
  const size_t smem = (size_t)KT * r * sizeof(double) + KT * sizeof(int64_t);
#define TRALS_RECON(XT_, OT_) \
  reconstruct_kernel<XT_, OT_><<<gridX, THREADS, smem, s>>>(ltab, utab, offL, offU, L, coreN, (OT_*)out, X, partials)
  if (out == nullptr || out_t == TRALS_X_F64) {
    if (xt == TRALS_X_F32)
      TRALS_RECON(float, double);
    else if (xt == TRALS_X_BF16)
      TRALS_RECON(__nv_bfloat16, double);
    else
      TRALS_RECON(double, double);
  } else if (out_t == TRALS_X_F32) {
    TRALS_RECON(double, float);
  } else {
    TRALS_RECON(double, __nv_bfloat16);
  }
#undef TRALS_RECON
}

}  // namespace trals
