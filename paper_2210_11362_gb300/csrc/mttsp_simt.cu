// MTTSP on CUDA cores (Alg. 2 lines 7-8): M_n = X_[n] G^{!=n}_[2], subchain rows generated on the
// fly from two partial-chain tables, never materialising G^{!=n}.  This is the FP64 path (and the
// generic fallback for the other element types on shapes the tensor-core kernel does not take).
// Also: the fused reconstruction / explicit residual pass over X (Sec. 4 error formula).
#include <algorithm>

#include "trals_internal.cuh"

namespace trals {

// ------------------------------------------------------------------ host: mode layout
ModeLayout make_mode_layout(int N, const int64_t* I, const int32_t* R, int n, const int64_t* Istore) {
  if (!Istore) Istore = I;
  ModeLayout L{};
  L.N = N;
  L.n = n;
  for (int t = 1; t < N; ++t) L.chain[t - 1] = (n + t) % N;
  L.Rn = R[n];
  L.Rn1 = R[(n + 1) % N];
  L.In = I[n];
  L.strideN = 1;
  L.Kpre = 1;
  for (int j = 0; j < n; ++j) {
    L.strideN *= Istore[j];
    L.Kpre *= I[j];
  }
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
                  std::vector<int64_t>& offU, const int64_t* Istore) {
  if (!Istore) Istore = I;
  int64_t stride[kMaxOrder];
  stride[0] = 1;
  for (int j = 1; j < N; ++j) stride[j] = stride[j - 1] * Istore[j - 1];
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

// Subchain rows of one tile: Gs[kk * r + (a + Rn b)] = sum_c Ltab[l][b + Rn1 c] Utab[u][c + Rs a], and
// base[kk] = the X offset of column kk.  (The FP64 kernels are bound by the FP64 pipe, so the
// per-element index arithmetic here runs on otherwise idle integer units.)
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
                                                              const void* __restrict__ X, double* __restrict__ partials,
                                                              int out_diff) {
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
      if (out != nullptr && !out_diff) out[off] = (OT)xh;
      if (X != nullptr) {
        const double xv = ld<XT>(X, off);
        const double d = xv - xh;
        if (out != nullptr && out_diff) out[off] = (OT)d;
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
    double a = 0.0, b = 0.0;  // per-block |X - X_hat|^2, |X|^2
    for (int w = 0; w < THREADS / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// ---- MTTSP on CUDA cores in FP32 arithmetic (reduced-precision modes, shapes the tensor-core
// kernel does not take).
//
// Columns of X_[n] are visited in memory order t = p + K_pre q (p over the modes before n, q over the
// modes after n), which is a permutation of the subchain order k = q + Q p; the sum over k does not
// depend on the order.  A tile holds FKT consecutive t: its X block is read coalesced, its subchain
// rows are generated from FP32 copies of the two partial-chain tables, and each thread accumulates
// a 4 x 4 block of M_n (rows i_n, columns a + R_n b) in FP32.  Per-CTA partials go out in FP64.
constexpr int FKT = 64;        // tile width (columns); 16 when the staged tables need the room
constexpr int kF32CtasPerSm = 6;

template <typename XT, int FKT>
__global__ void __launch_bounds__(THREADS, 4) mttsp_simt_f32_kernel(const void* __restrict__ X,
                                                                 const void* __restrict__ Xlo,
                                                                 const float* __restrict__ ltab,
                                                                 const float* __restrict__ utab,
                                                                 const int64_t* __restrict__ offL,
                                                                 const int64_t* __restrict__ offU, ModeLayout L,
                                                                 int64_t Kpre, int64_t Q, double* __restrict__ partials) {
  extern __shared__ float fs[];
  const int r = L.Rn * L.Rn1;
  const int In = (int)L.In;
  const int rp = (r + 3) & ~3, inp = (In + 3) & ~3;
  const int nLr = L.Rn1 * L.Rs, nUr = L.Rs * L.Rn;   // floats per Left / Right table row
  float* Gs = fs;                          // [FKT][rp]
  float* Xs = Gs + FKT * rp;               // [FKT][inp]
  float* Lt = Xs + FKT * inp;              // [FKT][nLr]: the tile columns' Left table rows
  float* Ut = Lt + FKT * nLr;              // [FKT][nUr]: and Right table rows
  int64_t* base = reinterpret_cast<int64_t*>(Ut + ((FKT * nUr + 1) & ~1));
  int64_t* lrow = base + FKT;              // table rows of column kk: Left l(k) and Right u(k)
  int64_t* urow = lrow + FKT;
  const int nrq = rp / 4, niq = inp / 4;
  const int mt = blockIdx.y * THREADS + threadIdx.x;
  const bool active = mt < nrq * niq;
  const int rq = mt % nrq, iq = mt / nrq;
  const int64_t chunk = (L.J + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * chunk;
  const int64_t t1 = min(L.J, t0 + chunk);
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
  for (int64_t tb = t0; tb < t1; tb += FKT) {
    // index arithmetic once per column (64-bit divisions are costly)
    for (int kk = threadIdx.x; kk < FKT; kk += blockDim.x) {
      const int64_t t = tb + kk;
      if (t < t1) {
        const int64_t k = t / Kpre + Q * (t % Kpre);
        const int64_t l = k % L.nL, u = k / L.nL;
        lrow[kk] = l;
        urow[kk] = u;
        base[kk] = offL[l] + offU[u];
      } else {
        base[kk] = -1;
      }
    }
    __syncthreads();
    // stage the two table rows of every tile column (contiguous rows: coalesced loads)
    for (int e = threadIdx.x; e < FKT * nLr; e += blockDim.x) {
      const int kk = e / nLr, q = e % nLr;
      Lt[e] = base[kk] >= 0 ? ltab[lrow[kk] * (int64_t)nLr + q] : 0.f;
    }
    for (int e = threadIdx.x; e < FKT * nUr; e += blockDim.x) {
      const int kk = e / nUr, q = e % nUr;
      Ut[e] = base[kk] >= 0 ? utab[urow[kk] * (int64_t)nUr + q] : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < FKT * rp; e += blockDim.x) {
      const int kk = e / rp, rr = e % rp;
      float g = 0.f;
      if (rr < r) {
        const int a = rr % L.Rn, b = rr / L.Rn;
        const float* Lp = Lt + kk * nLr;
        const float* Up = Ut + kk * nUr;
        for (int c = 0; c < L.Rs; ++c) g = fmaf(Lp[b + L.Rn1 * c], Up[c + L.Rs * a], g);
      }
      Gs[e] = g;
    }
    // X tile: four independent loads in flight per thread before any store
    for (int e0 = threadIdx.x; e0 < FKT * inp; e0 += 4 * blockDim.x) {
      float v[4];
      int dst[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = e0 + q * blockDim.x;
        int i = 0, kk = 0;
        if (Kpre == 1) {   // mode 0: memory is contiguous along i
          i = e % inp;
          kk = e / inp;
        } else {           // memory is contiguous along t
          kk = e % FKT;
          i = e / FKT;
        }
        dst[q] = e < FKT * inp ? kk * inp + i : -1;
        const int64_t bo = dst[q] >= 0 ? base[kk] : -1;
        v[q] = 0.f;
        if (i < In && bo >= 0) {
          const int64_t off = bo + (int64_t)i * L.strideN;
          v[q] = (float)ld<XT>(X, off);
          if (Xlo != nullptr) v[q] += (float)ld<XT>(Xlo, off);   // split-BF16 pair: hi + lo
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (dst[q] >= 0) Xs[dst[q]] = v[q];
    }
    __syncthreads();
    if (active) {
#pragma unroll 4
      for (int kk = 0; kk < FKT; ++kk) {
        const float4 xv = *reinterpret_cast<const float4*>(Xs + kk * inp + 4 * iq);
        const float4 gv = *reinterpret_cast<const float4*>(Gs + kk * rp + 4 * rq);
        const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc[u][0] = fmaf(xa[u], gv.x, acc[u][0]);
          acc[u][1] = fmaf(xa[u], gv.y, acc[u][1]);
          acc[u][2] = fmaf(xa[u], gv.z, acc[u][2]);
          acc[u][3] = fmaf(xa[u], gv.w, acc[u][3]);
        }
      }
    }
    __syncthreads();
  }
  if (!active) return;
  const int64_t outN = (int64_t)In * r;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = 4 * iq + u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int rr = 4 * rq + v;
      if (i < In && rr < r) partials[(int64_t)blockIdx.x * outN + i + (int64_t)In * rr] = (double)acc[u][v];
    }
  }
}

// ---- explicit residual with X_hat regenerated in FP32 (reduced-precision modes)
//
// |X - X_hat|^2 and |X|^2 against the caller's full-precision X, with X_hat = G_{n(2)} (G^{!=n}_[2])^T
// (Sec. 1 element formula, unfolded) evaluated in FP32 from FP32 copies of the subchain tables and
// of core n; the differences are formed and squared in FP64.  The FP32 regeneration error (about
// 1e-7 relative to |X_hat|) is far below what the residual is compared against (1e-4), while the
// FP64 arithmetic of the reconstruction above would cost ~100x more on GB300's FP64 pipe.
constexpr int RKT = 128;          // columns of X_[n] per tile
constexpr int GTS = RKT + 4;      // row stride of the transposed subchain rows (16-byte aligned, banks skewed)
constexpr int RIC = 32;           // rows of X_[n] per chunk: 8 warps x 4 rows

__global__ void tables_to_f32_kernel(const double* __restrict__ a, int64_t na, float* __restrict__ fa,
                                     const double* __restrict__ b, int64_t nb, float* __restrict__ fb) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < na + nb; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < na)
      fa[e] = (float)a[e];
    else
      fb[e - na] = (float)b[e - na];
  }
}

template <typename XT>
__global__ void __launch_bounds__(THREADS) residual_f32_kernel(const float* __restrict__ ltab,
                                                               const float* __restrict__ utab,
                                                               const int64_t* __restrict__ offL,
                                                               const int64_t* __restrict__ offU, ModeLayout L,
                                                               const double* __restrict__ coreN,
                                                               const void* __restrict__ X, double* __restrict__ partials,
                                                               float* __restrict__ Eout) {
  extern __shared__ float fsm[];
  __shared__ double red[2][THREADS / 32];
  const int r = L.Rn * L.Rn1;
  const int64_t In = L.In;
  float* Gt = fsm;                         // [r][GTS]: subchain rows, transposed
  float* Cs = Gt + (size_t)r * GTS;        // [RIC][r]: rows of G_{n(2)}
  int64_t* base = reinterpret_cast<int64_t*>(Cs + (size_t)RIC * r + 4);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t chunk = (L.J + gridDim.x - 1) / gridDim.x;
  const int64_t k0 = (int64_t)blockIdx.x * chunk;
  const int64_t k1 = min(L.J, k0 + chunk);
  double d2 = 0.0, x2 = 0.0;
  int64_t* lrow = base + RKT;
  int64_t* urow = lrow + RKT;
  for (int64_t kb = k0; kb < k1; kb += RKT) {
    for (int kk = threadIdx.x; kk < RKT; kk += blockDim.x) {
      const int64_t k = kb + kk;
      if (k < k1) {
        const int64_t l = k % L.nL, u = k / L.nL;
        lrow[kk] = l;
        urow[kk] = u;
        base[kk] = offL[l] + offU[u];
      } else {
        base[kk] = -1;
      }
    }
    __syncthreads();
    // lanes run along the row entries (a, b) of one column: the Left-table reads are then
    // contiguous (lanes along the columns touched 32 cache lines per warp load)
    for (int e = threadIdx.x; e < RKT * r; e += blockDim.x) {
      const int kk = e / r, rr = e % r;
      float acc = 0.f;
      if (base[kk] >= 0) {
        const int a = rr % L.Rn, b = rr / L.Rn;
        const float* Lp = ltab + lrow[kk] * (int64_t)L.Rn1 * L.Rs + b;
        const float* Up = utab + urow[kk] * (int64_t)L.Rs * L.Rn + L.Rs * a;
        // four independent chains: the table loads come from L2, and a single dependent chain
        // left the SMs waiting on them
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int c = 0;
        for (; c + 3 < L.Rs; c += 4) {
          a0 = fmaf(Lp[L.Rn1 * c], Up[c], a0);
          a1 = fmaf(Lp[L.Rn1 * (c + 1)], Up[c + 1], a1);
          a2 = fmaf(Lp[L.Rn1 * (c + 2)], Up[c + 2], a2);
          a3 = fmaf(Lp[L.Rn1 * (c + 3)], Up[c + 3], a3);
        }
        for (; c < L.Rs; ++c) a0 = fmaf(Lp[L.Rn1 * c], Up[c], a0);
        acc = (a0 + a1) + (a2 + a3);
      }
      Gt[rr * GTS + kk] = acc;
    }
    for (int64_t i0 = 0; i0 < In; i0 += RIC) {
      __syncthreads();   // Gt/base written; previous chunk's Cs reads done
      for (int e = threadIdx.x; e < RIC * r; e += blockDim.x) {
        const int ii = e / r, c = e % r;
        const int64_t i = i0 + ii;
        const int a = c % L.Rn, b = c / L.Rn;
        Cs[ii * r + c] = (i < In) ? (float)coreN[a + (int64_t)L.Rn * (i + In * b)] : 0.f;
      }
      __syncthreads();
      // micro-tile: rows i0 + 4 warp .. +3, columns 4 lane .. +3
      float acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
      const float* C0 = Cs + (warp * 4) * r;
      for (int c = 0; c < r; ++c) {
        const float4 g = *reinterpret_cast<const float4*>(Gt + c * GTS + 4 * lane);
        const float cv[4] = {C0[c], C0[r + c], C0[2 * r + c], C0[3 * r + c]};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc[u][0] = fmaf(cv[u], g.x, acc[u][0]);
          acc[u][1] = fmaf(cv[u], g.y, acc[u][1]);
          acc[u][2] = fmaf(cv[u], g.z, acc[u][2]);
          acc[u][3] = fmaf(cv[u], g.w, acc[u][3]);
        }
      }
      // issue all sixteen X loads before using any (they are independent; one DRAM latency per
      // chunk instead of one per element)
      double xv[4][4];
      int64_t off[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + warp * 4 + u;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int64_t bo = base[4 * lane + v];
          off[u][v] = (i < In && bo >= 0) ? bo + i * L.strideN : -1;
          xv[u][v] = off[u][v] >= 0 ? ld<XT>(X, off[u][v]) : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          if (off[u][v] < 0) continue;
          const double d = xv[u][v] - (double)acc[u][v];
          if (Eout != nullptr) Eout[off[u][v]] = (float)d;
          d2 = fma(d, d, d2);
          x2 = fma(xv[u][v], xv[u][v], x2);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    x2 += __shfl_xor_sync(0xffffffffu, x2, o);
  }
  if (lane == 0) {
    red[0][warp] = d2;
    red[1][warp] = x2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
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

static size_t f32_smem_w(const ModeLayout& L, int w) {
  const int r = L.Rn * L.Rn1;
  const int64_t rp = (r + 3) & ~3, inp = (L.In + 3) & ~3;
  const int64_t nLr = (int64_t)L.Rn1 * L.Rs, nUr = (int64_t)L.Rs * L.Rn;
  return (size_t)(w * (rp + inp + nLr) + ((w * nUr + 1) & ~1)) * sizeof(float) + 3 * w * sizeof(int64_t);
}

// tile width of the FP32 kernel for this layout: 64 columns, or 16 when that does not fit
static int f32_width(const ModeLayout& L) { return f32_smem_w(L, FKT) <= 200 * 1024 ? FKT : 16; }

size_t mttsp_simt_f32_smem(const ModeLayout& L) { return f32_smem_w(L, f32_width(L)); }

bool mttsp_simt_f32_fits(const ModeLayout& L) { return L.In <= 4096 && mttsp_simt_f32_smem(L) <= 200 * 1024; }

int mttsp_simt_f32_grid(const ModeLayout& L) {
  const int r = L.Rn * L.Rn1;
  const int64_t mts = (int64_t)((r + 3) / 4) * ((L.In + 3) / 4);
  const int64_t gy = (mts + THREADS - 1) / THREADS;
  // several CTAs per SM: each tile is a short chain of dependent steps, so SMs need many in flight
  const int64_t tiles = (L.J + f32_width(L) - 1) / f32_width(L);
  const int64_t by_partials = ((int64_t)8 << 20) / std::max<int64_t>(1, L.In * r);   // partials <= 64 MB
  return (int)std::max<int64_t>(
      1, std::min<int64_t>({tiles / 4, std::max<int64_t>(1, 152 * kF32CtasPerSm / gy), by_partials}));
}

void launch_mttsp_simt_f32(const MttspSimtArgs& a, const float* fl, const float* fu, cudaStream_t s) {
  const ModeLayout& L = a.L;
  const int r = L.Rn * L.Rn1;
  const int64_t outN = L.In * r;
  const int64_t mts = (int64_t)((r + 3) / 4) * ((L.In + 3) / 4);
  dim3 grid(a.gridX, (unsigned)((mts + THREADS - 1) / THREADS));
  const int64_t Kpre = L.Kpre;
  const int64_t Q = L.J / Kpre;
  const size_t smem = mttsp_simt_f32_smem(L);
  const bool wide = f32_width(L) == FKT;
  if (a.ev0) cudaEventRecord(a.ev0, s);
#define TRALS_F32(XT_, W_, LO_) \
  mttsp_simt_f32_kernel<XT_, W_><<<grid, THREADS, smem, s>>>(a.X, LO_, fl, fu, a.offL, a.offU, L, Kpre, Q, a.partials)
  if (a.xt == TRALS_X_F32) {
    if (wide) TRALS_F32(float, FKT, nullptr); else TRALS_F32(float, 16, nullptr);
  } else if (a.xt == TRALS_X_BF16) {
    if (wide) TRALS_F32(__nv_bfloat16, FKT, a.Xlo); else TRALS_F32(__nv_bfloat16, 16, a.Xlo);
  } else {
    if (wide) TRALS_F32(double, FKT, nullptr); else TRALS_F32(double, 16, nullptr);
  }
#undef TRALS_F32
  if (a.ev1) cudaEventRecord(a.ev1, s);
  const int rg = (int)std::min<int64_t>((outN + 255) / 256, 152 * 8);
  reduce_partials_kernel<<<rg, 256, 0, s>>>(a.partials, a.gridX, outN, a.M);
}

void launch_tables_to_f32(const double* a, int64_t na, float* fa, const double* b, int64_t nb, float* fb,
                          cudaStream_t s) {
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((na + nb + 255) / 256, 152 * 4));
  tables_to_f32_kernel<<<g, 256, 0, s>>>(a, na, fa, b, nb, fb);
}

size_t residual_f32_smem(const ModeLayout& L) {
  const int r = L.Rn * L.Rn1;
  return ((size_t)r * GTS + (size_t)RIC * r + 4) * sizeof(float) + 3 * RKT * sizeof(int64_t);
}

int residual_f32_grid(const ModeLayout& L) {
  const int64_t tiles = (L.J + RKT - 1) / RKT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 152 * 2));
}

void launch_residual_f32(const ModeLayout& L, const double* ltab, const double* utab, float* ftab, int64_t ltab_elems,
                         int64_t utab_elems, const int64_t* offL, const int64_t* offU, const double* coreN,
                         const void* X, int xt, double* partials, int gridX, cudaStream_t s, float* Eout) {
  float* fl = ftab;
  float* fu = ftab + ltab_elems;
  const int g = (int)std::min<int64_t>((ltab_elems + utab_elems + 255) / 256, 152 * 4);
  tables_to_f32_kernel<<<g, 256, 0, s>>>(ltab, ltab_elems, fl, utab, utab_elems, fu);
  const size_t smem = residual_f32_smem(L);
  if (xt == TRALS_X_F32)
    residual_f32_kernel<float><<<gridX, THREADS, smem, s>>>(fl, fu, offL, offU, L, coreN, X, partials, Eout);
  else if (xt == TRALS_X_BF16)
    residual_f32_kernel<__nv_bfloat16><<<gridX, THREADS, smem, s>>>(fl, fu, offL, offU, L, coreN, X, partials,
                                                                     Eout);
  else
    residual_f32_kernel<double><<<gridX, THREADS, smem, s>>>(fl, fu, offL, offU, L, coreN, X, partials, Eout);
}

size_t mttsp_simt_partials_elems(const ModeLayout& L, int gridX) {
  return (size_t)gridX * (size_t)(L.In * L.Rn * L.Rn1);
}

int mttsp_simt_default_grid(const ModeLayout& L) {
  const int64_t tiles = (L.J + KT - 1) / KT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 152 * 2));
}

static size_t simt_smem(const ModeLayout& L) {
  const int r = L.Rn * L.Rn1;
  return (size_t)KT * r * sizeof(double) + (size_t)L.In * KT * sizeof(double) + 3 * KT * sizeof(int64_t);
}

void launch_mttsp_simt(const MttspSimtArgs& a, cudaStream_t s) {
  const ModeLayout& L = a.L;
  const int64_t outN = L.In * L.Rn * L.Rn1;
  dim3 grid(a.gridX, (unsigned)((outN + OUTC - 1) / OUTC));
  const size_t smem = simt_smem(L);
  if (a.ev0) cudaEventRecord(a.ev0, s);
  if (a.xt == TRALS_X_F64)
    mttsp_simt_kernel<double><<<grid, THREADS, smem, s>>>(a.X, nullptr, a.ltab, a.utab, a.offL, a.offU, L, a.partials);
  else if (a.xt == TRALS_X_F32)
    mttsp_simt_kernel<float><<<grid, THREADS, smem, s>>>(a.X, nullptr, a.ltab, a.utab, a.offL, a.offU, L, a.partials);
  else
    mttsp_simt_kernel<__nv_bfloat16><<<grid, THREADS, smem, s>>>(a.X, a.Xlo, a.ltab, a.utab, a.offL, a.offU, L,
                                                                   a.partials);
  if (a.ev1) cudaEventRecord(a.ev1, s);
  const int rg = (int)std::min<int64_t>((outN + 255) / 256, 152 * 8);
  reduce_partials_kernel<<<rg, 256, 0, s>>>(a.partials, a.gridX, outN, a.M);
}

cudaError_t init_simt_attributes() {
  cudaError_t e = cudaFuncSetAttribute(mttsp_simt_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
#define TRALS_F32_ATTR(XT_, W_)                                                                           \
  if (e == cudaSuccess)                                                                                    \
    e = cudaFuncSetAttribute(mttsp_simt_f32_kernel<XT_, W_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             200 * 1024);
  TRALS_F32_ATTR(double, FKT)
  TRALS_F32_ATTR(float, FKT)
  TRALS_F32_ATTR(__nv_bfloat16, FKT)
  TRALS_F32_ATTR(double, 16)
  TRALS_F32_ATTR(float, 16)
  TRALS_F32_ATTR(__nv_bfloat16, 16)
#undef TRALS_F32_ATTR
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(residual_f32_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(residual_f32_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(residual_f32_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mttsp_simt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mttsp_simt_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return e;
}

void launch_reconstruct(const ModeLayout& L, const double* ltab, const double* utab, const int64_t* offL,
                        const int64_t* offU, const double* coreN, void* out, int out_t, const void* X, int xt,
                        double* partials, int gridX, cudaStream_t s, bool out_diff) {
  const int r = L.Rn * L.Rn1;
  const size_t smem = (size_t)KT * r * sizeof(double) + 3 * KT * sizeof(int64_t);
#define TRALS_RECON(XT_, OT_)                                                                                  \
  reconstruct_kernel<XT_, OT_><<<gridX, THREADS, smem, s>>>(ltab, utab, offL, offU, L, coreN, (OT_*)out, X, partials, \
                                                            out_diff ? 1 : 0)
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
