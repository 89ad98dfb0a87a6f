// Small, latency-bound steps of one TR-ALS-NE core update (Alg. 2 lines 2, 6, 9, 10) and the
// per-sweep residual (Sec. 4), all in FP64.
#include <math.h>

#include <algorithm>

#include "trals_internal.cuh"

namespace trals {

namespace {

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
    // four independent partial sums: the FP64 pipe has a long latency on this part
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t i = 0;
    for (; i + 3 < In; i += 4) {
      a0 = fma(gu[Rn * i], gv[Rn * i], a0);
      a1 = fma(gu[Rn * (i + 1)], gv[Rn * (i + 1)], a1);
      a2 = fma(gu[Rn * (i + 2)], gv[Rn * (i + 2)], a2);
      a3 = fma(gu[Rn * (i + 3)], gv[Rn * (i + 3)], a3);
    }
    for (; i < In; ++i) a0 = fma(gu[Rn * i], gv[Rn * i], a0);
    const double acc = (a0 + a1) + (a2 + a3);
    Gamma[(p * Rn + q) + rows * (int64_t)(s * Rn1 + t)] = acc;
    Gamma[(q * Rn + p) + rows * (int64_t)(t * Rn1 + s)] = acc;
  }
}

// The same Gram entries with the core staged in shared memory (cores up to kGammaSmemMax doubles):
// every block reads the core once, coalesced, instead of every thread gathering strided columns.
constexpr int kGammaSmemMax = 12288;
__global__ void gamma_smem_kernel(const double* __restrict__ G, int Rn, int In, int Rn1, double* __restrict__ Gamma) {
  extern __shared__ double Gs[];
  const int core = Rn * In * Rn1;
#pragma unroll 8
  for (int e = threadIdx.x; e < core; e += blockDim.x) Gs[e] = G[e];   // loads batched, not one round trip each
  __syncthreads();
  const int r = Rn * Rn1, rows = Rn * Rn;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
    const int u = e % r, v = e / r;
    if (u > v) continue;
    const int p = u % Rn, s = u / Rn;
    const int q = v % Rn, t = v / Rn;
    const double* gu = Gs + p + Rn * In * s;
    const double* gv = Gs + q + Rn * In * t;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int i = 0;
    for (; i + 3 < In; i += 4) {
      a0 = fma(gu[Rn * i], gv[Rn * i], a0);
      a1 = fma(gu[Rn * (i + 1)], gv[Rn * (i + 1)], a1);
      a2 = fma(gu[Rn * (i + 2)], gv[Rn * (i + 2)], a2);
      a3 = fma(gu[Rn * (i + 3)], gv[Rn * (i + 3)], a3);
    }
    for (; i < In; ++i) a0 = fma(gu[Rn * i], gv[Rn * i], a0);
    const double acc = (a0 + a1) + (a2 + a3);
    Gamma[(p * Rn + q) + rows * (s * Rn1 + t)] = acc;
    Gamma[(q * Rn + p) + rows * (t * Rn1 + s)] = acc;
  }
}

// The Gram entries as a small tiled product, for the sweep: Gamma is the Gram matrix of the mode-2
// unfolding G_[2] (I_n x r), (G_[2]^T G_[2])[(p + Rn s), (q + Rn t)] = sum_i G[p, i, s] G[q, i, t],
// stored regrouped.  Each block owns an 8 x 8 tile of (u, v) and its four 64-thread groups take
// interleaved quarters of i, summed in a fixed order; the whole square is formed (twice the work of
// the symmetric half, which is negligible) so no block idles.
__global__ void __launch_bounds__(256) gamma_tiled_kernel(const double* __restrict__ G, int Rn, int In, int Rn1,
                                                          double* __restrict__ Gamma) {
  __shared__ double part[4][64];
  const int t = threadIdx.x, o = t % 64, g = t / 64;
  const int r = Rn * Rn1;
  const int u = blockIdx.x * 8 + (o % 8), v = blockIdx.y * 8 + (o / 8);
  double a0 = 0.0, a1 = 0.0;
  if (u < r && v < r) {
    const int p = u % Rn, s = u / Rn, q = v % Rn, tt = v / Rn;
    const double* gu = G + p + (int64_t)Rn * In * s;
    const double* gv = G + q + (int64_t)Rn * In * tt;
    int i = g;
#pragma unroll 4
    for (; i + 4 < In; i += 8) {
      a0 = fma(gu[(int64_t)Rn * i], gv[(int64_t)Rn * i], a0);
      a1 = fma(gu[(int64_t)Rn * (i + 4)], gv[(int64_t)Rn * (i + 4)], a1);
    }
    if (i < In) a0 = fma(gu[(int64_t)Rn * i], gv[(int64_t)Rn * i], a0);
  }
  part[g][o] = a0 + a1;
  __syncthreads();
  if (g == 0 && u < r && v < r) {
    const int p = u % Rn, s = u / Rn, q = v % Rn, tt = v / Rn;
    Gamma[(p * Rn + q) + (int64_t)Rn * Rn * (s * Rn1 + tt)] = (part[0][o] + part[1][o]) + (part[2][o] + part[3][o]);
  }
}

// ------------------------------------------------------------------ FP64 GEMM (Gamma chain, K2)
// C = A B for the small Gamma-chain products (all dimensions <= 256).  The FP64 unit is shared by the
// whole SM (about one warp instruction per 19 cycles) and one warp issues at most one FP64 instruction
// per 64 cycles, so the work is spread over many blocks and short per-thread sums: a block owns an
// 8 x 8 output tile and its four 64-thread groups take interleaved quarters of k, combined in a fixed
// order.
constexpr int GT = 8;
constexpr int GK = 4;
// With regroup_Rn > 0 the product is Pi (R_{n+1}^2 x R_n^2) and the epilogue stores it regrouped as S_n
// (Prop. subchain_gram): S[(a + Rn b) + r (a' + Rn b')] = Pi[(b Rn1 + b') + Rn1^2 (a Rn + a')].
__global__ void __launch_bounds__(GT * GT * GK) gemm_f64_kernel(int m, int n, int k, const double* __restrict__ A,
                                                              const double* __restrict__ B, double* __restrict__ C,
                                                              int regroup_Rn, int regroup_Rn1) {
  __shared__ double part[GK][GT * GT];
  const int t = threadIdx.x;
  const int o = t % (GT * GT), g = t / (GT * GT);
  const int row = blockIdx.x * GT + (o % GT), col = blockIdx.y * GT + (o / GT);
  double a0 = 0.0, a1 = 0.0;
  if (row < m && col < n) {
    const double* Ar = A + row;
    const double* Bc = B + (int64_t)k * col;
    int kk = g;
#pragma unroll 8
    for (; kk + GK < k; kk += 2 * GK) {
      a0 = fma(Ar[(int64_t)m * kk], Bc[kk], a0);
      a1 = fma(Ar[(int64_t)m * (kk + GK)], Bc[kk + GK], a1);
    }
    if (kk < k) a0 = fma(Ar[(int64_t)m * kk], Bc[kk], a0);
  }
  part[g][o] = a0 + a1;
  __syncthreads();
  if (g == 0 && row < m && col < n) {
    const double v = (part[0][o] + part[1][o]) + (part[2][o] + part[3][o]);
    if (regroup_Rn > 0) {
      const int Rn = regroup_Rn, Rn1 = regroup_Rn1, r = Rn * Rn1;
      const int b = row / Rn1, b2 = row % Rn1, a = col / Rn, a2 = col % Rn;
      C[(a + Rn * b) + (int64_t)r * (a2 + Rn * b2)] = v;
    } else {
      C[row + (int64_t)m * col] = v;
    }
  }
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
// Right-looking column Cholesky of the lower triangle of S (r x r, r <= kCholSmemMax), the Golub & Van
// Loan Sec. 5.3.2 method cited for Alg. 2 line 9, in FP64 with the matrix in shared memory.  The
// reciprocal diagonal 1/L_jj is stored after the matrix (Lmat[r*r + j]) so the triangular solves never
// divide.
//
// On this part the SM's FP64 unit is shared by all its warps: it completes about one warp instruction per
// 19 cycles whatever the active lanes, and one warp issues at most one FP64 instruction per 64 cycles.
// The serial part of each column (update the next column, take its pivot, scale it) is a chain of
// dependent FP64 instructions, so it is latency-bound, and every FP64 instruction queued by other warps
// delays it.  The work is split so that few warps contend with it:
//   * warp 0 carries the chain: at step j it updates column j+1 with column j, forms the pivot of column
//     j+1 and scales it, holding the column in registers throughout;
//   * 24 warps (those with w mod 4 != 0, the arrangement measured fastest) apply column j to the
//     trailing columns k >= j+2.  Column j+2+c (length m - c, m = r - j - 2) is paired with column
//     r-1-c (length c + 1), so every pair is m + 1 entries long: a warp takes whole pairs and its lanes
//     run down the pair, with no lanes idle beyond the last chunk and no integer division;
//   * the remaining warps only load and store the matrix.
// One named barrier over the 800 working threads separates the steps.
//
// 1/sqrt(d) for d > 0 by Newton-Raphson on f(y) = y^-2 - d, y <- y (3 - d y^2) / 2, started from the
// FP32 hardware estimate of the exactly rescaled argument: each step doubles the correct bits, so two
// steps take the ~23-bit seed past the 53 of FP64.  d is first scaled by an even power of two into
// FP32 range, which changes neither the digits nor the result beyond that exact power.
__device__ __forceinline__ double rsqrt_newton(double d) {
  int e;
  const double m = frexp(d, &e);                  // d = m 2^e, m in [0.5, 1)
  const int h = (e >= 0 ? e : e - 1) / 2;          // floor(e / 2)
  const double m2 = ldexp(m, e - 2 * h);           // m 2^(e - 2h) in [0.5, 2)
  double y = (double)rsqrtf((float)m2);
  y = y * fma(-0.5 * m2, y * y, 1.5);
  y = y * fma(-0.5 * m2, y * y, 1.5);
  return ldexp(y, -h);                             // (m2 2^(2h))^(-1/2)
}

// 1/sqrt(d) for the pivots, d positive, finite, with a binary exponent in [-120, 120]: the FP32 hardware
// estimate of d truncated to 24 significant bits, widened exactly, then one third-order Householder
// step y <- y (1 + e/2 + 3e^2/8), e = 1 - d y^2, which cubes the relative error (2^-21 -> 2^-63) so the
// result is within the final roundings of the FP64 operations.  The FP32 copy and the widening are
// formed from the bit patterns, which keeps conversion instructions off the serial chain.  Other
// arguments take rsqrt_newton.
__device__ __forceinline__ double rsqrt_pivot(double d) {
  const long long b = __double_as_longlong(d);
  const int E = (int)((b >> 52) & 0x7ff) - 1023;
  if (E < -120 || E > 120) return rsqrt_newton(d);
  const unsigned fb = ((unsigned)(E + 127) << 23) | (unsigned)((b >> 29) & 0x7fffff);
  const unsigned yb = __float_as_uint(rsqrtf(__uint_as_float(fb)));
  const long long yd = ((long long)((int)((yb >> 23) & 0xff) - 127 + 1023) << 52) | ((long long)(yb & 0x7fffff) << 29);
  const double y0 = __longlong_as_double(yd);
  const double e = fma(-d, y0 * y0, 1.0);
  return fma(y0 * e, fma(0.375, e, 0.5), y0);
}

__global__ void pivot_rsqrt_check_kernel(const double* __restrict__ d, int64_t n, double* __restrict__ out,
                                         double* __restrict__ ref) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = rsqrt_pivot(d[i]);
    ref[i] = rsqrt(d[i]);
  }
}

constexpr int kCholSmemMax = 128;
// from this order on the blocked, many-SM factorization is used.  Measured warm on GB300, one-CTA kernel
// plus its block inverses against the blocked path: r = 64: 62.6 / 61.5 us; 80: 86.0 / 86.0;
// 96: 110.7 / 94.3; 120: 170.9 / 125.1; 128: 192.5 / 127.1.
constexpr int kCholBlockedMin = 88;
constexpr int kCholThreads = 1024;
constexpr int kCholWork = 800;       // warp 0 and the 24 trailing-update warps
constexpr int kCholTrail = 24;       // trailing-update warps

__device__ __forceinline__ void chol_step_barrier() {
  asm volatile("bar.sync 1, %0;" ::"r"(kCholWork) : "memory");
}

__global__ void __launch_bounds__(kCholThreads) cholesky_kernel(const double* __restrict__ S, double* __restrict__ Lmat,
                                                                 int r, DevStatus* st, const int* sweep_ctr, int mode) {
  extern __shared__ double A[];   // r x r, column-major
  __shared__ int bad[2];          // failure flag of the steps of each parity
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll 4
  for (int e = tid; e < r * r; e += kCholThreads) {
    const int i = e % r, j = e / r;
    A[e] = (i >= j) ? S[e] : 0.0;
  }
  if (tid < 2) bad[tid] = 0;
  __syncthreads();
  const bool chain = warp == 0, trail = (warp & 3) != 0;
  // pivot of column k from its updated diagonal d (lane 0); on failure the flag of step parity `slot`
  auto pivot = [&](int k, double d, int slot, double& y, double& l) -> bool {
    int ok = 1;
    if (lane == 0) {
      const long long b = __double_as_longlong(d);
      if (b > 0 && b < 0x7ff0000000000000LL) {
        y = rsqrt_pivot(d);
        l = d * y;
      } else {
        ok = 0;
        bad[slot] = 1;
        set_status(st, isfinite(d) ? TRALS_E_NOT_SPD : TRALS_E_NONFINITE, sweep_ctr ? *sweep_ctr : -1, mode, k, d);
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    y = __shfl_sync(0xffffffffu, y, 0);
    l = __shfl_sync(0xffffffffu, l, 0);
    return ok != 0;
  };
  if (chain || trail) {
    if (chain) {
      double y = 0.0, l = 0.0;
      if (pivot(0, A[0], 1, y, l)) {
        for (int i = 1 + lane; i < r; i += 32) A[i] *= y;
        if (lane == 0) {
          A[0] = l;
          Lmat[(int64_t)r * r] = y;
        }
      }
    }
    chol_step_barrier();
    // the flag written in step j is read after that step's barrier; the next write to the same slot
    // comes two barriers later, after every thread has read it
    if (!bad[1]) {
      const int tw = warp - (warp >> 2) - 1;   // trailing warp index 0..23
      for (int j = 0; j + 1 < r; ++j) {
        const double* Lj = A + r * j;
        if (chain) {
          const int k = j + 1;
          double* Ak = A + r * k;
          const double akj = Lj[k];
          double x[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
          for (int s = 0; s < 4; ++s)
            if (k + 32 * s < r) {
              const int i = k + lane + 32 * s;
              if (i < r) x[s] = fma(-Lj[i], akj, Ak[i]);
            }
          double y = 0.0, l = 0.0;
          if (pivot(k, x[0], j & 1, y, l)) {
#pragma unroll
            for (int s = 0; s < 4; ++s)
              if (k + 32 * s < r) {
                const int i = k + lane + 32 * s;
                if (i < r) Ak[i] = (i == k) ? l : x[s] * y;
              }
            if (lane == 0) Lmat[(int64_t)r * r + k] = y;
          }
        } else {
          const int m = r - j - 2, h = m + 1, np = (m + 1) >> 1;
          for (int c = tw; c < np; c += kCholTrail) {
            const int k1 = j + 2 + c, k2 = r - 1 - c, len = m - c;
            const double l1 = Lj[k1], l2 = Lj[k2];
            for (int rho = lane; rho < h; rho += 32) {
              const bool first = rho < len;
              const int k = first ? k1 : k2;
              const int i = first ? k1 + rho : k2 + rho - len;
              // the odd middle column pairs with itself: its second half is not there
              if (first || k2 != k1) A[i + r * k] = fma(-Lj[i], first ? l1 : l2, A[i + r * k]);
            }
          }
        }
        chol_step_barrier();
        if (bad[j & 1]) break;
      }
    }
  }
  __syncthreads();
  if (!bad[0] && !bad[1])
    for (int e = tid; e < r * r; e += kCholThreads) Lmat[e] = A[e];
}

// ------------------------------------------------------------------ K4: diagonal-block inverses
// W_q = D_q^{-1} for the 32 x 32 diagonal blocks D_q of L, so the triangular solves below need no serial
// substitution.  One CTA per block, by recursive doubling on the 2 x 2 block form of a lower-triangular
// inverse, [A 0; B C]^{-1} = [A^{-1} 0; -C^{-1} B A^{-1}  C^{-1}] (Higham, Accuracy and Stability of
// Numerical Algorithms, Sec. 14.2): level l merges pairs of 2^l x 2^l inverses, starting from the
// reciprocal diagonal.  The upper triangles of D and of every partial inverse are exact zeros, so the
// inner products run over whole blocks with no index tests.
template <int l>
__device__ __forceinline__ void block_inverse_level(double (*D)[kSolveBlock + 1], double (*W)[kSolveBlock + 1],
                                                    double (*T)[kSolveBlock + 1], int t) {
  constexpr int s = 1 << l;
  const bool act = t < (kSolveBlock / 2) * s;   // (32 / 2s) merges of s x s outputs
  const int j = t & (s - 1), i = (t >> l) & (s - 1), b = (t >> (2 * l)) * 2 * s;
  if (act) {   // T = B A^{-1}
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < s; ++q) acc = fma(D[b + s + i][b + q], W[b + q][b + j], acc);
    T[b + s + i][b + j] = acc;
  }
  __syncthreads();
  if (act) {   // lower-left block of the merged inverse: -C^{-1} T
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < s; ++q) acc = fma(W[b + s + i][b + s + q], T[b + s + q][b + j], acc);
    W[b + s + i][b + j] = -acc;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) chol_block_inverse_kernel(double* __restrict__ Lmat, int r) {
  __shared__ double D[kSolveBlock][kSolveBlock + 1], W[kSolveBlock][kSolveBlock + 1], T[kSolveBlock][kSolveBlock + 1];
  const int q = blockIdx.x, p0 = q * kSolveBlock, nb = min(kSolveBlock, r - p0);
  const double* inv = Lmat + (size_t)r * r;
  for (int e = threadIdx.x; e < kSolveBlock * kSolveBlock; e += blockDim.x) {
    const int i = e % kSolveBlock, j = e / kSolveBlock;
    double d = 0.0, w = 0.0;
    if (i < nb && j < nb) {
      d = (i >= j) ? Lmat[(p0 + i) + (size_t)r * (p0 + j)] : 0.0;
      if (i == j) w = inv[p0 + i];
    } else if (i == j) {   // identity past r
      d = 1.0;
      w = 1.0;
    }
    D[i][j] = d;
    W[i][j] = w;
  }
  __syncthreads();
  const int t = threadIdx.x;
  block_inverse_level<0>(D, W, T, t);
  block_inverse_level<1>(D, W, T, t);
  block_inverse_level<2>(D, W, T, t);
  block_inverse_level<3>(D, W, T, t);
  block_inverse_level<4>(D, W, T, t);
  double* Wq = Lmat + (size_t)r * r + r + (size_t)q * kSolveBlock * kSolveBlock;
  for (int e = threadIdx.x; e < kSolveBlock * kSolveBlock; e += blockDim.x)
    Wq[e] = W[e % kSolveBlock][e / kSolveBlock];
}

// ------------------------------------------------------------------ K4, blocked over many SMs
// Left-looking blocked Cholesky in 32-column panels (Golub & Van Loan Sec. 4.2, the same factorization),
// two kernels per panel so the FP64 work is spread over many SMs (the FP64 unit of a single SM is the
// bound of the one-CTA kernel above):
//   update: A[i][j] -= sum_{k < p0} L[i][k] L[j][k] for the panel's columns j and rows i >= j;
//   factor: every CTA factors the panel's diagonal block D redundantly in shared memory (the split
//           chain of cholesky_kernel at 32 x 32), inverts it by recursive doubling, and forms its share
//           of the rows below as L[i][p0:p1] = A[i][p0:p1] D^{-T}, a product with the inverse rather than
//           a substitution.  CTA 0 stores D, its reciprocal diagonal and W_q = D^{-1}: the factor's whole
//           layout, so no separate block-inverse pass follows.
constexpr int kPanel = kSolveBlock;

__global__ void __launch_bounds__(256) chol_panel_update_kernel(double* __restrict__ A, int r, int p0, int p1,
                                                                int move_prev) {
  __shared__ double part[4][64];
  const int t = threadIdx.x, o = t & 63, g = t >> 6;
  if (move_prev && blockIdx.x == 0 && blockIdx.y == 0) {
    // the previous panel's factored diagonal block, parked in the scratch after W by its factor kernel
    // (whose CTAs all read that block as input, so none of them could write it in place)
    const int q0 = p0 - kPanel;
    const double* scratch = A + lmat_scratch_offset(r);
    for (int e = t; e < kPanel * kPanel; e += blockDim.x) {
      const int i = e % kPanel, j = e / kPanel;
      if (i >= j) A[(q0 + i) + (int64_t)r * (q0 + j)] = scratch[e];
    }
  }
  const int i = p0 + blockIdx.x * 8 + (o & 7), j = p0 + blockIdx.y * 8 + (o >> 3);
  const bool live = i < r && j < p1 && i >= j;
  double a0 = 0.0, a1 = 0.0;
  if (live) {
    const double* Li = A + i;
    const double* Lj = A + j;
    int k = g;
#pragma unroll 4
    for (; k + 4 < p0; k += 8) {
      a0 = fma(Li[(int64_t)r * k], Lj[(int64_t)r * k], a0);
      a1 = fma(Li[(int64_t)r * (k + 4)], Lj[(int64_t)r * (k + 4)], a1);
    }
    if (k < p0) a0 = fma(Li[(int64_t)r * k], Lj[(int64_t)r * k], a0);
  }
  part[g][o] = a0 + a1;
  __syncthreads();
  if (g == 0 && live) A[i + (int64_t)r * j] -= (part[0][o] + part[1][o]) + (part[2][o] + part[3][o]);
}

__global__ void __launch_bounds__(256) chol_panel_factor_kernel(double* __restrict__ A, int r, int p0, DevStatus* st,
                                                                const int* sweep_ctr, int mode) {
  constexpr int B = kPanel;
  __shared__ double D[B][B + 1], W[B][B + 1], T[B][B + 1];
  __shared__ double yv[B];
  __shared__ int fail[2];   // failure flag of the steps of each parity
  const int p1 = min(r, p0 + B), nb = p1 - p0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < B * B; e += blockDim.x) {
    const int i = e % B, j = e / B;
    double v;
    if (i < nb && j < nb) v = (i >= j) ? A[(p0 + i) + (int64_t)r * (p0 + j)] : 0.0;
    else v = (i == j) ? 1.0 : 0.0;   // identity past the panel
    D[i][j] = v;
  }
  if (tid < 2) fail[tid] = 0;
  __syncthreads();
  // pivot of column k of the block from its updated diagonal d (every lane of warp 0 alike); a failure
  // goes to the flag of parity `slot`, read by everyone after that step's barrier
  auto pivot = [&](int k, double d, int slot, double& y) -> bool {
    const long long b = __double_as_longlong(d);
    if (b > 0 && b < 0x7ff0000000000000LL) {
      y = rsqrt_pivot(d);
      return true;
    }
    if (lane == 0) {
      fail[slot] = 1;
      if (blockIdx.x == 0)
        set_status(st, isfinite(d) ? TRALS_E_NOT_SPD : TRALS_E_NONFINITE, sweep_ctr ? *sweep_ctr : -1, mode, p0 + k, d);
    }
    return false;
  };
  if (warp == 0) {
    double y = 0.0;
    if (pivot(0, D[0][0], 1, y)) {
      if (lane < nb) D[lane][0] *= y;
      if (lane == 0) yv[0] = y;
    }
  }
  __syncthreads();
  // right-looking over the block: warp 0 carries column c+1 (update with column c, pivot, scale); warps
  // 1..7 apply column c to the columns after it.  One barrier per column; `fail` is read after it.
  for (int c = 0; c + 1 < nb; ++c) {
    // the flag of the previous step (slot 1 for the first column); the next write to that slot comes two
    // barriers later, after every thread has read it
    if (fail[(c + 1) & 1]) break;
    if (warp == 0) {
      const int k = c + 1;
      const double lkc = D[k][c];
      const double x = (lane >= k && lane < nb) ? fma(-D[lane][c], lkc, D[lane][k]) : 0.0;
      double y = 0.0;
      if (pivot(k, __shfl_sync(0xffffffffu, x, k), c & 1, y)) {
        if (lane >= k && lane < nb) D[lane][k] = x * y;
        if (lane == 0) yv[k] = y;
      }
    } else {
      for (int kk = c + 1 + warp; kk < nb; kk += 7) {
        const double lkc = D[kk][c];
        if (lane >= kk && lane < nb) D[lane][kk] = fma(-D[lane][c], lkc, D[lane][kk]);
      }
    }
    __syncthreads();
  }
  if (fail[0] || fail[1]) return;   // uniform: read after the last barrier
  for (int e = tid; e < B * B; e += blockDim.x) {
    const int i = e % B, j = e / B;
    W[i][j] = (i == j) ? (i < nb ? yv[i] : 1.0) : 0.0;
  }
  __syncthreads();
  block_inverse_level<0>(D, W, T, tid);
  block_inverse_level<1>(D, W, T, tid);
  block_inverse_level<2>(D, W, T, tid);
  block_inverse_level<3>(D, W, T, tid);
  block_inverse_level<4>(D, W, T, tid);
  if (blockIdx.x == 0) {
    if (gridDim.x == 1) {   // no other CTA reads the block: in place
      for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        if (i >= j) A[(p0 + i) + (int64_t)r * (p0 + j)] = D[i][j];
      }
    } else {                // parked; the next panel's update kernel moves it in place
      double* scratch = A + lmat_scratch_offset(r);
      for (int e = tid; e < B * B; e += blockDim.x) scratch[e] = D[e % B][e / B];
    }
    for (int c = tid; c < nb; c += blockDim.x) A[(int64_t)r * r + p0 + c] = yv[c];
    double* Wq = A + (int64_t)r * r + r + (int64_t)(p0 / B) * B * B;
    for (int e = tid; e < B * B; e += blockDim.x) Wq[e] = W[e % B][e / B];
  }
  // rows below: L[i][p0 + c] = sum_{t <= c} A[i][p0 + t] W[c][t], one warp per row
  for (int i = p1 + blockIdx.x * 8 + warp; i < r; i += gridDim.x * 8) {
    const double a = (lane < nb) ? A[i + (int64_t)r * (p0 + lane)] : 0.0;
    double acc = 0.0;
    for (int t = 0; t < nb; ++t) acc = fma(__shfl_sync(0xffffffffu, a, t), W[lane][t], acc);
    if (lane < nb) A[i + (int64_t)r * (p0 + lane)] = acc;
  }
}

// ------------------------------------------------------------------ K4: triangular solves
// Z S = M row by row: for right-hand side i (one CTA), L y = M[i,:]^T then L^T z = y, and
// G[a + Rn (i + In b)] = z[a + Rn b] (classical mode-2 folding).  Both sweeps go by 32-wide panels; a
// panel first subtracts the finished unknowns (a matrix-vector product over the solved part) and then
// multiplies by the diagonal block's inverse W_q (forward) or its transpose (backward): no serial
// substitution and no division.  Four warps carry the FP64 work: one warp issues at most one FP64
// instruction per 64 cycles, and four keep the SM's shared FP64 unit (about one per 19 cycles) busy
// with short reductions.  All eight stage L (row stride r | 1, odd, so the transposed reads of the
// backward sweep fall on distinct banks) and the W_q in shared memory when they fit.
template <bool kInSmem>
__global__ void __launch_bounds__(256) chol_solve_kernel(const double* __restrict__ Lmat, const double* __restrict__ M,
                                                         int Rn, int64_t In, int Rn1, double* __restrict__ G,
                                                         DevStatus* st, float* __restrict__ G32, int64_t Ist,
                                                         int which) {
  extern __shared__ double sh[];
  constexpr int B = kSolveBlock;
  const int r = Rn * Rn1, nblk = (r + B - 1) / B;
  const int lda = kInSmem ? (r | 1) : r;
  double* y = sh;                              // nblk * 32: right-hand side, then the unknowns
  double* part = y + nblk * B;                 // 4 x 32 partial sums
  double* Ls = part + 4 * B;                   // lda x r
  double* Ws = Ls + (size_t)lda * r;           // nblk blocks of 32 x 33
  const double* L = kInSmem ? Ls : Lmat;
  const double* Wg = Lmat + (size_t)r * r + r;
  const int64_t i0 = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (kInSmem) {
    // element e = i + r k of L to Ls[i + lda k] and the W_q entries, by 8-byte asynchronous copies:
    // every copy is in flight at once instead of a round trip per batch of loads; (i, k) advanced
    // without division
    int i = tid % r, k = tid / r;
    const int di = nt % r, dk = nt / r;
    for (int e = tid; e < r * r; e += nt) {
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(Ls + i + lda * k)),
                   "l"(Lmat + e)
                   : "memory");
      i += di;
      k += dk;
      if (i >= r) {
        i -= r;
        ++k;
      }
    }
    for (int e = tid; e < nblk * B * B; e += nt) {
      double* dst = Ws + (e / (B * B)) * (B * (B + 1)) + (e % B) + (B + 1) * ((e / B) % B);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                   "l"(Wg + e)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int j = tid; j < nblk * B; j += nt) y[j] = j < r ? M[i0 + In * (int64_t)j] : 0.0;
  if (kInSmem) asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  auto w_at = [&](int q, int a, int b) -> double {
    return kInSmem ? Ws[q * (B * (B + 1)) + a + (B + 1) * b] : Wg[q * (B * B) + a + B * b];
  };
  auto sum_parts = [&]() { return (part[lane] + part[B + lane]) + (part[2 * B + lane] + part[3 * B + lane]); };
  // forward: y_q = W_q (y_q - L[q, :p0] y[:p0])  (skipped for a backward solve alone)
  for (int q = 0; q < (which == 2 ? 0 : nblk); ++q) {
    const int p0 = q * B;
    if (p0 > 0) {
      if (warp < 4) {
        double acc = 0.0;
        const int i = p0 + lane;
        if (i < r)
          for (int k = warp; k < p0; k += 4) acc = fma(L[i + lda * k], y[k], acc);
        part[warp * B + lane] = acc;
      }
      __syncthreads();
      if (warp == 0) y[p0 + lane] -= sum_parts();
      __syncthreads();
    }
    if (warp < 4) {
      double acc = 0.0;
#pragma unroll
      for (int t = 8 * warp; t < 8 * warp + 8; ++t) acc = fma(w_at(q, lane, t), y[p0 + t], acc);
      part[warp * B + lane] = acc;
    }
    __syncthreads();
    if (warp == 0) y[p0 + lane] = sum_parts();
    __syncthreads();
  }
  // backward: z_q = W_q^T (y_q - L[p1:, q]^T z[p1:])  (skipped for a forward solve alone: z = y)
  for (int q = which == 1 ? -1 : nblk - 1; q >= 0; --q) {
    const int p0 = q * B, p1 = min(r, p0 + B);
    if (p1 < r) {
      if (warp < 4) {
        double acc = 0.0;
        const int i = p0 + lane;
        if (i < r)
          for (int k = p1 + warp; k < r; k += 4) acc = fma(L[k + lda * i], y[k], acc);
        part[warp * B + lane] = acc;
      }
      __syncthreads();
      if (warp == 0) y[p0 + lane] -= sum_parts();
      __syncthreads();
    }
    if (warp < 4) {
      double acc = 0.0;
#pragma unroll
      for (int t = 8 * warp; t < 8 * warp + 8; ++t) acc = fma(w_at(q, t, lane), y[p0 + t], acc);
      part[warp * B + lane] = acc;
    }
    __syncthreads();
    if (warp == 0) y[p0 + lane] = sum_parts();
    __syncthreads();
  }
  for (int c = tid; c < r; c += nt) {
    const double z = y[c];
    if (!isfinite(z)) set_status(st, TRALS_E_NONFINITE, -1, -1, (int)i0, z);
    const int a = c % Rn, b = c / Rn;
    G[a + (int64_t)Rn * (i0 + In * b)] = z;
    if (G32 != nullptr) G32[a + (int64_t)Rn * (i0 + Ist * b)] = (float)z;
  }
}

__global__ void core_to_f32_kernel(const double* __restrict__ G, int Rn, int64_t In, int64_t Ist, int Rn1,
                                   float* __restrict__ G32) {
  const int64_t total = (int64_t)Rn * In * Rn1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e % Rn, ib = e / Rn, i = ib % In, b = ib / In;
    G32[a + Rn * (i + Ist * b)] = (float)G[e];
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

template <typename XT>
__global__ void quantize_padded_kernel(const void* __restrict__ src, int64_t I0, int64_t I0p, int64_t rest,
                                       __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t count = I0p * rest;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = e % I0p, q = e / I0p;
    __nv_bfloat16 h = __float2bfloat16_rn(0.f), l = h;
    if (i0 < I0) {
      const double v = load_as_double<XT>(src, i0 + I0 * q);
      h = __float2bfloat16_rn((float)v);
      l = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
    }
    hi[e] = h;
    if (lo != nullptr) lo[e] = l;
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
  const int64_t core = (int64_t)Rn * In * Rn1;
  const int r = Rn * Rn1;
  if (In <= 4096) {
    const dim3 grid((r + 7) / 8, (r + 7) / 8);
    gamma_tiled_kernel<<<grid, 256, 0, s>>>(G, Rn, (int)In, Rn1, Gamma);
  } else if (core <= kGammaSmemMax)
    gamma_smem_kernel<<<grid_for(total, 128), 128, (size_t)core * sizeof(double), s>>>(G, Rn, (int)In, Rn1, Gamma);
  else
    gamma_kernel<<<grid_for(total, 256), 256, 0, s>>>(G, Rn, In, Rn1, Gamma);
}

void launch_gemm_f64(int m, int n, int k, const double* A, const double* B, double* C, cudaStream_t s) {
  dim3 grid((m + GT - 1) / GT, (n + GT - 1) / GT);
  gemm_f64_kernel<<<grid, GT * GT * GK, 0, s>>>(m, n, k, A, B, C, 0, 0);
}

void launch_gemm_f64_regroup(int k, const double* A, const double* B, int Rn, int Rn1, double* S, cudaStream_t s) {
  const int m = Rn1 * Rn1, n = Rn * Rn;
  dim3 grid((m + GT - 1) / GT, (n + GT - 1) / GT);
  gemm_f64_kernel<<<grid, GT * GT * GK, 0, s>>>(m, n, k, A, B, S, Rn, Rn1);
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

__global__ void copy_lower_kernel(const double* __restrict__ S, double* __restrict__ A, int r) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
    const int i = e % r, j = e / r;
    A[e] = (i >= j) ? S[e] : 0.0;
  }
}

int launch_cholesky_blocked(const double* S, double* Lmat, int r, DevStatus* st, const int* sweep_ctr, int mode,
                            cudaStream_t s) {
  int launches = 1;
  copy_lower_kernel<<<grid_for((int64_t)r * r, 256), 256, 0, s>>>(S, Lmat, r);
  int prev_blocks = 0;
  for (int p0 = 0; p0 < r; p0 += kPanel) {
    const int p1 = std::min(r, p0 + kPanel);
    if (p0 > 0) {
      const dim3 g((r - p0 + 7) / 8, (p1 - p0 + 7) / 8);
      chol_panel_update_kernel<<<g, 256, 0, s>>>(Lmat, r, p0, p1, prev_blocks > 1 ? 1 : 0);
      ++launches;
    }
    const int rows_below = r - p1;
    const int blocks = std::max(1, std::min(16, (rows_below + 7) / 8));
    chol_panel_factor_kernel<<<blocks, 256, 0, s>>>(Lmat, r, p0, st, sweep_ctr, mode);
    ++launches;
    prev_blocks = blocks;
  }
  return launches;
}

bool cholesky_is_blocked(int r) { return !(r <= kCholSmemMax && r < kCholBlockedMin); }

int launch_cholesky(const double* S, double* Lmat, int r, DevStatus* st, const int* sweep_ctr, int mode,
                    cudaStream_t s) {
  if (!cholesky_is_blocked(r)) {
    // one CTA, matrix in shared memory: the split chain of cholesky_kernel
    const size_t smem = (size_t)r * r * sizeof(double);
    cholesky_kernel<<<1, kCholThreads, smem, s>>>(S, Lmat, r, st, sweep_ctr, mode);
    launch_chol_block_inverse(Lmat, r, s);
    return 2;
  }
  return launch_cholesky_blocked(S, Lmat, r, st, sweep_ctr, mode, s);
}

void launch_pivot_rsqrt_check(const double* d, int64_t n, double* out, double* ref, cudaStream_t s) {
  pivot_rsqrt_check_kernel<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(d, n, out, ref);
}

size_t chol_solve_smem(int r, bool in_smem) {
  const int nblk = (r + kSolveBlock - 1) / kSolveBlock;
  size_t n = (size_t)nblk * kSolveBlock + 4 * kSolveBlock;
  if (in_smem) n += (size_t)(r | 1) * r + (size_t)nblk * kSolveBlock * (kSolveBlock + 1);
  return n * sizeof(double);
}

void launch_chol_solve(const double* Lmat, const double* M, int Rn, int64_t In, int Rn1, double* G, DevStatus* st,
                       cudaStream_t s, float* G32, int64_t Ist, int part) {
  const int r = Rn * Rn1;
  const size_t smem = chol_solve_smem(r, true);
  if (smem <= 227 * 1024)
    chol_solve_kernel<true><<<(unsigned)In, 256, smem, s>>>(Lmat, M, Rn, In, Rn1, G, st, G32, Ist, part);
  else
    chol_solve_kernel<false><<<(unsigned)In, 256, chol_solve_smem(r, false), s>>>(Lmat, M, Rn, In, Rn1, G, st, G32,
                                                                                 Ist, part);
}

void launch_core_to_f32(const double* G, int Rn, int64_t In, int64_t Ist, int Rn1, float* G32, cudaStream_t s) {
  core_to_f32_kernel<<<grid_for((int64_t)Rn * In * Rn1, 256), 256, 0, s>>>(G, Rn, In, Ist, Rn1, G32);
}

void launch_chol_block_inverse(double* Lmat, int r, cudaStream_t s) {
  chol_block_inverse_kernel<<<(r + kSolveBlock - 1) / kSolveBlock, 256, 0, s>>>(Lmat, r);
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

void launch_quantize_padded(const void* src, int src_t, int64_t I0, int64_t I0p, int64_t rest, __nv_bfloat16* hi,
                            __nv_bfloat16* lo, cudaStream_t s) {
  const int g = grid_for(I0p * rest, 256, 152 * 32);
  if (src_t == TRALS_X_F64)
    quantize_padded_kernel<double><<<g, 256, 0, s>>>(src, I0, I0p, rest, hi, lo);
  else if (src_t == TRALS_X_F32)
    quantize_padded_kernel<float><<<g, 256, 0, s>>>(src, I0, I0p, rest, hi, lo);
  else
    quantize_padded_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(src, I0, I0p, rest, hi, lo);
}

void launch_zero_status(DevStatus* st, cudaStream_t s) { zero_status_kernel<<<1, 1, 0, s>>>(st); }

void launch_convert_f32(const void* src_f64, int64_t count, float* dst, cudaStream_t s) {
  convert_f32_kernel<<<grid_for(count, 256, 152 * 32), 256, 0, s>>>(static_cast<const double*>(src_f64), count, dst);
}

cudaError_t init_small_attributes() {
  cudaError_t e = cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kCholSmemMax * kCholSmemMax * (int)sizeof(double));
  // solve: L (r x r) plus two vectors, r <= 160 (the QR path's solves use larger r from global memory)
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chol_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gamma_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kGammaSmemMax * (int)sizeof(double));
  return e;
}

}  // namespace trals
