// Explicit-subchain coefficient matrix (regular TR-ALS, Alg. 1): the comparison variant of the
// structured Gamma chain.  The subchain matrix G^{!=n}_[2] (J_n x R_n R_{n+1}, Def. subchain tensor
// and mode-2 unfolding) is formed explicitly in HBM, in row blocks of bounded size, and its Gram
// matrix S_n = (G^{!=n}_[2])^T G^{!=n}_[2] is accumulated by a blocked SYRK: FP64 rows and FP64
// sums in the FP64 mode, FP32 rows and FP32 tile sums (reduced in FP64) in the reduced modes.
#include <algorithm>

#include "trals_internal.cuh"

namespace trals {

namespace {

constexpr int RB = 32;    // subchain rows per generator block
constexpr int ST = 32;    // SYRK output tile (ST x ST) and k step

// A[(k - k0) * r + (a + Rn b)] = G^{!=n}(k)[b, a] = sum_c Ltab[l][b + Rn1 c] Utab[u][c + Rs a], k in [k0, k1)
template <typename T>
__global__ void subchain_rows_kernel(const double* __restrict__ ltab, const double* __restrict__ utab, ModeLayout L,
                                     int64_t k0, int64_t k1, T* __restrict__ A) {
  __shared__ int64_t lrow[RB], urow[RB];
  const int r = L.Rn * L.Rn1;
  const int64_t kb = k0 + (int64_t)blockIdx.x * RB;
  if (threadIdx.x < RB) {
    const int64_t k = kb + threadIdx.x;
    lrow[threadIdx.x] = k < k1 ? k % L.nL : 0;
    urow[threadIdx.x] = k < k1 ? k / L.nL : 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RB * r; e += blockDim.x) {
    const int kk = e / r, rr = e % r;
    const int64_t k = kb + kk;
    if (k >= k1) continue;
    const int a = rr % L.Rn, b = rr / L.Rn;
    const double* Lp = ltab + lrow[kk] * (int64_t)L.Rn1 * L.Rs;
    const double* Up = utab + urow[kk] * (int64_t)L.Rs * L.Rn;
    double g = 0.0;
    for (int c = 0; c < L.Rs; ++c) g = fma(Lp[b + L.Rn1 * c], Up[c + L.Rs * a], g);
    A[(k - k0) * r + rr] = (T)g;
  }
}

// Lower-triangle tiles (ti >= tj) of A^T A over this CTA's share of the block's rows, added into
// part[blockIdx.x][i + r j] (or stored there when `accumulate` is 0).
template <typename T>
__global__ void __launch_bounds__(256) syrk_tiles_kernel(const T* __restrict__ A, int64_t rows, int r,
                                                        double* __restrict__ part, int accumulate) {
  __shared__ T As[ST][ST + 1], Bs[ST][ST + 1];
  // decode the lower-triangle tile index
  int t = blockIdx.y, ti = 0;
  while (t > ti) {
    t -= ti + 1;
    ++ti;
  }
  const int tj = t;
  const int64_t chunk = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  const int li = threadIdx.x % ST, lj = (threadIdx.x / ST) * 4;
  T acc[4] = {0, 0, 0, 0};
  for (int64_t kb = r0; kb < r1; kb += ST) {
    for (int e = threadIdx.x; e < ST * ST; e += blockDim.x) {
      const int kk = e / ST, c = e % ST;
      const int64_t k = kb + kk;
      const int ci = ti * ST + c, cj = tj * ST + c;
      As[kk][c] = (k < r1 && ci < r) ? A[k * r + ci] : T(0);
      Bs[kk][c] = (k < r1 && cj < r) ? A[k * r + cj] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < ST; ++kk) {
      const T x = As[kk][li];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += x * Bs[kk][lj + q];
    }
    __syncthreads();
  }
  const int i = ti * ST + li;
  double* P = part + (int64_t)blockIdx.x * r * r;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = tj * ST + lj + q;
    if (i < r && j < r) {
      const double v = (double)acc[q];
      P[i + (int64_t)r * j] = accumulate ? P[i + (int64_t)r * j] + v : v;
    }
  }
}

// S[i + r j] = S[j + r i] = sum_g part[g][i + r j] for i >= j, in a fixed order over g
__global__ void syrk_reduce_kernel(const double* __restrict__ part, int groups, int r, double* __restrict__ S) {
  const int64_t total = (int64_t)r * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % r), j = (int)(e / r);
    if (i < j) continue;
    double s = 0.0;
    for (int g = 0; g < groups; ++g) s += part[(int64_t)g * total + e];
    S[e] = s;
    S[j + (int64_t)r * i] = s;
  }
}

}  // namespace

ExplicitGramSizes explicit_gram_sizes(const ModeLayout& L, bool fp64) {
  ExplicitGramSizes z;
  const int r = L.Rn * L.Rn1;
  const size_t es = fp64 ? 8 : 4;
  z.block_rows = std::max<int64_t>(1, std::min<int64_t>(L.J, ((int64_t)256 << 20) / ((int64_t)r * es)));
  const int nt = (r + ST - 1) / ST;
  const int tiles = nt * (nt + 1) / 2;
  int64_t g = std::max<int64_t>(1, 152 * 8 / tiles);
  g = std::min<int64_t>(g, (z.block_rows + ST - 1) / ST);
  g = std::min<int64_t>(g, std::max<int64_t>(1, ((int64_t)16 << 20) / ((int64_t)r * r)));
  z.groups = (int)std::max<int64_t>(1, g);
  z.A_bytes = (size_t)z.block_rows * r * es;
  z.part_elems = (size_t)z.groups * r * r;
  return z;
}

int launch_explicit_gram(const ModeLayout& L, const double* ltab, const double* utab, bool fp64, void* Ablk,
                         double* part, double* S, cudaStream_t s) {
  const ExplicitGramSizes z = explicit_gram_sizes(L, fp64);
  const int r = L.Rn * L.Rn1;
  const int nt = (r + ST - 1) / ST;
  const int tiles = nt * (nt + 1) / 2;
  int launches = 0;
  int first = 1;
  for (int64_t k0 = 0; k0 < L.J; k0 += z.block_rows) {
    const int64_t k1 = std::min<int64_t>(L.J, k0 + z.block_rows);
    const unsigned gb = (unsigned)((k1 - k0 + RB - 1) / RB);
    const dim3 sg(z.groups, tiles);
    if (fp64) {
      subchain_rows_kernel<double><<<gb, 256, 0, s>>>(ltab, utab, L, k0, k1, static_cast<double*>(Ablk));
      syrk_tiles_kernel<double><<<sg, 256, 0, s>>>(static_cast<const double*>(Ablk), k1 - k0, r, part, !first);
    } else {
      subchain_rows_kernel<float><<<gb, 256, 0, s>>>(ltab, utab, L, k0, k1, static_cast<float*>(Ablk));
      syrk_tiles_kernel<float><<<sg, 256, 0, s>>>(static_cast<const float*>(Ablk), k1 - k0, r, part, !first);
    }
    launches += 2;
    first = 0;
  }
  const int g = (int)std::min<int64_t>(((int64_t)r * r + 255) / 256, 152 * 4);
  syrk_reduce_kernel<<<g, 256, 0, s>>>(part, z.groups, r, S);
  return launches + 1;
}

}  // namespace trals
