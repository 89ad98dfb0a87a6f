// TR-ALS-QRNE (Alg. 4, Sec. 3.3) and the literal TR-ALS-QR (Alg. 3, Sec. 3.2) on the GPU, FP64: both
// work on the least-squares problem compressed by the mode-2 QR of every core.
//
// TR-ALS-QRNE solves the compressed problem through its normal equations:
// Every core is factored G_j = R_j x_2 Q_j (mode-2 QR).  A mode-n update then
//   * compresses X along every other mode, Y = X x_{j != n} Q_j^T (Multi-TTM, Alg. 4 line 8),
//   * contracts Y with the subchain of the R factors, M_n = Y_[n] V_n[2] (line 9; the FP64 MTTSP of
//     the NE path, run on Y and the R cores),
//   * forms S_n from the Gram tensors of the R factors (lines 3, 6, 12; the Gamma chain of the NE
//     path) and solves G_{n(2)} S_n = M_n by Cholesky (line 10),
//   * refactors the updated core (line 11).
// The mode-2 QR of a core whose unfolding G_{j(2)} (I_j x R_j R_{j+1}) is tall is computed by
// CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa & Yamamoto, 2014): R_1 from the Cholesky factor of
// G_{(2)}^T G_{(2)}, Q_1 = G_{(2)} R_1^{-1}, then once more on Q_1, R = R_2 R_1 and Q = Q_1 R_2^{-1};
// two passes give orthonormal columns to working accuracy for any condition number below about
// u^{-1/2}.  A mode with I_j <= R_j R_{j+1} has nothing to compress (case (2) of the mode-2 QR
// definition: Q_j square); it keeps Q_j = I and R_j = G_j, which leaves M_n and S_n unchanged, since
// the method needs only G_j = R_j x_2 Q_j with Q_j orthonormal.
//
// The literal TR-ALS-QR (Alg. 3) is meant for the compressible regime, where the subchain V_n of the R
// factors (Alg. 3 line 5) is small: V_n[2] is formed explicitly, factored by Householder QR with Q_0
// formed explicitly (line 6), W_n = Y_[n] Q_0 (line 8) and G_{n(2)} R^T = W_n is solved by substitution
// (line 9).  Its core QRs (lines 2 and 10) are Householder QRs too.
#include <algorithm>
#include <cstring>
#include <vector>

#include "trals_internal.cuh"

namespace trals {
namespace {

int grid_of(int64_t n, int threads, int cap = 152 * 16) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, cap));
}

// core G (R x I x R1, element a + R (i + I b)) -> G2 = G_(2) (I x R R1, column-major, column a + R b)
__global__ void unfold2_kernel(const double* __restrict__ G, int R, int64_t I, int R1, double* __restrict__ G2) {
  const int64_t total = (int64_t)R * I * R1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e % R, ib = e / R, i = ib % I, b = ib / I;
    G2[i + I * (a + (int64_t)R * b)] = G[e];
  }
}

// P = R^T (lower, r x r, column-major) -> the R core (R x r x R1): Rc[a + R (c + r b)] = R[c, a + R b]
__global__ void rcore_from_lower_kernel(const double* __restrict__ P, int R, int R1, double* __restrict__ Rc) {
  const int r = R * R1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
    const int a = e % R, cb = e / R, c = cb % r, b = cb / r;
    Rc[e] = P[(a + R * b) + (int64_t)r * c];
  }
}

// mode-j TTM with Q^T: out[a + A (c + C b)] = sum_d Q[d + D c] in[a + A (d + D b)].  Each thread owns one
// (a, b) pair and up to 8 consecutive c, and streams its column of `in` in order of d.
__global__ void ttm_kernel(const double* __restrict__ in, int64_t A, int64_t D, int64_t B, const double* __restrict__ Q,
                           int C, double* __restrict__ out) {
  const int c0 = blockIdx.y * 8;
  const int nc = min(8, C - c0);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < A * B; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = t % A, b = t / A;
    const double* x = in + a + A * D * b;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t d = 0; d < D; ++d) {
      const double v = x[A * d];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < nc) acc[k] = fma(Q[d + D * (c0 + k)], v, acc[k]);
    }
    for (int k = 0; k < nc; ++k) out[a + A * ((c0 + k) + (int64_t)C * b)] = acc[k];
  }
}

__global__ void finalize_ratio_kernel(const double* red2, double* out) { *out = sqrt(fmax(red2[0], 0.0) / red2[1]); }

// R (r x r upper, column-major) -> the R core (R x r x R1): Rc[a + R (c + r b)] = R[c, a + R b]
__global__ void rcore_from_upper_kernel(const double* __restrict__ Rm, int R, int R1, double* __restrict__ Rc) {
  const int r = R * R1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
    const int a = e % R, cb = e / R, c = cb % r, b = cb / r;
    Rc[e] = Rm[c + (int64_t)r * (a + R * b)];
  }
}

// V_n[2] explicitly (J' x r, column-major, column a + R_n b) from the two partial-chain tables of a mode
// layout: V[k, a + R_n b] = sum_s Ltab(l)[b, s] Utab(u)[s, a], k = l + nL u (eq. subchain_new)
__global__ void subchain_explicit_kernel(const double* __restrict__ ltab, const double* __restrict__ utab,
                                         const ModeLayout L, double* __restrict__ V) {
  const int64_t J = L.nL * L.nU;
  const int r = L.Rn * L.Rn1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < J * r; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e % J;
    const int c = (int)(e / J), a = c % L.Rn, b = c / L.Rn;
    const int64_t l = k % L.nL, u = k / L.nL;
    const double* Lt = ltab + l * (int64_t)L.Rn1 * L.Rs;
    const double* Ut = utab + u * (int64_t)L.Rs * L.Rn;
    double acc = 0.0;
    for (int t = 0; t < L.Rs; ++t) acc = fma(Lt[b + L.Rn1 * t], Ut[t + L.Rs * a], acc);
    V[e] = acc;
  }
}

// W_n = Y_[n] Q_0 (I_n x r): W[i + I_n c] = sum_k Y[offL[l] + offU[u] + i strideN] Q_0[k + J' c]
__global__ void wn_kernel(const double* __restrict__ Y, const int64_t* __restrict__ offL,
                          const int64_t* __restrict__ offU, const ModeLayout L, const double* __restrict__ Q0,
                          double* __restrict__ W) {
  const int64_t J = L.nL * L.nU;
  const int r = L.Rn * L.Rn1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L.In * r; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % L.In, c = e / L.In;
    const double* q = Q0 + J * c;
    double a0 = 0.0, a1 = 0.0;
    int64_t k = 0;
    for (int64_t u = 0; u < L.nU; ++u)
      for (int64_t l = 0; l < L.nL; ++l, ++k) {
        const double y = Y[offL[l] + offU[u] + i * L.strideN];
        if (k & 1) a1 = fma(y, q[k], a1);
        else a0 = fma(y, q[k], a0);
      }
    W[e] = a0 + a1;
  }
}

// L = R^T as a factor buffer (lower triangle, reciprocal diagonal; the diagonal-block inverses follow)
__global__ void upper_to_lmat_kernel(const double* __restrict__ Rm, int r, double* __restrict__ Lmat) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r + r; e += gridDim.x * blockDim.x) {
    if (e < r * r) {
      const int i = e % r, j = e / r;
      Lmat[e] = (i >= j) ? Rm[j + (int64_t)r * i] : 0.0;
    } else {
      const int j = e - r * r;
      Lmat[e] = 1.0 / Rm[j + (int64_t)r * j];
    }
  }
}

// core G (R x I x R1) from its unfolding G2 (I x R R1, column-major, column a + R b)
__global__ void fold2_kernel(const double* __restrict__ G2, int R, int64_t I, int R1, double* __restrict__ G) {
  const int64_t total = (int64_t)R * I * R1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e % R, ib = e / R, i = ib % I, b = ib / I;
    G[e] = G2[i + I * (a + (int64_t)R * b)];
  }
}

// column j of T (m x r) times sigma_j^+ (zero where the singular value is at the rounding level)
__global__ void scale_pinv_kernel(double* __restrict__ T, int64_t m, int r, const double* __restrict__ sig) {
  double smax = 0.0;
  for (int j = 0; j < r; ++j) smax = fmax(smax, sig[j]);
  const double tol = 32.0 * r * 1.1102230246251565e-16 * smax;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * r; e += (int64_t)gridDim.x * blockDim.x) {
    const double sg = sig[e / m];
    T[e] = sg > tol ? T[e] / sg : 0.0;
  }
}

constexpr int kSvdMaxR = 96;
// SVD of R (r x r, r <= kSvdMaxR) by one-sided Jacobi (Hestenes; Golub & Van Loan Sec. 8.6.4) in one CTA:
// rotations on pairs of columns of B = R accumulate in W until every pair is orthogonal to working
// accuracy; then R = U diag(sigma) V^T with sigma_j = |b_j|, u_j = b_j / sigma_j (zero for sigma_j = 0),
// V = W.  Each round treats r/2 disjoint pairs (round-robin order), one warp per pair; at most 30
// sweeps, fewer once a sweep rotates nothing.
__global__ void __launch_bounds__(256) jacobi_svd_kernel(const double* __restrict__ Rm, int r, double* __restrict__ U,
                                                         double* __restrict__ sig, double* __restrict__ Vm) {
  extern __shared__ double svd_sm[];   // B (r x r), then W (r x r)
  double* B = svd_sm;
  double* W = svd_sm + r * r;
  __shared__ int rotated;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < r * r; e += blockDim.x) {
    B[e] = Rm[e];
    W[e] = (e % r == e / r) ? 1.0 : 0.0;
  }
  const int P = (r + 1) & ~1;   // players, one dummy when r is odd
  const double eps = 1.1102230246251565e-16 * r;
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int t = 0; t < P - 1; ++t) {
      for (int i = warp; i < P / 2; i += nw) {
        // circle method: pair 0 is (t, P-1), pair i (t + i, t - i) mod (P - 1)
        int a = (i == 0) ? t : (t + i) % (P - 1);
        int b = (i == 0) ? P - 1 : (t - i + (P - 1)) % (P - 1);
        if (a > b) { const int x = a; a = b; b = x; }
        if (b >= r) continue;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int k = lane; k < r; k += 32) {
          const double x = B[k + r * a], y = B[k + r * b];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (fabs(ga) > eps * sqrt(al * be) && ga != 0.0) {
          const double zeta = (be - al) / (2.0 * ga);
          const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + tt * tt), sn = c * tt;
          for (int k = lane; k < r; k += 32) {
            const double x = B[k + r * a], y = B[k + r * b];
            B[k + r * a] = c * x - sn * y;
            B[k + r * b] = sn * x + c * y;
            const double wx = W[k + r * a], wy = W[k + r * b];
            W[k + r * a] = c * wx - sn * wy;
            W[k + r * b] = sn * wx + c * wy;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  for (int j = warp; j < r; j += nw) {
    double ss = 0.0;
    for (int k = lane; k < r; k += 32) ss = fma(B[k + r * j], B[k + r * j], ss);
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const double sj = sqrt(ss);
    if (lane == 0) sig[j] = sj;
    for (int k = lane; k < r; k += 32) {
      U[k + r * j] = sj > 0.0 ? B[k + r * j] / sj : 0.0;
      Vm[k + r * j] = W[k + r * j];
    }
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < nw; ++k) t += red[k];   // every thread, same fixed order
  return t;
}

// Householder QR of A (m x r, column-major, m >= r) in one CTA (Golub & Van Loan Sec. 5.2): A's columns
// are overwritten by the Householder vectors; R (r x r upper, column-major) and Q = H_0 ... H_{r-1} [I; 0]
// (m x r, column-major) are written, signs chosen so that R has a positive diagonal.  A column whose
// remaining part is at the rounding level, |R_kk| <= 32 r u max_j |a_j| (numerically rank deficient:
// a column that repeats earlier ones leaves a remainder of about u |a| rather than exact zeros), sets
// TRALS_E_NOT_SPD with its index and stops; with rd_flag given it is kept instead (R_kk = 0, no
// reflector: A = Q R still holds to that tolerance, Q orthonormal) and *rd_flag is set to 1.
__global__ void __launch_bounds__(256) householder_qr_kernel(double* __restrict__ A, int64_t m, int r,
                                                             double* __restrict__ Rm, double* __restrict__ Q,
                                                             double* __restrict__ tau, DevStatus* st, int mode,
                                                             int* __restrict__ rd_flag) {
  __shared__ double red[32];
  __shared__ double sc[2];
  __shared__ int fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) fail = 0;
  // the largest column norm of A, for the rank test
  double cmax = 0.0;
  for (int j = warp; j < r; j += nw) {
    double w = 0.0;
    for (int64_t i = lane; i < m; i += 32) w = fma(A[i + m * (int64_t)j], A[i + m * (int64_t)j], w);
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    cmax = fmax(cmax, w);
  }
  __syncthreads();
  if (lane == 0) red[warp] = cmax;
  __syncthreads();
  double norm0 = 0.0;
  for (int k = 0; k < nw; ++k) norm0 = fmax(norm0, red[k]);
  norm0 = sqrt(norm0);
  const double tol = 32.0 * r * 1.1102230246251565e-16 * norm0;
  for (int k = 0; k < r; ++k) {
    double* x = A + m * (int64_t)k;
    double ss = 0.0;
    for (int64_t i = k + tid; i < m; i += blockDim.x) ss = fma(x[i], x[i], ss);
    ss = block_sum(ss, red);
    if (tid == 0) {
      const double x0 = x[k], alpha = sqrt(ss);
      if (rd_flag != nullptr && isfinite(alpha) && !(alpha > tol)) {
        *rd_flag = 1;   // numerically dependent column: no reflector
        Rm[k + (int64_t)r * k] = 0.0;
        sc[0] = 0.0;
        tau[k] = 0.0;
      } else if (!(alpha > tol) || !isfinite(alpha)) {
        fail = 1;
        set_status(st, isfinite(alpha) ? TRALS_E_NOT_SPD : TRALS_E_NONFINITE, -1, mode, k, alpha);
      } else {
        const double beta = x0 >= 0.0 ? -alpha : alpha;
        const double v0 = x0 - beta;
        const double vtv = ss - x0 * x0 + v0 * v0;
        x[k] = v0;
        Rm[k + (int64_t)r * k] = beta;
        sc[0] = 2.0 / vtv;
        tau[k] = 2.0 / vtv;
      }
    }
    __syncthreads();
    if (fail) return;
    const double c = sc[0];
    // trailing columns: a_j -= c (v^T a_j) v, one warp per column
    for (int j = k + 1 + warp; j < r; j += nw) {
      double* y = A + m * (int64_t)j;
      double w = 0.0;
      for (int64_t i = k + lane; i < m; i += 32) w = fma(x[i], y[i], w);
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      const double f = c * w;
      for (int64_t i = k + lane; i < m; i += 32) y[i] = fma(-f, x[i], y[i]);
    }
    __syncthreads();
  }
  // R above the diagonal: row k of the reduced A
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    if (i < j) Rm[e] = A[i + m * (int64_t)j];
    else if (i > j) Rm[e] = 0.0;
  }
  // Q = H_0 ... H_{r-1} [I; 0], accumulated backwards (H_k touches rows >= k and, then, columns >= k)
  for (int64_t e = tid; e < m * r; e += blockDim.x) Q[e] = ((e % m) == (e / m)) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = r - 1; k >= 0; --k) {
    const double* v = A + m * (int64_t)k;
    const double c = tau[k];
    for (int j = k + warp; j < r; j += nw) {
      double* q = Q + m * (int64_t)j;
      double w = 0.0;
      for (int64_t i = k + lane; i < m; i += 32) w = fma(v[i], q[i], w);
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      const double f = c * w;
      for (int64_t i = k + lane; i < m; i += 32) q[i] = fma(-f, v[i], q[i]);
    }
    __syncthreads();
  }
  // positive diagonal: flip row k of R and column k of Q where R_kk < 0
  for (int k = warp; k < r; k += nw) {
    const bool neg = Rm[k + (int64_t)r * k] < 0.0;   // read by every lane before any lane flips it
    __syncwarp();
    if (neg) {
      for (int j = k + lane; j < r; j += 32) Rm[k + (int64_t)r * j] = -Rm[k + (int64_t)r * j];
      for (int64_t i = lane; i < m; i += 32) Q[i + m * (int64_t)k] = -Q[i + m * (int64_t)k];
    }
  }
}

struct Buf {
  std::vector<void*> all;
  cudaError_t e = cudaSuccess;
  template <class T>
  T* get(size_t n) {
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) all.push_back(p);
    return static_cast<T*>(p);
  }
  ~Buf() {
    for (void* p : all) cudaFree(p);
  }
};

}  // namespace

trals_status qrne_decompose(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R, const double* X,
                            double* const* cores_host, int sweeps, double* rel_res, bool literal) {
  cudaStream_t s = ctx->stream;
  Buf buf;
  int rr[kMaxOrder];
  bool comp[kMaxOrder];
  int64_t Yd[kMaxOrder];   // extents of the compressed modes (mode n keeps I_n)
  int64_t core_el[kMaxOrder], rcore_el[kMaxOrder];
  int rmax = 1;
  int64_t Imax = 1;
  for (int j = 0; j < N; ++j) {
    rr[j] = R[j] * R[(j + 1) % N];
    comp[j] = I[j] > rr[j];
    Yd[j] = comp[j] ? rr[j] : I[j];
    core_el[j] = (int64_t)R[j] * I[j] * R[(j + 1) % N];
    rcore_el[j] = (int64_t)R[j] * Yd[j] * R[(j + 1) % N];
    rmax = std::max(rmax, rr[j]);
    Imax = std::max(Imax, I[j]);
  }
  // ---- workspace
  double* G[kMaxOrder];
  double* Rc[kMaxOrder];
  double* Qm[kMaxOrder];
  double* gam[kMaxOrder];
  for (int j = 0; j < N; ++j) {
    G[j] = buf.get<double>(core_el[j]);
    Rc[j] = comp[j] ? buf.get<double>(rcore_el[j]) : G[j];
    Qm[j] = comp[j] ? buf.get<double>((size_t)I[j] * rr[j]) : nullptr;
    gam[j] = buf.get<double>((size_t)R[j] * R[j] * R[(j + 1) % N] * R[(j + 1) % N]);
  }
  double* G2 = buf.get<double>((size_t)Imax * rmax);
  double* Q1 = buf.get<double>((size_t)Imax * rmax);
  double* C = buf.get<double>((size_t)rmax * rmax);
  double* L1 = buf.get<double>(lmat_elems(rmax));
  double* L2 = buf.get<double>(lmat_elems(rmax));
  double* Pm = buf.get<double>((size_t)rmax * rmax);
  int64_t rsq = 1;
  for (int j = 0; j < N; ++j) rsq = std::max<int64_t>(rsq, (int64_t)R[j] * R[j]);
  double* chainA = buf.get<double>(rsq * rsq);   // Gamma-chain products: R_{n+1}^2 x R_c^2
  double* chainB = buf.get<double>(rsq * rsq);
  double* S = buf.get<double>((size_t)rmax * rmax);
  double* Lm = buf.get<double>(lmat_elems(rmax));
  // the Multi-TTM of mode n applies the most compressing modes first
  auto ttm_order = [&](int n) {
    std::vector<int> order;
    for (int j = 0; j < N; ++j)
      if (j != n && comp[j]) order.push_back(j);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return (double)rr[a] / I[a] < (double)rr[b] / I[b]; });
    return order;
  };
  // Multi-TTM ping-pong buffers: the largest intermediate of any mode's sequence
  int64_t ymax = 1;
  for (int n = 0; n < N; ++n) {
    int64_t cur[kMaxOrder];
    for (int j = 0; j < N; ++j) cur[j] = I[j];
    for (int j : ttm_order(n)) {
      cur[j] = rr[j];
      int64_t t = 1;
      for (int m = 0; m < N; ++m) t *= cur[m];
      ymax = std::max(ymax, t);
    }
  }
  double* Ya = buf.get<double>(ymax);
  double* Yb = buf.get<double>(ymax);
  // MTTSP of Y with the R cores: layouts, offsets and tables per mode
  ModeLayout LY[kMaxOrder];
  int64_t* offL[kMaxOrder];
  int64_t* offU[kMaxOrder];
  int64_t tab = 1;
  size_t part = 1;
  for (int n = 0; n < N; ++n) {
    int64_t d[kMaxOrder];
    for (int j = 0; j < N; ++j) d[j] = (j == n) ? I[j] : Yd[j];
    LY[n] = make_mode_layout(N, d, R, n);
    tab = std::max(tab, table_level_max_elems(LY[n], d, R));
    part = std::max(part, mttsp_simt_partials_elems(LY[n], mttsp_simt_default_grid(LY[n])));
    std::vector<int64_t> oL, oU;
    mode_offsets(N, d, LY[n], oL, oU);
    offL[n] = buf.get<int64_t>(oL.size());
    offU[n] = buf.get<int64_t>(oU.size());
    if (buf.e == cudaSuccess) buf.e = cudaMemcpy(offL[n], oL.data(), oL.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (buf.e == cudaSuccess) buf.e = cudaMemcpy(offU[n], oU.data(), oU.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  }
  // explicit residual of the G cores against X (layout of the last mode of X)
  const ModeLayout LX = make_mode_layout(N, I, R, N - 1);
  tab = std::max(tab, table_level_max_elems(LX, I, R));
  std::vector<int64_t> xoL, xoU;
  mode_offsets(N, I, LX, xoL, xoU);
  int64_t* xdL = buf.get<int64_t>(xoL.size());
  int64_t* xdU = buf.get<int64_t>(xoU.size());
  if (buf.e == cudaSuccess) buf.e = cudaMemcpy(xdL, xoL.data(), xoL.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (buf.e == cudaSuccess) buf.e = cudaMemcpy(xdU, xoU.data(), xoU.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  const int gridR = mttsp_simt_default_grid(LX);
  double* lt = buf.get<double>(tab);
  double* ut = buf.get<double>(tab);
  double* sc = buf.get<double>(tab);
  double* partials = buf.get<double>(std::max<size_t>(part, 2 * (size_t)gridR));
  double* M = buf.get<double>((size_t)Imax * rmax);
  double* tau = buf.get<double>(std::max<int64_t>(rmax, 1));
  // literal Alg. 3: V_n[2] and Q_0 (J' x r) of the largest mode
  int64_t vmax = 1;
  if (literal)
    for (int n = 0; n < N; ++n) vmax = std::max<int64_t>(vmax, LY[n].nL * LY[n].nU * rr[n]);
  if (literal) {
    for (int n = 0; n < N; ++n) {
      const int64_t Jc = LY[n].nL * LY[n].nU;
      if (Jc < rr[n] || Jc > ((int64_t)1 << 22)) {
        ctx->last_error = "literal TR-ALS-QR: the compressed subchain of mode " + std::to_string(n) + " has " +
                          std::to_string(Jc) + " rows (needs R_n R_{n+1} <= rows <= 2^22; use TRALS_SOLVE_QR)";
        return TRALS_E_ARG;
      }
    }
  }
  double* V = literal ? buf.get<double>(vmax) : nullptr;
  double* Q0 = literal ? buf.get<double>(vmax) : nullptr;
  // SVD option: U, sigma, V, V^T and W_n U of a rank-deficient subproblem; rank-deficiency flags
  double* Us = buf.get<double>((size_t)rmax * rmax);
  double* Vs = buf.get<double>((size_t)rmax * rmax);
  double* Vt = buf.get<double>((size_t)rmax * rmax);
  double* sig = buf.get<double>(rmax);
  double* T1 = buf.get<double>((size_t)Imax * rmax);
  int* rd_v = buf.get<int>(2);
  int* rd_core = rd_v + 1;
  double* red = buf.get<double>(2);
  double* res_dev = buf.get<double>(std::max(1, sweeps));
  TRALS_CUDA_TRY(ctx, buf.e);
  for (int j = 0; j < N; ++j)
    TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(G[j], cores_host[j], core_el[j] * sizeof(double), cudaMemcpyHostToDevice, s));

  // mode-2 QR of core j (Alg. 4 lines 2 and 11) and the Gram tensor of its R factor (lines 3 and 12)
  auto factor_core = [&](int j) {
    const int Rj = R[j], Rj1 = R[(j + 1) % N], r = rr[j];
    if (comp[j] && literal) {
      // Householder mode-2 QR (Alg. 3 lines 2 and 10)
      unfold2_kernel<<<grid_of(core_el[j], 256), 256, 0, s>>>(G[j], Rj, I[j], Rj1, G2);
      householder_qr_kernel<<<1, 256, 0, s>>>(G2, I[j], r, Pm, Qm[j], tau, ctx->d_status, j, rd_core);
      rcore_from_upper_kernel<<<grid_of((int64_t)r * r, 256), 256, 0, s>>>(Pm, Rj, Rj1, Rc[j]);
    } else if (comp[j]) {
      const int64_t Ij = I[j];
      unfold2_kernel<<<grid_of(core_el[j], 256), 256, 0, s>>>(G[j], Rj, Ij, Rj1, G2);
      // pass 1: C = G2^T G2 (the Gram of a 1 x I_j x r "core"), L1 L1^T = C, Q1 = G2 L1^{-T}
      launch_gamma(G2, 1, Ij, r, C, s);
      launch_cholesky(C, L1, r, ctx->d_status, nullptr, j, s);
      launch_chol_solve(L1, G2, 1, Ij, r, Q1, ctx->d_status, s, nullptr, 0, kSolveForward);
      // pass 2 on Q1
      launch_gamma(Q1, 1, Ij, r, C, s);
      launch_cholesky(C, L2, r, ctx->d_status, nullptr, j, s);
      launch_chol_solve(L2, Q1, 1, Ij, r, Qm[j], ctx->d_status, s, nullptr, 0, kSolveForward);
      // R = R2 R1 = (L1 L2)^T
      launch_gemm_f64(r, r, r, L1, L2, Pm, s);
      rcore_from_lower_kernel<<<grid_of((int64_t)r * r, 256), 256, 0, s>>>(Pm, Rj, Rj1, Rc[j]);
    }
    if (!literal) launch_gamma(Rc[j], Rj, Yd[j], Rj1, gam[j], s);
  };
  for (int j = 0; j < N; ++j) factor_core(j);

  for (int sw = 0; sw < sweeps; ++sw) {
    for (int n = 0; n < N; ++n) {
      const int Rn = R[n], Rn1 = R[(n + 1) % N], r = rr[n];
      // S_n from the Gram tensors of the R factors: Pi_n = Gamma_{n+1} ... Gamma_{n-1}, regrouped (line 7)
      if (!literal) {
        const int c0 = (n + 1) % N;
        const double* cur = gam[c0];
        const int rows = R[c0] * R[c0];
        double* bufs[2] = {chainA, chainB};
        for (int t = 2; t < N; ++t) {
          const int c = (n + t) % N;
          launch_gemm_f64(rows, R[(c + 1) % N] * R[(c + 1) % N], R[c] * R[c], cur, gam[c], bufs[t % 2], s);
          cur = bufs[t % 2];
        }
        launch_regroup_S(cur, Rn, Rn1, S, s);
      }
      // Y = X x_{j != n} Q_j^T, the most compressing modes first (line 8)
      int64_t cur[kMaxOrder];
      for (int j = 0; j < N; ++j) cur[j] = I[j];
      const std::vector<int> order = ttm_order(n);
      const double* src = X;
      double* dst = Ya;
      for (int j : order) {
        int64_t A = 1, B = 1;
        for (int m = 0; m < j; ++m) A *= cur[m];
        for (int m = j + 1; m < N; ++m) B *= cur[m];
        const dim3 g((unsigned)grid_of(A * B, 128), (unsigned)((rr[j] + 7) / 8));
        ttm_kernel<<<g, 128, 0, s>>>(src, A, I[j], B, Qm[j], rr[j], dst);
        cur[j] = rr[j];
        src = dst;
        dst = (dst == Ya) ? Yb : Ya;
      }
      if (literal) {
        // Alg. 3: V_n[2] explicitly from the R cores (line 5), its Householder QR V_n[2] = Q_0 R with Q_0
        // formed (line 6), W_n = Y_[n] Q_0 (line 8), then G_{n(2)} R^T = W_n by substitution (line 9):
        // G = W L^{-1} with L = R^T, the backward solve alone
        int64_t d[kMaxOrder];
        for (int j = 0; j < N; ++j) d[j] = (j == n) ? I[j] : Yd[j];
        const double* rc[kMaxOrder];
        for (int j = 0; j < N; ++j) rc[j] = Rc[j];
        build_tables(LY[n], rc, d, R, lt, ut, sc, s);
        const int64_t Jc = LY[n].nL * LY[n].nU;
        subchain_explicit_kernel<<<grid_of(Jc * r, 256), 256, 0, s>>>(lt, ut, LY[n], V);
        TRALS_CUDA_TRY(ctx, cudaMemsetAsync(rd_v, 0, sizeof(int), s));
        householder_qr_kernel<<<1, 256, 0, s>>>(V, Jc, r, Pm, Q0, tau, ctx->d_status, n, rd_v);
        wn_kernel<<<grid_of(I[n] * r, 128), 128, 0, s>>>(src, offL[n], offU[n], LY[n], Q0, M);
        int rd_host = 0;
        TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(&rd_host, rd_v, sizeof(int), cudaMemcpyDeviceToHost, s));
        TRALS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (rd_host && r <= kSvdMaxR) {
          // rank-deficient V_n: the SVD of R (remark after Alg. 3), G_{n(2)} = W_n U Sigma^+ V^T, the
          // minimum-norm solution of the compressed problem (and of the whole subproblem)
          const size_t svd_smem = 2 * (size_t)r * r * sizeof(double);
          TRALS_CUDA_TRY(ctx, cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)svd_smem));
          jacobi_svd_kernel<<<1, 256, svd_smem, s>>>(Pm, r, Us, sig, Vs);
          launch_gemm_f64((int)I[n], r, r, M, Us, T1, s);
          scale_pinv_kernel<<<grid_of(I[n] * r, 256), 256, 0, s>>>(T1, I[n], r, sig);
          launch_transpose(Vs, r, Vt, s);
          launch_gemm_f64((int)I[n], r, r, T1, Vt, G2, s);
          fold2_kernel<<<grid_of(core_el[n], 256), 256, 0, s>>>(G2, Rn, I[n], Rn1, G[n]);
        } else if (rd_host) {
          ctx->last_error = "literal TR-ALS-QR: rank-deficient subproblem with R_n R_{n+1} > 96 (SVD limit)";
          return TRALS_E_NOT_SPD;
        } else {
          upper_to_lmat_kernel<<<grid_of((int64_t)r * r + r, 256), 256, 0, s>>>(Pm, r, Lm);
          launch_chol_block_inverse(Lm, r, s);
          launch_chol_solve(Lm, M, Rn, I[n], Rn1, G[n], ctx->d_status, s, nullptr, 0, kSolveBackward);
        }
        factor_core(n);
        continue;
      }
      // M_n = Y_[n] V_n[2]: the FP64 MTTSP of Y with the R cores (line 9)
      {
        int64_t d[kMaxOrder];
        for (int j = 0; j < N; ++j) d[j] = (j == n) ? I[j] : Yd[j];
        const double* rc[kMaxOrder];
        for (int j = 0; j < N; ++j) rc[j] = Rc[j];
        build_tables(LY[n], rc, d, R, lt, ut, sc, s);
        MttspSimtArgs a;
        a.X = src;
        a.xt = TRALS_X_F64;
        a.ltab = lt;
        a.utab = ut;
        a.offL = offL[n];
        a.offU = offU[n];
        a.L = LY[n];
        a.partials = partials;
        a.M = M;
        a.gridX = mttsp_simt_default_grid(LY[n]);
        launch_mttsp_simt(a, s);
      }
      // G_{n(2)} S_n = M_n by Cholesky (line 10), then the new core's QR and Gram tensor (lines 11-12)
      launch_cholesky(S, Lm, r, ctx->d_status, nullptr, n, s);
      launch_chol_solve(Lm, M, Rn, I[n], Rn1, G[n], ctx->d_status, s);
      factor_core(n);
    }
    // explicit relative residual of the G cores against X (Sec. 4 error formula)
    const double* gc[kMaxOrder];
    for (int j = 0; j < N; ++j) gc[j] = G[j];
    build_tables(LX, gc, I, R, lt, ut, sc, s);
    launch_reconstruct(LX, lt, ut, xdL, xdU, G[N - 1], nullptr, TRALS_X_F64, X, TRALS_X_F64, partials, gridR, s);
    launch_reduce_pairs(partials, gridR, red, s);
    finalize_ratio_kernel<<<1, 1, 0, s>>>(red, res_dev + sw);
    TRALS_CUDA_TRY(ctx, cudaGetLastError());
  }
  for (int j = 0; j < N; ++j)
    TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(cores_host[j], G[j], core_el[j] * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (rel_res && sweeps > 0)
    TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(rel_res, res_dev, sweeps * sizeof(double), cudaMemcpyDeviceToHost, s));
  TRALS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  // a failed factorization (rank deficiency, non-finite values) was recorded in the status word
  DevStatus st{};
  TRALS_CUDA_TRY(ctx, cudaMemcpy(&st, ctx->d_status, sizeof st, cudaMemcpyDeviceToHost));
  if (st.code != 0) {
    ctx->last_error = std::string(st.code == TRALS_E_NOT_SPD ? "rank-deficient or non-positive factor"
                                                             : "non-finite value in a factorization") +
                      " at core " + std::to_string(st.mode) + ", index " + std::to_string(st.index);
    launch_zero_status(ctx->d_status, s);
    cudaStreamSynchronize(s);
    return (trals_status)st.code;
  }
  return TRALS_OK;
}

}  // namespace trals
