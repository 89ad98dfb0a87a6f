// QR-stabilised solve of the core subproblem (Sec. 3.2, TR-ALS-QR) without forming S_n.
//
// The R factor of the subchain matrix A = G^{!=n}_[2] is computed by a recursive structured QR along
// the subchain c_1 = n+1, ..., c_{N-1} = n-1 (eq. subchain_new).  The first step is the mode-2 QR of
// G_{c_1} (Def. mode-n QR).  Each later step writes the running product as
// (R_t x_2 Q_t) [x]_2 G_{c_{t+1}} = (R_t [x]_2 G_{c_{t+1}}) x_2 (I (x) Q_t) (Prop. slice_kron).  The
// factor I (x) Q_t has orthonormal columns, so the R factor of the product equals that of the
// small matrix (R_t [x]_2 G_{c_{t+1}})_[2].  That matrix has at most R_{n+1} R_{c_{t+1}} I_{c_{t+1}}
// rows and is factorised by a TSQR tree: Householder QR of row blocks, then pairwise QR of stacked
// R factors.  The paper's Alg. 3 reaches the same R by the QR of V_n (Alg. 3 line 6), whose size
// grows as R^{2N-2}; here every step stays R^2 I x R^2.
//
// With A = Q R, the normal equations G_{n(2)} A^T A = M_n read G_{n(2)} R^T R = M_n, so L = R^T
// takes the place of the Cholesky factor of S_n.  R comes from orthogonal transformations of the
// cores, so the squared condition number of S_n never enters the factor.
#include <algorithm>

#include "trals_internal.cuh"

namespace trals {

namespace {

// Threads per QR CTA.  A Householder step's columns are spread over 32 warps (a leaf: one column per
// warp and pass; a merge: eight columns per warp, four lanes each), so most steps are one pass and
// enough independent FP64 chains are in flight to keep the SM's FP64 unit issuing.
constexpr int QT = 1024;

// CTA-wide sum of each thread's part of a column's sum of squares; then one thread forms the
// Householder reflector of that column from it and from x0 (the entry on the diagonal, read by that
// thread after the first barrier): red[32] = the sum, red[33] = alpha (the new diagonal entry),
// red[34] = v0 (the reflector's entry on the diagonal), red[35] = tau = 2 / |v|^2.  kWithX0: the sum
// already includes x0^2 (else the sum runs over the entries below the diagonal only).  With v0_dst set
// that thread also stores v0 there.  The FP64 unit of an SM issues one warp instruction at a time
// whatever the number of active lanes, so the square root and the division are done once, not by
// every thread.
template <bool kWithX0>
__device__ __forceinline__ void householder_scalars(double part, const double* x0p, double* v0_dst, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = part;
  __syncthreads();
  if (w == 0) {
    double s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const double x0 = *x0p;
      const double below = kWithX0 ? s - x0 * x0 : s;
      const double nrm = sqrt(kWithX0 ? s : fma(x0, x0, s));
      const double alpha = x0 >= 0.0 ? -nrm : nrm;
      const double v0 = x0 - alpha;
      red[32] = s;
      red[33] = alpha;
      red[34] = v0;
      red[35] = 2.0 / (below + v0 * v0);
      if (v0_dst && s != 0.0) *v0_dst = v0;
    }
  }
  __syncthreads();
}

// Householder QR (GvL Alg. 5.2.1) of the m x C matrix W (column-major, leading dimension ld) in place,
// by one CTA.  On exit rows [0, min(m, C)) hold R (upper trapezoidal); everything below is zero.
__device__ void cta_householder_qr(double* W, int m, int C, int64_t ld, double* v, double* red) {
  const int kmax = min(m, C);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = 0; j < kmax; ++j) {
    double s = 0.0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
      const double x = W[i + (int64_t)ld * j];
      v[i] = x;
      s = fma(x, x, s);
    }
    householder_scalars<true>(s, &v[j], &v[j], red);   // v[j] <- v0
    if (red[32] == 0.0) {   // uniform: the column is already zero
      __syncthreads();
      continue;
    }
    const double alpha = red[33], tau = red[35];
    for (int c = j + 1 + warp; c < C; c += nw) {
      // two partial sums (rows i and i + 32 of each 64) halve the dependent chain
      double w0 = 0.0, w1 = 0.0;
      int i = j + lane;
      for (; i + 32 < m; i += 64) {
        w0 = fma(v[i], W[i + (int64_t)ld * c], w0);
        w1 = fma(v[i + 32], W[i + 32 + (int64_t)ld * c], w1);
      }
      if (i < m) w0 = fma(v[i], W[i + (int64_t)ld * c], w0);
      double w = w0 + w1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      const double f = tau * w;
      for (int i = j + lane; i < m; i += 32) W[i + (int64_t)ld * c] = fma(-f, v[i], W[i + (int64_t)ld * c]);
    }
    if (threadIdx.x == 0) W[j + (int64_t)ld * j] = alpha;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) W[i + (int64_t)ld * j] = 0.0;
    __syncthreads();
  }
}

// Householder QR of two stacked upper-triangular C x C factors, W = [R_top; R_bot] (2C x C, column-major,
// leading dimension ld), by one CTA.  The reflector of column j only involves row j and rows C .. C + j
// (the rows of R_bot that are not yet zero in column j), and the structure is kept: after step j the
// bottom block is zero in columns <= j and still upper triangular beyond.  Each step therefore costs
// (j + 2) rows instead of 2C - j, about a fifth of the dense QR's arithmetic.  On exit the top C rows
// hold R, the bottom block is zero.
__device__ void cta_householder_stacked(double* W, int C, int64_t ld, double* v, double* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int q = lane & 3;   // four lanes per column: a column's dot product and update
  double* Wb = W + C;       // bottom block: Wb[i + ld c]
  for (int j = 0; j < C; ++j) {
    double s = 0.0;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
      const double x = Wb[i + ld * j];
      v[i] = x;
      s = fma(x, x, s);
    }
    householder_scalars<false>(s, &W[j + ld * j], nullptr, red);
    if (red[32] == 0.0) {   // uniform: the bottom part of the column is already zero
      __syncthreads();
      continue;
    }
    const double alpha = red[33], v0 = red[34], tau = red[35];
    // eight columns per warp and pass (the loop bound is uniform per warp, so the shuffles see all lanes)
    for (int c0 = j + 1 + 8 * warp; c0 < C; c0 += 8 * nw) {
      const int c = c0 + (lane >> 2);
      const bool ok = c < C;
      double w0 = (ok && q == 0) ? v0 * W[j + ld * c] : 0.0, w1 = 0.0;
      if (ok) {
        int i = q;
        for (; i + 4 <= j; i += 8) {
          w0 = fma(v[i], Wb[i + ld * c], w0);
          w1 = fma(v[i + 4], Wb[i + 4 + ld * c], w1);
        }
        if (i <= j) w0 = fma(v[i], Wb[i + ld * c], w0);
      }
      double w = w0 + w1;
      w += __shfl_xor_sync(0xffffffffu, w, 1);
      w += __shfl_xor_sync(0xffffffffu, w, 2);
      if (ok) {
        const double f = tau * w;
        if (q == 0) W[j + ld * c] = fma(-f, v0, W[j + ld * c]);
        for (int i = q; i <= j; i += 4) Wb[i + ld * c] = fma(-f, v[i], Wb[i + ld * c]);
      }
    }
    if (threadIdx.x == 0) W[j + ld * j] = alpha;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) Wb[i + ld * j] = 0.0;
    __syncthreads();
  }
}

// B[(s + m i) + M (d + Rd b)] = sum_c P[s + ldp (c + Rc b)] G[c + Rc (i + I d)]: the mode-2 unfolding of
// (R_t [x]_2 G) with R_t given as an m x (Rc Rb) matrix (column c + Rc b).  With first != 0 the
// running product is the identity (m = 1): B[i + I (d + Rd b)] = G[b + Rc (i + I d)] (Rc = Rb).
__global__ void qr_form_kernel(const double* __restrict__ P, int m, int ldp, const double* __restrict__ G, int Rc,
                               int64_t I, int Rd, int Rb, int first, double* __restrict__ B) {
  const int64_t M = (int64_t)m * I;
  const int64_t total = M * Rd * Rb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e % M;
    const int col = (int)(e / M);
    const int d = col % Rd, b = col / Rd;
    const int s = (int)(row % m);
    const int64_t i = row / m;
    double acc;
    if (first) {
      acc = G[b + (int64_t)Rc * (i + I * d)];
    } else {
      acc = 0.0;
      for (int c = 0; c < Rc; ++c) acc = fma(P[s + (int64_t)ldp * (c + Rc * b)], G[c + (int64_t)Rc * (i + I * d)], acc);
    }
    B[e] = acc;
  }
}

// TSQR leaves: CTA b factorises rows [b Mb, min(M, (b+1) Mb)) of B (ld = M) in place and writes its
// R factor to Rout[b] (C x C, column-major, zero below the factor).
__global__ void __launch_bounds__(QT) tsqr_leaf_kernel(double* __restrict__ B, int64_t M, int C, int Mb,
                                                       double* __restrict__ Rout) {
  extern __shared__ double qsm[];
  double* red = qsm;          // 33
  double* v = qsm + 40;       // Mb
  const int64_t r0 = (int64_t)blockIdx.x * Mb;
  const int m = (int)min((int64_t)Mb, M - r0);
  double* W = B + r0;
  cta_householder_qr(W, m, C, M, v, red);
  double* R = Rout + (int64_t)blockIdx.x * C * C;
  for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
    const int i = e % C, j = e / C;
    R[e] = (i < m && i <= j) ? W[i + M * j] : 0.0;
  }
}

// TSQR tree level: CTA b stacks Rin[2b] over Rin[2b+1] (2C x C) in the workspace, factorises it and
// writes the R factor to Rout[b].  An unpaired last factor is copied through.
__global__ void __launch_bounds__(QT) tsqr_merge_kernel(const double* __restrict__ Rin, int nin, int C,
                                                        double* __restrict__ Wk, double* __restrict__ Rout) {
  extern __shared__ double qsm[];
  double* red = qsm;
  double* v = qsm + 40;       // 2C
  const int b = blockIdx.x;
  const double* A0 = Rin + (int64_t)(2 * b) * C * C;
  double* R = Rout + (int64_t)b * C * C;
  if (2 * b + 1 >= nin) {
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) R[e] = A0[e];
    return;
  }
  const double* A1 = A0 + (int64_t)C * C;
  double* W = Wk + (int64_t)b * 2 * C * C;
  for (int e = threadIdx.x; e < 2 * C * C; e += blockDim.x) {
    const int i = e % (2 * C), j = e / (2 * C);
    W[e] = i < C ? A0[i + C * j] : A1[(i - C) + C * j];
  }
  __syncthreads();
  cta_householder_stacked(W, C, 2 * C, v, red);
  for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
    const int i = e % C, j = e / C;
    R[e] = i <= j ? W[i + 2 * C * j] : 0.0;
  }
}

// Final factor: rows scaled to a positive diagonal, L = R^T with its reciprocal diagonal appended
// (the layout the Cholesky solve reads).  A zero or non-finite diagonal means G^{!=n}_[2] is rank
// deficient: reported like a failed Cholesky pivot.
__global__ void qr_to_l_kernel(const double* __restrict__ Rf, int r, double* __restrict__ Lmat, DevStatus* st,
                               const int* sweep_ctr, int mode) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
    const int i = e % r, j = e / r;   // L[i, j] = sign_j R[j, i]
    const double dj = Rf[j + (int64_t)r * j];
    Lmat[e] = i >= j ? (dj < 0.0 ? -Rf[j + (int64_t)r * i] : Rf[j + (int64_t)r * i]) : 0.0;
  }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < r; j += gridDim.x * blockDim.x) {
    const double d = fabs(Rf[j + (int64_t)r * j]);
    if (!(d > 0.0) || !isfinite(d)) set_status(st, TRALS_E_NOT_SPD, sweep_ctr ? *sweep_ctr : -1, mode, j, d);
    Lmat[(int64_t)r * r + j] = 1.0 / d;
  }
}

// S = L L^T (the coefficient matrix, for the residual identity of the QR path)
__global__ void llt_kernel(const double* __restrict__ Lmat, int r, double* __restrict__ S) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
    const int i = e % r, j = e / r;
    double acc = 0.0;
    for (int k = 0; k <= min(i, j); ++k) acc = fma(Lmat[i + (int64_t)r * k], Lmat[j + (int64_t)r * k], acc);
    S[e] = acc;
  }
}

__global__ void transpose_kernel(const double* __restrict__ A, int r, double* __restrict__ B) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x)
    B[(e / r) + (int64_t)r * (e % r)] = A[e];
}

__global__ void axpy_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] += x[e];
}

int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

// Chain steps of mode n: (rows M_t, columns C_t) of each step's matrix, and the TSQR leaf height.
static void qr_steps(int N, const int64_t* I, const int32_t* R, int n, int64_t* Ms, int* Cs) {
  const int Rb = R[(n + 1) % N];
  int64_t m = 1;
  for (int t = 1; t <= N - 1; ++t) {
    const int c = (n + t) % N;
    const int Rd = R[(c + 1) % N];
    Ms[t - 1] = m * I[c];
    Cs[t - 1] = Rd * Rb;
    m = std::min<int64_t>(Ms[t - 1], Cs[t - 1]);
  }
}

static int leaf_rows(int C) { return std::max(2 * C, 64); }

QrSizes qr_sizes(int N, const int64_t* I, const int32_t* R, int n) {
  QrSizes z;
  int64_t Ms[kMaxOrder];
  int Cs[kMaxOrder];
  qr_steps(N, I, R, n, Ms, Cs);
  for (int t = 0; t < N - 1; ++t) {
    const int64_t C = Cs[t];
    const int64_t nb = (Ms[t] + leaf_rows(Cs[t]) - 1) / leaf_rows(Cs[t]);
    z.B_elems = std::max<int64_t>(z.B_elems, Ms[t] * C);
    z.R_elems = std::max<int64_t>(z.R_elems, nb * C * C);
    z.W_elems = std::max<int64_t>(z.W_elems, ((nb + 1) / 2) * 2 * C * C);
  }
  return z;
}

size_t qr_smem_bytes(int C) { return (40 + (size_t)std::max(leaf_rows(C), 2 * C)) * sizeof(double); }

int launch_qr_factor(int N, const int64_t* I, const int32_t* R, int n, const double* const* cores, double* B,
                     double* R0, double* R1, double* Wk, double* Lmat, DevStatus* st, const int* sweep_ctr,
                     cudaStream_t s) {
  int64_t Ms[kMaxOrder];
  int Cs[kMaxOrder];
  qr_steps(N, I, R, n, Ms, Cs);
  const int Rb = R[(n + 1) % N];
  int launches = 0;
  const double* P = nullptr;
  int m = 1, ldp = 1;
  for (int t = 1; t <= N - 1; ++t) {
    const int c = (n + t) % N;
    const int Rc = R[c], Rd = R[(c + 1) % N];
    const int64_t M = Ms[t - 1];
    const int C = Cs[t - 1];
    qr_form_kernel<<<grid_of(M * C), 256, 0, s>>>(P, m, ldp, cores[c], Rc, I[c], Rd, Rb, t == 1, B);
    const int Mb = leaf_rows(C);
    int nb = (int)((M + Mb - 1) / Mb);
    const size_t smem = qr_smem_bytes(C);
    tsqr_leaf_kernel<<<nb, QT, smem, s>>>(B, M, C, Mb, R0);
    launches += 2;
    double* in = R0;
    double* out = R1;
    while (nb > 1) {
      const int nout = (nb + 1) / 2;
      tsqr_merge_kernel<<<nout, QT, smem, s>>>(in, nb, C, Wk, out);
      ++launches;
      std::swap(in, out);
      nb = nout;
    }
    P = in;   // C x C, rows >= min(M, C) zero
    m = (int)std::min<int64_t>(M, C);
    ldp = C;
  }
  const int r = Cs[N - 2];
  qr_to_l_kernel<<<grid_of((int64_t)r * r), 256, 0, s>>>(P, r, Lmat, st, sweep_ctr, n);
  launch_chol_block_inverse(Lmat, r, s);
  return launches + 2;
}

void launch_transpose(const double* A, int r, double* B, cudaStream_t s) {
  transpose_kernel<<<grid_of((int64_t)r * r), 256, 0, s>>>(A, r, B);
}

void launch_llt(const double* Lmat, int r, double* S, cudaStream_t s) {
  llt_kernel<<<grid_of((int64_t)r * r), 256, 0, s>>>(Lmat, r, S);
}

void launch_axpy(int64_t n, const double* x, double* y, cudaStream_t s) { axpy_kernel<<<grid_of(n), 256, 0, s>>>(n, x, y); }

cudaError_t init_qr_attributes() {
  cudaError_t e = cudaFuncSetAttribute(tsqr_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(tsqr_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  return e;
}

}  // namespace trals
