// Grouped step engine of the serving loop (interface in group.cuh).
//
// A step advances every active slot by one core update of Alg. 2 (its own mode n and sweep), or runs
// its set-up.  The step is one captured graph of seven kernels over a device table of the active slots:
//   K0 doorbell: one CTA waits, with a bound, until the host has published the step's table in mapped
//      host memory, then copies it into the device table (on a timeout the step has no slots);
//   K1 prepare: a slot's first step makes the BF16 copy of X (BF16 mode) and Gamma_k of every core
//      (Alg. 2 line 2); an update step builds the two FP32 subchain tables of mode n, A(j_A) =
//      G_{n+1}(i_{n+1}) ... G_m(i_m) and B(j_B) = G_{m+1}(i_{m+1}) ... G_{n-1}(i_{n-1}), and the first
//      product of the Gamma chain Gamma_{n+1} ... Gamma_{n-1} (Alg. 2 line 6);
//   K2 MTTSP (Alg. 2 lines 7-8): M_n(i_n, a + R_n b) = sum_j X(i_n, j) [A(j_A) B(j_B)](b, a), as partial
//      rows over chunks of 32 values of j_B, and the second chain product;
//   K3 M_n in FP64 (fixed-order sum of the chunks) and the third chain product; the last product is
//      stored as the regrouped S_n;
//   K4 Cholesky S_n = L L^T, one CTA per slot;
//   K5 the solve G_{n(2)} S_n = M_n (Alg. 2 line 9): forward and backward substitution, a warp per row;
//   K6 Gamma_n of the new core (Alg. 2 line 10) and, after the last sweep, the explicit relative
//      residual of the cores against the FP32 X (Sec. 4).
// K1-K3, K5 and K6 run a fixed grid that walks the step's units (pieces of work of one CTA) with a
// grid stride; a unit finds its slot in a prefix table of unit counts.  A slot's arithmetic depends on
// its own data only, in a fixed order, so its results do not depend on what else is in the step.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>

#include "group.cuh"

namespace trals {
namespace {

constexpr int kThreads = 256;
constexpr int kMP = 64;                             // (i_n, j_B) pairs per MTTSP / residual unit
constexpr int kE = 64;                              // FP64 entries per Gamma / chain-product unit
constexpr int kSolveRows = 2;                       // rows per solve unit
constexpr int kUnitA = 512;                         // j_A values per MTTSP / residual unit (16 tiles)
constexpr int kR2 = kGrpMaxRank * kGrpMaxRank;      // widest table row, Gamma side, S_n side
constexpr int kQuantChunk = 8192;                   // X entries per quantisation unit
constexpr int kKernels = 5;                         // unit tables: K1, K2, K3, K5, K6
constexpr int kRing = 64;                           // step timeout records kept in the control block
constexpr long long kDefaultSpin = 2000000000LL;    // doorbell wait bound (clock cycles, about a second)
constexpr int kLd = kR2 + 1;                        // leading dimension of L in shared memory

enum { kInit = 0, kUpdate = 1 };
enum { kLanesB = 0, kLanesA = 1, kLanesI = 2 };   // MTTSP unit geometries (see K2)

// One slot as a step sees it.
struct alignas(16) GrpSlot {
  int N, n, phase, fin, mode, sweep;
  int Ra, nA;                      // R at the split (rows of B); modes in A (chain[0 .. nA-1])
  int chain[kGrpMaxOrder - 1];     // n+1, ..., n-1 (cyclic)
  int R[kGrpMaxOrder];
  int64_t I[kGrpMaxOrder];
  int64_t str[kGrpMaxOrder];       // memory stride of i_k in X (I_0 fastest)
  int64_t KA, KB, numel;
  int cls;                         // MTTSP unit geometry
  int nchB, nchA;                  // units per i_n (or per block of 64 i_0): chunks of j_B and of j_A
  int cB;                          // kLanesI: j_B values per unit
  int pad0;
  const float* X;                  // FP32 X
  __nv_bfloat16* Xq;               // BF16 copy of X (BF16 mode)
  double* cores[kGrpMaxOrder];     // FP64 master cores, R_k x I_k x R_{k+1} column-major
  double* gam[kGrpMaxOrder];       // Gamma_k, R_k^2 x R_{k+1}^2
  float* Atab;                     // [j_A][b + R_{n+1} c]
  float* Btab;                     // [j_B][c + Ra a]
  int64_t* offA;                   // memory offset of X for j_A (i_n = 0, j_B = 0)
  int64_t* offB;
  float* part;                     // [i_n][chunk][col]
  double* chainbuf[2];
  double* S;                       // r x r
  double* L;                       // r x r lower, then the r reciprocal pivots
  double* M;                       // I_n x r, column-major
  double* rpart;                   // residual unit pairs (|X - X_hat|^2, |X|^2)
  unsigned* rctr;
  double* res;
  DevStatus* st;
  int uq, ug[kGrpMaxOrder + 1];    // set-up: quantisation units; Gamma_k units ug[k] .. ug[k+1]
  int ua, ub, uc1;                 // K1
  int um, uc2;                     // K2
  int ur, uc3;                     // K3
  int us;                          // K5
  int ugn, ures;                   // K6
};

struct alignas(16) GrpTable {
  unsigned seq;                    // doorbell: the step number once the table below is complete
  unsigned consumed;               // written by the device once it has taken the table
  long long spin;                  // wait bound of this step's doorbell (clock cycles)
  int nslots;
  int pad;
  int uoff[kKernels][kGrpMaxSlots + 1];
  GrpSlot slot[kGrpMaxSlots];
};

struct GrpCtl {                    // mapped host memory written by the device
  unsigned timeout[kRing];         // timeout[k % kRing] = k when the doorbell of step k gave up
};

__device__ __forceinline__ unsigned ld_acquire_sys(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(unsigned* p, unsigned v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Largest s < ns with uoff[s] <= u (uoff[ns] > u): the slot of unit u.
__device__ __forceinline__ int find_slot(const int* uoff, int ns, int u) {
  int lo = 0, hi = ns;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (uoff[mid] <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ float x_at(const GrpSlot& d, int64_t i) {
  return d.mode == TRALS_MODE_BF16 ? __bfloat162float(d.Xq[i]) : d.X[i];
}

// ------------------------------------------------------------------ K0
__global__ void grp_doorbell_kernel(GrpTable* h0, GrpTable* h1, GrpTable* dtab, unsigned* dseq, GrpCtl* ctl) {
  __shared__ int ok;
  const unsigned want = *dseq + 1;
  GrpTable* h = (want & 1) ? h1 : h0;
  if (threadIdx.x == 0) {
    const long long limit = *reinterpret_cast<volatile long long*>(&h->spin);
    const long long t0 = clock64();
    int good = 0;
    for (;;) {
      if (ld_acquire_sys(&h->seq) == want) {
        good = 1;
        break;
      }
      if (clock64() - t0 > limit) break;
      __nanosleep(256);
    }
    ok = good;
  }
  __syncthreads();
  if (ok) {
    __threadfence_system();
    const int ns = *reinterpret_cast<volatile int*>(&h->nslots);
    const size_t bytes = offsetof(GrpTable, slot) + (size_t)ns * sizeof(GrpSlot);
    const volatile uint4* src = reinterpret_cast<const volatile uint4*>(h);
    uint4* dst = reinterpret_cast<uint4*>(dtab);
    for (size_t w = threadIdx.x; w < bytes / 16; w += blockDim.x) {
      uint4 v;
      v.x = src[w].x;
      v.y = src[w].y;
      v.z = src[w].z;
      v.w = src[w].w;
      dst[w] = v;
    }
  } else if (threadIdx.x == 0) {
    dtab->nslots = 0;
    for (int k = 0; k < kKernels; ++k) dtab->uoff[k][0] = 0;
    reinterpret_cast<volatile unsigned*>(ctl->timeout)[want % kRing] = want;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_system();
    st_release_sys(&h->consumed, want);
    *dseq = want;
  }
}

// ------------------------------------------------------------------ FP64 entry units
// FP64 work (Gamma entries, Gamma-chain products) goes in units of kE entries, four threads per entry
// over interleaved quarters of the inner index, combined in a fixed order: the FP64 pipe of an SM is
// narrow, so units are kept small and spread over many SMs.
struct EntrySmem {
  double red[4][kE];
};

// The quarter sums of this thread's entry (t & 63, quarter t >> 6) -> the entry's sum on quarter 0.
__device__ __forceinline__ double combine4(double v, EntrySmem& sm) {
  const int e = threadIdx.x & (kE - 1), q = threadIdx.x >> 6;
  sm.red[q][e] = v;
  __syncthreads();
  double r = 0.0;
  if (q == 0) r = ((sm.red[0][e] + sm.red[1][e]) + sm.red[2][e]) + sm.red[3][e];
  __syncthreads();
  return r;
}

// Gamma entries of core k: Gamma[(p R + q) + R^2 (s R' + t)] = sum_i G[p,i,s] G[q,i,t].
__device__ void gamma_unit(const GrpSlot& d, int k, int lu, EntrySmem& sm) {
  const int N = d.N, Rk = d.R[k], Rk1 = d.R[(k + 1) % N];
  const int rows = Rk * Rk, total = rows * Rk1 * Rk1;
  const int e = lu * kE + (threadIdx.x & (kE - 1)), quarter = threadIdx.x >> 6;
  double acc = 0.0;
  if (e < total) {
    const int row = e % rows, col = e / rows;
    const int p = row / Rk, q = row % Rk, s = col / Rk1, t = col % Rk1;
    const int64_t Ik = d.I[k];
    const double* gu = d.cores[k] + p + (int64_t)Rk * Ik * s;
    const double* gv = d.cores[k] + q + (int64_t)Rk * Ik * t;
    for (int64_t i = quarter; i < Ik; i += 4) acc = fma(gu[Rk * i], gv[Rk * i], acc);
  }
  const double v = combine4(acc, sm);
  if (quarter == 0 && e < total) d.gam[k][e] = v;
}

// Product k (1-based) of the Gamma chain Gamma_{n+1} ... Gamma_{n-1}: P_k = P_{k-1} Gamma_{n+k+1}
// (P_0 = Gamma_{n+1}); the last (k = N - 2) is stored as the regrouped S_n,
// S[(a + R_n b) + r (a' + R_n b')] = Pi[(b R_{n+1} + b') + R_{n+1}^2 (a R_n + a')].
__device__ void chain_unit(const GrpSlot& d, int k, int lu, EntrySmem& sm) {
  const int N = d.N, n = d.n;
  const int c1 = (n + 1) % N, ck = (n + k + 1) % N, cn = (ck + 1) % N;
  const int rows = d.R[c1] * d.R[c1], inner = d.R[ck] * d.R[ck], cols = d.R[cn] * d.R[cn];
  const int e = lu * kE + (threadIdx.x & (kE - 1)), quarter = threadIdx.x >> 6;
  const int row = e % rows, col = e / rows;
  double acc = 0.0;
  if (e < rows * cols) {
    const double* A = (k == 1) ? d.gam[c1] : d.chainbuf[(k - 2) & 1];
    const double* B = d.gam[ck];
    for (int t = quarter; t < inner; t += 4) acc = fma(A[row + rows * t], B[t + inner * col], acc);
  }
  const double v = combine4(acc, sm);
  if (quarter != 0 || e >= rows * cols) return;
  if (k < N - 2) {
    d.chainbuf[(k - 1) & 1][e] = v;
  } else {
    const int Rn = d.R[n], Rn1 = d.R[c1], r = Rn * Rn1;
    const int b = row / Rn1, b2 = row % Rn1, a = col / Rn, a2 = col % Rn;
    d.S[(a + Rn * b) + r * (a2 + Rn * b2)] = v;
  }
}

// ------------------------------------------------------------------ pieces of K1
// Row `row` of the subchain product G_{c_t0}(i) G_{c_t0+1}(i) ... over the modes chain[t0 .. t1-1] at
// index j (first mode fastest), in FP32, into v; returns the memory offset of the index in X.
__device__ __forceinline__ int64_t chain_row(const GrpSlot& d, int t0, int t1, int64_t j, int row, float* v) {
  const int N = d.N;
  float w[kGrpMaxRank];
  int k = d.chain[t0];
  int64_t i = j % d.I[k];
  j /= d.I[k];
  int64_t off = i * d.str[k];
  {
    const int Rc = d.R[(k + 1) % N];
    const double* G = d.cores[k] + row + (int64_t)d.R[k] * i;
    const int64_t cs = (int64_t)d.R[k] * d.I[k];
#pragma unroll
    for (int s = 0; s < kGrpMaxRank; ++s) v[s] = s < Rc ? (float)G[cs * s] : 0.0f;
  }
  for (int t = t0 + 1; t < t1; ++t) {
    k = d.chain[t];
    i = j % d.I[k];
    j /= d.I[k];
    off += i * d.str[k];
    const int Rk = d.R[k], Rk1 = d.R[(k + 1) % N];
    const double* G = d.cores[k] + (int64_t)Rk * i;
    const int64_t cs = (int64_t)Rk * d.I[k];
#pragma unroll
    for (int y = 0; y < kGrpMaxRank; ++y) {
      float acc = 0.0f;
      if (y < Rk1) {
#pragma unroll
        for (int x = 0; x < kGrpMaxRank; ++x)
          if (x < Rk) acc = fmaf(v[x], (float)G[x + cs * y], acc);
      }
      w[y] = acc;
    }
#pragma unroll
    for (int y = 0; y < kGrpMaxRank; ++y) v[y] = w[y];
  }
  return off;
}

__device__ void table_a_unit(const GrpSlot& d, int lu) {
  const int Rb = d.R[d.chain[0]];
  const int64_t e = (int64_t)lu * kThreads + threadIdx.x;
  if (e >= d.KA * Rb) return;
  const int b = (int)(e % Rb);
  const int64_t jA = e / Rb;
  float v[kGrpMaxRank];
  const int64_t off = chain_row(d, 0, d.nA, jA, b, v);
  float* out = d.Atab + jA * (int64_t)(Rb * d.Ra) + b;
#pragma unroll
  for (int c = 0; c < kGrpMaxRank; ++c)
    if (c < d.Ra) out[Rb * c] = v[c];
  if (b == 0) d.offA[jA] = off;
}

__device__ void table_b_unit(const GrpSlot& d, int lu) {
  const int Ra = d.Ra, Rn = d.R[d.n];
  const int64_t e = (int64_t)lu * kThreads + threadIdx.x;
  if (e >= d.KB * Ra) return;
  const int c = (int)(e % Ra);
  const int64_t jB = e / Ra;
  float v[kGrpMaxRank];
  const int64_t off = chain_row(d, d.nA, d.N - 1, jB, c, v);
  float* out = d.Btab + jB * (int64_t)(Ra * Rn) + c;
#pragma unroll
  for (int a = 0; a < kGrpMaxRank; ++a)
    if (a < Rn) out[Ra * a] = v[a];
  if (c == 0) d.offB[jB] = off;
}

__global__ void __launch_bounds__(kThreads) grp_prepare_kernel(const GrpTable* __restrict__ T) {
  __shared__ EntrySmem sm;
  const int ns = T->nslots;
  const int total = T->uoff[0][ns];
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int s = find_slot(T->uoff[0], ns, u);
    const GrpSlot& d = T->slot[s];
    int lu = u - T->uoff[0][s];
    if (d.st->code != 0) continue;
    if (d.phase == kInit) {
      if (lu < d.uq) {
        const int64_t e0 = (int64_t)lu * kQuantChunk, e1 = min(d.numel, e0 + kQuantChunk);
        for (int64_t e = e0 + threadIdx.x; e < e1; e += kThreads) d.Xq[e] = __float2bfloat16_rn(d.X[e]);
        continue;
      }
      lu -= d.uq;
      int k = 0;
      while (k + 1 < d.N && lu >= d.ug[k + 1]) ++k;
      gamma_unit(d, k, lu - d.ug[k], sm);
      continue;
    }
    if (lu < d.ua) {
      table_a_unit(d, lu);
      continue;
    }
    lu -= d.ua;
    if (lu < d.ub) {
      table_b_unit(d, lu);
      continue;
    }
    chain_unit(d, 1, lu - d.ub, sm);
  }
}

// ------------------------------------------------------------------ K2
// Stage 1, T[p][bc] = sum_{j_A} X(i_n, j_A, j_B) A(j_A)[bc] over a set of 64 "pairs" p, is a small GEMM
// per unit (64 pairs x 64 columns, K = j_A in tiles of 32); each thread keeps a 4 x 4 block of it in
// registers and reads its operands as 16-byte shared-memory vectors.  Stage 2 contracts T with B(j_B)
// over c.  The unit geometry follows the memory order of X, so that consecutive lanes load consecutive
// elements:
//   kLanesB (0 < n < N-1): B = modes 0 .. n-1, pairs = 64 consecutive j_B at one i_n, a range of j_A;
//   kLanesA (n = N-1): A starts with mode 0, the same pairs, and the tiles are loaded along j_A;
//   kLanesI (n = 0): pairs = 64 consecutive i_0 at one j_B, looping over a range of j_B whose stage-2
//      results each pair accumulates.
struct MttspSmem {
  union {
    struct {
      float Xs[32][kMP + 4];   // padded rows: stores along j_A spread over the banks
      float As[32][kR2];
    } t;
    float Bs[kMP][kR2 + 1];
  } u;
  float Ts[kMP][kR2 + 1];
  float red[4][kR2];
  float Brow[kR2];
  int64_t offA[kUnitA];
  EntrySmem e;
};

// Stage 1 over the j_A range [ja0, ja1) for 64 pairs with X offsets pbase[p] + offA[j_A] (lanes along
// pairs, or along j_A when along_a), accumulated into acc.  The offsets of each 512-value chunk of j_A are
// staged in shared memory, and the next tile's X and A values are loaded into registers while the
// current tile is multiplied.
__device__ __forceinline__ void stage1(const GrpSlot& d, MttspSmem& sm, int64_t ja0, int64_t ja1, int np,
                                       const int64_t* pbase, bool along_a, float (&acc)[4][4]) {
  const int RA2 = d.R[d.chain[0]] * d.Ra;
  const float* Atab = d.Atab;
  const int64_t* offA = d.offA;
  const bool bf = d.mode == TRALS_MODE_BF16;
  const float* X = d.X;
  const __nv_bfloat16* Xq = d.Xq;
  const int bg = threadIdx.x & 15, pg = threadIdx.x >> 4;
  for (int64_t c0 = ja0; c0 < ja1; c0 += kUnitA) {
    const int64_t c1 = min(ja1, c0 + kUnitA);
    for (int e = threadIdx.x; e < (int)(c1 - c0); e += kThreads) sm.offA[e] = offA[c0 + e];
    __syncthreads();
    float xr[8], ar[8];
    auto load = [&](int64_t j0) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = threadIdx.x + kThreads * q;
        const int p = along_a ? (e >> 5) : (e & (kMP - 1));
        const int jj = along_a ? (e & 31) : (e >> 6);
        float x = 0.0f;
        if (p < np && j0 + jj < c1) {
          const int64_t at = pbase[p] + sm.offA[j0 - c0 + jj];
          x = bf ? __bfloat162float(Xq[at]) : X[at];
        }
        xr[q] = x;
        const int ja = e >> 6, bc = e & 63;
        ar[q] = (j0 + ja < c1 && bc < RA2) ? Atab[(j0 + ja) * RA2 + bc] : 0.0f;
      }
    };
    load(c0);
    for (int64_t j0 = c0; j0 < c1; j0 += 32) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = threadIdx.x + kThreads * q;
        const int p = along_a ? (e >> 5) : (e & (kMP - 1));
        const int jj = along_a ? (e & 31) : (e >> 6);
        sm.u.t.Xs[jj][p] = xr[q];
        sm.u.t.As[e >> 6][e & 63] = ar[q];
      }
      __syncthreads();
      if (j0 + 32 < c1) load(j0 + 32);
#pragma unroll 4
      for (int jj = 0; jj < 32; ++jj) {
        const float4 x = *reinterpret_cast<const float4*>(&sm.u.t.Xs[jj][4 * pg]);
        const float4 a = *reinterpret_cast<const float4*>(&sm.u.t.As[jj][4 * bg]);
        const float xv[4] = {x.x, x.y, x.z, x.w}, av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], av[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
}

__device__ void mttsp_unit(const GrpSlot& d, int lu, MttspSmem& sm, int64_t* pbase) {
  const int N = d.N, n = d.n;
  const int Rb = d.R[(n + 1) % N], Ra = d.Ra, Rn = d.R[n];
  const int RB2 = Ra * Rn, r = Rn * Rb;
  const int bg = threadIdx.x & 15, pg = threadIdx.x >> 4;
  const int col = threadIdx.x & 63, quarter = threadIdx.x >> 6;
  float acc[4][4];
  if (d.cls != kLanesI) {
    const int per = d.nchB * d.nchA;
    const int in = lu / per, rem = lu % per, chB = rem / d.nchA, chA = rem % d.nchA;
    const int64_t jB0 = (int64_t)chB * kMP;
    const int np = (int)min((int64_t)kMP, d.KB - jB0);
    const int64_t ja0 = (int64_t)chA * kUnitA, ja1 = min(d.KA, ja0 + kUnitA);
    if (threadIdx.x < kMP) pbase[threadIdx.x] = threadIdx.x < np ? in * d.str[n] + d.offB[jB0 + threadIdx.x] : 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    __syncthreads();
    stage1(d, sm, ja0, ja1, np, pbase, d.cls == kLanesA, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) sm.Ts[4 * pg + i][4 * bg + j] = acc[i][j];
    for (int e = threadIdx.x; e < kMP * kR2; e += kThreads) {
      const int pp = e >> 6, x = e & 63;
      sm.u.Bs[pp][x] = (pp < np && x < RB2) ? d.Btab[(jB0 + pp) * RB2 + x] : 0.0f;
    }
    __syncthreads();
    float sum = 0.0f;
    if (col < r) {
      const int a = col % Rn, b = col / Rn;
      const int p1 = min(np, 16 * quarter + 16);
      for (int pp = 16 * quarter; pp < p1; ++pp)
        for (int c = 0; c < Ra; ++c) sum = fmaf(sm.Ts[pp][b + Rb * c], sm.u.Bs[pp][c + Ra * a], sum);
    }
    sm.red[quarter][col] = sum;
    __syncthreads();
    if (threadIdx.x < r)
      d.part[(((int64_t)in * d.nchB + chB) * d.nchA + chA) * r + threadIdx.x] =
          ((sm.red[0][threadIdx.x] + sm.red[1][threadIdx.x]) + sm.red[2][threadIdx.x]) + sm.red[3][threadIdx.x];
    __syncthreads();
    return;
  }
  // kLanesI: 64 consecutive i_0, the j_B range of chunk chB
  const int blk = lu / d.nchB, chB = lu % d.nchB;
  const int64_t i0 = (int64_t)blk * kMP;
  const int np = (int)min((int64_t)kMP, d.I[0] - i0);
  const int64_t jb0 = (int64_t)chB * d.cB, jb1 = min(d.KB, jb0 + d.cB);
  float out[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) out[k] = 0.0f;
  const int a = col % Rn, b = col / Rn;
  for (int64_t jB = jb0; jB < jb1; ++jB) {
    if (threadIdx.x < kMP) pbase[threadIdx.x] = i0 + threadIdx.x + d.offB[jB];
    if (threadIdx.x < kR2) sm.Brow[threadIdx.x] = threadIdx.x < RB2 ? d.Btab[jB * RB2 + threadIdx.x] : 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    __syncthreads();
    stage1(d, sm, 0, d.KA, np, pbase, false, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) sm.Ts[4 * pg + i][4 * bg + j] = acc[i][j];
    __syncthreads();
    if (col < r) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        float v = out[k];
        for (int c = 0; c < Ra; ++c) v = fmaf(sm.Ts[16 * quarter + k][b + Rb * c], sm.Brow[c + Ra * a], v);
        out[k] = v;
      }
    }
    __syncthreads();
  }
  if (col < r) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int p = 16 * quarter + k;
      if (p < np) d.part[((i0 + p) * d.nchB + chB) * r + col] = out[k];
    }
  }
}

__global__ void __launch_bounds__(kThreads, 2) grp_mttsp_kernel(const GrpTable* __restrict__ T) {
  __shared__ __align__(16) MttspSmem sm;
  __shared__ int64_t pbase[kMP];
  const int ns = T->nslots;
  const int total = T->uoff[1][ns];
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int s = find_slot(T->uoff[1], ns, u);
    const GrpSlot& d = T->slot[s];
    const int lu = u - T->uoff[1][s];
    if (d.st->code != 0) continue;
    if (lu < d.um) mttsp_unit(d, lu, sm, pbase);
    else chain_unit(d, 2, lu - d.um, sm.e);
  }
}

// ------------------------------------------------------------------ K3
__global__ void __launch_bounds__(kThreads) grp_reduce_kernel(const GrpTable* __restrict__ T) {
  __shared__ EntrySmem sm;
  const int ns = T->nslots;
  const int total = T->uoff[2][ns];
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int s = find_slot(T->uoff[2], ns, u);
    const GrpSlot& d = T->slot[s];
    const int lu = u - T->uoff[2][s];
    if (d.st->code != 0) continue;
    if (lu < d.ur) {
      const int N = d.N, n = d.n, r = d.R[n] * d.R[(n + 1) % N];
      const int In = (int)d.I[n];
      const int e = lu * kThreads + threadIdx.x;
      if (e < In * r) {
        const int i = e % In, col = e / In;
        const int nch = d.nchB * d.nchA;
        const float* src = d.part + (int64_t)i * nch * r + col;
        double sum = 0.0;
        for (int ch = 0; ch < nch; ++ch) sum += (double)src[(int64_t)ch * r];
        d.M[e] = sum;
      }
    } else {
      chain_unit(d, 3, lu - d.ur, sm);
    }
  }
}

// ------------------------------------------------------------------ K4
// Right-looking Cholesky in shared memory.  Per column j: the pivot (thread 0), then, from the unscaled
// column, L(i, j) = A(i, j) y_j written out and the trailing update A(i, k) -= A(i, j) A(k, j) y_j^2 for
// j < k <= i, on a 16 x 16 thread grid.
__global__ void __launch_bounds__(kThreads) grp_chol_kernel(const GrpTable* __restrict__ T) {
  __shared__ double A[kR2 * kR2];
  __shared__ double ys[kR2];
  __shared__ int bad;
  const int s = blockIdx.x;
  if (s >= T->nslots) return;
  const GrpSlot& d = T->slot[s];
  if (d.phase != kUpdate || d.st->code != 0) return;
  const int N = d.N, n = d.n, r = d.R[n] * d.R[(n + 1) % N];
  const int tid = threadIdx.x, ti = tid & 15, tk = tid >> 4;
  double* L = d.L;
  for (int e = tid; e < r * r; e += kThreads) {
    A[e] = d.S[e];
    L[e] = 0.0;
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (tid == 0) {
      const double dj = A[j + r * j];
      if (dj > 0.0 && isfinite(dj)) {
        const double y = rsqrt(dj);
        ys[j] = y;
        L[j + r * j] = dj * y;
      } else {
        bad = 1;
        set_status(d.st, isfinite(dj) ? TRALS_E_NOT_SPD : TRALS_E_NONFINITE, d.sweep, n, j, dj);
      }
    }
    __syncthreads();
    if (bad) break;
    const double y = ys[j], y2 = y * y;
    for (int i = j + 1 + tid; i < r; i += kThreads) L[i + r * j] = A[i + r * j] * y;
    for (int k = j + 1 + tk; k < r; k += 16) {
      const double akj = A[k + r * j] * y2;
      for (int i = k + ti; i < r; i += 16) A[i + r * k] = fma(-A[i + r * j], akj, A[i + r * k]);
    }
    __syncthreads();
  }
  if (bad) return;
  for (int j = tid; j < r; j += kThreads) L[r * r + j] = ys[j];
}

// ------------------------------------------------------------------ K5
// Row g of G_{n(2)} from S_n g^T = m^T: L w = m (forward), then L^T g = w (backward), with the
// reciprocal pivots; a unit solves two rows (warps 0 and 1; lane l holds entries l and l + 32) after
// the whole CTA has staged L.
__global__ void __launch_bounds__(kThreads) grp_solve_kernel(const GrpTable* __restrict__ T) {
  __shared__ double Ls[kLd * kR2];
  __shared__ double ys[kR2];
  const int ns = T->nslots;
  const int total = T->uoff[3][ns];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int s = find_slot(T->uoff[3], ns, u);
    const GrpSlot& d = T->slot[s];
    const int lu = u - T->uoff[3][s];
    if (d.st->code != 0) continue;
    const int N = d.N, n = d.n, Rn = d.R[n], r = Rn * d.R[(n + 1) % N];
    const int In = (int)d.I[n];
    for (int e = threadIdx.x; e < r * r; e += kThreads) Ls[(e % r) + kLd * (e / r)] = d.L[e];
    for (int j = threadIdx.x; j < r; j += kThreads) ys[j] = d.L[r * r + j];
    __syncthreads();
    const int row = lu * kSolveRows + warp;
    if (warp < kSolveRows && row < In) {
      double t0 = lane < r ? d.M[row + (int64_t)In * lane] : 0.0;
      double t1 = lane + 32 < r ? d.M[row + (int64_t)In * (lane + 32)] : 0.0;
      for (int k = 0; k < r; ++k) {
        const double wk = __shfl_sync(0xffffffffu, k < 32 ? t0 : t1, k & 31) * ys[k];
        if (lane == (k & 31)) {
          if (k < 32) t0 = wk;
          else t1 = wk;
        }
        if (lane > k) t0 = fma(-Ls[lane + kLd * k], wk, t0);
        if (lane + 32 > k && lane + 32 < r) t1 = fma(-Ls[lane + 32 + kLd * k], wk, t1);
      }
      for (int k = r - 1; k >= 0; --k) {
        const double gk = __shfl_sync(0xffffffffu, k < 32 ? t0 : t1, k & 31) * ys[k];
        if (lane == (k & 31)) {
          if (k < 32) t0 = gk;
          else t1 = gk;
        }
        if (lane < k) t0 = fma(-Ls[k + kLd * lane], gk, t0);
        if (lane + 32 < k) t1 = fma(-Ls[k + kLd * (lane + 32)], gk, t1);
      }
      double* G = d.cores[n];
      if (lane < r) G[(lane % Rn) + (int64_t)Rn * (row + (int64_t)In * (lane / Rn))] = t0;
      if (lane + 32 < r) G[((lane + 32) % Rn) + (int64_t)Rn * (row + (int64_t)In * ((lane + 32) / Rn))] = t1;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ K6
struct ResSmem {
  float Cs[kMP][kR2 + 1];
  float As[32][kR2 + 1];
  double red[2][kThreads];
  EntrySmem e;
};

// Explicit residual (n = N-1, so A starts with mode 0) over the unit's pairs and j_A range:
// X_hat(i_n, j_A, j_B) = sum_{b,c} A(j_A)[b, c] C[c, b] with C = B(j_B) G_n(i_n), lanes along j_A; the
// unit's (|X - X_hat|^2, |X|^2) go to rpart, and the last unit of the slot to finish adds all units in
// order.
__device__ void residual_unit(const GrpSlot& d, int lu, ResSmem& sm) {
  const int N = d.N, n = d.n;
  const int per = d.nchB * d.nchA;
  const int in = lu / per, rem = lu % per, chB = rem / d.nchA, chA = rem % d.nchA;
  const int64_t jB0 = (int64_t)chB * kMP;
  const int np = (int)min((int64_t)kMP, d.KB - jB0);
  const int64_t ja0 = (int64_t)chA * kUnitA, ja1 = min(d.KA, ja0 + kUnitA);
  const int Rb = d.R[(n + 1) % N], Ra = d.Ra, Rn = d.R[n];
  const int RA2 = Rb * Ra, RB2 = Ra * Rn;
  const int64_t In = d.I[n];
  const double* G = d.cores[n];
  for (int e = threadIdx.x; e < kMP * kR2; e += kThreads) {
    const int pp = e >> 6, x = e & 63;
    float v = 0.0f;
    if (pp < np && x < RA2) {
      const int b = x % Rb, c = x / Rb;
      const float* Brow = d.Btab + (jB0 + pp) * RB2 + c;
      for (int a = 0; a < Rn; ++a) v = fmaf(Brow[Ra * a], (float)G[a + (int64_t)Rn * (in + In * b)], v);
    }
    sm.Cs[pp][x] = v;
  }
  const int jj = threadIdx.x & 31, pb = threadIdx.x >> 5;
  double sse = 0.0, sxx = 0.0;
  for (int64_t j0 = ja0; j0 < ja1; j0 += 32) {
    for (int e = threadIdx.x; e < 32 * kR2; e += kThreads) {
      const int r0 = e >> 6, x = e & 63;
      sm.As[r0][x] = (j0 + r0 < ja1 && x < RA2) ? d.Atab[(j0 + r0) * RA2 + x] : 0.0f;
    }
    __syncthreads();
    if (j0 + jj < ja1) {
      const int64_t oa = in * d.str[n] + d.offA[j0 + jj];
      for (int p = pb; p < np; p += 8) {
        float xh = 0.0f;
        for (int x = 0; x < RA2; ++x) xh = fmaf(sm.As[jj][x], sm.Cs[p][x], xh);
        const float xv = d.X[oa + d.offB[jB0 + p]];
        const double df = (double)xv - (double)xh;
        sse = fma(df, df, sse);
        sxx = fma((double)xv, (double)xv, sxx);
      }
    }
    __syncthreads();
  }
  sm.red[0][threadIdx.x] = sse;
  sm.red[1][threadIdx.x] = sxx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int t = 0; t < kThreads; ++t) {
      a += sm.red[0][t];
      b += sm.red[1][t];
    }
    d.rpart[2 * lu] = a;
    d.rpart[2 * lu + 1] = b;
    __threadfence();
    const unsigned ticket = atomicAdd(d.rctr, 1u);
    if (ticket == (unsigned)d.ures - 1) {
      __threadfence();
      double sa = 0.0, sb = 0.0;
      const volatile double* rp = d.rpart;
      for (int w = 0; w < d.ures; ++w) {
        sa += rp[2 * w];
        sb += rp[2 * w + 1];
      }
      *d.res = sqrt(fmax(sa, 0.0) / sb);
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) grp_finish_kernel(const GrpTable* __restrict__ T) {
  __shared__ ResSmem sm;
  const int ns = T->nslots;
  const int total = T->uoff[4][ns];
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int s = find_slot(T->uoff[4], ns, u);
    const GrpSlot& d = T->slot[s];
    const int lu = u - T->uoff[4][s];
    if (d.st->code != 0) continue;
    if (lu < d.ugn) gamma_unit(d, d.n, lu, sm.e);
    else residual_unit(d, lu - d.ugn, sm);
  }
}

int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Host view of one slot.
struct HostSlot {
  int state = 0;                   // 0 free, 1 active, 2 draining, 3 done
  int N = 0, mode = 0, sweeps = 0;
  int64_t I[kGrpMaxOrder] = {};
  int32_t R[kGrpMaxOrder] = {};
  int64_t numel = 0;
  int idx = 0;                     // next step of the request: 0 set-up, 1 .. N * sweeps updates
  void* ws = nullptr;
  GrpSlot base{};                  // static fields and pointers
  struct Mode {
    int nA, Ra, cls, nchB, nchA, cB, units;
    int64_t KA, KB;
  } md[kGrpMaxOrder] = {};
  size_t core_elems = 0;
  double* h_cores = nullptr;       // pinned: initial cores in, fitted cores out
  size_t h_cap = 0;
  double* h_misc = nullptr;        // pinned: DevStatus (4 doubles) then the residual
  cudaEvent_t done = nullptr;
  unsigned seq_first = 0, seq_last = 0;
  bool timed_out = false;
};

// MTTSP geometry of mode n: the split of the chain n+1, ..., n-1 into A (first nA modes) and B, and the
// unit grid.  Middle modes split at mode 0 (B = modes 0 .. n-1, contiguous in X); the first and last
// modes take the split with the smaller larger table.
void choose_split(int N, const int64_t* I, const int32_t* R, int n, HostSlot::Mode& m) {
  auto sizes = [&](int nA, int64_t& KA, int64_t& KB) {
    KA = 1;
    KB = 1;
    for (int t = 0; t < N - 1; ++t) (t < nA ? KA : KB) *= I[(n + 1 + t) % N];
  };
  if (n >= 1 && n <= N - 2) {
    m.cls = kLanesB;
    m.nA = N - 1 - n;
    sizes(m.nA, m.KA, m.KB);
  } else {
    m.cls = n == 0 ? kLanesI : kLanesA;
    int64_t best = -1;
    for (int nA = 1; nA <= N - 2; ++nA) {
      int64_t KA, KB;
      sizes(nA, KA, KB);
      if (best < 0 || std::max(KA, KB) < best) {
        best = std::max(KA, KB);
        m.nA = nA;
        m.KA = KA;
        m.KB = KB;
      }
    }
  }
  m.Ra = R[(n + 1 + m.nA) % N];
  if (m.cls == kLanesI) {
    // about 16 tiles of 32 j_A per unit
    m.cB = std::max(1, 16 / cdiv(m.KA, 32));
    m.nchB = cdiv(m.KB, m.cB);
    m.nchA = 1;
    m.units = cdiv(I[0], kMP) * m.nchB;
  } else {
    m.cB = 0;
    m.nchB = cdiv(m.KB, kMP);
    m.nchA = cdiv(m.KA, kUnitA);
    m.units = (int)(I[n] * m.nchB * m.nchA);
  }
}

// Workspace carve-up (byte offsets), shared by the footprint count and the admission.
struct Carve {
  size_t xq, xcopy, cores, gam, atab, btab, offa, offb, part, chain, S, L, M, rpart, misc, total;
};

Carve carve(int N, const int64_t* I, const int32_t* R, int mode, bool x_on_host) {
  int64_t numel = 1;
  for (int k = 0; k < N; ++k) numel *= I[k];
  size_t cores = 0, gam = 0, atab = 0, btab = 0, offa = 0, offb = 0, part = 0, M = 0, rmax = 0, rpart = 0;
  size_t r2max = 0;
  for (int k = 0; k < N; ++k) {
    const size_t Rk = R[k], Rk1 = R[(k + 1) % N];
    cores += Rk * I[k] * Rk1;
    gam += Rk * Rk * Rk1 * Rk1;
    r2max = std::max(r2max, Rk * Rk);
    HostSlot::Mode m;
    choose_split(N, I, R, k, m);
    atab = std::max(atab, (size_t)m.KA * Rk1 * m.Ra);
    btab = std::max(btab, (size_t)m.KB * m.Ra * Rk);
    offa = std::max(offa, (size_t)m.KA);
    offb = std::max(offb, (size_t)m.KB);
    part = std::max(part, (size_t)(m.cls == kLanesI ? I[0] * m.nchB : I[k] * m.nchB * m.nchA) * Rk * Rk1);
    M = std::max(M, (size_t)I[k] * Rk * Rk1);
    rmax = std::max(rmax, Rk * Rk1);
    if (k == N - 1) rpart = (size_t)m.units;
  }
  Carve c{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += al256(bytes);
    return at;
  };
  c.xq = take(mode == TRALS_MODE_BF16 ? (size_t)numel * 2 : 0);
  c.xcopy = take(x_on_host ? (size_t)numel * 4 : 0);
  c.cores = take(cores * 8);
  c.gam = take(gam * 8);
  c.atab = take(atab * 4);
  c.btab = take(btab * 4);
  c.offa = take(offa * 8);
  c.offb = take(offb * 8);
  c.part = take(part * 4);
  c.chain = take(2 * r2max * r2max * 8);
  c.S = take(rmax * rmax * 8);
  c.L = take((rmax * rmax + rmax) * 8);
  c.M = take(M * 8);
  c.rpart = take(rpart * 2 * 8);
  c.misc = take(64);
  c.total = o;
  return c;
}

}  // namespace

struct GroupEngine {
  int device = 0;
  int nsm = 152;
  cudaStream_t stream = nullptr;
  GrpTable* htab[2] = {nullptr, nullptr};   // pinned, mapped
  GrpTable* htab_dev[2] = {nullptr, nullptr};
  GrpCtl* ctl = nullptr;
  GrpCtl* ctl_dev = nullptr;
  GrpTable* dtab = nullptr;
  unsigned* dseq = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // kernel nodes whose grids follow the step's work (K1, K2, K3, K4, K5, K6), their functions, and the
  // one argument they all take (the device table), held here so that a node update never points into
  // storage the graph owns
  cudaGraphNode_t knode[6] = {};
  const void* kfunc[6] = {};
  const GrpTable* karg = nullptr;
  void* kargv[1] = {nullptr};
  unsigned kgrid[6] = {};
  cudaEvent_t step_ev[4] = {};
  unsigned seq = 0;                 // last step launched
  unsigned done_seq = 0;            // last step seen complete
  std::vector<HostSlot> slots;
  std::vector<unsigned> timeouts;   // steps whose doorbell gave up, not yet matched to slots
  int withhold = 0;
  long long withhold_spin = 0;
};

bool grp_eligible(int N, const int64_t* I, const int32_t* R, int xt, const trals_opts& o, int sweeps,
                  int64_t max_elems) {
  if (N < 3 || N > kGrpMaxOrder || xt != TRALS_X_F32 || sweeps < 1 || max_elems <= 0) return false;
  if (o.mode != TRALS_MODE_FP32 && o.mode != TRALS_MODE_BF16) return false;
  if (o.solver != TRALS_SOLVE_CHOL || o.gram != TRALS_GRAM_STRUCTURED || o.explicit_residual) return false;
  int64_t numel = 1;
  for (int k = 0; k < N; ++k) {
    if (R[k] < 1 || R[k] > kGrpMaxRank || I[k] < 1) return false;
    numel *= I[k];
    if (numel > max_elems) return false;
  }
  return numel <= (int64_t)1 << 30;
}

size_t grp_footprint(int N, const int64_t* I, const int32_t* R, int mode, bool x_on_host) {
  return carve(N, I, R, mode, x_on_host).total;
}

GroupEngine* grp_create(int device, std::string* err) {
  GroupEngine* e = new GroupEngine();
  e->device = device;
  e->slots.resize(kGrpMaxSlots);
  auto fail = [&](const char* what, cudaError_t c) -> GroupEngine* {
    if (err) *err = std::string("grouped engine: ") + what + ": " + cudaGetErrorString(c);
    grp_destroy(e);
    return nullptr;
  };
  cudaError_t c = cudaSetDevice(device);
  if (c != cudaSuccess) return fail("device", c);
  cudaDeviceGetAttribute(&e->nsm, cudaDevAttrMultiProcessorCount, device);
  // the highest priority: a step's CTAs are dispatched ahead of the queued CTAs of the plans' kernels
  // (the large requests' tensor-core MTTSPs fill every SM), so small requests keep a short step time
  int prio_low = 0, prio_high = 0;
  cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  if ((c = cudaStreamCreateWithPriority(&e->stream, cudaStreamNonBlocking, prio_high)) != cudaSuccess)
    return fail("stream", c);
  for (int b = 0; b < 2; ++b) {
    if ((c = cudaHostAlloc(reinterpret_cast<void**>(&e->htab[b]), sizeof(GrpTable), cudaHostAllocMapped)) != cudaSuccess)
      return fail("pinned table", c);
    std::memset(e->htab[b], 0, sizeof(GrpTable));
    if ((c = cudaHostGetDevicePointer(reinterpret_cast<void**>(&e->htab_dev[b]), e->htab[b], 0)) != cudaSuccess)
      return fail("mapped table", c);
  }
  if ((c = cudaHostAlloc(reinterpret_cast<void**>(&e->ctl), sizeof(GrpCtl), cudaHostAllocMapped)) != cudaSuccess)
    return fail("pinned control block", c);
  std::memset(e->ctl, 0, sizeof(GrpCtl));
  if ((c = cudaHostGetDevicePointer(reinterpret_cast<void**>(&e->ctl_dev), e->ctl, 0)) != cudaSuccess)
    return fail("mapped control block", c);
  if ((c = cudaMalloc(&e->dtab, sizeof(GrpTable))) != cudaSuccess) return fail("device table", c);
  if ((c = cudaMalloc(&e->dseq, sizeof(unsigned))) != cudaSuccess) return fail("step counter", c);
  if ((c = cudaMemsetAsync(e->dtab, 0, sizeof(GrpTable), e->stream)) != cudaSuccess ||
      (c = cudaMemsetAsync(e->dseq, 0, sizeof(unsigned), e->stream)) != cudaSuccess)
    return fail("device table init", c);
  for (int k = 0; k < 4; ++k)
    if ((c = cudaEventCreateWithFlags(&e->step_ev[k], cudaEventDisableTiming)) != cudaSuccess) return fail("event", c);
  // pinned result buffers sized for the usual requests up front: allocating (and freeing) pinned memory
  // while the device is busy stalls the worker
  constexpr size_t kCoresCap = (size_t)1 << 16;
  for (HostSlot& h : e->slots) {
    if ((c = cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming)) != cudaSuccess ||
        (c = cudaHostAlloc(reinterpret_cast<void**>(&h.h_misc), 64, cudaHostAllocDefault)) != cudaSuccess ||
        (c = cudaHostAlloc(reinterpret_cast<void**>(&h.h_cores), kCoresCap * sizeof(double), cudaHostAllocDefault)) !=
            cudaSuccess)
      return fail("slot buffers", c);
    h.h_cap = kCoresCap;
  }
  // the step graph
  cudaGraph_t g = nullptr;
  const int grid = 2 * e->nsm;
  if ((c = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return fail("capture", c);
  grp_doorbell_kernel<<<1, kThreads, 0, e->stream>>>(e->htab_dev[0], e->htab_dev[1], e->dtab, e->dseq, e->ctl_dev);
  grp_prepare_kernel<<<grid, kThreads, 0, e->stream>>>(e->dtab);
  grp_mttsp_kernel<<<grid, kThreads, 0, e->stream>>>(e->dtab);
  grp_reduce_kernel<<<grid, kThreads, 0, e->stream>>>(e->dtab);
  grp_chol_kernel<<<kGrpMaxSlots, kThreads, 0, e->stream>>>(e->dtab);
  grp_solve_kernel<<<grid, kThreads, 0, e->stream>>>(e->dtab);
  grp_finish_kernel<<<grid, kThreads, 0, e->stream>>>(e->dtab);
  c = cudaStreamEndCapture(e->stream, &g);
  if (c != cudaSuccess) return fail("capture", c);
  e->graph = g;
  c = cudaGraphInstantiate(&e->exec, g, 0);
  if (c != cudaSuccess) return fail("graph", c);
  {
    const void* funcs[6] = {reinterpret_cast<const void*>(grp_prepare_kernel),
                            reinterpret_cast<const void*>(grp_mttsp_kernel),
                            reinterpret_cast<const void*>(grp_reduce_kernel),
                            reinterpret_cast<const void*>(grp_chol_kernel),
                            reinterpret_cast<const void*>(grp_solve_kernel),
                            reinterpret_cast<const void*>(grp_finish_kernel)};
    size_t count = 0;
    cudaGraphGetNodes(g, nullptr, &count);
    std::vector<cudaGraphNode_t> nodes(count);
    cudaGraphGetNodes(g, nodes.data(), &count);
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
      cudaKernelNodeParams kp{};
      if ((c = cudaGraphKernelNodeGetParams(nd, &kp)) != cudaSuccess) return fail("graph nodes", c);
      for (int k = 0; k < 6; ++k)
        if (kp.func == funcs[k]) {
          e->knode[k] = nd;
          e->kfunc[k] = funcs[k];
          e->kgrid[k] = kp.gridDim.x;
        }
    }
    for (int k = 0; k < 6; ++k)
      if (!e->knode[k]) return fail("graph nodes", cudaErrorInvalidValue);
    e->karg = e->dtab;
    e->kargv[0] = &e->karg;
  }
  if ((c = cudaStreamSynchronize(e->stream)) != cudaSuccess) return fail("init", c);
  return e;
}

void grp_destroy(GroupEngine* e) {
  if (!e) return;
  if (e->stream) cudaStreamSynchronize(e->stream);
  for (HostSlot& h : e->slots) {
    if (h.ws) cudaFree(h.ws);
    if (h.done) cudaEventDestroy(h.done);
    if (h.h_cores) cudaFreeHost(h.h_cores);
    if (h.h_misc) cudaFreeHost(h.h_misc);
  }
  for (int k = 0; k < 4; ++k)
    if (e->step_ev[k]) cudaEventDestroy(e->step_ev[k]);
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  if (e->dtab) cudaFree(e->dtab);
  if (e->dseq) cudaFree(e->dseq);
  for (int b = 0; b < 2; ++b)
    if (e->htab[b]) cudaFreeHost(e->htab[b]);
  if (e->ctl) cudaFreeHost(e->ctl);
  if (e->stream) cudaStreamDestroy(e->stream);
  delete e;
}

uint64_t grp_steps(const GroupEngine* e) { return e->seq; }

int grp_free_slots(const GroupEngine* e) {
  int f = 0;
  for (const HostSlot& h : e->slots) f += h.state == 0;
  return f;
}

bool grp_busy(const GroupEngine* e) {
  for (const HostSlot& h : e->slots)
    if (h.state == 1 || h.state == 2) return true;
  return false;
}

int grp_admit(GroupEngine* e, int N, const int64_t* I, const int32_t* R, const float* X, bool x_on_host, int mode,
              int sweeps, const double* const* init_cores, std::string* err) {
  int id = -1;
  for (int k = 0; k < (int)e->slots.size(); ++k)
    if (e->slots[k].state == 0) {
      id = k;
      break;
    }
  if (id < 0) {
    if (err) *err = "grouped engine: no free slot";
    return -1;
  }
  HostSlot& h = e->slots[id];
  h.N = N;
  h.mode = mode;
  h.sweeps = sweeps;
  h.numel = 1;
  for (int k = 0; k < N; ++k) {
    h.I[k] = I[k];
    h.R[k] = R[k];
    h.numel *= I[k];
  }
  h.idx = 0;
  h.timed_out = false;
  h.seq_first = h.seq_last = 0;
  h.core_elems = 0;
  for (int k = 0; k < N; ++k) h.core_elems += (size_t)R[k] * I[k] * R[(k + 1) % N];
  const Carve cv = carve(N, I, R, mode, x_on_host);
  auto cuda_fail = [&](const char* what, cudaError_t c) {
    if (err) *err = std::string("grouped engine: ") + what + ": " + cudaGetErrorString(c);
    return -1;
  };
  cudaError_t c;
  if (h.h_cap < h.core_elems) {
    if (h.h_cores) cudaFreeHost(h.h_cores);
    h.h_cores = nullptr;
    h.h_cap = 0;
    const size_t cap = std::max<size_t>(h.core_elems, 4096);
    if ((c = cudaHostAlloc(reinterpret_cast<void**>(&h.h_cores), cap * sizeof(double), cudaHostAllocDefault)) != cudaSuccess)
      return cuda_fail("pinned cores", c);
    h.h_cap = cap;
  }
  if ((c = cudaMallocAsync(&h.ws, cv.total, e->stream)) != cudaSuccess) {
    h.ws = nullptr;
    return cuda_fail("workspace", c);
  }
  char* w = static_cast<char*>(h.ws);
  GrpSlot& b = h.base;
  std::memset(&b, 0, sizeof b);
  b.N = N;
  b.mode = mode;
  b.numel = h.numel;
  int64_t st = 1;
  for (int k = 0; k < N; ++k) {
    b.I[k] = I[k];
    b.R[k] = R[k];
    b.str[k] = st;
    st *= I[k];
  }
  b.X = x_on_host ? reinterpret_cast<const float*>(w + cv.xcopy) : X;
  b.Xq = mode == TRALS_MODE_BF16 ? reinterpret_cast<__nv_bfloat16*>(w + cv.xq) : nullptr;
  size_t co = 0, go = 0;
  for (int k = 0; k < N; ++k) {
    b.cores[k] = reinterpret_cast<double*>(w + cv.cores) + co;
    b.gam[k] = reinterpret_cast<double*>(w + cv.gam) + go;
    co += (size_t)R[k] * I[k] * R[(k + 1) % N];
    go += (size_t)R[k] * R[k] * R[(k + 1) % N] * R[(k + 1) % N];
  }
  b.Atab = reinterpret_cast<float*>(w + cv.atab);
  b.Btab = reinterpret_cast<float*>(w + cv.btab);
  b.offA = reinterpret_cast<int64_t*>(w + cv.offa);
  b.offB = reinterpret_cast<int64_t*>(w + cv.offb);
  b.part = reinterpret_cast<float*>(w + cv.part);
  size_t r2max = 0;
  for (int k = 0; k < N; ++k) r2max = std::max(r2max, (size_t)R[k] * R[k]);
  b.chainbuf[0] = reinterpret_cast<double*>(w + cv.chain);
  b.chainbuf[1] = b.chainbuf[0] + r2max * r2max;
  b.S = reinterpret_cast<double*>(w + cv.S);
  b.L = reinterpret_cast<double*>(w + cv.L);
  b.M = reinterpret_cast<double*>(w + cv.M);
  b.rpart = reinterpret_cast<double*>(w + cv.rpart);
  b.st = reinterpret_cast<DevStatus*>(w + cv.misc);
  b.rctr = reinterpret_cast<unsigned*>(w + cv.misc + 32);
  b.res = reinterpret_cast<double*>(w + cv.misc + 40);
  for (int k = 0; k < N; ++k) choose_split(N, I, R, k, h.md[k]);
  // initial cores through the pinned buffer, X from the host, the status word, counter and result zeroed
  size_t off = 0;
  for (int k = 0; k < N; ++k) {
    const size_t cnt = (size_t)R[k] * I[k] * R[(k + 1) % N];
    std::memcpy(h.h_cores + off, init_cores[k], cnt * sizeof(double));
    off += cnt;
  }
  if ((c = cudaMemcpyAsync(w + cv.cores, h.h_cores, h.core_elems * sizeof(double), cudaMemcpyHostToDevice,
                           e->stream)) != cudaSuccess)
    return cuda_fail("initial cores", c);
  if (x_on_host &&
      (c = cudaMemcpyAsync(w + cv.xcopy, X, (size_t)h.numel * 4, cudaMemcpyHostToDevice, e->stream)) != cudaSuccess)
    return cuda_fail("copy of X", c);
  if ((c = cudaMemsetAsync(w + cv.misc, 0, 64, e->stream)) != cudaSuccess) return cuda_fail("status word", c);
  h.state = 1;
  return id;
}

namespace {

// Note the steps that completed: a step whose doorbell gave up fails the requests it carried.
void note_completed(GroupEngine* e, bool wait_all) {
  while (e->done_seq < e->seq) {
    const unsigned k = e->done_seq + 1;
    cudaEvent_t ev = e->step_ev[k % 4];
    if (wait_all) cudaEventSynchronize(ev);
    else if (cudaEventQuery(ev) != cudaSuccess) break;
    e->done_seq = k;
    if (reinterpret_cast<volatile unsigned*>(e->ctl->timeout)[k % kRing] == k) {
      for (HostSlot& h : e->slots)
        if ((h.state == 1 || h.state == 2) && h.seq_first != 0 && h.seq_first <= k && k <= h.seq_last)
          h.timed_out = true;
    }
  }
}

}  // namespace

bool grp_step(GroupEngine* e, std::string* err) {
  note_completed(e, false);
  if (e->seq - e->done_seq >= 2) return false;   // two steps in flight
  std::vector<int> act;
  for (int k = 0; k < (int)e->slots.size(); ++k)
    if (e->slots[k].state == 1) act.push_back(k);
  if (act.empty()) return false;
  const unsigned seq = e->seq + 1;
  GrpTable* T = e->htab[seq & 1];
  // the device took this buffer's previous table (two steps back, seen complete above)
  if (seq > 2 && __atomic_load_n(&T->consumed, __ATOMIC_ACQUIRE) != seq - 2) {
    if (err) *err = "grouped engine: descriptor buffer still in use";
    return false;
  }
  const int ns = (int)act.size();
  T->nslots = ns;
  for (int k = 0; k < kKernels; ++k) T->uoff[k][0] = 0;
  for (int s = 0; s < ns; ++s) {
    HostSlot& h = e->slots[act[s]];
    GrpSlot d = h.base;
    const int N = h.N;
    if (h.idx == 0) {
      d.phase = kInit;
      d.uq = h.mode == TRALS_MODE_BF16 ? cdiv(h.numel, kQuantChunk) : 0;
      d.ug[0] = 0;
      for (int k = 0; k < N; ++k) {
        const int64_t Rk = h.R[k], Rk1 = h.R[(k + 1) % N];
        d.ug[k + 1] = d.ug[k] + cdiv(Rk * Rk * Rk1 * Rk1, kE);
      }
      T->uoff[0][s + 1] = T->uoff[0][s] + d.uq + d.ug[N];
      for (int k = 1; k < kKernels; ++k) T->uoff[k][s + 1] = T->uoff[k][s];
    } else {
      const int u = h.idx - 1, n = u % N;
      d.phase = kUpdate;
      d.n = n;
      d.sweep = u / N;
      d.fin = h.idx == N * h.sweeps;
      const HostSlot::Mode& m = h.md[n];
      d.nA = m.nA;
      d.Ra = m.Ra;
      d.KA = m.KA;
      d.KB = m.KB;
      d.cls = m.cls;
      d.nchB = m.nchB;
      d.nchA = m.nchA;
      d.cB = m.cB;
      for (int t = 0; t < N - 1; ++t) d.chain[t] = (n + 1 + t) % N;
      const int64_t Rn = h.R[n], Rn1 = h.R[(n + 1) % N], r = Rn * Rn1;
      auto prod_units = [&](int k) -> int {   // units of chain product k (0 if the chain is shorter)
        if (k > N - 2) return 0;
        const int64_t rows = Rn1 * Rn1, ck = h.R[(n + k + 2) % N];
        return cdiv(rows * ck * ck, kE);
      };
      d.ua = cdiv(m.KA * Rn1, kThreads);
      d.ub = cdiv(m.KB * m.Ra, kThreads);
      d.uc1 = prod_units(1);
      d.um = m.units;
      d.uc2 = prod_units(2);
      d.ur = cdiv(h.I[n] * r, kThreads);
      d.uc3 = prod_units(3);
      d.us = cdiv(h.I[n], kSolveRows);
      d.ugn = cdiv(r * r, kE);
      d.ures = d.fin ? d.um : 0;
      T->uoff[0][s + 1] = T->uoff[0][s] + d.ua + d.ub + d.uc1;
      T->uoff[1][s + 1] = T->uoff[1][s] + d.um + d.uc2;
      T->uoff[2][s + 1] = T->uoff[2][s] + d.ur + d.uc3;
      T->uoff[3][s + 1] = T->uoff[3][s] + d.us;
      T->uoff[4][s + 1] = T->uoff[4][s] + d.ugn + d.ures;
    }
    T->slot[s] = d;
  }
  // grids sized to the step's units (at most two CTAs per SM): CTAs without work would still have to be
  // placed on SMs, which the large requests' kernels may hold for a while
  {
    const unsigned want[6] = {(unsigned)T->uoff[0][ns], (unsigned)T->uoff[1][ns], (unsigned)T->uoff[2][ns],
                              (unsigned)ns, (unsigned)T->uoff[3][ns], (unsigned)T->uoff[4][ns]};
    for (int k = 0; k < 6; ++k) {
      const unsigned g = std::max(1u, std::min(want[k], (unsigned)(k == 3 ? kGrpMaxSlots : 2 * e->nsm)));
      if (g == e->kgrid[k]) continue;
      cudaKernelNodeParams kp{};
      kp.func = const_cast<void*>(e->kfunc[k]);
      kp.gridDim = dim3(g, 1, 1);
      kp.blockDim = dim3(kThreads, 1, 1);
      kp.sharedMemBytes = 0;
      kp.kernelParams = e->kargv;
      kp.extra = nullptr;
      const cudaError_t c = cudaGraphExecKernelNodeSetParams(e->exec, e->knode[k], &kp);
      if (c != cudaSuccess) {
        if (err) *err = std::string("grouped engine: step grid: ") + cudaGetErrorString(c);
        return false;
      }
      e->kgrid[k] = g;
    }
  }
  const bool withheld = e->withhold > 0;
  T->spin = withheld ? e->withhold_spin : kDefaultSpin;
  if (withheld) --e->withhold;
  else __atomic_store_n(&T->seq, seq, __ATOMIC_RELEASE);
  cudaError_t c = cudaGraphLaunch(e->exec, e->stream);
  if (c == cudaSuccess) c = cudaEventRecord(e->step_ev[seq % 4], e->stream);
  if (c != cudaSuccess) {
    if (err) *err = std::string("grouped engine: step launch: ") + cudaGetErrorString(c);
    return false;
  }
  e->seq = seq;
  for (int id : act) {
    HostSlot& h = e->slots[id];
    if (h.seq_first == 0) h.seq_first = seq;
    h.seq_last = seq;
    ++h.idx;
    if (h.idx > h.N * h.sweeps) {
      // last update done in this step: results to the pinned buffers, then the slot drains
      cudaMemcpyAsync(h.h_cores, h.base.cores[0], h.core_elems * sizeof(double), cudaMemcpyDeviceToHost, e->stream);
      cudaMemcpyAsync(h.h_misc, h.base.st, 48, cudaMemcpyDeviceToHost, e->stream);
      cudaEventRecord(h.done, e->stream);
      h.state = 2;
    }
  }
  return true;
}

void grp_poll(GroupEngine* e, std::vector<int>* done) {
  std::vector<int> ready;
  for (int k = 0; k < (int)e->slots.size(); ++k)
    if (e->slots[k].state == 2 && cudaEventQuery(e->slots[k].done) == cudaSuccess) ready.push_back(k);
  note_completed(e, !ready.empty());
  for (int k : ready) {
    e->slots[k].state = 3;
    done->push_back(k);
  }
}

int grp_result(GroupEngine* e, int slot, const double** cores, double* rel_res, std::string* msg) {
  HostSlot& h = e->slots[slot];
  *cores = h.h_cores;
  *rel_res = h.h_misc[5];
  if (h.timed_out) {
    if (msg) *msg = "grouped step: the wait for the step's descriptor table gave up";
    return TRALS_E_TIMEOUT;
  }
  const int code = status_code(h.h_misc);
  if (code != TRALS_OK && msg) *msg = status_message(h.h_misc);
  return code;
}

void grp_release(GroupEngine* e, int slot) {
  HostSlot& h = e->slots[slot];
  if (h.ws) cudaFreeAsync(h.ws, e->stream);
  h.ws = nullptr;
  h.state = 0;
}

void grp_withhold(GroupEngine* e, int steps, long long spin_cycles) {
  e->withhold = steps;
  e->withhold_spin = spin_cycles > 0 ? spin_cycles : kDefaultSpin;
}

}  // namespace trals
