// Tensor-core MTTSP (Alg. 2 lines 7-8) for the BF16 mode on sm_103a: tcgen05.mma with TMEM
// accumulators, operands staged by TMA (cp.async.bulk.tensor) into 128B-swizzled shared memory.
//
// The contraction M_n[i_n, a + R_n b] = sum_k X_[n][i_n, k] G^{!=n}(k)[b, a] runs in two stages so
// that X is streamed from HBM exactly once and G^{!=n} is never formed:
//   stage 1 (tensor cores):  T[row, w] = sum_{s in S} X(row, s) Tab[w, s]
//       S is a block of modes that is contiguous both in memory and in the subchain order
//       (eq. subchain_new); Tab(s) is the product of the cores of S (a table rebuilt per update),
//       a "row" fixes i_n and every mode outside S.
//   stage 2 (CUDA cores):    M[i_n(row), :] += F(row) applied to T[row, :]
//       where F(row) is the product of the remaining cores (one small matrix per row, from a
//       second table), on one side of T only (the other side is the identity).
// Three tile geometries (chosen per mode on the host):
//   KM-L : S = modes 0..n-1 (K-major X), F = G_{n+1}...G_N on the left   (n < N-1)
//   KM-R : S = modes 0..s,    (K-major X), F = G_{s+1}...G_{N-1} on the right (n = N-1)
//   MM   : S = modes n+1..m  (MN-major X), F = G_{m+1}...G_N G_1...G_{n-1} on the right
//   MM-L : n = 0, S = modes m..N-1 (MN-major X), F = G_1...G_{m-1} on the left; a tile is 128
//          consecutive elements of X in memory, (i_0, i_1 .. i_{m-1}), so every TMA row is one aligned
//          pair of 128-byte lines even when I_0 < 64; the row -> i_0 map then changes from tile to tile,
//          so each unit's rows are combined into a shared-memory I_0 x r accumulator in a fixed order
// Rows of a tile map to distinct (i_n, factor) pairs; stage 2 reduces rows with equal i_n in a
// fixed order into a per-CTA FP32 accumulator; CTA partials are summed in FP64 by a second kernel.
#include <cuda.h>

#include <algorithm>
#include <cstdio>

#include "mttsp_tc.cuh"

namespace trals {

namespace {

constexpr int kRows = 128;                    // MMA M (TMEM lanes)
constexpr int kKT = 64;                       // K elements per stage (one 128-byte swizzle row of BF16)
constexpr int kNSMax = 8;                     // pipeline stages (upper bound; the host picks what fits)
constexpr int kThreads = 192;                 // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int kABytes = kRows * 128;          // X tile: 128 rows x 128 B
constexpr int kAtomBytes = 64 * 128;          // MN-major atom: 64 K rows x 128 B (64 MN elements)
constexpr int kMaxW = 128;                    // stage-1 table width (MMA N) limit
constexpr int kSmemBudget = 227 * 1024;
constexpr long long kSpinLimit = 4000000000LL;  // ~2 s at 2 GHz: the default bound of every wait

enum { KM_L = 0, KM_R = 1, MM = 2, MM_L = 3 };

struct TcArgs {
  int variant;
  int ksteps;
  int64_t n_tiles;   // KM: row tiles (each ksteps K steps)
  int whole;         // split the work at tile boundaries only (shares of several tiles)
  int In;
  int nrep;          // KM: factor values per tile
  int64_t n_fac;     // KM: factor entries along the tiled mode (K_post or K_mid)
  int64_t P, K_pre, K_hi, pchunks;   // MM
  int64_t opairs;                    // MM: ceil(K_hi / 2) o-pairs per p-chunk
  int NX, NY, Sy, Rn, r, W_pad, fs_stride, ms_stride, ns;
  int fac_shared;    // KM-L, KM-R, MM-L: the factor blocks of a tile are staged once (double buffered);
                     // MM: one block per row
  int nslot;         // factor blocks per tile (KM: nrep; MM-L: distinct i_1.. values in 128 elements)
  int64_t Pp;        // MM-L: elements per K row (I_0 ... I_{m-1})
  int ksync;         // K-synchronous work split (see get_unit)
  long long spin_limit;   // bound of every mbarrier wait, in clock cycles
  int withhold;      // fault injection for tests: the producer skips its first copy (see tc_set_fault)
  uint32_t tx_bytes;
  uint32_t idesc;
  int x3;            // split-BF16 planes: 0 none; 1 bf16x2, the table as hi/lo (two products per K step);
                     // 2 bf16x3, X and the table as hi/lo (three products)
  const float* F;    // [fac][NX][SYP]
  float* partials;   // [grid][In * r]
  DevStatus* status;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the limit passes or another role raised the abort flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) return false;
  }
}

// TMA tile loads with an L2 cache policy: X is read once per launch (evict first), the stage-1 table
// by every tile (evict last), so the stream of X does not push the table out of L2.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%3, "
      "%4}], [%2], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "l"(policy)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%3, "
      "%4, %5}], [%2], %6;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, 128-byte swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;          // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;          // SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ void raise_timeout(DevStatus* st, int where) {
  if (st != nullptr && atomicCAS(&st->code, 0, (int)TRALS_E_TIMEOUT) == 0) {
    st->sweep = -1;
    st->mode = -2;
    st->index = where;
    st->value = 0.0;
  }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Work split: a CTA owns one contiguous, equal share of the K steps of all its tiles (tile-major), so
// every CTA streams the same amount of X; the share is cut at tile boundaries into units, the j-th
// being (tile, K steps [ks0, ks1)).  When the shares span several tiles (a.whole) they are rounded to
// whole tiles instead: each unit costs an epilogue, and splitting would add one per CTA.  Every unit's contribution is additive, so a tile may be split
// between CTAs anywhere in K.  K-major tiles are shared by the whole grid; MN-major tiles pin CTA c
// to p-chunk pc = c % pchunks (each lane keeps its rows, hence its i_n, for the whole launch) and the
// CTAs of a p-chunk share that chunk's o-pairs.  Producer, MMA issuer and epilogue call this alike.
__device__ __forceinline__ bool get_unit(const TcArgs& a, int64_t j, int64_t& tile, int64_t& op, int64_t& pc,
                                         int& ks0, int& ks1) {
  if (a.ksync) {
    // K-synchronous split (grid = n_tiles x groups): CTA c takes tile c % n_tiles and the (c / n_tiles)-th
    // K range of it, one unit per CTA, so the CTAs of all tiles walk the same K rows of X together and
    // jointly read whole DRAM rows (each tile holds only a 256-byte piece of a K row)
    if (j > 0) return false;
    const int64_t T = a.n_tiles, groups = gridDim.x / T, g = blockIdx.x / T;
    tile = blockIdx.x % T;
    op = 0;
    pc = 0;
    ks0 = (int)(g * a.ksteps / groups);
    ks1 = (int)((g + 1) * a.ksteps / groups);
    return ks0 < ks1;
  }
  int64_t ntile, g, G;
  if (a.variant != MM) {
    ntile = a.n_tiles;
    g = blockIdx.x;
    G = gridDim.x;
    pc = 0;
  } else {
    pc = blockIdx.x % a.pchunks;
    g = blockIdx.x / a.pchunks;
    G = (gridDim.x - pc + a.pchunks - 1) / a.pchunks;   // CTAs sharing this p-chunk
    ntile = a.opairs;
  }
  if (a.whole) {   // contiguous whole tiles: no tile is split, so every unit carries a full K range
    const int64_t t = g * ntile / G + j;
    if (t >= (g + 1) * ntile / G) return false;
    ks0 = 0;
    ks1 = a.ksteps;
    tile = (a.variant != MM) ? t : 0;
    op = (a.variant != MM) ? 0 : t;
    return true;
  }
  const int64_t W = ntile * a.ksteps;
  const int64_t s0 = g * W / G, s1 = (g + 1) * W / G;   // this CTA's K steps
  const int64_t t = s0 / a.ksteps + j;
  const int64_t ts = t * a.ksteps;
  if (s0 >= s1 || ts >= s1) return false;
  ks0 = (int)(max(s0, ts) - ts);
  ks1 = (int)(min(s1, ts + a.ksteps) - ts);
  tile = (a.variant != MM) ? t : 0;
  op = (a.variant != MM) ? 0 : t;
  return true;
}

// SYP: the stage-2 dot length (inner subchain rank padded to a multiple of 4); the stage-1 result of a
// row is T[y * SYP + z] (y < NY, z < SYP) and is held in registers.  SPLIT: the split-BF16 modes
// (a.x3 != 0), compiled apart so that the plain BF16 kernel carries none of their code.
template <int SYP, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    mttsp_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmT,
                    const __grid_constant__ CUtensorMap tmXl, const __grid_constant__ CUtensorMap tmTl, const TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int bBytes = ((a.W_pad * 128) + 1023) & ~1023;
  const int planes = SPLIT ? 2 : 1;                // stage: X hi [, X lo], table hi [, table lo]
  // (bf16x2 leaves the X lo slot of its stages unused)
  const int stageBytes = planes * (kABytes + bBytes);
  const int NS = a.ns;
  // stage-2 factor blocks: per row (MM), or the blocks of a tile, double buffered
  float* F_s = reinterpret_cast<float*>(base + NS * stageBytes);
  const int fs_rows = a.fac_shared ? 2 * a.nslot : kRows;
  // MM-L: one x-column of every row's stage-2 result (rows 128, stride NY | 1), and the CTA's I_0 x r sums
  float* U_s = F_s + ((fs_rows * a.fs_stride + 1) & ~1);
  const int us = a.NY | 1;
  float* Macc = U_s + (a.variant == MM_L ? ((kRows * us + 1) & ~1) : 0);
  uint64_t* bars = reinterpret_cast<uint64_t*>(Macc + (a.variant == MM_L ? ((a.In * a.ms_stride + 1) & ~1) : 0));
  uint64_t* full = bars;
  uint64_t* empty = bars + kNSMax;
  uint64_t* accf = bars + 2 * kNSMax;
  uint64_t* acce = bars + 2 * kNSMax + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * kNSMax + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  volatile int* epi_stop = reinterpret_cast<volatile int*>(tmem_holder + 2);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int E = a.In * a.r;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 128);
    }
    *abort_flag = 0;
    epi_stop[0] = 0;
    epi_stop[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_holder))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued[kNSMax] = {};
      const uint64_t pol_x = policy_evict_first(), pol_tab = policy_evict_last();
      int64_t tile, op, pc;
      int ks0, ks1;
      for (int64_t j = 0; get_unit(a, j, tile, op, pc, ks0, ks1) && !*abort_flag; ++j) {
        for (int ks = ks0; ks < ks1; ++ks) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.spin_limit)) {
            *abort_flag = 1;
            raise_timeout(a.status, 1);
            break;
          }
          // fault injection (tests only): the first copy of the CTA's first unit is never issued, so the
          // MMA issuer's wait for it runs out and the kernel reports TRALS_E_TIMEOUT
          if (!(a.withhold && j == 0 && ks == ks0)) {
            uint8_t* A = base + stage * stageBytes;
            uint8_t* B = A + planes * kABytes;
            mbar_expect_tx(&full[stage], a.tx_bytes);
            const int k0 = ks * kKT;
            for (int pl = 0; pl < planes; ++pl) {
              const CUtensorMap* mx = pl ? &tmXl : &tmX;
              if (SPLIT && pl == 1 && a.x3 == 1) {   // bf16x2: the table's lo plane only
                tma_load_2d(B + bBytes, &tmTl, &full[stage], k0, 0, pol_tab);
                continue;
              }
              uint8_t* Ap = A + pl * kABytes;
              if (a.variant == KM_L) {
                tma_load_3d(Ap, mx, &full[stage], k0, 0, (int)(tile * a.nrep), pol_x);
              } else if (a.variant == KM_R) {
                tma_load_3d(Ap, mx, &full[stage], k0, (int)(tile * a.nrep), 0, pol_x);
              } else if (a.variant == MM_L) {
                for (int at = 0; at < 2; ++at)
                  tma_load_2d(Ap + at * kAtomBytes, mx, &full[stage], (int)(tile * kRows + 64 * at), k0, pol_x);
              } else {
                for (int at = 0; at < 2; ++at)
                  tma_load_3d(Ap + at * kAtomBytes, mx, &full[stage], (int)(pc * 64), k0, (int)(2 * op + at), pol_x);
              }
              tma_load_2d(B + pl * bBytes, pl ? &tmTl : &tmT, &full[stage], k0, 0, pol_tab);
            }
            ++issued[stage];
          }
          if (++stage == NS) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (*abort_flag) {
        // Do not leave copies in flight into this CTA's shared memory: wait (bounded) for the last
        // load issued into every stage.
        volatile int never = 0;
        for (int st = 0; st < NS; ++st)
          if (issued[st] > 0) mbar_wait(&full[st], (uint32_t)((issued[st] - 1) & 1), &never, kSpinLimit);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int64_t tile, op, pc;
      int ks0, ks1;
      for (int64_t j = 0; get_unit(a, j, tile, op, pc, ks0, ks1) && !*abort_flag; ++j) {
        const int buf = (int)(j & 1);
        if (!mbar_wait(&acce[buf], (uint32_t)(((j >> 1) & 1) ^ 1), abort_flag, a.spin_limit)) {
          *abort_flag = 1;
          raise_timeout(a.status, 2);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * 128);
        bool ok = true;
        for (int ks = ks0; ks < ks1; ++ks) {
          if (!mbar_wait(&full[stage], phase, abort_flag, a.spin_limit)) {
            *abort_flag = 1;
            raise_timeout(a.status, 3);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t A = smem_u32(base + stage * stageBytes);
          const uint32_t B = A + (uint32_t)(planes * kABytes);
#pragma unroll
          for (int jj = 0; jj < kKT / 16; ++jj) {
            const bool mn = a.variant == MM || a.variant == MM_L;
            const uint64_t ad = mn ? sdesc(A + 2048u * jj, kAtomBytes, 1024) : sdesc(A + 32u * jj, 16, 1024);
            const uint64_t bd = sdesc(B + 32u * jj, 16, 1024);
            umma_bf16(d, ad, bd, a.idesc, (ks > ks0 || jj > 0) ? 1u : 0u);
            if (SPLIT) {
              // split-BF16 products: X_hi T_lo (bf16x2, bf16x3) + X_lo T_hi (bf16x3); X_lo T_lo is below
              // FP32 rounding
              const uint64_t bdl = sdesc(B + (uint32_t)bBytes + 32u * jj, 16, 1024);
              umma_bf16(d, ad, bdl, a.idesc, 1u);
              if (a.x3 == 2) {
                const uint32_t Al = A + (uint32_t)kABytes;
                const uint64_t adl = mn ? sdesc(Al + 2048u * jj, kAtomBytes, 1024) : sdesc(Al + 32u * jj, 16, 1024);
                umma_bf16(d, adl, bd, a.idesc, 1u);
              }
            }
          }
          umma_commit(&empty[stage]);
          if (++stage == NS) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(&accf[buf]);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (stage 2)
    const int q = warp & 3;            // TMEM lane quarter of this warp
    const int row = 32 * q + lane;
    const int fblk = a.NX * SYP;       // floats per factor block
    float* myF = F_s + row * a.fs_stride;   // MM; the shared blocks are picked per unit below
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    const uint32_t vacc = lane_base + 256u;   // this lane's running V[x][y] at column 256 + 16 x + y
    // Fixed row geometry: the i_n of this lane never changes (see get_unit).
    bool lane_ok;
    int my_i, rep = 0;
    int64_t k_pre = 0;
    int at = 0;
    if (a.variant == KM_L || a.variant == MM_L) {
      rep = row / a.In;
      my_i = row % a.In;
      lane_ok = rep < a.nrep;
    } else if (a.variant == KM_R) {
      rep = row % a.nrep;
      my_i = row / a.nrep;
      lane_ok = my_i < a.In;
    } else {
      at = row / 64;
      const int64_t pc0 = blockIdx.x % a.pchunks;
      const int64_t p = pc0 * 64 + (row % 64);
      lane_ok = p < a.P;
      my_i = lane_ok ? (int)(p / a.K_pre) : 0;
      k_pre = p % a.K_pre;
    }
    const bool accum_rows = a.variant == MM_L;   // per-unit row combine instead of per-lane running sums
    if (accum_rows) {
      for (int e = row; e < a.In * a.ms_stride; e += kRows) Macc[e] = 0.0f;
    } else {
      uint32_t z[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = 0u;
      for (int x = 0; x < a.NX; ++x) tmem_st16(vacc + 16u * x, z);
      tmem_wait_st();
    }
    int64_t tile, op, pc;
    int ks0, ks1;
    for (int64_t j = 0; get_unit(a, j, tile, op, pc, ks0, ks1); ++j) {
      const int buf = (int)(j & 1);
      bool valid;
      int64_t fi;
      int slot = rep;
      bool copier = my_i == 0;
      if (a.variant == MM) {
        const int64_t o = 2 * op + at;
        valid = lane_ok && o < a.K_hi;
        fi = o + a.K_hi * k_pre;
      } else if (accum_rows) {
        const int64_t e = tile * kRows + row;
        valid = e < a.Pp;
        my_i = (int)(e % a.In);
        fi = e / a.In;
        slot = (int)(fi - (tile * kRows) / a.In);
        copier = row == 0 || my_i == 0;
      } else {
        fi = tile * a.nrep + rep;
        valid = lane_ok && fi < a.n_fac;
      }
      // prefetch the factor blocks into shared memory while the MMAs run: each row its own (MM), or
      // the first row of each repetition its repetition's block into the buffer of this unit's parity
      if (a.fac_shared) {
        myF = F_s + (2 * slot + (int)(j & 1)) * a.fs_stride;
        if (valid && copier) {
          const float* src = a.F + (size_t)fi * fblk;
          for (int c = 0; c < fblk; c += 4) cp_async16(myF + c, src + c);
        }
      } else if (valid) {
        const float* src = a.F + (size_t)fi * fblk;
        for (int c = 0; c < fblk; c += 4) cp_async16(myF + c, src + c);
      }
      cp_async_commit();
      const bool got = mbar_wait(&accf[buf], (uint32_t)((j >> 1) & 1), abort_flag, a.spin_limit);
      if (!got) {
        *abort_flag = 1;
        epi_stop[j & 1] = 1;
        raise_timeout(a.status, 4);
      }
      // Uniform decision: slot (j & 1) is written only before this unit's barrier and read right after
      // it; the next write to the same slot comes two units later, after every thread has passed the
      // following unit's barrier, i.e. after every thread has read this slot.
      epi_bar();
      if (epi_stop[j & 1]) {
        cp_async_wait_all();
        break;
      }
      tc_fence_after();
      // this row's stage-1 result: TMEM -> registers
      float T[128];
      const uint32_t taddr = lane_base + (uint32_t)(buf * 128);
#pragma unroll
      for (int c0 = 0; c0 < 128; c0 += 32) {
        if (c0 < a.W_pad) {
          uint32_t v[32];
          tmem_ld32(taddr + (uint32_t)c0, v);
          tmem_wait_ld();
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) T[c0 + jj] = __uint_as_float(v[jj]);
        }
      }
      tc_fence_before();
      mbar_arrive(&acce[buf]);
      cp_async_wait_all();
      if (a.fac_shared) epi_bar();   // the copying row's block is visible to the other rows
      // stage 2: V[x][y] += f_x . T[y]  (independent accumulators over y), kept per lane in TMEM
      constexpr int YMAX = (128 / SYP) < 16 ? (128 / SYP) : 16;
      for (int x = 0; x < a.NX; ++x) {
        float f[SYP];
#pragma unroll
        for (int jj = 0; jj < SYP / 4; ++jj) {
          float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
          if (valid) t = *reinterpret_cast<const float4*>(myF + x * SYP + 4 * jj);
          f[4 * jj] = t.x;
          f[4 * jj + 1] = t.y;
          f[4 * jj + 2] = t.z;
          f[4 * jj + 3] = t.w;
        }
        float acc[YMAX];
#pragma unroll
        for (int y = 0; y < YMAX; ++y) acc[y] = 0.0f;
        if (valid) {
#pragma unroll
          for (int z = 0; z < SYP; ++z) {
#pragma unroll
            for (int y = 0; y < YMAX; ++y) acc[y] = fmaf(f[z], T[y * SYP + z], acc[y]);
          }
        }
        if (accum_rows) {
          // this x-column of every row to shared memory, then each output (i_0, y) adds the rows of
          // its i_0 in ascending order into the CTA's sums
#pragma unroll
          for (int y = 0; y < YMAX; ++y)
            if (y < a.NY) U_s[row * us + y] = acc[y];
          epi_bar();
          const int base_i = (int)((tile * kRows) % a.In);
          const int64_t rows_left = a.Pp - tile * kRows;
          for (int o = row; o < a.In * a.NY; o += kRows) {
            const int i = o / a.NY, y = o - i * a.NY;
            float sum = 0.0f;
            for (int r = (i - base_i + a.In) % a.In; r < kRows && r < rows_left; r += a.In) sum += U_s[r * us + y];
            Macc[i * a.ms_stride + y + a.Rn * x] += sum;
          }
          epi_bar();
          continue;
        }
        uint32_t v[16];
        tmem_ld16(vacc + 16u * x, v);
        tmem_wait_ld();
#pragma unroll
        for (int y = 0; y < YMAX; ++y) v[y] = __float_as_uint(__uint_as_float(v[y]) + acc[y]);
        tmem_st16(vacc + 16u * x, v);
      }
      tmem_wait_st();
    }
    // Stage the lanes' running sums V[x][y] in the pipeline buffers, which are idle now (every MMA
    // and copy has been consumed).
    epi_bar();
    if (!accum_rows) {
    float* S = reinterpret_cast<float*>(base);
    const int nv = a.NX * a.NY, ss = nv | 1;
    float* myS = S + row * ss;
    for (int x = 0; x < a.NX; ++x) {
      uint32_t v[16];
      tmem_ld16(vacc + 16u * x, v);
      tmem_wait_ld();
#pragma unroll
      for (int y = 0; y < 16; ++y)
        if (y < a.NY) myS[x * a.NY + y] = lane_ok ? __uint_as_float(v[y]) : 0.0f;
    }
    }
  }
  // Combine: all warps (the producer and MMA warps are done) own outputs (i_n, x, y) and add the rows
  // of their i_n in a fixed order; then the CTA's partial (column-major I_n x r) goes out.
  __syncthreads();
  if (!*abort_flag && a.variant == MM_L) {
    // MM-L: the sums are already combined
    float* out = a.partials + (size_t)blockIdx.x * E;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
      const int i = e % a.In, c = e / a.In;
      out[e] = Macc[i * a.ms_stride + c];
    }
  } else if (!*abort_flag) {
    float* S = reinterpret_cast<float*>(base);
    const int nv = a.NX * a.NY, ss = nv | 1;
    int* colmap = reinterpret_cast<int*>(S + kRows * ss);   // xy -> column of M_s
    float* M_s = reinterpret_cast<float*>(colmap + ((nv + 3) & ~3));
    const bool left = a.variant == KM_L || a.variant == MM_L;
    for (int xy = threadIdx.x; xy < nv; xy += blockDim.x) {
      const int x = xy / a.NY, y = xy % a.NY;
      colmap[xy] = left ? (y + a.Rn * x) : (x + a.Rn * y);
    }
    for (int e = threadIdx.x; e < a.In * a.ms_stride; e += blockDim.x) M_s[e] = 0.0f;
    int64_t i_lo = 0, i_hi = a.In - 1, p0 = 0, p1 = 0;
    if (a.variant == MM) {
      p0 = (blockIdx.x % a.pchunks) * 64;
      p1 = min(a.P, p0 + 64);
      i_lo = p0 / a.K_pre;
      i_hi = (p1 - 1) / a.K_pre;
    }
    __syncthreads();
    const int cnt = (int)(i_hi - i_lo + 1) * nv;
    const int step = blockDim.x;
    int g = (int)threadIdx.x / nv, xy = (int)threadIdx.x % nv;
    const int dg = step / nv, dxy = step % nv;
    for (int o = threadIdx.x; o < cnt; o += step) {
      const int64_t i = i_lo + g;
      float sum = 0.0f;
      if (left) {
        for (int rp = 0; rp < a.nrep; ++rp) sum += S[(i + a.In * rp) * ss + xy];
      } else if (a.variant == KM_R) {
        for (int rp = 0; rp < a.nrep; ++rp) sum += S[(rp + a.nrep * i) * ss + xy];
      } else {
        const int r0 = (int)(max(p0, i * a.K_pre) - p0), r1 = (int)(min(p1, (i + 1) * a.K_pre) - p0);
        for (int at2 = 0; at2 < 2; ++at2)
          for (int rr = r0; rr < r1; ++rr) sum += S[(at2 * 64 + rr) * ss + xy];
      }
      M_s[i * a.ms_stride + colmap[xy]] = sum;
      g += dg;
      xy += dxy;
      if (xy >= nv) {
        xy -= nv;
        ++g;
      }
    }
    __syncthreads();
    float* out = a.partials + (size_t)blockIdx.x * E;
    int i = (int)threadIdx.x % a.In, c = (int)threadIdx.x / a.In;
    const int di = step % a.In, dc = step / a.In;
    for (int e = threadIdx.x; e < E; e += step) {
      out[e] = M_s[i * a.ms_stride + c];
      i += di;
      c += dc;
      if (i >= a.In) {
        i -= a.In;
        ++c;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

using TcKernel = void (*)(CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, TcArgs);

// The instantiation for a stage-2 dot length (4, 8, 12, 16) and split mode.
static TcKernel tc_kernel_for(int syp, bool split) {
  switch (syp) {
    case 4: return split ? mttsp_tc_kernel<4, true> : mttsp_tc_kernel<4, false>;
    case 8: return split ? mttsp_tc_kernel<8, true> : mttsp_tc_kernel<8, false>;
    case 12: return split ? mttsp_tc_kernel<12, true> : mttsp_tc_kernel<12, false>;
    default: return split ? mttsp_tc_kernel<16, true> : mttsp_tc_kernel<16, false>;
  }
}

// M[e] = sum_g partials[g * E + e] in FP64: a block takes 32 consecutive e; warp w sums g = w, w+8, ...
// (coalesced 128-byte rows), then the 8 warp sums are added in a fixed order.
// M[i + In_out c] = sum over CTAs of partials[g][i + In c] for i < In_out (In_out < In when the rows
// beyond In_out are the zero padding of a padded leading mode).
__global__ void tc_reduce_kernel(const float* __restrict__ partials, int G, int64_t E, int In, int In_out,
                                 double* __restrict__ M) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int64_t e = blockIdx.x * 32LL + lane;   // output index i + In_out c
  const int64_t Eout = E / In * In_out;
  const int64_t src = (e % In_out) + (int64_t)In * (e / In_out);
  double s = 0.0;
  if (e < Eout) {
    // four loads in flight per thread; the sums stay in ascending g
    const float* P = partials + src;
    int g = w;
    for (; g + 24 < G; g += 32) {
      const float v0 = P[(int64_t)g * E], v1 = P[(int64_t)(g + 8) * E], v2 = P[(int64_t)(g + 16) * E],
                  v3 = P[(int64_t)(g + 24) * E];
      s += (double)v0;
      s += (double)v1;
      s += (double)v2;
      s += (double)v3;
    }
    for (; g < G; g += 8) s += (double)P[(int64_t)g * E];
  }
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && e < Eout) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k][lane];
    M[e] = t;
  }
}

// The FP32 subchain tables below are stored entry-fastest ("structure of arrays"): element (x, y) of
// entry l sits at P[(x + Ra y) * count + l], so consecutive threads touch consecutive addresses.

// Stage-1 table: Tab[w * Kpad + k] = bf16(P_k(...)) with w = z + SYP y (z: inner/dot index, y: outer):
// kindL (factor on the left): P = c x a (Ra = Sy rows), element (z, y); otherwise P = b x d (Ra = NY rows),
// element (y, z).  Zero for z >= Sy, y >= NY or k >= K.
// grid: x over k (Kpad) in groups of four, y over the packed column w (W_pad); no per-element division.
// 16-byte loads when the source columns are 16-byte aligned (K a multiple of 4).
__global__ void pack_tab_kernel(const float* __restrict__ src, int64_t K, int64_t Kpad, int Ra, int Rb, int kindL,
                                int Sy, int SYP, int NY, int W_pad, __nv_bfloat16* __restrict__ dst,
                                __nv_bfloat16* __restrict__ dst_lo) {
  const int w = blockIdx.y;
  const int z = w % SYP, y = w / SYP;
  const bool live = z < Sy && y < NY;
  const float* col = src + (int64_t)(kindL ? (z + Ra * y) : (y + Ra * z)) * K;
  const bool vec = (K & 3) == 0;
  for (int64_t k0 = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); k0 < Kpad;
       k0 += 4 * (int64_t)gridDim.x * blockDim.x) {
    float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (live) {
      if (vec && k0 + 3 < K) {
        const float4 q = *reinterpret_cast<const float4*>(col + k0);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
      } else {
        for (int t = 0; t < 4; ++t) v[t] = (k0 + t < K) ? col[k0 + t] : 0.0f;
      }
    }
    const int64_t e = (int64_t)w * Kpad + k0;   // Kpad is a multiple of 8
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v[t]);
      dst[e + t] = h;
      if (dst_lo != nullptr) dst_lo[e + t] = __float2bfloat16_rn(v[t] - __bfloat162float(h));   // split-BF16 remainder
    }
  }
}

// Stage-2 factors: F[(f * NX + x) * SYP + z] = kindL ? P_f(x, z) (L[b=x][c=z]) : P_f(z, x) (Rm[d=z][a=x]).
// grid: x over f, y over (x, z); no per-element division
__global__ void pack_fac_kernel(const float* __restrict__ src, int64_t nf, int Ra, int Rb, int kindL, int NX, int Sy,
                                int SYP, float* __restrict__ dst) {
  const int xz = blockIdx.y;
  const int z = xz % SYP, x = xz / SYP;
  const float* col = src + (int64_t)(kindL ? (x + Ra * z) : (z + Ra * x)) * nf;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x)
    dst[(f * NX + x) * SYP + z] = (z < Sy) ? col[f] : 0.0f;
}

// FP32 subchain table level (reduced precision is enough here: the table is rounded to BF16 for the
// tensor cores, and the factors feed an FP32 stage):
// out(l + nPrev i)[x + Ra y] = sum_c prev(l)[x + Ra c] G[c + Rc (i + Ii y)]   (prev == nullptr: core slices)
// Small levels: grid x over the output rows ent = l + nPrev i, y over the output column x + Ra y.
__global__ void chain_level_f32_small_kernel(const float* __restrict__ prev, int64_t nPrev, int Ra, int Rc,
                                             const float* __restrict__ G, int64_t Ii, int Rb, float* __restrict__ out) {
  const int64_t nOut = nPrev * Ii;
  const int xy = blockIdx.y;
  const int x = xy % Ra, y = xy / Ra;
  float* o = out + (int64_t)xy * nOut;
  for (int64_t ent = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ent < nOut;
       ent += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)((uint32_t)ent / (uint32_t)nPrev), l = ent - i * nPrev;   // tables < 2^31 entries
    float acc;
    if (prev == nullptr) {
      acc = G[x + (int64_t)Rc * (i + Ii * y)];
    } else {
      acc = 0.0f;
      for (int c = 0; c < Rc; ++c)
        acc = fmaf(prev[(int64_t)(x + Ra * c) * nPrev + l], G[c + (int64_t)Rc * (i + Ii * y)], acc);
    }
    o[ent] = acc;
  }
}

// Large levels: grid x over the output rows, y over x; each thread keeps prev(l)[x + Ra c] (c < Rc) in
// registers and forms all Rb outputs of its row, so prev is read once per x rather than once per (x, y).
constexpr int kChainMaxR = 16;
__global__ void chain_level_f32_kernel(const float* __restrict__ prev, int64_t nPrev, int Ra, int Rc,
                                       const float* __restrict__ G, int64_t Ii, int Rb, float* __restrict__ out) {
  const int64_t nOut = nPrev * Ii;
  const int x = blockIdx.y;
  for (int64_t ent = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ent < nOut;
       ent += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)((uint32_t)ent / (uint32_t)nPrev), l = ent - i * nPrev;   // tables < 2^31 entries
    if (prev == nullptr) {
      for (int y = 0; y < Rb; ++y) out[(int64_t)(x + Ra * y) * nOut + ent] = G[x + (int64_t)Rc * (i + Ii * y)];
      continue;
    }
    float pv[kChainMaxR];
#pragma unroll
    for (int c = 0; c < kChainMaxR; ++c) pv[c] = c < Rc ? prev[(int64_t)(x + Ra * c) * nPrev + l] : 0.0f;
    const float* Gi = G + (int64_t)Rc * i;
    for (int y = 0; y < Rb; ++y) {
      const float* g = Gi + (int64_t)Rc * Ii * y;
      float acc = 0.0f;
#pragma unroll
      for (int c = 0; c < kChainMaxR; ++c)
        if (c < Rc) acc = fmaf(pv[c], g[c], acc);
      out[(int64_t)(x + Ra * y) * nOut + ent] = acc;
    }
  }
}

// The last level of a chain fused with its packing (for the core the previous mode updated): the level's
// sums run in the order of chain_level_f32_kernel, and each result goes straight to the packed stage-1
// table (kTab: BF16 hi and optional lo planes, row w = z + SYP y, column k = the level's row) or to the
// packed stage-2 factor (F[(f NX + x) SYP + z], f = the level's row).  Padding entries are never
// written: the plan zeroes those buffers once.
template <bool kTab>
__global__ void chain_last_pack_kernel(const float* __restrict__ prev, int64_t nPrev, int Ra, int Rc,
                                       const float* __restrict__ G, int64_t Ii, int Rb, int kindL,
                                       int SYP, int Sy, int NY, int64_t Kpad, int NX, __nv_bfloat16* __restrict__ tab,
                                       __nv_bfloat16* __restrict__ tab_lo, float* __restrict__ F) {
  const int64_t nOut = nPrev * Ii;
  const int x = blockIdx.y;
  for (int64_t ent = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ent < nOut;
       ent += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)((uint32_t)ent / (uint32_t)nPrev), l = ent - i * nPrev;
    float pv[kChainMaxR];
#pragma unroll
    for (int c = 0; c < kChainMaxR; ++c)
      pv[c] = (prev != nullptr && c < Rc) ? prev[(int64_t)(x + Ra * c) * nPrev + l] : 0.0f;
    for (int y = 0; y < Rb; ++y) {
      const float* g = G + (int64_t)Rc * (i + Ii * y);
      float v;
      if (prev == nullptr) {
        v = g[x];
      } else {
        v = 0.0f;
#pragma unroll
        for (int c = 0; c < kChainMaxR; ++c)
          if (c < Rc) v = fmaf(pv[c], g[c], v);
      }
      if (kTab) {
        const int z = kindL ? x : y, yy = kindL ? y : x;
        if (z < Sy && yy < NY) {
          const int64_t e = (int64_t)(z + SYP * yy) * Kpad + ent;
          const __nv_bfloat16 h = __float2bfloat16_rn(v);
          tab[e] = h;
          if (tab_lo != nullptr) tab_lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
      } else {
        const int z = kindL ? y : x, xx = kindL ? x : y;
        if (z < Sy) F[(ent * NX + xx) * SYP + z] = v;
      }
    }
  }
}

// FP64 cores -> one FP32 copy (conversions run once per update, not once per table element).
// FP32 copies of all cores, concatenated (offsets off[]).  Core 0 may be stored with I0p >= I0
// slices (R0 x I0p x R1), the extra slices zero, to match a zero-padded leading mode of X.
struct CorePtrs {
  const double* p[kMaxOrder];
  int64_t off[kMaxOrder + 1];
  int N;
  int R0;
  int64_t I0, I0p;
};
__global__ void cores_to_f32_kernel(const CorePtrs c, float* __restrict__ dst) {
  const int64_t total = c.off[c.N];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int j = 0;
    while (e >= c.off[j + 1]) ++j;
    const int64_t q = e - c.off[j];
    if (j == 0 && c.I0p != c.I0) {
      const int64_t a = q % c.R0, rest = q / c.R0;
      const int64_t i = rest % c.I0p, b = rest / c.I0p;
      dst[e] = i < c.I0 ? (float)c.p[0][a + c.R0 * (i + c.I0 * b)] : 0.f;
    } else {
      dst[e] = (float)c.p[j][q];
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  // looked up once, thread-safely (plans may be built by several host threads at once)
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return nullptr;
  }();
  return fn;
}

// 128-byte promotion for X: tiles whose rows start off a 256-byte boundary (mode 0 with the factor on
// the left) would otherwise fetch lines they do not read (measured: 77 -> 68 us on that mode).
constexpr CUtensorMapL2promotion kXPromotion = CU_TENSOR_MAP_L2_PROMOTION_L2_128B;

bool encode_bf16(CUtensorMap* m, const void* ptr, int rank, const uint64_t* dims, const uint64_t* strides_bytes,
                 const uint32_t* box, CUtensorMapL2promotion promotion = CU_TENSOR_MAP_L2_PROMOTION_L2_256B) {
  EncodeTiledFn fn = get_encode();
  if (!fn) return false;
  cuuint64_t gd[5], gs[4];
  cuuint32_t bd[5], es[5];
  for (int i = 0; i < rank; ++i) {
    gd[i] = dims[i];
    bd[i] = box[i];
    es[i] = 1;
  }
  for (int i = 0; i + 1 < rank; ++i) gs[i] = strides_bytes[i];
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(ptr), gd, gs, bd, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, promotion,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Host-side plan of one mode.
struct TcImpl {
  TcArgs args{};
  CUtensorMap tmX{}, tmT{}, tmXl{}, tmTl{};
  int grid = 0;
  size_t smem = 0;
  // stage-1 table build: chain modes S (cyclic order), FP64 scratch, packed BF16 table
  std::vector<int> s_modes, f_modes;
  int tabRa = 0, tabRb = 0, kindL = 0;
  int64_t K_S = 0, Kpad = 0;
  int facRa = 0, facRb = 0;
  int64_t n_fac_total = 0;
  float* chainA = nullptr;
  float* chainB = nullptr;
  float* cores32 = nullptr;                 // FP32 copy of every core, concatenated
  int64_t core_off[kMaxOrder + 1] = {};
  int SYP = 4;
  __nv_bfloat16* tab = nullptr;
  __nv_bfloat16* tab_lo = nullptr;   // split-table modes (bf16x2, bf16x3) only
  float* F = nullptr;
  float* partials = nullptr;
  int64_t E = 0;
  const int64_t* I = nullptr;
  int64_t Icopy[kMaxOrder];   // extents as stored (mode 0 possibly padded)
  int64_t I0real = 0;         // the true extent of mode 0
  int n = 0;                  // the mode this plan contracts for
  int32_t Rcopy[kMaxOrder];
  int N = 0;
  // the core the previous mode of a sweep updates is the last link of one chain: everything else is
  // built by tc_enqueue_pre, that link (fused with its packing) by tc_enqueue_main
  int late = 0;
  bool late_in_s = false;
};

int64_t prod_range(const int64_t* I, int lo, int hi) {  // prod I[lo..hi-1]
  int64_t p = 1;
  for (int j = lo; j < hi; ++j) p *= I[j];
  return p;
}

// Level sizes of a chain build over consecutive cyclic modes `modes`; returns the largest level.
int64_t chain_max_elems(const std::vector<int>& modes, const int64_t* I, const int32_t* R, int N) {
  int64_t n = 1, mx = 0;
  const int Ra = R[modes[0]];
  for (int m : modes) {
    n *= I[m];
    mx = std::max<int64_t>(mx, n * Ra * R[(m + 1) % N]);
  }
  return mx;
}

// Build the FP32 chain table over consecutive cyclic `modes` (ping-ponging bufA/bufB); returns the result.
const float* build_chain(const std::vector<int>& modes, const float* const* cores, const int64_t* I, const int32_t* R,
                         int N, float* bufA, float* bufB, cudaStream_t s, int* launches) {
  const float* prev = nullptr;
  int64_t nPrev = 1;
  const int Ra = R[modes[0]];
  float* bufs[2] = {bufA, bufB};
  int t = 0;
  for (int m : modes) {
    float* out = bufs[t++ % 2];
    const int64_t nOut = nPrev * I[m];
    if (nOut * Ra >= (int64_t)152 * 2048) {   // enough rows to fill the GPU with one thread per (row, x)
      const dim3 g((unsigned)std::min<int64_t>((nOut + 255) / 256, 4096), (unsigned)Ra);
      chain_level_f32_kernel<<<g, 256, 0, s>>>(prev, nPrev, Ra, R[m], cores[m], I[m], R[(m + 1) % N], out);
    } else {
      const dim3 g((unsigned)((nOut + 255) / 256), (unsigned)(Ra * R[(m + 1) % N]));
      chain_level_f32_small_kernel<<<g, 256, 0, s>>>(prev, nPrev, Ra, R[m], cores[m], I[m], R[(m + 1) % N], out);
    }
    ++*launches;
    prev = out;
    nPrev *= I[m];
  }
  return prev;
}

// The first `count` levels of a chain; *nPrev_out gets the row count of the last level built.
const float* build_chain_levels(const std::vector<int>& modes, int count, const float* const* cores, const int64_t* I,
                                const int32_t* R, int N, float* bufA, float* bufB, cudaStream_t s, int* launches,
                                int64_t* nPrev_out) {
  std::vector<int> sub(modes.begin(), modes.begin() + count);
  int64_t nPrev = 1;
  for (int m : sub) nPrev *= I[m];
  *nPrev_out = nPrev;
  if (count == 0) return nullptr;
  return build_chain(sub, cores, I, R, N, bufA, bufB, s, launches);
}

}  // namespace

TcChoice tc_choose(int N, const int64_t* I, const int32_t* R, int n) {
  TcChoice best;
  int maxR = 0;
  for (int j = 0; j < N; ++j) maxR = std::max(maxR, (int)R[j]);
  const int Rn = R[n], Rn1 = R[(n + 1) % N];
  const int r = Rn * Rn1;
  const int64_t In = I[n];
  if (maxR > 16 || r > 256 || In * r > 8192) return best;
  auto consider = [&](TcChoice c, int W, int64_t extra_cost = 0) {
    if (c.K_S < 256 || W > kMaxW) return;
    const int64_t tabBytes = c.K_S * (int64_t)((W + 15) / 16 * 16) * 2;
    if (tabBytes > (int64_t)64 << 20) return;
    c.cost = (c.variant == MM) ? tabBytes + tabBytes / 4 + 1 : tabBytes;   // prefer K-major X unless MN-major is clearly cheaper
    c.cost += extra_cost;
    if (best.variant < 0 || c.cost < best.cost) best = c;
  };
  // MN-major tiles over a contiguous run P = I_0 ... I_n shorter than a 64-element TMA row read part
  // of every 128-byte row out of bounds, which the copy engine streams at about half the rate of full
  // rows (measured): such an MM tile counts as costly as a 1 GB table.
  constexpr int64_t kShortRunPenalty = (int64_t)1 << 30;
  // KM-L: S = modes 0..n-1 (needs post modes)
  if (n >= 1 && n <= N - 2) {
    TcChoice c;
    c.variant = KM_L;
    c.s_lo = 0;
    c.s_hi = n - 1;
    c.K_S = prod_range(I, 0, n);
    // rows i + I_n rep: each repetition's factor block is staged in shared memory per unit, so at
    // most 16 repetitions (I_n >= 8)
    if ((c.K_S * 2) % 16 == 0 && In <= kRows && In >= 8) consider(c, (R[0] + 3) / 4 * 4 * Rn);
  }
  // KM-R: n = N-1, S = modes 0..s with s <= N-3
  if (n == N - 1) {
    for (int s = 0; s <= N - 3; ++s) {
      TcChoice c;
      c.variant = KM_R;
      c.s_lo = 0;
      c.s_hi = s;
      c.K_S = prod_range(I, 0, s + 1);
      if ((c.K_S * 2) % 16 == 0 && In <= kRows) consider(c, (R[s + 1] + 3) / 4 * 4 * R[0]);
    }
  }
  // MM: S = modes n+1..m, not the whole chain
  {
    const int64_t P = prod_range(I, 0, n + 1);
    if ((P * 2) % 16 == 0 && (P + 63) / 64 <= 128) {   // one p-chunk per CTA
      for (int m = n + 1; m <= N - 1; ++m) {
        if (n == 0 && m == N - 1) continue;
        TcChoice c;
        c.variant = MM;
        c.s_lo = n + 1;
        c.s_hi = m;
        c.K_S = prod_range(I, n + 1, m + 1);
        consider(c, (R[(m + 1) % N] + 3) / 4 * 4 * Rn1, P < 64 ? kShortRunPenalty : 0);
      }
    }
  }
  // MM-L (n = 0): S = modes m..N-1, a tile = 128 consecutive elements (i_0, l), l over modes 1..m-1,
  // the left factor G_1(i_1)...G_{m-1}(i_{m-1}); K rows are P' = I_0 ... I_{m-1} elements apart (a
  // multiple of 8 for the 16-byte stride rule).
  if (n == 0 && In <= kRows) {
    for (int m = 2; m <= N - 1; ++m) {
      const int64_t Pp = prod_range(I, 0, m);
      if ((Pp * 2) % 16 != 0 || Pp > ((int64_t)1 << 30)) continue;
      TcChoice c;
      c.variant = MM_L;
      c.s_lo = m;
      c.s_hi = N - 1;
      c.K_S = prod_range(I, m, N);
      // only the smallest m whose table fits: K rows of X are P' elements apart, and with a short P'
      // the CTAs of all tiles read each K row together (whole DRAM rows); a larger m makes the table
      // smaller but scatters every tile's 256-byte pieces over K rows megabytes apart
      const int W = (R[m] + 3) / 4 * 4 * R[0];
      if (c.K_S < 256 || W > kMaxW || c.K_S * (int64_t)((W + 15) / 16 * 16) * 2 > ((int64_t)64 << 20)) continue;
      consider(c, W);
      break;
    }
  }
  return best;
}

int tc_plan(TcPlan& p, int N, const int64_t* I, const int32_t* R, int n, int mode, const void* X, int64_t numel,
            cudaError_t* err, cudaStream_t s, size_t* count_bytes, int64_t I0_real, const void* Xlo, int free_sms) {
  if (err) *err = cudaSuccess;
  p.valid = false;
  const bool x3 = mode == TRALS_MODE_BF16X3;
  const bool tlo = x3 || mode == TRALS_MODE_BF16X2;   // the table as hi/lo planes
  if (mode != TRALS_MODE_BF16 && mode != TRALS_MODE_BF16X2 && !(x3 && Xlo != nullptr)) return 0;
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) return 0;
  if (x3 && (reinterpret_cast<uintptr_t>(Xlo) & 15) != 0) return 0;
  if (!get_encode()) return 0;
  const int Rn = R[n], Rn1 = R[(n + 1) % N];
  const int r = Rn * Rn1;
  const int64_t In = I[n];

  const TcChoice best = tc_choose(N, I, R, n);
  if (best.variant < 0) return 0;

  TcImpl* impl = new TcImpl();
  impl->N = N;
  impl->I0real = I0_real > 0 ? I0_real : I[0];
  impl->n = n;
  for (int j = 0; j < N; ++j) {
    impl->Icopy[j] = I[j];
    impl->Rcopy[j] = R[j];
  }
  TcArgs& A = impl->args;
  A.variant = best.variant;
  A.In = (int)In;
  A.Rn = Rn;
  A.r = r;
  impl->K_S = best.K_S;
  impl->Kpad = (best.K_S + 7) / 8 * 8;
  A.ksteps = (int)((best.K_S + kKT - 1) / kKT);
  for (int m = best.s_lo; m <= best.s_hi; ++m) impl->s_modes.push_back(m);
  impl->tabRa = R[best.s_lo];
  impl->tabRb = R[(best.s_hi + 1) % N];
  uint64_t dims[3], strides[2];
  uint32_t box[3];
  int64_t n_tiles = 0;
  if (A.variant == KM_L) {
    // T = c x a (c = dot index, Sy = R_0); F = L = G_{n+1}..G_{N-1} (R_{n+1} x R_0) on the left
    impl->kindL = 1;
    for (int m = n + 1; m <= N - 1; ++m) impl->f_modes.push_back(m);
    impl->facRa = Rn1;
    impl->facRb = R[0];
    A.NX = Rn1;
    A.NY = Rn;
    A.Sy = R[0];
    const int64_t K_post = prod_range(I, n + 1, N);
    A.nrep = std::max<int>(1, (int)(kRows / In));
    A.n_fac = K_post;
    n_tiles = (K_post + A.nrep - 1) / A.nrep;
    dims[0] = best.K_S; dims[1] = In; dims[2] = K_post;
    strides[0] = best.K_S * 2; strides[1] = best.K_S * In * 2;
    box[0] = kKT; box[1] = (uint32_t)In; box[2] = (uint32_t)A.nrep;
    A.tx_bytes = (uint32_t)(kKT * 2 * In * A.nrep);
  } else if (A.variant == KM_R) {
    // T = b x d (d = dot index, Sy = R_{s+1}); F = Rm = G_{s+1}..G_{N-2} (R_{s+1} x R_n) on the right
    impl->kindL = 0;
    for (int m = best.s_hi + 1; m <= N - 2; ++m) impl->f_modes.push_back(m);
    impl->facRa = R[best.s_hi + 1];
    impl->facRb = Rn;
    A.NX = Rn;
    A.NY = Rn1;
    A.Sy = impl->tabRb;
    const int64_t K_mid = prod_range(I, best.s_hi + 1, N - 1);
    A.nrep = std::max<int>(1, (int)(kRows / In));
    A.n_fac = K_mid;
    n_tiles = (K_mid + A.nrep - 1) / A.nrep;
    dims[0] = best.K_S; dims[1] = K_mid; dims[2] = In;
    strides[0] = best.K_S * 2; strides[1] = best.K_S * K_mid * 2;
    box[0] = kKT; box[1] = (uint32_t)A.nrep; box[2] = (uint32_t)In;
    A.tx_bytes = (uint32_t)(kKT * 2 * In * A.nrep);
  } else if (A.variant == MM_L) {
    // T = c x a (c = dot index, Sy = R_m); F = L = G_1..G_{m-1} (R_1 x R_m) on the left; a tile = 128
    // consecutive elements e = i_0 + I_0 l of a K row
    impl->kindL = 1;
    for (int m = 1; m < best.s_lo; ++m) impl->f_modes.push_back(m);
    impl->facRa = R[1];
    impl->facRb = R[best.s_lo];
    A.NX = R[1];
    A.NY = Rn;
    A.Sy = R[best.s_lo];
    const int64_t Lf = prod_range(I, 1, best.s_lo);
    A.nrep = 1;
    A.nslot = (int)((kRows + In - 1) / In) + 1;   // values of l that 128 consecutive elements can touch
    A.Pp = In * Lf;
    A.n_fac = Lf;
    n_tiles = (A.Pp + kRows - 1) / kRows;
    dims[0] = In * Lf; dims[1] = best.K_S; dims[2] = 1;
    strides[0] = In * Lf * 2; strides[1] = In * Lf * best.K_S * 2;
    box[0] = 64; box[1] = kKT; box[2] = 1;
    A.tx_bytes = (uint32_t)(2 * kAtomBytes);
  } else {
    // T = b x d (d = dot index, Sy = R_{m+1}); F = Rm = G_{m+1}..G_{N-1} G_0..G_{n-1} (R_{m+1} x R_n) on the right
    impl->kindL = 0;
    for (int m = best.s_hi + 1; m <= N - 1; ++m) impl->f_modes.push_back(m);
    for (int m = 0; m <= n - 1; ++m) impl->f_modes.push_back(m);
    impl->facRa = R[(best.s_hi + 1) % N];
    impl->facRb = Rn;
    A.NX = Rn;
    A.NY = Rn1;
    A.Sy = impl->tabRb;
    A.P = prod_range(I, 0, n + 1);
    A.K_pre = prod_range(I, 0, n);
    A.K_hi = prod_range(I, best.s_hi + 1, N);
    A.pchunks = (A.P + 63) / 64;
    A.opairs = (A.K_hi + 1) / 2;
    n_tiles = A.pchunks * A.opairs;
    dims[0] = A.P; dims[1] = best.K_S; dims[2] = A.K_hi;
    strides[0] = A.P * 2; strides[1] = A.P * best.K_S * 2;
    box[0] = 64; box[1] = kKT; box[2] = 1;
    A.tx_bytes = (uint32_t)(2 * kAtomBytes);
  }
  impl->SYP = (A.Sy + 3) / 4 * 4;
  A.fac_shared = (A.variant == MM) ? 0 : 1;
  if (A.variant == KM_L || A.variant == KM_R) A.nslot = A.nrep;
  impl->late = (n + N - 1) % N;
  impl->late_in_s = !impl->s_modes.empty() && impl->s_modes.back() == impl->late;
  if (!impl->late_in_s && (impl->f_modes.empty() || impl->f_modes.back() != impl->late)) {
    delete impl;   // every geometry ends one chain with the previous mode; anything else is not planned for
    return 0;
  }
  const int W = impl->SYP * A.NY;
  A.W_pad = (W + 15) / 16 * 16;
  A.fs_stride = (A.NX * impl->SYP + 7) / 8 * 8 + 4;
  A.ms_stride = A.r | 1;   // odd row stride: lanes with different i_n hit different banks

  A.x3 = x3 ? 2 : tlo ? 1 : 0;
  // X box(es) (hi, and lo in bf16x3), then table box(es) (hi, and lo in both split modes)
  A.tx_bytes = (uint32_t)((x3 ? 2 : 1) * A.tx_bytes + (tlo ? 2 : 1) * A.W_pad * 128);
  // MMA instruction descriptor: D=F32, A=B=BF16, A major per variant, B K-major, N=W_pad, M=128
  A.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((A.variant == MM || A.variant == MM_L ? 1u : 0u) << 15) |
            ((uint32_t)(A.W_pad >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);

  // units: split K so that the grid gets a few units per SM
  int nsm = 152;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  // SMs left free for the FP64 coefficient-matrix branch that runs concurrently in the sweep (its
  // one-CTA Cholesky needs one; the blocked factorization's panel kernels need more)
  nsm = std::max(1, nsm - std::max(0, free_sms));
  A.n_tiles = n_tiles;
  {
    // shares of at least four tiles: whole tiles (at most a quarter of imbalance, one epilogue fewer)
    const int64_t per_chunk = (A.variant == MM) ? A.opairs : n_tiles;
    const int64_t ctas = (A.variant == MM) ? std::max<int64_t>(1, nsm / std::max<int64_t>(1, A.pchunks))
                                           : std::min<int64_t>(n_tiles * A.ksteps, nsm);
    A.whole = per_chunk >= 4 * ctas ? 1 : 0;
  }
  A.ksync = 0;
  A.spin_limit = kSpinLimit;
  A.withhold = 0;
  if (A.variant == MM) {
    if (A.pchunks > nsm) {   // each CTA keeps a single p-chunk
      delete impl;
      return 0;
    }
    impl->grid = nsm;
  } else if (A.variant == MM_L && n_tiles <= nsm && A.ksteps >= nsm / n_tiles) {
    A.ksync = 1;
    A.whole = 0;
    impl->grid = (int)(n_tiles * (nsm / n_tiles));
  } else {
    impl->grid = (int)std::min<int64_t>(n_tiles * A.ksteps, nsm);
  }
  impl->E = In * r;

  // ---- shared-memory plan (checked before anything is allocated)
  const int bBytes = ((A.W_pad * 128) + 1023) & ~1023;
  const int fs_rows = A.fac_shared ? 2 * A.nslot : kRows;
  size_t fixed = 1024 + (size_t)((fs_rows * A.fs_stride + 1) & ~1) * 4 + (2 * kNSMax + 4) * 8 + 64;
  if (A.variant == MM_L)   // one x-column of every row, and the I_0 x r sums
    fixed += (size_t)((kRows * (A.NY | 1) + 1) & ~1) * 4 + (size_t)((In * A.ms_stride + 1) & ~1) * 4;
  const size_t stage = (size_t)(tlo ? 2 : 1) * ((size_t)kABytes + bBytes);
  const int ns = (int)std::min<size_t>(kNSMax, fixed < (size_t)kSmemBudget ? (kSmemBudget - fixed) / stage : 0);
  if (ns < 2) {
    delete impl;
    return 0;
  }
  A.ns = ns;
  impl->smem = fixed + (size_t)ns * stage;
  {
    // the end-of-kernel lane staging, its column map and the CTA's I_n x r sums reuse the pipeline
    // buffers (idle by then)
    const size_t stage_area = (size_t)ns * stage;
    const int nv = A.NX * A.NY;
    const size_t need = (size_t)kRows * (nv | 1) * 4 + (size_t)((nv + 3) & ~3) * 4 + (size_t)In * A.ms_stride * 4;
    if (need > stage_area) {
      delete impl;
      return 0;
    }
  }

  // ---- tensor maps: validated before anything is allocated, so that the counting pass and the real
  // plan agree on whether this mode runs on the tensor cores (the table's map is encoded again once
  // the table exists; the encoder only checks the address's alignment)
  const uint64_t tdims[2] = {(uint64_t)impl->Kpad, (uint64_t)A.W_pad};
  const uint64_t tstrides[1] = {(uint64_t)impl->Kpad * 2};
  const uint32_t tbox[2] = {kKT, (uint32_t)A.W_pad};
  const int xrank = (A.variant == MM_L) ? 2 : 3;
  if (!encode_bf16(&impl->tmX, X, xrank, dims, strides, box, kXPromotion) ||
      !encode_bf16(&impl->tmT, reinterpret_cast<const void*>(uintptr_t(1) << 40), 2, tdims, tstrides, tbox) ||
      (x3 && !encode_bf16(&impl->tmXl, Xlo, xrank, dims, strides, box, kXPromotion))) {
    delete impl;
    return 0;
  }

  // ---- allocations (stream-ordered on s; in the counting pass only summed)
  const int64_t chainMax = std::max(chain_max_elems(impl->s_modes, I, R, N), chain_max_elems(impl->f_modes, I, R, N));
  int64_t nfac = 1;
  for (int m : impl->f_modes) nfac *= I[m];
  impl->n_fac_total = nfac;
  for (int j = 0; j < N; ++j) impl->core_off[j + 1] = impl->core_off[j] + (int64_t)R[j] * I[j] * R[(j + 1) % N];
  const size_t sizes[7] = {(size_t)impl->core_off[N] * sizeof(float), chainMax * sizeof(float),
                           chainMax * sizeof(float), (size_t)A.W_pad * impl->Kpad * sizeof(__nv_bfloat16),
                           (size_t)nfac * A.NX * impl->SYP * sizeof(float),
                           (size_t)impl->grid * impl->E * sizeof(float),
                           tlo ? (size_t)A.W_pad * impl->Kpad * sizeof(__nv_bfloat16) : 0};
  const int nalloc = tlo ? 7 : 6;
  if (count_bytes) {
    for (int k = 0; k < nalloc; ++k) *count_bytes += (std::max<size_t>(sizes[k], 16) + 255) & ~(size_t)255;
    delete impl;
    return 1;
  }
  p.stream = s;
  cudaError_t e = cudaSuccess;
  void* q[7] = {};
  p.bytes = 0;
  for (int k = 0; k < nalloc && e == cudaSuccess; ++k) {
    const size_t b = (std::max<size_t>(sizes[k], 16) + 255) & ~(size_t)255;
    e = cudaMallocAsync(&q[k], b, s);
    if (e == cudaSuccess) {
      p.allocs.push_back(q[k]);
      p.bytes += b;
    }
  }
  if (e != cudaSuccess) {
    if (err) *err = e;
    delete impl;
    for (void* a : p.allocs) cudaFreeAsync(a, s);
    p.allocs.clear();
    return 0;
  }
  impl->cores32 = static_cast<float*>(q[0]);
  impl->chainA = static_cast<float*>(q[1]);
  impl->chainB = static_cast<float*>(q[2]);
  impl->tab = static_cast<__nv_bfloat16*>(q[3]);
  impl->F = static_cast<float*>(q[4]);
  impl->partials = static_cast<float*>(q[5]);
  impl->tab_lo = tlo ? static_cast<__nv_bfloat16*>(q[6]) : nullptr;
  A.F = impl->F;
  A.partials = impl->partials;
  // padding of the packed table and factor stays zero: the fused last-link kernel writes live entries only
  e = cudaMemsetAsync(impl->tab, 0, sizes[3], s);
  if (e == cudaSuccess) e = cudaMemsetAsync(impl->F, 0, sizes[4], s);
  if (e == cudaSuccess && tlo) e = cudaMemsetAsync(impl->tab_lo, 0, sizes[6], s);
  if (e != cudaSuccess) {
    if (err) *err = e;
    delete impl;
    for (void* a : p.allocs) cudaFreeAsync(a, s);
    p.allocs.clear();
    return 0;
  }
  if (!encode_bf16(&impl->tmT, impl->tab, 2, tdims, tstrides, tbox) ||
      (tlo && !encode_bf16(&impl->tmTl, impl->tab_lo, 2, tdims, tstrides, tbox))) {
    delete impl;
    for (void* a : p.allocs) cudaFreeAsync(a, s);
    p.allocs.clear();
    return 0;
  }
  p.impl = impl;
  p.valid = true;
  p.N = N;
  p.n = n;
  p.mode = mode;
  (void)numel;
  return 1;
}

int tc_enqueue_pre(TcPlan& p, double* const* cores, cudaStream_t s, const float* const* c32_ext) {
  TcImpl* impl = static_cast<TcImpl*>(p.impl);
  int launches = 0;
  const int64_t* I = impl->Icopy;
  const int32_t* R = impl->Rcopy;
  const int N = impl->N;
  TcArgs A = impl->args;
  const float* c32[kMaxOrder];
  if (c32_ext != nullptr) {
    for (int j = 0; j < N; ++j) c32[j] = c32_ext[j];
  } else {
    CorePtrs cp;
    cp.N = N;
    for (int j = 0; j <= N; ++j) cp.off[j] = impl->core_off[j];
    cp.R0 = R[0];
    cp.I0 = impl->I0real;
    cp.I0p = I[0];
    for (int j = 0; j < N; ++j) {
      cp.p[j] = cores[j];
      c32[j] = impl->cores32 + impl->core_off[j];
    }
    cores_to_f32_kernel<<<(unsigned)std::min<int64_t>((impl->core_off[N] + 255) / 256, 152), 256, 0, s>>>(cp,
                                                                                                     impl->cores32);
    ++launches;
  }
  // the chain without the late core, whole, and its packing
  if (impl->late_in_s) {
    const float* fsrc = build_chain(impl->f_modes, c32, I, R, N, impl->chainA, impl->chainB, s, &launches);
    const dim3 g((unsigned)std::min<int64_t>((impl->n_fac_total + 255) / 256, 1024), (unsigned)(A.NX * impl->SYP));
    pack_fac_kernel<<<g, 256, 0, s>>>(fsrc, impl->n_fac_total, impl->facRa, impl->facRb, impl->kindL, A.NX, A.Sy,
                                      impl->SYP, impl->F);
    ++launches;
  } else {
    const float* tsrc = build_chain(impl->s_modes, c32, I, R, N, impl->chainA, impl->chainB, s, &launches);
    const dim3 g((unsigned)std::min<int64_t>((impl->Kpad / 4 + 255) / 256, 1024), (unsigned)A.W_pad);
    pack_tab_kernel<<<g, 256, 0, s>>>(tsrc, impl->K_S, impl->Kpad, impl->tabRa, impl->tabRb, impl->kindL, A.Sy,
                                      impl->SYP, A.NY, A.W_pad, impl->tab, impl->tab_lo);
    ++launches;
  }
  // the other chain up to its last link (left in chainA / chainB for tc_enqueue_main)
  const std::vector<int>& lc = impl->late_in_s ? impl->s_modes : impl->f_modes;
  int64_t nPrev = 1;
  build_chain_levels(lc, (int)lc.size() - 1, c32, I, R, N, impl->chainA, impl->chainB, s, &launches, &nPrev);
  return launches;
}

int tc_enqueue_main(TcPlan& p, double* const* cores, double* M, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                    const float* const* c32_ext, cudaEvent_t before_kernel) {
  (void)cores;
  TcImpl* impl = static_cast<TcImpl*>(p.impl);
  int launches = 0;
  const int64_t* I = impl->Icopy;
  const int32_t* R = impl->Rcopy;
  const int N = impl->N;
  TcArgs A = impl->args;
  {
    // the last link: the level built by tc_enqueue_pre sits in chainA or chainB by the parity of its levels
    const std::vector<int>& lc = impl->late_in_s ? impl->s_modes : impl->f_modes;
    const int nl = (int)lc.size() - 1;
    int64_t nPrev = 1;
    for (int j = 0; j < nl; ++j) nPrev *= I[lc[j]];
    const float* prev = nl == 0 ? nullptr : ((nl - 1) % 2 == 0 ? impl->chainA : impl->chainB);
    const int m = lc.back();
    const int Ra = R[lc[0]], Rc = R[m], Rb = R[(m + 1) % N];
    const float* G = c32_ext != nullptr ? c32_ext[m] : impl->cores32 + impl->core_off[m];
    const int64_t nOut = nPrev * I[m];
    const dim3 g((unsigned)std::min<int64_t>((nOut + 255) / 256, 4096), (unsigned)Ra);
    if (impl->late_in_s)
      chain_last_pack_kernel<true><<<g, 256, 0, s>>>(prev, nPrev, Ra, Rc, G, I[m], Rb, impl->kindL,
                                                      impl->SYP, A.Sy, A.NY, impl->Kpad, A.NX, impl->tab,
                                                      impl->tab_lo, nullptr);
    else
      chain_last_pack_kernel<false><<<g, 256, 0, s>>>(prev, nPrev, Ra, Rc, G, I[m], Rb, impl->kindL,
                                                       impl->SYP, A.Sy, A.NY, impl->Kpad, A.NX, nullptr, nullptr,
                                                       impl->F);
    ++launches;
  }
  if (before_kernel) cudaStreamWaitEvent(s, before_kernel, 0);
  if (ev0) cudaEventRecord(ev0, s);
  const CUtensorMap& xl = A.x3 == 2 ? impl->tmXl : impl->tmX;   // unread unless bf16x3
  const CUtensorMap& tl = A.x3 ? impl->tmTl : impl->tmT;         // unread without a split table
  tc_kernel_for(impl->SYP, A.x3 != 0)<<<impl->grid, kThreads, impl->smem, s>>>(impl->tmX, impl->tmT, xl, tl, A);
  ++launches;
  if (ev1) cudaEventRecord(ev1, s);
  {
    const int In_out = (impl->n == 0) ? (int)impl->I0real : A.In;
    const int64_t Eout = impl->E / A.In * In_out;
    tc_reduce_kernel<<<(unsigned)((Eout + 31) / 32), 256, 0, s>>>(impl->partials, impl->grid, impl->E, A.In, In_out,
                                                                  M);
  }
  ++launches;
  return launches;
}

int tc_enqueue(TcPlan& p, const void* X, double* const* cores, double* M, cudaStream_t s, cudaEvent_t ev0,
               cudaEvent_t ev1) {
  (void)X;
  return tc_enqueue_pre(p, cores, s, nullptr) + tc_enqueue_main(p, cores, M, s, ev0, ev1, nullptr);
}

void launch_cores_to_f32(double* const* cores, int N, const int32_t* R, const int64_t* Ist, int64_t I0real,
                         float* dst, cudaStream_t s) {
  CorePtrs cp;
  cp.N = N;
  cp.off[0] = 0;
  for (int j = 0; j < N; ++j) {
    cp.p[j] = cores[j];
    cp.off[j + 1] = cp.off[j] + (int64_t)R[j] * Ist[j] * R[(j + 1) % N];
  }
  cp.R0 = R[0];
  cp.I0 = I0real;
  cp.I0p = Ist[0];
  cores_to_f32_kernel<<<(unsigned)std::min<int64_t>((cp.off[N] + 255) / 256, 152 * 4), 256, 0, s>>>(cp, dst);
}

int tc_variant(const TcPlan& p) { return p.impl ? static_cast<const TcImpl*>(p.impl)->args.variant : -1; }

void tc_set_status(TcPlan& p, DevStatus* st) {
  if (p.impl) static_cast<TcImpl*>(p.impl)->args.status = st;
}

void tc_set_fault(TcPlan& p, int withhold_first_copy, long long spin_limit_cycles) {
  if (!p.impl) return;
  TcArgs& A = static_cast<TcImpl*>(p.impl)->args;
  A.withhold = withhold_first_copy ? 1 : 0;
  A.spin_limit = spin_limit_cycles > 0 ? spin_limit_cycles : kSpinLimit;
}

void tc_destroy(TcPlan& p) {
  for (void* q : p.allocs) cudaFreeAsync(q, p.stream);
  p.allocs.clear();
  delete static_cast<TcImpl*>(p.impl);
  p.impl = nullptr;
  p.valid = false;
}

cudaError_t init_tc_attributes() {
  cudaError_t e = cudaSuccess;
  for (int syp = 4; syp <= 16 && e == cudaSuccess; syp += 4)
    for (int sp = 0; sp < 2 && e == cudaSuccess; ++sp)
      e = cudaFuncSetAttribute(tc_kernel_for(syp, sp != 0), cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget);
  return e;
}

}  // namespace trals
