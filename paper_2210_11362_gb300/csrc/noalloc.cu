// trals_mttsp_noalloc: the FP64 MTTSP (the CUDA-core kernel behind trals_mttsp in FP64 mode) for
// callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc/cudaFree are unavailable or forbidden, for example a
// host callback or a custom allocator hook that must not re-enter the CUDA allocator, a real-time
// loop with a fixed memory budget that may not grow, or an embedding runtime that owns all device
// memory itself.  trals_mttsp allocates its subchain tables, offsets and per-block partial sums on
// every call; this variant places them in one static device array instead.
//
// The scratch array (kNoAllocScratchBytes) exists on every GPU that loads the library, from load to
// process exit.  Its device address is looked up once per device with cudaGetSymbolAddress on the
// first call made while that device is current; make that first call before any stream capture.
// Every call shares the array: concurrent or overlapping calls on the GPU race, so issue calls on one
// stream (or otherwise serialise them).  Nothing in the array needs to start at zero: each call
// rewrites every table entry, offset and partial sum it reads.
#include <algorithm>
#include <cstring>
#include <vector>

#include "trals_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" trals_status trals_mttsp_noalloc(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                                            const void* X_dev, const double* const* cores_dev, int n,
                                            double* M_dev) {
  using namespace trals;
  if (!ctx || !I || !R || !X_dev || !cores_dev || !M_dev || N < 3 || N > TRALS_MAX_ORDER || n < 0 || n >= N)
    return TRALS_E_ARG;
  for (int k = 0; k < N; ++k) {
    if (I[k] < 1 || R[k] < 1 || R[k] > 64) {
      ctx->last_error = "trals_mttsp_noalloc: invalid mode size or rank";
      return TRALS_E_ARG;
    }
  }
  if (ctx->device < 0 || ctx->device >= kMaxDevices) return TRALS_E_ARG;
  // size check first: a shape that does not fit is rejected before any CUDA call
  const ModeLayout L = make_mode_layout(N, I, R, n);
  const int64_t tab = table_level_max_elems(L, I, R);
  const size_t tab_b = align256((size_t)tab * sizeof(double));
  const size_t offL_b = align256((size_t)L.nL * sizeof(int64_t));
  const size_t offU_b = align256((size_t)L.nU * sizeof(int64_t));
  const size_t fixed = 3 * tab_b + offL_b + offU_b;
  const size_t per_block = (size_t)(L.In * L.Rn * L.Rn1) * sizeof(double);
  if (fixed + per_block > kNoAllocScratchBytes) {
    ctx->last_error = "trals_mttsp_noalloc: the subchain tables and one block's partial sums need " +
                      std::to_string(fixed + per_block) + " bytes, more than the " +
                      std::to_string(kNoAllocScratchBytes) + "-byte static scratch (use trals_mttsp)";
    return TRALS_E_ARG;
  }
  TRALS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (g_scratch_addr[ctx->device] == nullptr) {
    void* ptr = nullptr;
    TRALS_CUDA_TRY(ctx, cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_scratch_addr[ctx->device] = ptr;
  }
  unsigned char* scratch = static_cast<unsigned char*>(g_scratch_addr[ctx->device]);
  std::vector<int64_t> offL, offU;
  mode_offsets(N, I, L, offL, offU);
  const int gridX = (int)std::max<size_t>(
      1, std::min<size_t>((size_t)mttsp_simt_default_grid(L), (kNoAllocScratchBytes - fixed) / per_block));
  double* lt = reinterpret_cast<double*>(scratch);
  double* ut = reinterpret_cast<double*>(scratch + tab_b);
  double* sc = reinterpret_cast<double*>(scratch + 2 * tab_b);
  int64_t* dL = reinterpret_cast<int64_t*>(scratch + 3 * tab_b);
  int64_t* dU = reinterpret_cast<int64_t*>(scratch + 3 * tab_b + offL_b);
  double* part = reinterpret_cast<double*>(scratch + fixed);

  cudaStream_t s = ctx->stream;
  TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(dL, offL.data(), offL.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  TRALS_CUDA_TRY(ctx, cudaMemcpyAsync(dU, offU.data(), offU.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  build_tables(L, cores_dev, I, R, lt, ut, sc, s);
  MttspSimtArgs a;
  a.X = X_dev;
  a.xt = TRALS_X_F64;
  a.ltab = lt;
  a.utab = ut;
  a.offL = dL;
  a.offU = dU;
  a.L = L;
  a.partials = part;
  a.M = M_dev;
  a.gridX = gridX;
  launch_mttsp_simt(a, s);
  TRALS_CUDA_TRY(ctx, cudaGetLastError());
  // the host offset vectors must outlive their copies
  TRALS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return TRALS_OK;
}
