// trals_mttsp_noalloc: the FP64 MTTSP (the CUDA-core kernel behind trals_mttsp in FP64 mode) for
// callers that must not allocate device memory.
//
// Who needs it: code that may not call cudaMalloc/cudaFree, for example a custom allocator hook
// that must not re-enter the CUDA allocator, a real-time loop with a fixed memory budget that may
// not grow, or an embedding runtime that owns all device memory itself and passes the library only
// its inputs and outputs.  trals_mttsp allocates its subchain tables, offsets and per-block partial
// sums on every call; this variant places them in one static device array instead.
//
// The scratch array (kNoAllocScratchBytes) exists on every GPU that loads the library, from load to
// process exit.  Its device address is looked up once per device with cudaGetSymbolAddress on the
// first call made while that device is current.  The call is synchronous: it copies the index
// offsets from host memory and waits for its stream, so it is not for stream callbacks (where CUDA
// calls are not allowed) nor for a stream that is being captured.  Every call shares the array:
// calls that overlap on the GPU race, so serialise them.  Nothing in the array needs to start at
// zero: each call rewrites every table entry, offset and partial sum it reads.
#include <algorithm>
#include <cstring>
#include <vector>

#include "trals_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

void* g_scratch_addr[kMaxDevices] = {};

constexpr size_t kSat = ~(size_t)0;
// products and sums that stick at SIZE_MAX instead of wrapping
size_t mul_sat(size_t a, size_t b) { return (a != 0 && b > kSat / a) ? kSat : a * b; }
size_t add_sat(size_t a, size_t b) { return b > kSat - a ? kSat : a + b; }
size_t align256(size_t b) { return b > kSat - 255 ? kSat : (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" trals_status trals_mttsp_noalloc(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                                            const void* X_dev, const double* const* cores_dev, int n,
                                            double* M_dev) {
  using namespace trals;
  if (!ctx) return TRALS_E_ARG;
  if (!X_dev || !cores_dev || !M_dev) {
    ctx->last_error = "trals_mttsp_noalloc: null buffer";
    return TRALS_E_ARG;
  }
  // the shapes trals_mttsp accepts, no others (this also caps prod I_n at 2^46)
  const trals_status st = check_shape(ctx, N, I, R);
  if (st != TRALS_OK) return st;
  if (n < 0 || n >= N) {
    ctx->last_error = "trals_mttsp_noalloc: mode index out of range";
    return TRALS_E_ARG;
  }
  if (ctx->device < 0 || ctx->device >= kMaxDevices) {
    ctx->last_error = "trals_mttsp_noalloc: device index beyond the supported range";
    return TRALS_E_ARG;
  }
  // size check first, in saturating arithmetic: a shape that does not fit is rejected before any
  // CUDA call, and no wrapped product can pass the comparison
  const ModeLayout L = make_mode_layout(N, I, R, n);
  const size_t tab_b = align256(mul_sat((size_t)table_level_max_elems(L, I, R), sizeof(double)));
  const size_t offL_b = align256(mul_sat((size_t)L.nL, sizeof(int64_t)));
  const size_t offU_b = align256(mul_sat((size_t)L.nU, sizeof(int64_t)));
  const size_t fixed = add_sat(add_sat(mul_sat(3, tab_b), offL_b), offU_b);
  const size_t per_block = mul_sat(mul_sat((size_t)L.In, (size_t)L.Rn * L.Rn1), sizeof(double));
  if (add_sat(fixed, per_block) > kNoAllocScratchBytes) {
    ctx->last_error = "trals_mttsp_noalloc: the subchain tables and one block's partial sums need " +
                      std::to_string(add_sat(fixed, per_block)) + " bytes, more than the " +
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
