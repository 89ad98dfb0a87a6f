// Tensor-core (tcgen05) MTTSP for the reduced-precision modes: interface used by the sweep driver.
#pragma once

#include "trals_internal.cuh"

namespace trals {

// Per-mode plan of the tensor-core MTTSP.  Owns its device workspace.
struct TcPlan {
  bool valid = false;
  int N = 0, n = 0, mode = 0;
  std::vector<void*> allocs;    // stream-ordered allocations on `stream`
  cudaStream_t stream = nullptr;
  size_t bytes = 0;             // device workspace held
  void* impl = nullptr;
};

// Geometry the tensor-core MTTSP would use for mode n (host only; variant -1 = not supported):
// 0 = K-major X with the factor on the left, 1 = K-major X with the factor on the right,
// 2 = MN-major X with the factor on the right, 3 = MN-major X with the factor on the left (mode 0).
// S = modes [s_lo, s_hi] is contracted on the tensor cores.
struct TcChoice {
  int variant = -1;
  int s_lo = 0, s_hi = 0;
  int64_t K_S = 0;
  int64_t cost = 0;
};
TcChoice tc_choose(int N, const int64_t* I, const int32_t* R, int n);

// Prepare the tensor-core MTTSP of mode n for X (element type implied by `mode`).  Returns 1 when
// the shape is supported (then tc_enqueue is used), 0 otherwise (the caller falls back to the
// CUDA-core MTTSP).  *err is set on a CUDA failure.  Workspace is allocated stream-ordered on s.
// With count_bytes set nothing is allocated: the workspace bytes are added to *count_bytes.
// I are the extents of X as stored; I0_real (0: I[0]) is the true extent of mode 0 when X is stored
// with mode 0 zero-padded to I[0] (the rows of M_0 beyond it are dropped).
// In the bf16x3 mode Xlo is the lo plane of the split-BF16 X (same layout as X).  The grid leaves
// free_sms SMs free for concurrent work (the coefficient branch of the sweep).
int tc_plan(TcPlan& p, int N, const int64_t* I, const int32_t* R, int n, int mode, const void* X, int64_t numel,
            cudaError_t* err, cudaStream_t s = nullptr, size_t* count_bytes = nullptr, int64_t I0_real = 0,
            const void* Xlo = nullptr, int free_sms = 1);
// Enqueue M_n (FP64, I_n x R_n R_{n+1}) on stream s; returns the number of kernel launches.  When
// given, ev0/ev1 are recorded on s directly before and after the main contraction kernel.
int tc_enqueue(TcPlan& p, const void* X, double* const* cores, double* M, cudaStream_t s, cudaEvent_t ev0 = nullptr,
               cudaEvent_t ev1 = nullptr);
// tc_enqueue in two parts.  The core of the mode before p.n (the one a sweep updates just before this
// MTTSP) ends one of the two subchain products.  tc_enqueue_pre builds everything that does not read
// it (so it may run while that core is being updated, on another stream); tc_enqueue_main builds the
// last link from that core, then runs the MTTSP and its reduction.  Both return their launch counts.
// c32 (optional): FP32 copies of the cores kept by the caller, laid out as launch_cores_to_f32 writes
// them; without it, tc_enqueue_pre converts the cores into the plan's own copy (all of them, so the
// two parts must then see the same cores).
int tc_enqueue_pre(TcPlan& p, double* const* cores, cudaStream_t s, const float* const* c32 = nullptr);
// before_kernel (optional): an event the MTTSP kernel itself waits for.  Its persistent CTAs fill every
// SM but one, so work that must not be squeezed onto that SM is better finished first.
int tc_enqueue_main(TcPlan& p, double* const* cores, double* M, cudaStream_t s, cudaEvent_t ev0 = nullptr,
                    cudaEvent_t ev1 = nullptr, const float* const* c32 = nullptr,
                    cudaEvent_t before_kernel = nullptr);
// FP32 copies of all N cores into dst, concatenated in order; core j holds R_j x Ist[j] x R_{j+1} values,
// the slices of core 0 from I0real to Ist[0] zero (a zero-padded leading mode of the BF16 copy of X).
void launch_cores_to_f32(double* const* cores, int N, const int32_t* R, const int64_t* Ist, int64_t I0real,
                         float* dst, cudaStream_t s);
void tc_destroy(TcPlan& p);
// Geometry of a valid plan (0 KM-L, 1 KM-R, 2 MM, 3 MM-L), -1 if none.
int tc_variant(const TcPlan& p);
// Device status word the kernel reports a bounded-wait timeout into.
void tc_set_status(TcPlan& p, DevStatus* st);
// Fault injection for tests: with withhold_first_copy set, the producer of every CTA skips the first
// copy of its first unit, so the MMA issuer's wait for it gives up after spin_limit_cycles clock cycles
// (<= 0: the default of about 2 s); the kernel then stops every role, drains the copies it did issue,
// frees its tensor memory and reports TRALS_E_TIMEOUT in the status word.
void tc_set_fault(TcPlan& p, int withhold_first_copy, long long spin_limit_cycles);
cudaError_t init_tc_attributes();

}  // namespace trals
