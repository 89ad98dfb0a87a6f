// Grouped step engine of the serving loop: small requests advance together, one core update
// (Alg. 2 for one mode n) per request per step, as one captured graph of grouped kernels over a
// device table of the active slots.
#pragma once

#include <string>
#include <vector>

#include "trals_internal.cuh"

namespace trals {

constexpr int kGrpMaxSlots = 64;   // requests in one step
constexpr int kGrpMaxOrder = 5;    // the Gamma chain of S_n (N - 2 products) is spread over three kernels
constexpr int kGrpMaxRank = 8;     // r = R_n R_{n+1} <= 64: S_n, L and a Gamma_k fit one CTA's shared memory

// Whether a request is served by the grouped engine: order 3..5, ranks <= 8, at most max_elems
// entries of FP32 X, the FP32 or BF16 mode with the Cholesky solve of the structured Gram chain, no
// per-sweep explicit residual, at least one sweep.
bool grp_eligible(int N, const int64_t* I, const int32_t* R, int xt, const trals_opts& o, int sweeps,
                  int64_t max_elems);
// Device bytes the engine holds for such a request (its workspace plus the copy of a host X).
size_t grp_footprint(int N, const int64_t* I, const int32_t* R, int mode, bool x_on_host);

struct GroupEngine;

// Create the engine on `device` (its own stream, graph and pinned tables).  On failure returns null and
// sets *err.
GroupEngine* grp_create(int device, std::string* err);
void grp_destroy(GroupEngine* e);
int grp_free_slots(const GroupEngine* e);
// Admit a request into a free slot: allocates its workspace on the engine's stream and enqueues the
// copies of its initial cores (and of X when X is on the host); the request starts with the next
// step.  X (FP32, I_0 fastest) must stay valid until the request is collected.  Returns the slot id,
// or -1 with *err set.
int grp_admit(GroupEngine* e, int N, const int64_t* I, const int32_t* R, const float* X, bool x_on_host, int mode,
              int sweeps, const double* const* init_cores, std::string* err);
// Launch the next step when there is work and fewer than two steps are in flight; returns true if
// one was launched, false otherwise (*err set on a CUDA failure).
bool grp_step(GroupEngine* e, std::string* err);
// Slots whose requests are done (results in the slot's pinned buffers).
void grp_poll(GroupEngine* e, std::vector<int>* done);
// Results of a done slot: status code (trals_status), message, cores (concatenated, FP64), relative
// residual after the last sweep.
int grp_result(GroupEngine* e, int slot, const double** cores, double* rel_res, std::string* msg);
// Release a done slot (frees its workspace, stream-ordered).
void grp_release(GroupEngine* e, int slot);
// True while any slot is active or draining.
bool grp_busy(const GroupEngine* e);
// Steps launched so far.
uint64_t grp_steps(const GroupEngine* e);
// Testing: the next `steps` steps are launched without their descriptor table being published, and
// the step's bounded wait for it gives up after spin_cycles clock cycles; the requests in those steps
// report TRALS_E_TIMEOUT.
void grp_withhold(GroupEngine* e, int steps, long long spin_cycles);

}  // namespace trals
