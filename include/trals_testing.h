/*
 * trals_testing.h -- fault-injection hooks of libtrals for tests.  None is a step of the method (the
 * paper has no counterpart); they exist so that error paths the kernels guard against can be exercised
 * without faulting, trapping or hanging a GPU.
 */
#ifndef TRALS_TESTING_H
#define TRALS_TESTING_H

#include "trals.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Runs the tensor-core MTTSP of mode n (BF16 mode; arguments and layouts as trals_mttsp, X_dev BF16) with
 * a copy withheld: in every CTA the TMA producer never issues the first copy of its first unit, and every
 * bounded mbarrier wait of the kernel gives up after spin_cycles clock cycles (> 0; 2e6 is about 1 ms).
 * The MMA issuer's wait for the missing copy therefore runs out: the kernel raises its abort flag, every
 * role leaves its loop, the copies that were issued are waited for (bounded), the tensor memory is freed
 * and TRALS_E_TIMEOUT is written to the device status word, which this call returns (the message of
 * trals_last_error names the wait).  The context stays usable.  M_dev receives no defined values.
 * TRALS_E_ARG for invalid shapes or when the mode has no tensor-core geometry.  Synchronous. */
trals_status trals_testing_mttsp_withheld_copy(trals_ctx* ctx, int N, const int64_t* I, const int32_t* R,
                                               const void* X_dev, int mode, const double* const* cores_dev, int n,
                                               double* M_dev, long long spin_cycles);

/* The next `steps` steps of the server's grouped step engine are launched without their descriptor table
 * being published: the step's first kernel waits for it, gives up after spin_cycles clock cycles (> 0),
 * and the step then does no work.  Every request that was in one of those steps completes with
 * TRALS_E_TIMEOUT (its result names the wait); later requests are served normally.  TRALS_E_ARG for a
 * null server, steps < 0 or spin_cycles <= 0. */
trals_status trals_testing_server_withhold_steps(trals_server* server, int steps, long long spin_cycles);

#ifdef __cplusplus
}
#endif
#endif /* TRALS_TESTING_H */
