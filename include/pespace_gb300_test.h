/* pespace_gb300_test.h -- entry points of the TEST BUILD of the library only
 * (paper_2602_12011_gb300/lib/libpespace_gb300_test.so, compiled with -DPE_FAULT_INJECTION
 * -DPE_CHECKED); the product library libpespace_gb300.so does not export them. They make the
 * library's failure handling testable without faulting a GPU. No counterpart in the paper.
 *
 * Fault injection (host side). Every device allocation, host-to-device upload and kernel
 * launch-status read of the library is an event of its kind (0 allocation, 1 upload, 2 launch).
 *   pe_test_fault_arm(kind, nth): reset the event counts; the nth event of `kind` from now (1-based)
 *     fails instead of doing its work -- an allocation returns out-of-memory and allocates nothing,
 *     an upload copies nothing, a launch has run and only its status reads as failed. nth = 0 (or
 *     kind = -1) disarms and only counts. PE_EINVAL outside kind -1..2, nth >= 0. The environment
 *     variable PE_FAULT = "alloc[:n]", "upload[:n]" or "launch[:n]", read once, arms the same way
 *     at the first event.
 *   pe_test_fault_count(kind): events of that kind since the last arm (-1 for a bad kind).
 *   pe_test_fault_fired(): armed faults that have fired since the last arm.
 *   pe_test_live_allocations(): device allocations the library holds now (handles, scratch not
 *     yet released; stream-ordered frees count when they are enqueued).
 * Index checks (device side). In this build the log-likelihood, gradient and Fisher kernels test
 * the indices they derive from the work lists (pair index, partial-sum range, bin count against
 * the grid); a failing check skips the access and ORs a code into an error word.
 *   pe_test_checked_take(): the OR of the codes since the last call (0 none, -1 unreadable),
 *     cleared when read. Synchronous. */
#ifndef PESPACE_GB300_TEST_H
#define PESPACE_GB300_TEST_H
#include "pespace_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

pe_status pe_test_fault_arm(int kind, long nth);
long pe_test_fault_count(int kind);
long pe_test_fault_fired(void);
long pe_test_live_allocations(void);
int pe_test_checked_take(void);

#ifdef __cplusplus
}
#endif
#endif /* PESPACE_GB300_TEST_H */
