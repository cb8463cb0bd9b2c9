// pe_measure.h -- internal hooks of the profiling helpers (pe_profile_enable / pe_profile_read).
#pragma once
#include <cuda_runtime.h>

namespace pe {
// Record a start event on st if profiling is on; *token is NULL otherwise.
void profile_begin(cudaStream_t st, void** token);
// Record the matching end event and keep the pair for pe_profile_read.
void profile_end(cudaStream_t st, void* token);
}  // namespace pe
