// pe_plan.h -- autotuner and tuning cache shared by pe_plan.cu and the direct entry points.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "pe_internal.h"

namespace pe {

struct TuneChoice {
  int variant;      // forward-kernel register-budget variant (0..kFwdVariants-1)
  int ctas_per_sm;  // persistent grid = SMs x ctas_per_sm CTAs
  int subtiles;     // 128-bin sub-tiles per work item (1, 2, 4, 8)
  double ms;        // measured forward-kernel time of the choice (0 for the default)
};

std::string tune_key(const DetSet& ds, int B, unsigned mask);
bool lookup_tuned(const DetSet& ds, int B, unsigned mask, TuneChoice* out);
TuneChoice default_choice(int prec);
int grid_for(const TuneChoice& c, long long max_tiles);
// Times the candidates on the prepared work list (coefficients, active counts and sub-tile offsets
// off on the device; offi: scratch for the work-item offsets, P + 1 entries) and returns the fastest.
cudaError_t autotune_fwd(const DetSet& ds, int B, unsigned mask, const SampleCoef* coef, const int* nend,
                         const long long* off, long long* offi, double* part, long long max_tiles, cudaStream_t st,
                         TuneChoice* best);
void store_tuned(const DetSet& ds, int B, unsigned mask, const TuneChoice& c);

}  // namespace pe
