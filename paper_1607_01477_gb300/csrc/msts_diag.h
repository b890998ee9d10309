// msts_diag.h -- internal launcher of the diagonal-block step (msts_diag.cu).
#pragma once
#include <cuda_runtime.h>

#include "msts_common.cuh"

namespace msts {
// Lanes per shift for a launch over `total_cols` shifts (all problems).
int diag_lanes(int nb, long long total_cols, bool safe);
// Launches the diagonal-block step of block step `step` for every problem of
// `tab`; ncols_max is the largest number of active shifts of one problem.
// gen: generalized problems (every problem of the table has V).
cudaError_t launch_diag(const ProbTable &tab, int nb, bool safe, bool conj, int step, int shortcut,
                        int ncols_max, long long total_cols, uint32_t *status, cudaStream_t st,
                        bool gen = false);
}  // namespace msts
