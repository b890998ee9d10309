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
// The four-warp layout of the step (msts_diagw.cu; n_b = 32, standard
// problems): `lanes` = 1, 2 or 4 lanes per shift.
cudaError_t launch_diagw(const ProbTable &tab, bool safe, bool conj, int step, int shortcut, int ncols_max,
                         int lanes, uint32_t *status, cudaStream_t st);
// Lanes per shift of the four-warp layout for a launch over total_cols
// shifts, or 0 where the one-warp layout is faster.
int diagw_lanes(long long total_cols, bool safe);
// Tuning override (0 = automatic): lanes per shift of every four-warp launch,
// or -1 to take the one-warp layout for n_b = 32 as well.
void set_diag_override(int lanes);
// Tuning knob of the four-warp layout: 1 takes Alg. 4's decisions by the
// serial chain in every block (the one-warp layout's flag is in msts_diag.cu).
cudaError_t set_alg4_chain_w(int on);
}  // namespace msts
