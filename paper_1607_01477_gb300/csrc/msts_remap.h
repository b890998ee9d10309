// msts_remap.h -- exact permutation/conjugation copies of column-major
// complex matrices (used by the triangular variants and the 1-norm
// pseudospectra).
#pragma once
#include <cuda_runtime.h>

namespace msts {
// dst(r, c) = [conj] src(p, q) for r < rows, c < cols, where
//   r' = rev_r ? rows-1-r : r,  c' = rev_c ? cols-1-c : c,
//   (p, q) = tr ? (c', r') : (r', c');
// with `upper`, only r <= c is written.  dst must not alias src.
cudaError_t remap(const double2 *src, long long lds, double2 *dst, long long ldd, int rows, int cols, bool tr,
                  bool rev_r, bool rev_c, bool conj, bool upper, cudaStream_t st);
}  // namespace msts
