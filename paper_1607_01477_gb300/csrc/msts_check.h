// msts_check.h -- host-side pointer alignment check of the C entry points.
#pragma once
#include <stdint.h>

#include <initializer_list>

namespace msts {
// True when a complex array is not 16-byte aligned (the kernels move complex
// values as 16-byte vectors) or the workspace is not 256-byte aligned.  NULL
// passes: the entry points check missing arrays themselves.
inline bool bad_alignment(std::initializer_list<const void *> complex_arrays, const void *workspace) {
  for (const void *p : complex_arrays)
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return true;
  return reinterpret_cast<uintptr_t>(workspace) % 256 != 0;
}
}  // namespace msts
