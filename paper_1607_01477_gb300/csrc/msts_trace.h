// msts_trace.h -- internal hooks for launch counting and kernel timing.
#pragma once
#include <cuda_runtime.h>

namespace msts {
constexpr int kTraceKernels = 5;   // MSTS_KERNEL_GEMM, _DIAG, _OZAKI, _RESIDUAL, _LANCZOS
void count_launches(int n);
bool trace_on();
// Records a start event on `st` for one launch of `kernel` doing `flops`
// algorithmic FLOPs over `bytes` algorithmic bytes; returns a handle or null.
void *trace_start(int kernel, double flops, double bytes, cudaStream_t st);
void trace_stop(void *h, cudaStream_t st);
}  // namespace msts
