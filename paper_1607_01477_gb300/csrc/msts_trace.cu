// msts_trace.cu -- launch counting and per-kernel CUDA-event timing.
//
// Every kernel launch of the library bumps a process-wide counter.  Between
// msts_trace_begin() and msts_trace_end() the launches of the hot kernels
// (the substitution GEMM on either path, the diagonal-block solve, the
// tensor-core residual and the Lanczos step) are also bracketed by
// CUDA events on the launching stream, together with the algorithmic work of
// each launch, so that a caller can compute achieved FLOP/s per kernel.
#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/msts.h"
#include "msts_trace.h"

namespace msts {

namespace {
std::atomic<unsigned long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
long long g_cap = 0;
struct Rec { int kernel; cudaEvent_t a, b; double flops, bytes; };
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;   // 2 x capacity events, created by msts_trace_begin
struct Tot { double ms = 0, flops = 0, bytes = 0; long long n = 0; };
Tot g_tot[kTraceKernels];
}  // namespace

void count_launches(int n) { g_launches.fetch_add((unsigned long long)n); }

bool trace_on() { return g_on; }

void *trace_start(int kernel, double flops, double bytes, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || (long long)g_recs.size() >= g_cap) return nullptr;
  const size_t k = g_recs.size();
  Rec r{kernel, g_pool[2 * k], g_pool[2 * k + 1], flops, bytes};
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  return &g_recs.back();
}

void trace_stop(void *h, cudaStream_t st) {
  if (!h) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(static_cast<Rec *>(h)->b, st);
}

}  // namespace msts

extern "C" {

uint64_t msts_launch_count(void) { return msts::g_launches.load(); }

int msts_trace_begin(int64_t capacity) {
  std::lock_guard<std::mutex> lk(msts::g_mu);
  if (capacity < 0 || capacity > (1 << 22)) return -1;
  msts::g_recs.clear();
  msts::g_recs.reserve((size_t)capacity);   // pointers handed out stay valid
  // the events are created here, outside the traced region
  while (msts::g_pool.size() < 2 * (size_t)capacity) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return MSTS_ERR_CUDA;
    msts::g_pool.push_back(e);
  }
  for (auto &t : msts::g_tot) t = msts::Tot{};
  msts::g_cap = capacity;
  msts::g_on = true;
  return 0;
}

int msts_trace_end(void) {
  std::lock_guard<std::mutex> lk(msts::g_mu);
  msts::g_on = false;
  int rc = 0;
  for (auto &r : msts::g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) rc = MSTS_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) rc = MSTS_ERR_CUDA;
    auto &t = msts::g_tot[r.kernel];
    t.ms += ms; t.flops += r.flops; t.bytes += r.bytes; t.n += 1;
  }
  msts::g_recs.clear();
  for (cudaEvent_t e : msts::g_pool) cudaEventDestroy(e);   // outside the traced region too
  msts::g_pool.clear();
  return rc;
}

int msts_trace_query(int32_t kernel, double *total_ms, int64_t *launches, double *flops,
                     double *bytes) {
  if (kernel < 0 || kernel >= msts::kTraceKernels) return -1;
  std::lock_guard<std::mutex> lk(msts::g_mu);
  const auto &t = msts::g_tot[kernel];
  if (total_ms) *total_ms = t.ms;
  if (launches) *launches = t.n;
  if (flops) *flops = t.flops;
  if (bytes) *bytes = t.bytes;
  return 0;
}

}  // extern "C"
