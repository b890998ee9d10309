// msts_noalloc.cu -- the safe multi-shift solve with its scratch memory in a
// fixed, library-owned device array instead of a caller-provided workspace.
//
// Who this is for: callers that cannot allocate device memory at the point
// where they need the solve.  cudaMalloc synchronises the whole device and can
// fail at run time, so code with a fixed memory budget (long-running services,
// plug-ins whose host framework owns every allocation, callers running on a
// schedule that must not stall the device) often may not call it, or any
// routine that calls it.  msts_solve needs scratch for the per-column bounds
// and exponents of Alg. 5; this variant takes that scratch from a static
// __device__ array, so the call itself allocates nothing.  The caller still
// provides U, the shifts, B, scales, scale_exp and (optionally) status.
//
// Cost of the array: every GPU that loads this library holds
// kStaticScratchBytes of device memory until the process exits.
#include <mutex>

#include "../../include/msts.h"
#include "msts_check.h"
#include "msts_engine.h"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};   // device address of g_static_scratch, per device

// The name g_static_scratch in host code is only a host-side stand-in for the
// device array; its device address must be looked up, once per device, with
// that device current.
int scratch_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MSTS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return MSTS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return MSTS_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return 0;
}

}  // namespace

extern "C" int msts_safe_solve_static(const msts_z *U, int64_t ldu, int64_t m,
                                      const msts_z *shifts, int64_t n, msts_z *B, int64_t ldb,
                                      double *scales, int32_t *scale_exp, int32_t nb,
                                      uint32_t *status, void *stream) {
  const int64_t kMaxDim = (int64_t)1 << 30;
  if (m < 0 || m > kMaxDim) return -3;
  if (m > 0 && !U) return -1;
  if (ldu < (m > 1 ? m : 1)) return -2;
  if (n < 0 || n > kMaxDim) return -5;
  if (n > 0 && !shifts) return -4;
  if (m > 0 && n > 0 && !B) return -6;
  if (ldb < (m > 1 ? m : 1)) return -7;
  if (n > 0 && !scales) return -8;
  if (n > 0 && !scale_exp) return -9;
  if (nb != 16 && nb != 32 && nb != 64) return -10;
  const size_t need = msts_solve_workspace_size(m, n, nb, MSTS_SAFE);
  if (msts::bad_alignment({U, shifts, B}, nullptr)) return MSTS_ERR_ALIGN;
  if (need > kStaticScratchBytes) return MSTS_ERR_STATIC_SCRATCH;
  if (m == 0 || n == 0) return 0;
  void *scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != 0) return rc;
  msts::EngineProblem p{};
  p.U = reinterpret_cast<const double2 *>(U);
  p.ldu = ldu;
  p.m = (int)m;
  p.shifts = reinterpret_cast<const double2 *>(shifts);
  p.shift_stride = 1;
  p.n = (int)n;
  p.B = reinterpret_cast<double2 *>(B);
  p.ldb = ldb;
  p.scales = scales;
  p.scale_exp = scale_exp;
  const cudaError_t e = msts::engine_run(&p, 1, nb, true, false, false, scratch, status,
                                         static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? 0 : MSTS_ERR_CUDA;
}
