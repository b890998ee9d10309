// msts_adjoint.cu -- reverse-mode derivative of X = (U - s_j I)^{-1} B(:,j)
// (not in the paper).  For a real loss with complex gradient
// GX = dL/dRe X + i dL/dIm X:
//   Lambda(:,j) = (U - s_j I)^{-H} GX(:,j)    -- a conjugate-transposed
//                                               multi-shift solve (engine)
//   dB = Lambda,  dU = -triu(Lambda X^H),  ds_j = X(:,j)^H Lambda(:,j),
// from dx_j = (U - s_j I)^{-1}(db_j - dU x_j + ds_j x_j).  X is not an input:
// it is recomputed by a forward multi-shift solve into the workspace.
#include <algorithm>
#include <vector>

#include "msts_check.h"
#include "msts_common.cuh"
#include "msts_engine.h"
#include "msts_ozaki.h"
#include "msts_trace.h"

namespace msts {

struct AdjProb {
  const double2 *L; long long ldl;   // Lambda (= dB)
  const double2 *X; long long ldx;   // recomputed solution
  double2 *dU; long long lddu;
  double2 *ds;
  int m, n;
};
struct AdjTable {
  int count;
  AdjProb p[kMaxProbs];
};

constexpr int kTBM = 64, kTBN = 32, kTKC = 16, kTThreads = 256;

// Copies B -> X and GX -> dB for every problem (grid.z = problem).
struct CopyProb { const double2 *src; long long lds; double2 *dst; long long ldd; int m, n; };
struct CopyTable { int count; CopyProb p[2 * kMaxProbs]; };

__global__ void k_copy_cols(const __grid_constant__ CopyTable tab) {
  const CopyProb &c = tab.p[blockIdx.z];
  const int j = blockIdx.y;
  if (j >= c.n) return;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < c.m; r += gridDim.x * blockDim.x)
    c.dst[r + (long long)j * c.ldd] = c.src[r + (long long)j * c.lds];
}

// dU(r, c) = -sum_j Lambda(r, j) conj(X(c, j)) for r <= c, zero for r > c.
__global__ void __launch_bounds__(kTThreads) k_triu_gemm(const __grid_constant__ AdjTable tab) {
  __shared__ double2 sL[kTKC][kTBM + 1];
  __shared__ double2 sX[kTKC][kTBN + 1];
  const AdjProb &P = tab.p[blockIdx.z];
  const int r0 = blockIdx.y * kTBM, c0 = blockIdx.x * kTBN;
  if (r0 >= P.m || c0 >= P.m) return;
  const int tid = threadIdx.x, tr = tid & 31, tc = tid >> 5;
  double2 acc[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = make_double2(0.0, 0.0);
  const bool below = r0 > c0 + kTBN - 1;   // tile entirely below the diagonal
  if (!below) {
    for (int j0 = 0; j0 < P.n; j0 += kTKC) {
      for (int idx = tid; idx < kTKC * kTBM; idx += kTThreads) {
        const int j = idx / kTBM, r = idx - j * kTBM;
        sL[j][r] = (j0 + j < P.n && r0 + r < P.m) ? P.L[(r0 + r) + (long long)(j0 + j) * P.ldl]
                                                  : make_double2(0.0, 0.0);
      }
      for (int idx = tid; idx < kTKC * kTBN; idx += kTThreads) {
        const int j = idx / kTBN, c = idx - j * kTBN;
        sX[j][c] = (j0 + j < P.n && c0 + c < P.m) ? P.X[(c0 + c) + (long long)(j0 + j) * P.ldx]
                                                  : make_double2(0.0, 0.0);
      }
      __syncthreads();
#pragma unroll 4
      for (int j = 0; j < kTKC; ++j) {
        const double2 l0 = sL[j][tr], l1 = sL[j][tr + 32];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double2 xc = zconj(sX[j][tc + 8 * c]);
          acc[0][c] = zfma(acc[0][c], l0, xc);
          acc[1][c] = zfma(acc[1][c], l1, xc);
        }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int col = c0 + tc + 8 * c;
    if (col >= P.m) continue;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int row = r0 + tr + 32 * i;
      if (row >= P.m) continue;
      P.dU[row + (long long)col * P.lddu] =
          row <= col ? make_double2(-acc[i][c].x, -acc[i][c].y) : make_double2(0.0, 0.0);
    }
  }
}

// ds_j = X(:,j)^H Lambda(:,j): one warp per column.
__global__ void k_ds(const __grid_constant__ AdjTable tab) {
  const AdjProb &P = tab.p[blockIdx.z];
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= P.n) return;
  double2 s = make_double2(0.0, 0.0);
  for (int r = lane; r < P.m; r += 32)
    s = zfma_cj(s, P.X[r + (long long)j * P.ldx], P.L[r + (long long)j * P.ldl]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
  }
  if (lane == 0) P.ds[j] = s;
}

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// X per problem, then (tensor) the digit-plane plans of U for the forward
// solve and of U^H for the adjoint solve.
size_t adjoint_workspace_bytes(const msts_adjoint_problem *probs, int64_t batch, int nb, bool tensor) {
  size_t s = 0;
  for (int64_t i = 0; i < batch; ++i) {
    s += a256(sizeof(double2) * (size_t)probs[i].m * probs[i].n);
    if (tensor && probs[i].m > 0 && probs[i].n > 0) s += 2 * a256(ozaki_plan_bytes((int)probs[i].m, (int)probs[i].n, nb));
    if (tensor && probs[i].m > 0) s += a256(ozaki_neg_triu_bytes((int)probs[i].m, (int)probs[i].n));
  }
  return s;
}

cudaError_t adjoint_run(const msts_adjoint_problem *probs, int64_t batch, int nb, void *ws,
                        uint32_t *status, cudaStream_t st, bool tensor) {
  char *cur = static_cast<char *>(ws);
  std::vector<OzPlan> plans(tensor ? 2 * (size_t)std::min<int64_t>(batch, kMaxProbs) : 0);
  for (int64_t base = 0; base < batch; base += kMaxProbs) {
    const int cnt = (int)std::min<int64_t>(kMaxProbs, batch - base);
    std::vector<EngineProblem> fwd(cnt), adj(cnt);
    CopyTable ct;
    ct.count = 2 * cnt;
    AdjTable at;
    at.count = cnt;
    int maxm = 0, maxn = 0;
    std::vector<OzPlanSrc> src;                // the U planes of the chunk, prepared in one launch each way
    for (int i = 0; i < cnt; ++i) {
      const msts_adjoint_problem &q = probs[base + i];
      double2 *X = reinterpret_cast<double2 *>(cur);
      cur += a256(sizeof(double2) * (size_t)q.m * q.n);
      const long long ldx = std::max<long long>(1, q.m);
      ct.p[2 * i] = CopyProb{reinterpret_cast<const double2 *>(q.B), q.ldb, X, ldx, (int)q.m, (int)q.n};
      ct.p[2 * i + 1] = CopyProb{reinterpret_cast<const double2 *>(q.GX), q.ldg,
                                 reinterpret_cast<double2 *>(q.dB), q.lddb, (int)q.m, (int)q.n};
      EngineProblem e{};
      e.U = reinterpret_cast<const double2 *>(q.U); e.ldu = q.ldu; e.m = (int)q.m;
      e.shifts = reinterpret_cast<const double2 *>(q.shifts); e.shift_stride = 1; e.n = (int)q.n;
      e.B = X; e.ldb = ldx;
      fwd[i] = e;
      e.B = reinterpret_cast<double2 *>(q.dB); e.ldb = q.lddb;
      adj[i] = e;
      at.p[i] = AdjProb{reinterpret_cast<const double2 *>(q.dB), q.lddb, X, ldx,
                        reinterpret_cast<double2 *>(q.dU), q.lddu, reinterpret_cast<double2 *>(q.ds),
                        (int)q.m, (int)q.n};
      if (tensor && q.m > 0 && q.n > 0) {
        const size_t pb = a256(ozaki_plan_bytes((int)q.m, (int)q.n, nb));
        cudaError_t e = ozaki_plan_init(&plans[2 * i], (int)q.m, (int)q.n, nb, false, cur);
        if (e != cudaSuccess) return e;
        cur += pb;
        e = ozaki_plan_init(&plans[2 * i + 1], (int)q.m, (int)q.n, nb, true, cur);
        if (e != cudaSuccess) return e;
        cur += pb;
        src.push_back(OzPlanSrc{&plans[2 * i], fwd[i].U, q.ldu});
        src.push_back(OzPlanSrc{&plans[2 * i + 1], fwd[i].U, q.ldu});
        fwd[i].oz = &plans[2 * i];
        adj[i].oz = &plans[2 * i + 1];
      }
      maxm = std::max<int>(maxm, (int)q.m);
      maxn = std::max<int>(maxn, (int)q.n);
    }
    if (maxm == 0) continue;
    if (!src.empty()) {
      const cudaError_t e = ozaki_plans_prepare(src.data(), (int)src.size(), st);
      if (e != cudaSuccess) return e;
    }
    if (maxn > 0) {
      k_copy_cols<<<dim3(std::max(1, std::min(16, (maxm + 255) / 256)), maxn, 2 * cnt), 256, 0, st>>>(ct);
      cudaError_t e = engine_run(fwd.data(), cnt, nb, false, false, false, nullptr, status, st);
      if (e != cudaSuccess) return e;
      e = engine_run(adj.data(), cnt, nb, false, true, false, nullptr, status, st);
      if (e != cudaSuccess) return e;
      k_ds<<<dim3((maxn + 7) / 8, 1, cnt), 256, 0, st>>>(at);
      count_launches(2);
    }
    if (tensor) {                              // dU = -triu(Lambda X^H) on the tensor cores
      OzNegTriuItem it[kMaxProbs];
      size_t bytes = 0;
      for (int i = 0; i < cnt; ++i) {
        const AdjProb &P = at.p[i];
        it[i] = OzNegTriuItem{P.L, P.ldl, P.X, P.ldx, P.dU, P.lddu, P.m, P.n};
        if (P.m > 0) bytes += a256(ozaki_neg_triu_bytes(P.m, P.n));
      }
      const cudaError_t e = ozaki_neg_triu_batched(it, cnt, cur, status, st);
      if (e != cudaSuccess) return e;
      cur += bytes;
    } else {
      k_triu_gemm<<<dim3((maxm + kTBN - 1) / kTBN, (maxm + kTBM - 1) / kTBM, cnt), kTThreads, 0, st>>>(at);
      count_launches(1);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace msts

extern "C" {

size_t msts_adjoint_batched_flags_workspace_size(const msts_adjoint_problem *probs, int64_t batch,
                                                 int32_t nb, uint32_t flags) {
  if (!probs || batch < 0 || (nb != 16 && nb != 32 && nb != 64)) return 0;
  if ((flags & ~(uint32_t)MSTS_TENSOR_GEMM) != 0) return 0;
  return msts::adjoint_workspace_bytes(probs, batch, nb, (flags & MSTS_TENSOR_GEMM) != 0);
}

size_t msts_adjoint_batched_workspace_size(const msts_adjoint_problem *probs, int64_t batch,
                                           int32_t nb) {
  return msts_adjoint_batched_flags_workspace_size(probs, batch, nb, 0);
}

int msts_adjoint_batched(const msts_adjoint_problem *probs, int64_t batch, int32_t nb,
                         void *workspace, size_t workspace_bytes, uint32_t *status, void *stream) {
  return msts_adjoint_batched_flags(probs, batch, nb, workspace, workspace_bytes, status, 0, stream);
}

int msts_adjoint_batched_flags(const msts_adjoint_problem *probs, int64_t batch, int32_t nb,
                               void *workspace, size_t workspace_bytes, uint32_t *status, uint32_t flags,
                               void *stream) {
  const int64_t kMax = (int64_t)1 << 30;
  if (batch < 0 || batch > kMax) return -2;
  if (batch > 0 && !probs) return -1;
  if (nb != 16 && nb != 32 && nb != 64) return -3;
  if ((flags & ~(uint32_t)MSTS_TENSOR_GEMM) != 0) return -8;
  for (int64_t i = 0; i < batch; ++i) {
    const msts_adjoint_problem &q = probs[i];
    const int64_t mm = q.m > 1 ? q.m : 1;
    if (q.m < 0 || q.m > kMax || q.n < 0 || q.n > kMax) return -1;
    if (q.ldu < mm || q.ldb < mm || q.ldg < mm || q.lddu < mm || q.lddb < mm) return -1;
    if (q.m > 0 && (!q.U || !q.dU)) return -1;
    if (q.n > 0 && (!q.shifts || !q.ds)) return -1;
    if (q.m > 0 && q.n > 0 && (!q.B || !q.GX || !q.dB)) return -1;
    if (msts::bad_alignment({q.U, q.shifts, q.B, q.GX, q.dU, q.dB, q.ds}, nullptr)) return MSTS_ERR_ALIGN;
  }
  const bool tensor = (flags & MSTS_TENSOR_GEMM) != 0;
  const size_t need = msts::adjoint_workspace_bytes(probs, batch, nb, tensor);
  if (need > 0 && (!workspace || workspace_bytes < need)) return workspace ? -5 : -4;
  if (msts::bad_alignment({}, workspace)) return MSTS_ERR_ALIGN;
  if (batch == 0) return 0;
  const cudaError_t e = msts::adjoint_run(probs, batch, nb, workspace, status,
                                          static_cast<cudaStream_t>(stream), tensor);
  return e == cudaSuccess ? 0 : MSTS_ERR_CUDA;
}

size_t msts_adjoint_workspace_size(int64_t m, int64_t n, int32_t nb) {
  msts_adjoint_problem q{};
  q.m = m; q.n = n;
  if (m < 0 || n < 0) return 0;
  return msts_adjoint_batched_workspace_size(&q, 1, nb);
}

int msts_adjoint(const msts_z *U, int64_t ldu, int64_t m, const msts_z *shifts, int64_t n,
                 const msts_z *B, int64_t ldb, const msts_z *GX, int64_t ldg, msts_z *dU,
                 int64_t lddu, msts_z *dB, int64_t lddb, msts_z *ds, int32_t nb, void *workspace,
                 size_t workspace_bytes, uint32_t *status, void *stream) {
  if (m < 0) return -3;
  if (n < 0) return -5;
  msts_adjoint_problem q{U, ldu, m, shifts, n, B, ldb, GX, ldg, dU, lddu, dB, lddb, ds};
  const int rc = msts_adjoint_batched(&q, 1, nb, workspace, workspace_bytes, status, stream);
  return rc == -1 ? -1 : rc;
}

}  // extern "C"
