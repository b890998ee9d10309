// msts_abi.cu -- argument checking and the extern "C" entry points for the
// multi-shift solve, its batched form and TREVC (see include/msts.h).
#include <algorithm>
#include <vector>

#include "../../include/msts.h"
#include "msts_check.h"
#include "msts_engine.h"
#include "msts_ozaki.h"

namespace {

bool nb_ok(int32_t nb) { return nb == 16 || nb == 32 || nb == 64; }

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? 0 : MSTS_ERR_CUDA; }

msts::EngineProblem make_problem(const msts_z *U, int64_t ldu, int64_t m, const msts_z *shifts,
                                 int64_t shift_stride, int64_t n, msts_z *B, int64_t ldb,
                                 double *scales, int32_t *scale_exp, int diag_z) {
  msts::EngineProblem p;
  p.U = reinterpret_cast<const double2 *>(U);
  p.ldu = ldu;
  p.m = (int)m;
  p.shifts = reinterpret_cast<const double2 *>(shifts);
  p.shift_stride = shift_stride;
  p.n = (int)n;
  p.B = reinterpret_cast<double2 *>(B);
  p.ldb = ldb;
  p.scales = scales;
  p.scale_exp = scale_exp;
  p.diag_z = diag_z;
  p.oz = nullptr;
  return p;
}

constexpr int64_t kMaxDim = (int64_t)1 << 30;

}  // namespace

extern "C" {

int msts_version(void) { return 10000; }

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t msts_solve_workspace_size(int64_t m, int64_t n, int32_t nb, uint32_t flags) {
  if (m < 0 || n < 0 || !nb_ok(nb)) return 0;
  msts::EngineProblem p = make_problem(nullptr, 1, m, nullptr, 1, n, nullptr, 1, nullptr, nullptr, 0);
  size_t s = align256(msts::engine_workspace_bytes(&p, 1, nb, (flags & MSTS_SAFE) != 0));
  if ((flags & MSTS_TENSOR_GEMM) && m > 0 && n > 0) s += msts::ozaki_plan_bytes((int)m, (int)n, nb);
  return s;
}

int msts_solve(const msts_z *U, int64_t ldu, int64_t m, const msts_z *shifts, int64_t n,
               msts_z *B, int64_t ldb, double *scales, int32_t *scale_exp, int32_t nb,
               void *workspace, size_t workspace_bytes, uint32_t *status, uint32_t flags,
               void *stream) {
  const bool safe = (flags & MSTS_SAFE) != 0, conj = (flags & MSTS_CONJ_TRANS) != 0;
  if (m < 0 || m > kMaxDim) return -3;
  if (m > 0 && !U) return -1;
  if (ldu < std::max<int64_t>(1, m)) return -2;
  if (n < 0 || n > kMaxDim) return -5;
  if (n > 0 && !shifts) return -4;
  if (m > 0 && n > 0 && !B) return -6;
  if (ldb < std::max<int64_t>(1, m)) return -7;
  if (safe && n > 0 && (!scales || !scale_exp)) return scales ? -9 : -8;
  if (!nb_ok(nb)) return -10;
  if ((flags & ~(MSTS_SAFE | MSTS_CONJ_TRANS | MSTS_TENSOR_GEMM)) != 0 || (safe && conj)) return -14;
  const size_t need = msts_solve_workspace_size(m, n, nb, flags);
  if (need > 0 && (!workspace || workspace_bytes < need)) return workspace ? -12 : -11;
  if (msts::bad_alignment({U, shifts, B}, workspace)) return MSTS_ERR_ALIGN;
  if (m == 0 || n == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  msts::EngineProblem p = make_problem(U, ldu, m, shifts, 1, n, B, ldb, scales, scale_exp, 0);
  msts::OzPlan plan;
  char *ws = static_cast<char *>(workspace);
  if (flags & MSTS_TENSOR_GEMM) {
    const size_t eng = align256(msts::engine_workspace_bytes(&p, 1, nb, safe));
    if (msts::ozaki_plan_prepare(&plan, p.U, ldu, (int)m, (int)n, nb, conj, ws + eng, st) != cudaSuccess)
      return MSTS_ERR_CUDA;
    p.oz = &plan;
  }
  return cuda_rc(msts::engine_run(&p, 1, nb, safe, conj, false, workspace, status, st));
}

// Tensor-core plans of a batch: one per problem with work, after the engine's
// own workspace.
static size_t batched_plan_bytes(const msts_problem *probs, int64_t batch, int32_t nb) {
  size_t s = 0;
  for (int64_t i = 0; i < batch; ++i)
    if (probs[i].m > 0 && probs[i].n > 0) s += align256(msts::ozaki_plan_bytes((int)probs[i].m, (int)probs[i].n, nb));
  return s;
}

size_t msts_solve_batched_workspace_size(const msts_problem *probs, int64_t batch, int32_t nb,
                                         uint32_t flags) {
  if (!probs || batch < 0 || !nb_ok(nb)) return 0;
  std::vector<msts::EngineProblem> v;
  for (int64_t i = 0; i < batch; ++i)
    v.push_back(make_problem(nullptr, 1, probs[i].m, nullptr, 1, probs[i].n, nullptr, 1, nullptr,
                             nullptr, 0));
  size_t s = msts::engine_workspace_bytes(v.data(), (int)batch, nb, (flags & MSTS_SAFE) != 0);
  if (flags & MSTS_TENSOR_GEMM) s = align256(s) + batched_plan_bytes(probs, batch, nb);
  return s;
}

int msts_solve_batched(const msts_problem *probs, int64_t batch, int32_t nb, void *workspace,
                       size_t workspace_bytes, uint32_t *status, uint32_t flags, void *stream) {
  const bool safe = (flags & MSTS_SAFE) != 0, conj = (flags & MSTS_CONJ_TRANS) != 0;
  if (batch < 0 || batch > kMaxDim) return -2;
  if (batch > 0 && !probs) return -1;
  if (!nb_ok(nb)) return -3;
  if ((flags & ~(MSTS_SAFE | MSTS_CONJ_TRANS | MSTS_TENSOR_GEMM)) != 0 || (safe && conj)) return -7;
  std::vector<msts::EngineProblem> v;
  for (int64_t i = 0; i < batch; ++i) {
    const msts_problem &q = probs[i];
    if (q.m < 0 || q.m > kMaxDim || q.n < 0 || q.n > kMaxDim) return -1;
    if (q.ldu < std::max<int64_t>(1, q.m) || q.ldb < std::max<int64_t>(1, q.m)) return -1;
    if ((q.m > 0 && !q.U) || (q.n > 0 && !q.shifts) || (q.m > 0 && q.n > 0 && !q.B)) return -1;
    if (safe && q.n > 0 && (!q.scales || !q.scale_exp)) return -1;
    if (msts::bad_alignment({q.U, q.shifts, q.B}, nullptr)) return MSTS_ERR_ALIGN;
    v.push_back(make_problem(q.U, q.ldu, q.m, q.shifts, 1, q.n, q.B, q.ldb, q.scales,
                             q.scale_exp, 0));
  }
  const size_t need = msts_solve_batched_workspace_size(probs, batch, nb, flags);
  if (need > 0 && (!workspace || workspace_bytes < need)) return workspace ? -5 : -4;
  if (msts::bad_alignment({}, workspace)) return MSTS_ERR_ALIGN;
  if (batch == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<msts::OzPlan> plans;
  if (flags & MSTS_TENSOR_GEMM) {
    plans.resize((size_t)batch);
    char *cur = static_cast<char *>(workspace) + align256(msts::engine_workspace_bytes(v.data(), (int)batch, nb, safe));
    std::vector<msts::OzPlanSrc> src;
    for (int64_t i = 0; i < batch; ++i) {
      if (probs[i].m == 0 || probs[i].n == 0) continue;
      if (msts::ozaki_plan_init(&plans[(size_t)i], (int)probs[i].m, (int)probs[i].n, nb, conj, cur) != cudaSuccess)
        return MSTS_ERR_CUDA;
      src.push_back(msts::OzPlanSrc{&plans[(size_t)i], v[(size_t)i].U, probs[i].ldu});
      cur += align256(msts::ozaki_plan_bytes((int)probs[i].m, (int)probs[i].n, nb));
      v[(size_t)i].oz = &plans[(size_t)i];
    }
    // the U planes of the whole batch in one launch
    if (msts::ozaki_plans_prepare(src.data(), (int)src.size(), st) != cudaSuccess) return MSTS_ERR_CUDA;
  }
  return cuda_rc(msts::engine_run(v.data(), (int)batch, nb, safe, conj, false, workspace, status, st));
}

size_t msts_trevc_workspace_size(int64_t m, int32_t nb, uint32_t flags) {
  if (m < 0 || !nb_ok(nb)) return 0;
  return msts_solve_workspace_size(m, m, nb, MSTS_SAFE | (flags & MSTS_TENSOR_GEMM));
}

int msts_trevc(const msts_z *T, int64_t ldt, int64_t m, msts_z *Z, int64_t ldz, double *scales,
               int32_t *scale_exp, int32_t nb, void *workspace, size_t workspace_bytes,
               uint32_t *status, uint32_t flags, void *stream) {
  if (m < 0 || m > kMaxDim) return -3;
  if (m > 0 && !T) return -1;
  if (ldt < std::max<int64_t>(1, m)) return -2;
  if (m > 0 && !Z) return -4;
  if (ldz < std::max<int64_t>(1, m)) return -5;
  if (m > 0 && !scales) return -6;
  if (m > 0 && !scale_exp) return -7;
  if (!nb_ok(nb)) return -8;
  if ((flags & ~(uint32_t)MSTS_TENSOR_GEMM) != 0) return -12;
  const size_t need = msts_trevc_workspace_size(m, nb, flags);
  if (need > 0 && (!workspace || workspace_bytes < need)) return workspace ? -10 : -9;
  if (msts::bad_alignment({T, Z}, workspace)) return MSTS_ERR_ALIGN;
  if (m == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = msts::engine_trevc_setup(reinterpret_cast<const double2 *>(T), ldt, (int)m,
                                           reinterpret_cast<double2 *>(Z), ldz, st);
  if (e != cudaSuccess) return MSTS_ERR_CUDA;
  // Shifts are the diagonal of T, read with stride ldt + 1.
  msts::EngineProblem p = make_problem(T, ldt, m, T, ldt + 1, m, Z, ldz, scales, scale_exp, 1);
  msts::OzPlan plan;
  if (flags & MSTS_TENSOR_GEMM) {
    const size_t eng = align256(msts::engine_workspace_bytes(&p, 1, nb, true));
    if (msts::ozaki_plan_prepare(&plan, p.U, ldt, (int)m, (int)m, nb, false,
                                 static_cast<char *>(workspace) + eng, st) != cudaSuccess)
      return MSTS_ERR_CUDA;
    p.oz = &plan;
  }
  return cuda_rc(msts::engine_run(&p, 1, nb, true, false, true, workspace, status, st));
}

// ----- generalized problems (appendix, Alg. 8-10) ----------------------------
size_t msts_gsolve_workspace_size(int64_t m, int64_t n, int32_t nb, uint32_t flags) {
  if (m < 0 || n < 0 || !nb_ok(nb)) return 0;
  msts::EngineProblem p = make_problem(nullptr, 1, m, nullptr, 1, n, nullptr, 1, nullptr, nullptr, 0);
  p.V = reinterpret_cast<const double2 *>(16);     // sizes of the generalized form (never read)
  size_t s = align256(msts::engine_workspace_bytes(&p, 1, nb, (flags & MSTS_SAFE) != 0));
  if ((flags & MSTS_TENSOR_GEMM) && m > 0 && n > 0) s += msts::ozaki_plan_bytes((int)m, (int)n, nb, true);
  return s;
}

int msts_gsolve(const msts_z *U, int64_t ldu, const msts_z *V, int64_t ldv, int64_t m, const msts_z *shifts,
                int64_t n, msts_z *B, int64_t ldb, double *scales, int32_t *scale_exp, int32_t nb,
                void *workspace, size_t workspace_bytes, uint32_t *status, uint32_t flags, void *stream) {
  const bool safe = (flags & MSTS_SAFE) != 0;
  if (m < 0 || m > kMaxDim) return -5;
  if (m > 0 && !U) return -1;
  if (ldu < std::max<int64_t>(1, m)) return -2;
  if (m > 0 && !V) return -3;
  if (ldv < std::max<int64_t>(1, m)) return -4;
  if (n < 0 || n > kMaxDim) return -7;
  if (n > 0 && !shifts) return -6;
  if (m > 0 && n > 0 && !B) return -8;
  if (ldb < std::max<int64_t>(1, m)) return -9;
  if (safe && n > 0 && (!scales || !scale_exp)) return scales ? -11 : -10;
  if (!nb_ok(nb)) return -12;
  if ((flags & ~(uint32_t)(MSTS_SAFE | MSTS_TENSOR_GEMM)) != 0) return -16;
  const size_t need = msts_gsolve_workspace_size(m, n, nb, flags);
  if (need > 0 && (!workspace || workspace_bytes < need)) return workspace ? -14 : -13;
  if (msts::bad_alignment({U, V, shifts, B}, workspace)) return MSTS_ERR_ALIGN;
  if (m == 0 || n == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  msts::EngineProblem p = make_problem(U, ldu, m, shifts, 1, n, B, ldb, scales, scale_exp, 0);
  p.V = reinterpret_cast<const double2 *>(V);
  p.ldv = ldv;
  msts::OzPlan plan;
  if (flags & MSTS_TENSOR_GEMM) {
    const size_t eng = align256(msts::engine_workspace_bytes(&p, 1, nb, safe));
    if (msts::ozaki_plan_prepare(&plan, p.U, ldu, (int)m, (int)n, nb, false, static_cast<char *>(workspace) + eng,
                                 st, p.V, ldv) != cudaSuccess)
      return MSTS_ERR_CUDA;
    p.oz = &plan;
  }
  return cuda_rc(msts::engine_run(&p, 1, nb, safe, false, false, workspace, status, st));
}

size_t msts_gtrevc_workspace_size(int64_t m, int32_t nb, uint32_t flags) {
  if (m < 0 || !nb_ok(nb) || (flags & ~(uint32_t)MSTS_TENSOR_GEMM) != 0) return 0;
  return msts_gsolve_workspace_size(m, m, nb, MSTS_SAFE | flags);
}

int msts_gtrevc(const msts_z *T, int64_t ldt, const msts_z *S, int64_t lds, int64_t m, msts_z *Z, int64_t ldz,
                msts_z *lambda, double *scales, int32_t *scale_exp, int32_t nb, void *workspace,
                size_t workspace_bytes, uint32_t *status, uint32_t flags, void *stream) {
  if (m < 0 || m > kMaxDim) return -5;
  if (m > 0 && !T) return -1;
  if (ldt < std::max<int64_t>(1, m)) return -2;
  if (m > 0 && !S) return -3;
  if (lds < std::max<int64_t>(1, m)) return -4;
  if (m > 0 && !Z) return -6;
  if (ldz < std::max<int64_t>(1, m)) return -7;
  if (m > 0 && !lambda) return -8;
  if (m > 0 && !scales) return -9;
  if (m > 0 && !scale_exp) return -10;
  if (!nb_ok(nb)) return -11;
  if ((flags & ~(uint32_t)MSTS_TENSOR_GEMM) != 0) return -15;
  const size_t need = msts_gtrevc_workspace_size(m, nb, flags);
  if (need > 0 && (!workspace || workspace_bytes < need)) return workspace ? -13 : -12;
  if (msts::bad_alignment({T, S, Z, lambda}, workspace)) return MSTS_ERR_ALIGN;
  if (m == 0) return 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double2 *lam = reinterpret_cast<double2 *>(lambda);
  cudaError_t e = msts::engine_gtrevc_setup(reinterpret_cast<const double2 *>(T), ldt,
                                            reinterpret_cast<const double2 *>(S), lds, (int)m,
                                            reinterpret_cast<double2 *>(Z), ldz, lam, st);
  if (e != cudaSuccess) return MSTS_ERR_CUDA;
  msts::EngineProblem p = make_problem(T, ldt, m, lambda, 1, m, Z, ldz, scales, scale_exp, 1);
  p.V = reinterpret_cast<const double2 *>(S);
  p.ldv = lds;
  msts::OzPlan plan;
  if (flags & MSTS_TENSOR_GEMM) {
    const size_t eng = align256(msts::engine_workspace_bytes(&p, 1, nb, true));
    if (msts::ozaki_plan_prepare(&plan, p.U, ldt, (int)m, (int)m, nb, false, static_cast<char *>(workspace) + eng,
                                 st, p.V, lds) != cudaSuccess)
      return MSTS_ERR_CUDA;
    p.oz = &plan;
  }
  return cuda_rc(msts::engine_run(&p, 1, nb, true, false, true, workspace, status, st));
}

}  // extern "C"
