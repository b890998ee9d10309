// msts_engine.h -- internal interface between the C ABI layer and the solve
// engine (msts_solve.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace msts {
struct OzPlan;

// One multi-shift problem as the host driver describes it.  Shift j is read
// from shifts[j * shift_stride] (TREVC passes the diagonal of T this way).
struct EngineProblem {
  const double2 *U;
  long long ldu;
  int m;
  const double2 *shifts;
  long long shift_stride;
  int n;
  double2 *B;
  long long ldb;
  double *scales;
  int *scale_exp;
  int diag_z;  // write Z(j,j) = s_j at the end (TREVC)
  const struct OzPlan *oz;  // non-null: substitution GEMM on the tensor cores (one plan per problem)
  // Generalized problem (appendix, Alg. 8/9): (U - s_j V) x_j = b_j with V
  // upper triangular; null for the standard one.
  const double2 *V = nullptr;
  long long ldv = 1;
};

size_t engine_workspace_bytes(const EngineProblem *probs, int count, int nb, bool safe);

// Runs Alg. 3 (plain), Alg. 5 (safe) or the conjugate-transposed plain solve
// on all problems; `shortcut` declares column j of B zero in rows >= j.
// lp: the substitution GEMM multiplies in FP32 (the low-precision solve of the
// mixed-precision form; plain upper solves only).
cudaError_t engine_run(const EngineProblem *probs, int count, int nb, bool safe, bool conj,
                       bool shortcut, void *ws, uint32_t *status, cudaStream_t st, bool lp = false);

cudaError_t engine_trevc_setup(const double2 *T, long long ldt, int m, double2 *Z, long long ldz,
                               cudaStream_t st);
// Alg. 10's set-up: lam[j] = T(j,j) / S(j,j); Z = -T + S diag(lam) strictly
// above the diagonal, zero elsewhere.
cudaError_t engine_gtrevc_setup(const double2 *T, long long ldt, const double2 *S, long long lds, int m,
                                double2 *Z, long long ldz, double2 *lam, cudaStream_t st);

}  // namespace msts
