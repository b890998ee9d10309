// msts_ozaki.h -- internal interface of the tensor-core FP64-accurate residual.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <cuda.h>
#include <cuda_bf16.h>

namespace msts {
// The status word a tensor-core call publishes its timeouts in: `status`
// itself, or (status == NULL) a library word on the current device, cleared
// on `st` first.  One call that runs several tensor-core launches takes it
// once and passes it to all of them.
uint32_t *ozaki_call_status(uint32_t *status, cudaStream_t st);
// Workspace for the digit planes of triu(U) and X and their exponents.
size_t ozaki_workspace_bytes(int m, int n);
// Splits triu(U) into BF16 digit planes (once per matrix).
cudaError_t ozaki_prepare(const double2 *U, long long ldu, int m, int n, void *ws, cudaStream_t st);
// R = B - triu(U) X + X diag(s) with the product on the tensor cores; needs a
// prior ozaki_prepare of U into the same workspace.
cudaError_t ozaki_residual(const double2 *U, long long ldu, int m, const double2 *s, int n,
                           const double2 *B, long long ldb, const double2 *X, long long ldx,
                           double2 *R, long long ldr, void *ws, uint32_t *status, cudaStream_t st);
// C = A B (m x m dense A, m x n B; B upper triangular when triu_b), FP64-accurate
// on the tensor cores; workspace ozaki_workspace_bytes(m, n).
cudaError_t ozaki_product(const double2 *A, long long lda, int m, const double2 *Bm, long long ldbm, int n,
                          bool triu_b, double2 *C, long long ldc, void *ws, uint32_t *status, cudaStream_t st);
// Tensor-core substitution step of the blocked solve: the block-layout digit
// planes of U (upper, or conjugate-transposed for forward substitution) and
// a per-step buffer for the planes of the solved block X(I1,:).
struct OzPlan {
  __nv_bfloat16 *planes;
  int *rexp;
  __nv_bfloat16 *bp;
  int *cexp;
  int m, nb, nblk, KB, nmax;
  bool conj;
  CUtensorMap tmA;
  CUtensorMap tmB;   // the X planes of a step that updates all nmax columns
};
// gen: a generalized problem (U - lambda_j V), whose panels are [U | V].
size_t ozaki_plan_bytes(int m, int n, int nb, bool gen = false);
cudaError_t ozaki_plan_prepare(OzPlan *plan, const double2 *U, long long ldu, int m, int n, int nb,
                               bool conj, void *ws, cudaStream_t st, const double2 *V = nullptr,
                               long long ldv = 0);
// The two halves of ozaki_plan_prepare for a batch: ozaki_plan_init carves a
// plan's buffers from ws and encodes its tensor maps (host only);
// ozaki_plans_prepare then writes the U planes of every plan of the batch,
// one launch per 64 plans of each orientation.
cudaError_t ozaki_plan_init(OzPlan *plan, int m, int n, int nb, bool conj, void *ws, bool gen = false);
struct OzPlanSrc {
  const OzPlan *plan;
  const double2 *U;
  long long ldu;
};
cudaError_t ozaki_plans_prepare(const OzPlanSrc *src, int count, cudaStream_t st);
// B(rows, jstart..jstart+ncols) = 2^-pend B - U-panel(b) X(I1, .), rows above the
// block (upper) or below it (conj); `flops` is recorded by the tracer.
// planes_ready: the X digit planes and exponents of this block were written by
// the diagonal-block step (otherwise they are sliced here first).  lam (a
// generalized plan): the shifts, column j's at lam[j lam_stride]; the update
// is then B(I0,:) -= U(I0,I1) X(I1,:) - V(I0,I1) (lam X(I1,:)).
// lp: the low-precision product of the mixed solve (3 digit planes per
// operand, FP32 accumulation; n_b <= 32, else the FP64-accurate product).
cudaError_t ozaki_update(const OzPlan &plan, int b, int lo, int hi, double2 *B, long long ldb,
                         int jstart, int ncols, const int *pend, uint32_t *status, double flops,
                         cudaStream_t st, bool planes_ready = false, const double2 *lam = nullptr,
                         long long lam_stride = 0, bool lp = false);
// One problem's substitution step inside a batched launch (see ozaki_update;
// the X planes of this block were written by the diagonal-block step).
struct OzBatchStep {
  const OzPlan *plan;
  int b, lo, hi;
  double2 *B; long long ldb;
  int jstart, ncols;
  const int *pend;
};
// The steps of `count` (<= 64) problems as one launch of the chunked kernel,
// problem i in grid slice z = i.
cudaError_t ozaki_update_batched(const OzBatchStep *steps, int count, uint32_t *status, cudaStream_t st);
// dU = -triu(L X^H) (L, X m x n, dU m x m, strictly lower part set to zero) for
// `count` (<= 64) problems, FP64-accurate on the tensor cores; the workspace
// holds sum over problems of ozaki_neg_triu_bytes(m, n).
struct OzNegTriuItem {
  const double2 *L; long long ldl;
  const double2 *X; long long ldx;
  double2 *dU; long long lddu;
  int m, n;
};
size_t ozaki_neg_triu_bytes(int m, int n);
cudaError_t ozaki_neg_triu_batched(const OzNegTriuItem *items, int count, void *ws, uint32_t *status,
                                   cudaStream_t st);
}  // namespace msts
