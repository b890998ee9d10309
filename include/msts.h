/*
 * msts.h -- C ABI of libmsts, a GB300 (sm_103a) implementation of the blocked
 * multi-shift triangular solve of Moon & Poulson, "Accelerating eigenvector
 * and pseudospectra computation using blocked multi-shift triangular solves"
 * (arXiv:1607.01477).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Complex numbers are msts_z = {double re, im} (binary compatible with
 *    std::complex<double>, C99 double _Complex and torch.complex128).
 *  - Matrices are column-major with a leading dimension: element (r, c) of A
 *    is A[r + c * lda]; lda >= max(1, rows).
 *  - Every array argument is a DEVICE pointer unless its comment says "host".
 *    The caller owns all memory; the library never allocates, frees or keeps
 *    a pointer after the call returns.
 *  - Only the upper triangle of U / T is read; the strictly lower part may
 *    hold anything.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  They do not synchronise and can be captured in a CUDA graph.
 *  - `workspace` is caller-owned device scratch of at least the size returned
 *    by the matching *_workspace_size function, aligned to 256 bytes.  It must
 *    not be used by anything else until the work queued on `stream` finishes.
 *  - Complex arrays must be 16-byte aligned (the kernels move complex values
 *    as 16-byte vectors; cudaMalloc, torch and numpy allocations are) and the
 *    workspace 256-byte aligned.
 *  - Return value: 0 on success; a negative value -k means argument k (1-based)
 *    is invalid and nothing was launched; MSTS_ERR_ALIGN means a complex array
 *    or the workspace is not aligned as above (nothing was launched);
 *    MSTS_ERR_CUDA means a CUDA launch failed (cudaGetLastError() tells why).
 *  - `status` (device, may be NULL) receives, asynchronously, the OR of the
 *    MSTS_STATUS_* bits below raised by the kernels.  The library only ORs
 *    bits into it: clear it before the call.
 *  - Block size n_b: blocks of rows are cut from the bottom of the matrix; if
 *    m is not a multiple of n_b the ragged block of m mod n_b rows is the top
 *    one.  Allowed n_b: 16, 32, 64.
 *
 * Safe variant (Alg. 4, Alg. 5 of the paper): readings fixed by this library
 *  - Omega = 2^960; growth bounds use complex moduli |z|; every scale factor
 *    is a power of two 2^-k with the smallest k >= 1 that brings the quantity
 *    below Omega; s_j = 2^-scale_exp[j] exactly (scales[j] underflows to 0
 *    once scale_exp[j] > 1074, scale_exp keeps the exact value).
 *  - An exactly zero pivot U(i,i) - s_j is replaced by the real number
 *    delta = max(2^-52 * ||U||_inf, DBL_MIN) (Sec. 3).
 *  - The bounds are guaranteed overflow-free for |U(i,k)| < 2^48 and
 *    |B(i,j)| < Omega; inputs outside that range raise MSTS_STATUS_RANGE.
 */
#ifndef MSTS_H_
#define MSTS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } msts_z;

/* flags */
#define MSTS_SAFE        1u  /* Alg. 5: (U - s_j I) x_j = scale_j b_j with scale_j in [0,1]  */
#define MSTS_CONJ_TRANS  2u  /* solve (U^H - conj(s_j) I) x_j = b_j (forward substitution)  */
#define MSTS_RESIDUAL_OZAKI 4u /* msts_solve_mixed / msts_residual: FP64-accurate product on the
                                  BF16 tensor cores (error-free digit splitting) instead of FP64 FMA */
#define MSTS_TENSOR_GEMM 8u    /* msts_solve / msts_trevc / msts_pseudospectra: the substitution GEMM
                                  of every block step as the same FP64-accurate digit-plane product
                                  on the BF16 tensor cores instead of FP64 FMA (single problem);
                                  msts_back_transform: the product X = Q Z likewise */
#define MSTS_NORMALIZE_COLUMNS 16u /* msts_back_transform: scale every column of X to unit 2-norm */
#define MSTS_MIXED_FP32_GEMM 32u   /* msts_solve_mixed: the low-precision substitution product with FP32
                                      FMAs on the CUDA cores instead of the tensor cores' 3-plane
                                      split-BF16 product */

/* status bits */
#define MSTS_STATUS_ZERO_PIVOT  1u  /* plain solve: some U(i,i) - s_j == 0 exactly (X is undefined) */
#define MSTS_STATUS_NONFINITE   2u  /* a NaN or Inf was found in U or B                        */
#define MSTS_STATUS_RANGE       4u  /* safe solve: |U(i,k)| >= 2^48 or |B(i,j)| >= Omega           */
#define MSTS_STATUS_SCALED      8u  /* safe solve: some scale_j < 1                              */
#define MSTS_STATUS_DELTA      16u  /* safe solve: a zero pivot was replaced by delta            */
#define MSTS_STATUS_NOT_CONVERGED 32u /* mixed solve: refinement stopped at its iteration cap   */
#define MSTS_STATUS_TIMEOUT    64u  /* a bounded wait inside a tensor-core kernel expired: the
                                       results of that call are invalid                     */

#define MSTS_ERR_CUDA (-1000)
#define MSTS_ERR_ALIGN (-1002)

/* Library version as 10000*major + 100*minor + patch. */
int msts_version(void);

/* Tuning knobs (no counterpart in the paper; the choices change no result bit,
 * only the speed).  Process-wide; set them between calls, not while a call is
 * being launched from another host thread.
 * MSTS_TUNE_DIAG_LANES: the diagonal-block step for n_b = 32 of the standard
 *   solves spreads each shift's rows over four warps with 1, 2 or 4 lanes per
 *   shift; 0 (default) picks the width per launch from the number of active
 *   shifts, 1 / 2 / 4 force it, -1 takes the one-warp layout (a group of
 *   lanes per shift inside one warp) instead.
 * MSTS_TUNE_ALG4_CHAIN: the safe solves take Alg. 4's rescaling decisions on
 *   each diagonal block from a closed form (the final rescale exponent is the
 *   largest of the ratio tests' and of the exponent of the bound's full sum,
 *   estimated in FP32 and checked) and run the serial decision chain only
 *   where that estimate cannot decide; 1 runs the chain in every block, 0
 *   (default) restores the closed form.  Both give the same bits.  Set on the
 *   current device; synchronises it.
 * Returns 0, -1 (unknown knob), -2 (invalid value) or -3 (CUDA error). */
#define MSTS_TUNE_DIAG_LANES 1
#define MSTS_TUNE_ALG4_CHAIN 2
int msts_tune_set(int32_t knob, int32_t value);

/* ---------------------------------------------------------------------------
 * Multi-shift triangular solve (Sec. 2, Eq. 2, Alg. 3) and its safe variant
 * (Sec. 3, Eq. 3 generalised to many shifts, Alg. 4 and Alg. 5).
 *
 *   plain:            (U - shifts[j] I) X(:,j) = B(:,j),          j = 0..n-1
 *   MSTS_SAFE:        (U - shifts[j] I) X(:,j) = scales[j] B(:,j), scales[j] in [0,1]
 *   MSTS_CONJ_TRANS:  (U^H - conj(shifts[j]) I) X(:,j) = B(:,j)    (plain only)
 *
 * U        m x m, leading dimension ldu, upper triangle read.
 * shifts   n complex shifts lambda_j.
 * B        m x n, leading dimension ldb; overwritten with X.
 * scales   n doubles (MSTS_SAFE only, else may be NULL): s_j = 2^-scale_exp[j].
 * scale_exp n int32 (MSTS_SAFE only, else may be NULL).
 * nb       block size n_b (16, 32 or 64).
 * A plain solve that meets an exactly zero pivot raises MSTS_STATUS_ZERO_PIVOT
 * and leaves X undefined (Inf/NaN), as back substitution does.
 * m == 0 or n == 0 is a no-op.  Returns 0, -k, or MSTS_ERR_CUDA.
 * ------------------------------------------------------------------------- */
size_t msts_solve_workspace_size(int64_t m, int64_t n, int32_t nb, uint32_t flags);
int msts_solve(const msts_z *U, int64_t ldu, int64_t m,
               const msts_z *shifts, int64_t n,
               msts_z *B, int64_t ldb,
               double *scales, int32_t *scale_exp,
               int32_t nb, void *workspace, size_t workspace_bytes,
               uint32_t *status, uint32_t flags, void *stream);

/* ---------------------------------------------------------------------------
 * The other triangular variants (footnote to Sec. 2: the lower-triangular and
 * right-hand cases of the multi-shift solve).  With op(A) = A, A^T or A^H
 * (trans = MSTS_OP_N, MSTS_OP_T, MSTS_OP_C) and A upper or lower triangular
 * (uplo = MSTS_UPLO_UPPER / MSTS_UPLO_LOWER; only that triangle is read):
 *
 *   side = MSTS_SIDE_LEFT:  (op(A) - shifts[j] I) X(:,j) = scale_j B(:,j)
 *                           B is m x n (ldb >= m), one column per shift;
 *   side = MSTS_SIDE_RIGHT: X(j,:) (op(A) - shifts[j] I) = scale_j B(j,:)
 *                           B is n x m (ldb >= n), one row per shift;
 *
 * scale_j = 1 for the plain solve; with MSTS_SAFE, scale_j = scales[j] =
 * 2^-scale_exp[j] from Alg. 5 run in the variant's own substitution order
 * (the operator written as an upper-triangular matrix in that order, blocks
 * of n_b cut from where the substitution starts).  The shifts are not
 * conjugated for MSTS_OP_C.  Left/upper/N is msts_solve itself; every other
 * variant is mapped onto it by exact permutations (and conjugation) of A and
 * B in the workspace: msts_solve_variant_workspace_size(side, uplo, trans, m,
 * n, nb, flags) bytes, up to 16 m^2 + 16 m n bytes more than msts_solve.
 * flags: MSTS_SAFE, MSTS_TENSOR_GEMM.  B is overwritten with X.  Returns 0,
 * -15 for an unknown side/uplo/trans, the other codes of msts_solve (ldb
 * checked against the row count of B), or MSTS_ERR_CUDA.
 * ------------------------------------------------------------------------- */
#define MSTS_SIDE_LEFT  0
#define MSTS_SIDE_RIGHT 1
#define MSTS_UPLO_UPPER 0
#define MSTS_UPLO_LOWER 1
#define MSTS_OP_N 0
#define MSTS_OP_T 1
#define MSTS_OP_C 2
size_t msts_solve_variant_workspace_size(int32_t side, int32_t uplo, int32_t trans, int64_t m, int64_t n,
                                         int32_t nb, uint32_t flags);
int msts_solve_variant(int32_t side, int32_t uplo, int32_t trans,
                       const msts_z *A, int64_t lda, int64_t m,
                       const msts_z *shifts, int64_t n,
                       msts_z *B, int64_t ldb,
                       double *scales, int32_t *scale_exp,
                       int32_t nb, void *workspace, size_t workspace_bytes,
                       uint32_t *status, uint32_t flags, void *stream);

/* ---------------------------------------------------------------------------
 * Batched multi-shift solves of uneven sizes: problem p is solved exactly as
 * msts_solve would with the fields of probs[p] (host array of `batch`
 * descriptors; the pointers inside are device pointers).  All problems share
 * n_b, flags and stream; their block steps run together, one launch per step
 * for all problems.  flags: MSTS_SAFE, MSTS_CONJ_TRANS (plain only) and
 * MSTS_TENSOR_GEMM (each problem's U split into digit planes in the workspace,
 * every problem's substitution step in one tensor-core launch per block step).
 * ------------------------------------------------------------------------- */
typedef struct {
  const msts_z *U; int64_t ldu; int64_t m;
  const msts_z *shifts; int64_t n;
  msts_z *B; int64_t ldb;
  double *scales; int32_t *scale_exp;
} msts_problem;

size_t msts_solve_batched_workspace_size(const msts_problem *probs, int64_t batch,
                                         int32_t nb, uint32_t flags);
int msts_solve_batched(const msts_problem *probs, int64_t batch, int32_t nb,
                       void *workspace, size_t workspace_bytes,
                       uint32_t *status, uint32_t flags, void *stream);

/* ---------------------------------------------------------------------------
 * Triangular eigenvectors (Sec. 4, Alg. 6 "TriangEig"): for the upper
 * triangular Schur factor T (m x m), writes the upper triangular Z (m x m,
 * leading dimension ldz, the strictly lower part is set to zero) with
 *   T Z(:,j) = T(j,j) Z(:,j),   Z(j,j) = scales[j] = 2^-scale_exp[j],
 * computed as the safe multi-shift solve with shifts T(j,j) and right-hand
 * sides -T(0:j-1, j), shortcut so that column j only visits rows < j.
 * Columns are returned unnormalised, as Alg. 6 returns them.
 * ------------------------------------------------------------------------- */
size_t msts_trevc_workspace_size(int64_t m, int32_t nb, uint32_t flags);
int msts_trevc(const msts_z *T, int64_t ldt, int64_t m,
               msts_z *Z, int64_t ldz,
               double *scales, int32_t *scale_exp,
               int32_t nb, void *workspace, size_t workspace_bytes,
               uint32_t *status, uint32_t flags, void *stream);   /* flags: 0 or MSTS_TENSOR_GEMM */

/* ---------------------------------------------------------------------------
 * Generalized multi-shift triangular solve (appendix, Alg. 8; safe form
 * Alg. 9): for U, V upper triangular (m x m; only their upper triangles are
 * read),
 *   (U - shifts[j] V) X(:,j) = scale_j B(:,j),
 * B (m x n, ldb) overwritten with X. flags: 0 (Alg. 8, scale_j = 1) or
 * MSTS_SAFE (Alg. 9 with Alg. 4 on each shifted diagonal block; scales and
 * scale_exp as for msts_solve). Readings: the column bounds of U - s_j V are
 * ||U(.,k)|| + |s_j| ||V(.,k)|| (rigorous upper bounds), and an exactly zero
 * pivot U(i,i) - s_j V(i,i) becomes delta_j = max(2^-52 (||U||_inf +
 * |s_j| ||V||_inf), DBL_MIN). MSTS_TENSOR_GEMM runs the substitution step
 * B(I0,:) -= U(I0,I1) X(I1,:) - V(I0,I1) (s X(I1,:)) on the tensor cores as one
 * FP64-accurate digit-plane product of [U | V] and [X; -s X] (s X rounded once
 * in FP64); otherwise FP64 FMA.
 * workspace: msts_gsolve_workspace_size(m, n, nb, flags) bytes.
 * Returns 0, -k for invalid argument k (nothing launched; -13/-14 for a
 * missing / too small workspace, -16 for unsupported flags), MSTS_ERR_CUDA.
 * ------------------------------------------------------------------------- */
size_t msts_gsolve_workspace_size(int64_t m, int64_t n, int32_t nb, uint32_t flags);
int msts_gsolve(const msts_z *U, int64_t ldu, const msts_z *V, int64_t ldv, int64_t m,
                const msts_z *shifts, int64_t n,
                msts_z *B, int64_t ldb,
                double *scales, int32_t *scale_exp,
                int32_t nb, void *workspace, size_t workspace_bytes,
                uint32_t *status, uint32_t flags, void *stream);

/* ---------------------------------------------------------------------------
 * Generalized triangular eigenvectors (appendix, Alg. 10
 * "GeneralizedTriangEig"): for the generalized Schur pair (T, S), both upper
 * triangular with S(j,j) != 0, writes lambda[j] = T(j,j) / S(j,j) and the upper
 * triangular Z with T Z(:,j) = lambda[j] S Z(:,j), Z(j,j) = scales[j] =
 * 2^-scale_exp[j] (right-hand sides -T(0:j-1,j) + lambda[j] S(0:j-1,j), the
 * strictly-upper shortcut as in msts_trevc). flags: 0 or MSTS_TENSOR_GEMM
 * (the substitution step as in msts_gsolve).
 * workspace: msts_gtrevc_workspace_size(m, nb, flags) bytes.
 * ------------------------------------------------------------------------- */
size_t msts_gtrevc_workspace_size(int64_t m, int32_t nb, uint32_t flags);
int msts_gtrevc(const msts_z *T, int64_t ldt, const msts_z *S, int64_t lds, int64_t m,
                msts_z *Z, int64_t ldz, msts_z *lambda,
                double *scales, int32_t *scale_exp,
                int32_t nb, void *workspace, size_t workspace_bytes,
                uint32_t *status, uint32_t flags, void *stream);

/* ---------------------------------------------------------------------------
 * Back-transformation (Sec. 4, Alg. 6 "Eig", second half): the eigenvectors
 * of A = Q T Q^H are the columns of X = Q Z, with Z the upper triangular
 * eigenvectors of T from msts_trevc.
 * Q   m x m (leading dimension ldq), typically the unitary Schur vectors.
 * Z   m x m upper triangular (ldz); only the upper triangle is read.
 * X   m x m output (ldx); must not overlap Q or Z.
 * flags: MSTS_TENSOR_GEMM runs the product on the tensor cores through the
 *   exact digit splitting (FP64-accurate: the error is below 2^-46 m times
 *   max|Q(i,:)| max|Z(:,j)| per entry), else FP64 FMA; MSTS_NORMALIZE_COLUMNS
 *   then scales every column to unit 2-norm (zero columns stay zero).
 * workspace: msts_back_transform_workspace_size(m, flags) bytes (0 without
 *   MSTS_TENSOR_GEMM), device memory owned by the caller.
 * status: device word, only MSTS_STATUS_TIMEOUT can be set.
 * Returns 0, or -k for an invalid argument k (nothing launched; -8/-9 for a
 * missing / too small workspace), or MSTS_ERR_CUDA.
 * ------------------------------------------------------------------------- */
size_t msts_back_transform_workspace_size(int64_t m, uint32_t flags);
int msts_back_transform(const msts_z *Q, int64_t ldq, int64_t m,
                        const msts_z *Z, int64_t ldz,
                        msts_z *X, int64_t ldx,
                        void *workspace, size_t workspace_bytes,
                        uint32_t *status, uint32_t flags, void *stream);

/* ---------------------------------------------------------------------------
 * Pseudospectra (Sec. 5, Alg. 7, Van Loan / Lui): for each grid point z[p],
 *   sigma_min[p] = sigma_min(T - z[p] I) = 1 / ||(z[p] I - A)^{-1}||_2
 * for A = Q T Q^H, from the largest eigenvalue of (T - zI)^{-H} (T - zI)^{-1}
 * estimated by `iters` (1..64) Lanczos steps; every operator application is a pair of
 * multi-shift solves over all N grid points at once (upper with T - zI, then
 * lower with its conjugate transpose).
 * V0       m x N start vectors (leading dimension ldv), normalised inside.
 * Lanczos readings: full reorthogonalisation by classical Gram-Schmidt, run a
 * second time when the first pass removed more than half of ||w||^2 ("twice
 * is enough"); exactly min(iters, m) steps unless beta_k <= 1e-14 max_i |alpha_i|.
 * alpha, beta (optional, may be NULL): N x iters tridiagonal entries, point p
 * at [p*iters, (p+1)*iters); steps (optional): the tridiagonal order per point.
 * ------------------------------------------------------------------------- */
size_t msts_pseudospectra_workspace_size(int64_t m, int64_t N, int32_t iters, int32_t nb,
                                         uint32_t flags);
int msts_pseudospectra(const msts_z *T, int64_t ldt, int64_t m,
                       const msts_z *z, int64_t N,
                       const msts_z *V0, int64_t ldv, int32_t iters,
                       double *sigma_min, double *alpha, double *beta, int32_t *steps,
                       int32_t nb, void *workspace, size_t workspace_bytes,
                       uint32_t *status, uint32_t flags, void *stream);   /* flags: 0 or MSTS_TENSOR_GEMM */

/* ---------------------------------------------------------------------------
 * 1-norm pseudospectra (footnote to Sec. 5: Hager's estimator with Higham's
 * refinements, driven by multi-shift solves with the grid points as shifts):
 *   est[p] <= ||(z[p] I - A)^{-1}||_1,  A = Q T Q^H (Q may be NULL: A = T),
 * a lower-bound estimate of the resolvent 1-norm from the start vector e/m,
 * at most five gradient steps (each one solve with (T - zI)^H and one with
 * T - zI, between products with Q^H and Q), and the alternative vector
 * x(i) = (-1)^i (1 + i/(m-1)) scaled by 2/(3m).  Points leave the iteration
 * as they converge; each step solves only the points still iterating.
 * kind[p] = j >= 0 when est[p] = ||R e_j||_1, -1 for the start vector, -2 for
 * the alternative vector; steps[p] = the number of (T - zI)^H solves.
 * T        m x m upper triangular (ldt), Q m x m unitary (ldq) or NULL.
 * z, est, kind, steps: N grid points and the three outputs (device).
 * flags    0 or MSTS_TENSOR_GEMM (the substitution and the Q products on the
 *          tensor cores, FP64-accurate).
 * workspace: msts_pseudospectra_1norm_workspace_size(m, N, nb, Q != NULL,
 * flags) bytes.  The call synchronises the stream once per step (the number
 * of live points decides the next launch).  A grid point equal to a
 * diagonal entry of T raises MSTS_STATUS_ZERO_PIVOT.  Returns 0, -k for an
 * invalid argument k (-9/-10 missing / small workspace), or MSTS_ERR_CUDA.
 * ------------------------------------------------------------------------- */
size_t msts_pseudospectra_1norm_workspace_size(int64_t m, int64_t N, int32_t nb, int32_t with_q, uint32_t flags);
int msts_pseudospectra_1norm(const msts_z *T, int64_t ldt, int64_t m,
                             const msts_z *Q, int64_t ldq,
                             const msts_z *z, int64_t N,
                             double *est, int32_t *kind, int32_t *steps,
                             int32_t nb, void *workspace, size_t workspace_bytes,
                             uint32_t *status, uint32_t flags, void *stream);

/* ---------------------------------------------------------------------------
 * Automatic grid of a spectral portrait (the SpectralPortrait driver listed in
 * Sec. 6): box = (x0, x1, y0, y1) is the bounding box of diag(T) widened on
 * every side by h = max(max(x-side, y-side)/4, 2^-20 max(1, max_i max(|Re
 * T(i,i)|, |Im T(i,i)|))); z[k + l nx] = (x0 + k dx) + i (y0 + l dy) with
 * dx = (x1 - x0)/(nx - 1) (0 for nx == 1), likewise dy, each operation one
 * rounding.  T (device, ldt >= m >= 1); z: nx*ny points, box: 4 doubles
 * (device).  Returns 0, -k for an invalid argument k, or MSTS_ERR_CUDA.
 * ------------------------------------------------------------------------- */
int msts_portrait_grid(const msts_z *T, int64_t ldt, int64_t m, int64_t nx, int64_t ny,
                       msts_z *z, double *box, void *stream);

/* ---------------------------------------------------------------------------
 * Adjoint of X = (U - s_j I)^{-1} B(:,j) (not in the paper): given
 * GX = dL/dRe X + i dL/dIm X for a real loss L, returns
 *   dB = Lambda,  Lambda(:,j) = (U - s_j I)^{-H} GX(:,j)
 *   dU = -triu(Lambda X^H)   (m x m, strictly lower part set to zero)
 *   ds_j = X(:,j)^H Lambda(:,j)
 * X is recomputed from U, shifts and B block by block; it is not an input.
 * B and GX are read only.  dB (m x n, lddb) and dU (lddu) are written.
 * ------------------------------------------------------------------------- */
size_t msts_adjoint_workspace_size(int64_t m, int64_t n, int32_t nb);
/* Single problem; the batched form below takes one descriptor per problem. */
int msts_adjoint(const msts_z *U, int64_t ldu, int64_t m,
                 const msts_z *shifts, int64_t n,
                 const msts_z *B, int64_t ldb, const msts_z *GX, int64_t ldg,
                 msts_z *dU, int64_t lddu, msts_z *dB, int64_t lddb, msts_z *ds,
                 int32_t nb, void *workspace, size_t workspace_bytes,
                 uint32_t *status, void *stream);

/* ---------------------------------------------------------------------------
 * Batched adjoint: problem p is processed exactly as msts_adjoint would with
 * the fields of probs[p] (host array; pointers inside are device pointers).
 * All problems share n_b and stream; their solves run in shared launches.
 * ------------------------------------------------------------------------- */
typedef struct {
  const msts_z *U; int64_t ldu; int64_t m;
  const msts_z *shifts; int64_t n;
  const msts_z *B; int64_t ldb;
  const msts_z *GX; int64_t ldg;
  msts_z *dU; int64_t lddu;
  msts_z *dB; int64_t lddb;
  msts_z *ds;
} msts_adjoint_problem;

size_t msts_adjoint_batched_workspace_size(const msts_adjoint_problem *probs, int64_t batch,
                                           int32_t nb);
int msts_adjoint_batched(const msts_adjoint_problem *probs, int64_t batch, int32_t nb,
                         void *workspace, size_t workspace_bytes,
                         uint32_t *status, void *stream);
/* The same with flags: MSTS_TENSOR_GEMM runs the substitution steps of both
 * internal solves (X recomputed, and Lambda) and the product dU = -triu(Lambda
 * X^H) on the tensor cores (FP64-accurate digit planes), all problems of a step
 * in one launch; workspace from the _flags size query (it adds the digit planes
 * of U, U^H, Lambda and X^H per problem).  Returns -8 for unknown flags. */
size_t msts_adjoint_batched_flags_workspace_size(const msts_adjoint_problem *probs, int64_t batch,
                                                 int32_t nb, uint32_t flags);
int msts_adjoint_batched_flags(const msts_adjoint_problem *probs, int64_t batch, int32_t nb,
                               void *workspace, size_t workspace_bytes,
                               uint32_t *status, uint32_t flags, void *stream);

/* ---------------------------------------------------------------------------
 * Mixed-precision multi-shift solve with FP64 iterative refinement (not in the
 * paper, which is FP64 throughout).  Solves (U - s_j I) X(:,j) = B(:,j) with
 *   X_0 = solve_lp(B);  repeat  R = B - (U - S) X  (FP64),
 *                               eta = max_j ||R_j||_inf / (||U - s_j I||_inf ||x_j||_inf + ||b_j||_inf),
 *                               stop if eta <= tol or after max_iter corrections,
 *                               X += solve_lp(R)
 * where solve_lp is the blocked solve of Alg. 3 whose substitution GEMM is
 * a low-precision product (diagonal blocks in FP64).  By default that product
 * runs on the BF16 tensor cores: U(I0,I1) and X(I1,:) are split into their 3
 * leading signed 7-bit digit planes (3 BF16 pieces per entry below a power of
 * two per row of U and per column of X), the 6 plane pairs with s + t <= 4 are
 * multiplied with FP32 accumulation in tensor memory and their sum is formed
 * in FP32 (about 2^-20 relative to K max|U(r,:)| max|X(:,j)|; n_b = 16 or 32;
 * with n_b = 64 the substitution step is the FP64-accurate 8-plane product);
 * with MSTS_MIXED_FP32_GEMM it is an FP32 FMA product on the CUDA cores.
 * B (read only) and X (written, ldx) are m x n.  Residual: without
 * MSTS_RESIDUAL_OZAKI it is computed with FP64 FMAs; MSTS_RESIDUAL_OZAKI computes the product triu(U) X
 * on the BF16 tensor cores from 8 seven-bit digit planes per operand with
 * exact FP32 accumulation per 64-wide K chunk and integer accumulation across
 * chunks (accurate to ~2^-50 relative to K max|U(r,:)| max|X(:,j)|), and
 * needs about 32 m (m + n) bytes more workspace; the tensor-core
 * low-precision product needs the digit planes of U's block panels (about
 * 32 m^2 bytes for n_b = 32); msts_solve_mixed_workspace_size(m, n, nb,
 * flags) gives the total.
 * SYNCHRONOUS: the convergence test reads eta on the host every iteration, so
 * the call returns after the work is done.  *iters (host, may be NULL)
 * receives the number of corrections, *eta the final max eta and
 * *eta_before the max eta of X_0 (host pointers).  If eta > tol at the cap,
 * MSTS_STATUS_NOT_CONVERGED is OR-ed into *status.
 * ------------------------------------------------------------------------- */
size_t msts_solve_mixed_workspace_size(int64_t m, int64_t n, int32_t nb, uint32_t flags);
int msts_solve_mixed(const msts_z *U, int64_t ldu, int64_t m,
                     const msts_z *shifts, int64_t n,
                     const msts_z *B, int64_t ldb, msts_z *X, int64_t ldx,
                     double tol, int32_t max_iter,
                     int32_t nb, void *workspace, size_t workspace_bytes,
                     uint32_t *status, uint32_t flags,
                     int32_t *iters, double *eta, double *eta_before, void *stream);

/* ---------------------------------------------------------------------------
 * Residual R = B - (U - diag(s)) X of a multi-shift solve (not in the paper):
 * R(:,j) = B(:,j) - triu(U) X(:,j) + s_j X(:,j), all m x n, asynchronous.
 * flags = 0: FP64 FMA; MSTS_RESIDUAL_OZAKI: the tensor-core product described
 * under msts_solve_mixed (workspace from msts_residual_workspace_size).
 * ------------------------------------------------------------------------- */
size_t msts_residual_workspace_size(int64_t m, int64_t n, uint32_t flags);
int msts_residual(const msts_z *U, int64_t ldu, int64_t m,
                  const msts_z *shifts, int64_t n,
                  const msts_z *B, int64_t ldb, const msts_z *X, int64_t ldx,
                  msts_z *R, int64_t ldr,
                  void *workspace, size_t workspace_bytes,
                  uint32_t *status, uint32_t flags, void *stream);

/* ---------------------------------------------------------------------------
 * Instrumentation (not in the paper).
 * msts_launch_count: number of kernels the library has launched in this
 *   process so far (all entry points).
 * msts_trace_begin(capacity): from now on, bracket each launch of the hot
 *   kernels (MSTS_KERNEL_GEMM: the substitution GEMM or FP64 residual,
 *   MSTS_KERNEL_DIAG: the diagonal-block solve, MSTS_KERNEL_OZAKI: the
 *   tensor-core substitution step and products, MSTS_KERNEL_RESIDUAL: the
 *   tensor-core residual, MSTS_KERNEL_LANCZOS: the Lanczos step) with CUDA
 *   events on its stream, for at most
 *   `capacity` launches, recording the algorithmic FLOPs (8 per complex
 *   multiply-add) and algorithmic bytes of each launch.  The 2 x capacity
 *   events are created by this call and destroyed by msts_trace_end, so the
 *   traced region only records them; capacity <= 2^22.  Host-side; not for
 *   use inside stream capture.
 * msts_trace_end: waits for the recorded events, accumulates per-kernel
 *   totals and stops recording.  msts_trace_query reads the totals.
 * ------------------------------------------------------------------------- */
#define MSTS_KERNEL_GEMM 0
#define MSTS_KERNEL_DIAG 1
#define MSTS_KERNEL_OZAKI 2   /* tensor-core substitution step or product; FLOPs = BF16 MMA FLOPs issued */
#define MSTS_KERNEL_RESIDUAL 3 /* tensor-core residual of the mixed solve; FLOPs = BF16 MMA FLOPs issued */
#define MSTS_KERNEL_LANCZOS 4  /* Lanczos step of the pseudospectra (vector passes, HBM-bound) */
uint64_t msts_launch_count(void);
int msts_trace_begin(int64_t capacity);
int msts_trace_end(void);
int msts_trace_query(int32_t kernel, double *total_ms, int64_t *launches, double *flops,
                     double *bytes);

/* Failure injection for tests (host side; no counterpart in the paper).  The
 * tensor-core kernels publish a timeout of a bounded wait in the caller's
 * status word, or, for a call made with status == NULL, in a word of the
 * library's own on the current device, which every such call clears on its
 * stream before its first launch.  msts_inject_fallback_status ORs `bits`
 * into that word (ordered on `stream`, synchronising it), so a test can check
 * that a later call without a status word is not cut short by an earlier
 * give-up.  Returns 0 or MSTS_ERR_CUDA. */
int msts_inject_fallback_status(uint32_t bits, void *stream);

/* ---------------------------------------------------------------------------
 * Safe multi-shift solve without any allocation (the paper has no
 * counterpart; this is a convenience of this library).
 *
 * For callers that cannot allocate device memory when they need the solve:
 * cudaMalloc synchronises the device and may fail at run time, so code with a
 * fixed memory budget, or whose host framework owns every allocation, often
 * may not call it.  This entry point computes exactly what msts_solve with
 * flags = MSTS_SAFE computes (same arguments, same meaning), but takes its
 * scratch from a 16 MiB array that the library keeps in device memory on
 * every GPU that loads it, until the process exits.  It calls no allocator.
 *  - The caller still passes U, shifts, B, scales, scale_exp (and status).
 *  - Problems whose scratch need (msts_solve_workspace_size(m, n, nb,
 *    MSTS_SAFE)) exceeds 16 MiB are rejected with MSTS_ERR_STATIC_SCRATCH
 *    before anything is launched (e.g. m = n = 4096 at n_b = 32 needs ~2.2 MiB).
 *  - The first call on a device looks up the array's device address with that
 *    device current (cudaGetSymbolAddress); make that first call before any
 *    stream capture.
 *  - Every call shares the one array and the kernels write every scratch word
 *    before reading it, so nothing needs clearing between calls; but calls
 *    whose work overlaps on the GPU (different streams, or concurrent host
 *    threads without ordering) race on it.  Order such calls on one stream.
 * Returns 0, -k for invalid argument k (numbering as msts_solve without the
 * workspace arguments), MSTS_ERR_STATIC_SCRATCH, MSTS_ERR_ALIGN or MSTS_ERR_CUDA.
 * ------------------------------------------------------------------------- */
#define MSTS_ERR_STATIC_SCRATCH (-1001)
int msts_safe_solve_static(const msts_z *U, int64_t ldu, int64_t m,
                           const msts_z *shifts, int64_t n,
                           msts_z *B, int64_t ldb,
                           double *scales, int32_t *scale_exp,
                           int32_t nb, uint32_t *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MSTS_H_ */
