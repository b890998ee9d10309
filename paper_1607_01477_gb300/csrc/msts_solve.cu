// msts_solve.cu -- the blocked multi-shift triangular solve (Sec. 2, Alg. 3)
// and its safe variant (Sec. 3, Alg. 4 and Alg. 5) on GB300, FP64 complex.
//
// Schedule (the paper's right-looking order): for every block of n_b rows,
// bottom to top,
//   k_diag : each shift j solves its shifted n_b x n_b diagonal block with one
//            warp (lane = row), U(I1,I1) staged once per CTA in shared memory;
//            the safe variant also runs the Alg. 4 bounds, the careful
//            back substitution and the Alg. 5 column bound update in the same
//            pass (per-column state lives in the workspace);
//   k_gemm : the substitution step B(I0,:) -= U(I0,I1) X(I1,:) shared by all
//            shifts, an FP64 DFMA tile kernel.  In the safe variant its
//            epilogue also applies the power-of-two rescaling that Alg. 5
//            owes B(I0,j) for this block (lazy xSCAL, exact).
// Rows below the current block (I2) are rescaled lazily too: the exponent of
// each column at the time each block was finished is recorded and a final
// k_fixup pass multiplies every block by the power of two it still owes.
//
// Many problems (uneven sizes) run in the same launches: each launch receives
// a table of problem descriptors and grid.z indexes the problem.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "msts_common.cuh"
#include "msts_diag.h"
#include "msts_engine.h"
#include "msts_ozaki.h"
#include "msts_trace.h"

namespace msts {

constexpr int kNumSMs = 152;


// ---------------------------------------------------------------------------
// Safe-variant preprocessing (Alg. 5 set-up, the column norms of Sec. 3).
// ---------------------------------------------------------------------------

// |Re z|, |Im z| bit patterns: the larger one (as a nonnegative int64, ordered
// like the magnitudes) and whether both are finite.  max(|Re|, |Im|) <=
// |z| <= sqrt 2 max(|Re|, |Im|), so an element whose larger component is
// below half the largest seen cannot have the largest modulus: only the few
// others need the FP64 square sum (FP64 arithmetic is slow on this part, the
// integer tests are not).
__device__ __forceinline__ long long zmaxbits(double2 z) {
  return max(__double_as_longlong(z.x) & 0x7fffffffffffffffLL, __double_as_longlong(z.y) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool zfinite_bits(double2 z) {
  return ((__double2hiint(z.x) & 0x7ff00000) != 0x7ff00000) && ((__double2hiint(z.y) & 0x7ff00000) != 0x7ff00000);
}
__device__ __forceinline__ long long half_bits(long long m) {   // bits of m / 2 (or 0)
  return m >= (1LL << 53) ? m - (1LL << 52) : 0;
}

// The set-up and fix-up kernels below give each column a CTA of kColThreads
// threads (the columns of a triangle differ in length; one warp per column
// left them bound by the latency of its serial loop).
constexpr int kColThreads = 256;
// Maximum of v over the CTA (every thread gets it); red holds kColThreads / 32 values.
__device__ __forceinline__ long long cta_max_ll(long long v, long long *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, (long long)__shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();                                       // red free from an earlier call
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  v = red[0];
#pragma unroll
  for (int w = 1; w < kColThreads / 32; ++w) v = max(v, red[w]);
  return v;
}

// One CTA per column k: cin[k] = max_{lo(k) <= r < k} |U(r,k)| (within its own
// block, diagonal excluded) and cup[k] = max_{r < lo(k)} |U(r,k)| (above it);
// with useV the same for V into cinV, cupV (generalized problem).
__global__ void __launch_bounds__(kColThreads)
k_colnorms(const __grid_constant__ ProbTable tab, int nb, uint32_t *status, int useV) {
  const Prob &P = tab.p[blockIdx.z];
  __shared__ long long red[kColThreads / 32];
  if (P.n == 0 || (useV && !P.V)) return;
  if (!useV && blockIdx.x == 0 && threadIdx.x == 0) *P.delta = 0.0;   // the zero-pivot flag of k_zero_scan
  const int k = blockIdx.x;
  if (k >= P.m) return;
  const int b = (P.m - 1 - k) / nb;
  int lo, hi;
  block_range(P, b, nb, lo, hi);
  // Maxima of squared moduli (as bits: nonnegative doubles order like their
  // bits), one square root per column at the end (|U(i,k)| < 2^48 is the
  // documented range, so the squares cannot overflow).  Each thread's running
  // maxima of the larger components select its candidates: the element of
  // largest modulus in each range is one of them.
  long long Min = 0, Mup = 0, Mall = 0, cin = 0, cup = 0, amax = 0;
  bool finite = true;
  const double2 *col = useV ? P.V + (long long)k * P.ldv : P.U + (long long)k * P.ldu;
#pragma unroll 4
  for (int r = threadIdx.x; r <= k; r += kColThreads) {
    const double2 u = col[r];
    finite &= zfinite_bits(u);
    const long long m = zmaxbits(u);
    const bool in_in = r >= lo && r < k, in_up = r < lo;
    Mall = max(Mall, m);
    if (in_in) Min = max(Min, m);
    if (in_up) Mup = max(Mup, m);
    const bool cand = m != 0 && (m >= half_bits(Mall) || (in_in && m >= half_bits(Min)) ||
                                 (in_up && m >= half_bits(Mup)));
    if (cand) {
      const long long a2 = __double_as_longlong(fma(u.x, u.x, u.y * u.y));
      amax = max(amax, a2);
      if (in_in) cin = max(cin, a2);
      if (in_up) cup = max(cup, a2);
    }
  }
  const bool all_finite = __syncthreads_and(finite);
  cin = cta_max_ll(cin, red);
  cup = cta_max_ll(cup, red);
  amax = cta_max_ll(amax, red);
  if (threadIdx.x == 0) {
    (useV ? P.cinV : P.cin)[k] = sqrt(__longlong_as_double(cin));
    (useV ? P.cupV : P.cup)[k] = sqrt(__longlong_as_double(cup));
    if (!all_finite) raise_status(status, MSTS_STATUS_NONFINITE);
    if (sqrt(__longlong_as_double(amax)) >= kRangeLimitU) raise_status(status, MSTS_STATUS_RANGE);
  }
}

// a == b for doubles, on the bit patterns (+0 == -0; a NaN equals nothing).
__device__ __forceinline__ bool deq_bits(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  if (((ia | ib) & 0x7fffffffffffffffLL) == 0) return true;
  const bool nan = (((unsigned)__double2hiint(a) >> 20) & 0x7ffu) == 0x7ffu &&
                   ((__double2hiint(a) & 0xfffff) | __double2loint(a)) != 0;
  return !nan && ia == ib;
}

// delta (Sec. 3) replaces a pivot U(i,i) - lambda_j that is exactly zero, so
// ||U||_inf is needed only if some shift equals a diagonal entry of a row it
// visits (rows i < j for Alg. 6's right-hand sides, all rows otherwise).
// One thread per shift and CTA per 256 diagonal entries (staged in shared
// memory); *delta is
// set nonzero (k_colnorms zeroed it) when such a pair exists.
__global__ void k_zero_scan(const __grid_constant__ ProbTable tab, int shortcut) {
  const Prob &P = tab.p[blockIdx.z];
  __shared__ double2 dg[256], dv[256];
  if (P.m == 0 || P.n == 0) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = j < P.n;
  const double2 lam = act ? P.shifts[(long long)j * P.shift_stride] : make_double2(0.0, 0.0);
  const int end = !act ? 0 : (shortcut ? min(j, P.m) : P.m);
  const int i0 = 256 * blockIdx.y;                       // this CTA's 256 diagonal entries
  if (i0 >= P.m) return;
  if (i0 + (int)threadIdx.x < P.m) dg[threadIdx.x] = P.U[(long long)(i0 + threadIdx.x) * (P.ldu + 1)];
  if (P.V && i0 + (int)threadIdx.x < P.m) dv[threadIdx.x] = P.V[(long long)(i0 + threadIdx.x) * (P.ldv + 1)];
  __syncthreads();
  bool hit = false;
  const int cnt = min(256, end - i0);
  if (!P.V) {
    for (int t = 0; t < cnt; ++t) hit |= deq_bits(dg[t].x, lam.x) && deq_bits(dg[t].y, lam.y);
  } else {                                               // U(i,i) - lambda V(i,i), as the diagonal step forms it
    for (int t = 0; t < cnt; ++t) {
      const double2 p = zsub(dg[t], zmul_rn(lam, dv[t]));
      hit |= deq_bits(p.x, 0.0) && deq_bits(p.y, 0.0);
    }
  }
  if (hit) *P.delta = 1.0;
}

// One warp per row: rowsum[r] = sum_{c >= r} |U(r,c)| (lanes stride over the
// columns, then a fixed-order warp reduction: deterministic); only when a zero
// pivot can occur (k_zero_scan).
__global__ void k_rowsums(const __grid_constant__ ProbTable tab, int useV) {
  const Prob &P = tab.p[blockIdx.z];
  if (P.n == 0 || *P.delta == 0.0 || (useV && !P.V)) return;
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= P.m) return;
  double s = 0.0;
  const double2 *row = useV ? P.V + r : P.U + r;
  const long long ld = useV ? P.ldv : P.ldu;
  for (int c = r + lane; c < P.m; c += 32) {
    const double2 u = row[(long long)c * ld];
    s += sqrt(fma(u.x, u.x, u.y * u.y));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) (useV ? P.rowsumV : P.rowsum)[r] = s;
}

// C_blk per block (Alg. 5; and of V, Alg. 9), and delta = max(eps ||U||_inf,
// DBL_MIN) when a zero pivot can occur (otherwise delta is never read; DBL_MIN
// is stored).  Generalized: delta = eps ||U||_inf and deltaV = eps ||V||_inf,
// delta_j = max(delta + |s_j| deltaV, DBL_MIN) being formed per shift.
__global__ void k_safe_finish(const __grid_constant__ ProbTable tab, int nb) {
  const Prob &P = tab.p[blockIdx.z];
  __shared__ double red[32];
  if (P.m == 0 || P.n == 0) return;
  for (int b = threadIdx.x; b < P.nblk; b += blockDim.x) {
    int lo, hi;
    block_range(P, b, nb, lo, hi);
    double c = 0.0, cv = 0.0;
    for (int k = lo; k < hi; ++k) c += P.cup[k];
    P.cblk[b] = c;
    if (P.V) {
      for (int k = lo; k < hi; ++k) cv += P.cupV[k];
      P.cblkV[b] = cv;
    }
  }
  const bool need = *P.delta != 0.0;                     // uniform
  __syncthreads();
  if (!need) {
    if (threadIdx.x == 0) {
      *P.delta = kDblMin;
      if (P.V) *P.deltaV = 0.0;
    }
    return;
  }
  // max row sum of U (and of V): eps ||U||_inf, eps ||V||_inf
  for (int w = 0; w < (P.V ? 2 : 1); ++w) {
    const double *rs = w ? P.rowsumV : P.rowsum;
    double mx = 0.0;
    for (int r = threadIdx.x; r < P.m; r += blockDim.x) mx = fmax(mx, rs[r]);
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
      v = warp_max(v);
      if (threadIdx.x == 0) {
        const double d = kEps * v;
        if (w) *P.deltaV = d;
        else *P.delta = P.V ? d : (d < kDblMin ? kDblMin : d);   // generalized: capped per shift
      }
    }
    __syncthreads();
  }
}

// One CTA per column: G(j) = ||B(:,j)||_inf over the active rows, e_j = 0.
// The scaled square sums are formed only for the candidates of the maximum
// (see zmaxbits), with the same values as for all elements.
__global__ void __launch_bounds__(kColThreads)
k_safe_init(const __grid_constant__ ProbTable tab, int shortcut, uint32_t *status) {
  const Prob &P = tab.p[blockIdx.z];
  __shared__ long long red[kColThreads / 32];
  const int j = blockIdx.x;
  if (j >= P.n) return;
  const int end = shortcut ? min(j, P.m) : P.m;
  bool finite = true;
  const double2 *col = P.B + (long long)j * P.ldb;
  long long M = 0;
#pragma unroll 4
  for (int r = threadIdx.x; r < end; r += kColThreads) {
    const double2 v = col[r];
    finite &= zfinite_bits(v);
    M = max(M, zmaxbits(v));
  }
  const bool all_finite = __syncthreads_and(finite);
  M = cta_max_ll(M, red);
  const int E = min(max((int)(M >> 52) - 1023, -1022), 1022);   // zexp of the largest component
  const double sc = pow2i(-E);
  const long long thr = half_bits(M);
  long long g2 = 0;
#pragma unroll 4
  for (int r = threadIdx.x; r < end; r += kColThreads) {  // the column again, from L2
    const double2 v = col[r];
    if (M != 0 && zmaxbits(v) >= thr) {
      const double a = v.x * sc, bb = v.y * sc;
      g2 = max(g2, __double_as_longlong(fma(a, a, bb * bb)));
    }
  }
  g2 = cta_max_ll(g2, red);
  if (threadIdx.x == 0) {
    const double g = sqrt(__longlong_as_double(g2)) * pow2i(E);
    P.G[j] = g;
    P.e[j] = 0;
    P.pend[j] = 0;
    if (!all_finite) raise_status(status, MSTS_STATUS_NONFINITE);
    if (g >= omega()) raise_status(status, MSTS_STATUS_RANGE);
  }
}

// TREVC set-up (Alg. 6): Z = -T strictly above the diagonal, zero elsewhere.
__global__ void k_trevc_setup(const double2 *T, long long ldt, int m, double2 *Z, long long ldz) {
  const int j = blockIdx.x;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (r < j) {
      const double2 t = T[r + (long long)j * ldt];
      v = make_double2(-t.x, -t.y);
    }
    Z[r + (long long)j * ldz] = v;
  }
}

template <int BM, int BN>
struct GemmCfg {
  static constexpr int kThreads = 256;
  static constexpr int LDA = BM + 1, LDX = BN + 1;
  static constexpr int TM = BM / 32, TN = BN / 8;   // outputs per thread
  template <int NB>
  static constexpr size_t smem() { return (size_t)NB * (LDA + LDX) * sizeof(double2); }
};

template <int NB, int BM, int BN, bool SAFE, bool CONJ, bool GEN = false>
__global__ void __launch_bounds__(256)
k_gemm(const __grid_constant__ ProbTable tab, int step, int shortcut) {
  using C = GemmCfg<BM, BN>;
  constexpr int LDA = C::LDA, LDX = C::LDX, TM = C::TM, TN = C::TN, NT = C::kThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *sA = reinterpret_cast<double2 *>(smem_raw);   // [NB][LDA]
  double2 *sX = sA + NB * LDA;                            // [NB][LDX]
  const Prob &P = tab.p[blockIdx.z];
  if (step >= P.nblk) return;
  const int b = CONJ ? P.nblk - 1 - step : step;
  int lo, hi;
  block_range(P, b, NB, lo, hi);
  const int K = hi - lo;
  const int rend = CONJ ? P.m : lo;
  const int r0 = (CONJ ? hi : 0) + blockIdx.y * BM;
  if (r0 >= rend) return;
  const int c0 = (shortcut ? lo + 1 : 0) + blockIdx.x * BN;
  if (c0 >= P.n) return;
  const int tid = threadIdx.x;

  for (int idx = tid; idx < NB * BM; idx += NT) {
    int k, r;
    if (!CONJ) { k = idx / BM; r = idx - k * BM; }   // coalesced along U's rows
    else { r = idx / NB; k = idx - r * NB; }          // coalesced along U's rows (= k)
    double2 v = make_double2(0.0, 0.0);
    if (k < K && r0 + r < rend)
      v = CONJ ? zconj(P.U[(lo + k) + (long long)(r0 + r) * P.ldu])
               : P.U[(r0 + r) + (long long)(lo + k) * P.ldu];
    sA[k * LDA + r] = v;
  }
  for (int idx = tid; idx < NB * BN; idx += NT) {
    const int c = idx / NB, k = idx - c * NB;
    double2 v = make_double2(0.0, 0.0);
    if (k < K && c0 + c < P.n) v = P.B[(lo + k) + (long long)(c0 + c) * P.ldb];
    sX[k * LDX + c] = v;
  }
  // Generalized problem (Alg. 8/9): also V(I0,I1), for B(I0,:) += V(I0,I1) (s X(I1,:)).
  constexpr bool gen = GEN && !CONJ;
  double2 *sV = sX + NB * LDX;                           // [NB][LDA]
  if constexpr (gen)
    for (int idx = tid; idx < NB * BM; idx += NT) {
      const int kk = idx / BM, r = idx - kk * BM;
      sV[kk * LDA + r] = (kk < K && r0 + r < rend) ? P.V[(r0 + r) + (long long)(lo + kk) * P.ldv]
                                                   : make_double2(0.0, 0.0);
    }
  __syncthreads();

  const int tr = tid & 31, tc = tid >> 5;
  double2 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[i][c] = make_double2(0.0, 0.0);
  double2 accv[TM][TN];                                  // V(I0,I1) X(I1,:) (generalized)
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int c = 0; c < TN; ++c) accv[i][c] = make_double2(0.0, 0.0);
  if constexpr (!gen) {
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      double2 a[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = sA[k * LDA + tr + 32 * i];
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        const double2 x = sX[k * LDX + tc + 8 * c];
#pragma unroll
        for (int i = 0; i < TM; ++i) acc[i][c] = zfma(acc[i][c], a[i], x);
      }
    }
  } else {
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
      double2 a[TM], w[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        a[i] = sA[k * LDA + tr + 32 * i];
        w[i] = sV[k * LDA + tr + 32 * i];
      }
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        const double2 x = sX[k * LDX + tc + 8 * c];
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          acc[i][c] = zfma(acc[i][c], a[i], x);
          accv[i][c] = zfma(accv[i][c], w[i], x);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < TN; ++c) {
    const int col = c0 + tc + 8 * c;
    if (col >= P.n) continue;
    const int pend = SAFE ? P.pend[col] : 0;
    const double2 lam = gen ? P.shifts[(long long)col * P.shift_stride] : make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int row = r0 + tr + 32 * i;
      if (row >= rend) continue;
      double2 *p = P.B + row + (long long)col * P.ldb;
      double2 v = *p;
      if (SAFE && pend) v = zshift(v, pend);
      v = zsub(v, acc[i][c]);
      if (gen) v = zfma(v, lam, accv[i][c]);             // + s_j V(I0,I1) X(I1,j)
      *p = v;
    }
  }
}

// The same substitution step with the product in FP32 (operands rounded to
// float, FP32 accumulation, the update applied to the FP64 B): the
// low-precision solve of the mixed-precision form.  Plain upper solves only.
template <int NB, int BM, int BN, bool SAFE, bool CONJ>
__global__ void __launch_bounds__(256)
k_gemm_f32(const __grid_constant__ ProbTable tab, int step, int shortcut) {
  using C = GemmCfg<BM, BN>;
  constexpr int LDA = C::LDA, LDX = C::LDX, TM = C::TM, TN = C::TN, NT = C::kThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sA = reinterpret_cast<float2 *>(smem_raw);     // [NB][LDA]
  float2 *sX = sA + NB * LDA;                             // [NB][LDX]
  const Prob &P = tab.p[blockIdx.z];
  if (step >= P.nblk) return;
  const int b = CONJ ? P.nblk - 1 - step : step;
  int lo, hi;
  block_range(P, b, NB, lo, hi);
  const int K = hi - lo;
  const int rend = CONJ ? P.m : lo;
  const int r0 = (CONJ ? hi : 0) + blockIdx.y * BM;
  if (r0 >= rend) return;
  const int c0 = (shortcut ? lo + 1 : 0) + blockIdx.x * BN;
  if (c0 >= P.n) return;
  const int tid = threadIdx.x;

  for (int idx = tid; idx < NB * BM; idx += NT) {
    int k, r;
    if (!CONJ) { k = idx / BM; r = idx - k * BM; }   // coalesced along U's rows
    else { r = idx / NB; k = idx - r * NB; }          // coalesced along U's rows (= k)
    double2 v = make_double2(0.0, 0.0);
    if (k < K && r0 + r < rend)
      v = CONJ ? zconj(P.U[(lo + k) + (long long)(r0 + r) * P.ldu])
               : P.U[(r0 + r) + (long long)(lo + k) * P.ldu];
    sA[k * LDA + r] = make_float2((float)v.x, (float)v.y);
  }
  for (int idx = tid; idx < NB * BN; idx += NT) {
    const int c = idx / NB, k = idx - c * NB;
    double2 v = make_double2(0.0, 0.0);
    if (k < K && c0 + c < P.n) v = P.B[(lo + k) + (long long)(c0 + c) * P.ldb];
    sX[k * LDX + c] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();

  const int tr = tid & 31, tc = tid >> 5;
  float2 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[i][c] = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    float2 a[TM];
#pragma unroll
    for (int i = 0; i < TM; ++i) a[i] = sA[k * LDA + tr + 32 * i];
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const float2 x = sX[k * LDX + tc + 8 * c];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        acc[i][c].x = fmaf(a[i].x, x.x, fmaf(-a[i].y, x.y, acc[i][c].x));
        acc[i][c].y = fmaf(a[i].x, x.y, fmaf(a[i].y, x.x, acc[i][c].y));
      }
    }
  }
#pragma unroll
  for (int c = 0; c < TN; ++c) {
    const int col = c0 + tc + 8 * c;
    if (col >= P.n) continue;
    const int pend = SAFE ? P.pend[col] : 0;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int row = r0 + tr + 32 * i;
      if (row >= rend) continue;
      double2 *p = P.B + row + (long long)col * P.ldb;
      double2 v = *p;
      if (SAFE && pend) v = zshift(v, pend);
      *p = make_double2(v.x - (double)acc[i][c].x, v.y - (double)acc[i][c].y);
    }
  }
}

// Final lazy rescale (safe variant): block b of column j was finished with
// exponent E[b][j]; it still owes 2^-(e_j - E[b][j]).  Also writes s_j.
__global__ void __launch_bounds__(kColThreads)
k_fixup(const __grid_constant__ ProbTable tab, int nb, int shortcut) {
  const Prob &P = tab.p[blockIdx.z];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x;                              // one CTA per column, its warps over the blocks
  if (j >= P.n) return;
  const int ej = P.e[j];
  const int end = shortcut ? min(j, P.m) : P.m;
  double2 *col = P.B + (long long)j * P.ldb;
  for (int b = warp; b < P.nblk; b += kColThreads / 32) {
    int lo, hi;
    block_range(P, b, nb, lo, hi);
    if (lo >= end) continue;
    const int d = ej - P.E[(long long)b * P.n + j];
    if (d == 0) continue;
    const int top = min(hi, end);
    for (int r = lo + lane; r < top; r += 32) col[r] = zshift(col[r], d);
  }
  if (threadIdx.x == 0) {
    const double s = scalbn(1.0, -ej);
    if (P.scales) P.scales[j] = s;
    if (P.scale_exp) P.scale_exp[j] = ej;
    if (P.diag_z) col[j] = make_double2(s, 0.0);
  }
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static size_t prob_ws_bytes(int m, int n, int nb, bool safe, bool gen) {
  if (!safe || m == 0 || n == 0) return 0;
  const size_t nblk = (size_t)(m + nb - 1) / nb;
  size_t s = 0;
  if (gen) {
    s += align256(sizeof(double) * m) * 3;      // cinV, cupV, rowsumV
    s += align256(sizeof(double) * nblk);       // cblkV
    s += align256(sizeof(double));              // deltaV
  }
  s += align256(sizeof(double) * n);            // G
  s += align256(sizeof(int) * n) * 2;           // e, pend
  s += align256(sizeof(int) * nblk * n);        // E
  s += align256(sizeof(double) * m) * 3;        // cin, cup, rowsum
  s += align256(sizeof(double) * nblk);         // cblk
  s += align256(sizeof(double));                // delta
  return s;
}

size_t engine_workspace_bytes(const EngineProblem *probs, int count, int nb, bool safe) {
  size_t s = 0;
  for (int p = 0; p < count; ++p) s += prob_ws_bytes(probs[p].m, probs[p].n, nb, safe, probs[p].V != nullptr);
  return s;
}

template <typename T>
static T *carve(char *&cur, size_t count) {
  T *p = reinterpret_cast<T *>(cur);
  cur += align256(sizeof(T) * count);
  return p;
}

template <int NB, int BM, int BN, bool SAFE, bool CONJ>
static void launch_gemm(const ProbTable &tab, int gx, int gy, int s, bool shortcut, bool lp,
                        cudaStream_t st, bool gen = false) {
  // the generalized form also stages V(I0,I1) (NB x LDA)
  const size_t smem = GemmCfg<BM, BN>::template smem<NB>() +
                      (gen ? (size_t)NB * GemmCfg<BM, BN>::LDA * sizeof(double2) : 0);
  if (lp && !SAFE && !CONJ) {
    cudaFuncSetAttribute(k_gemm_f32<NB, BM, BN, SAFE, CONJ>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gemm_f32<NB, BM, BN, SAFE, CONJ><<<dim3(gx, gy, tab.count), 256, smem, st>>>(tab, s, shortcut ? 1 : 0);
    return;
  }
  if constexpr (!CONJ) {
    if (gen) {
      cudaFuncSetAttribute(k_gemm<NB, BM, BN, SAFE, CONJ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      k_gemm<NB, BM, BN, SAFE, CONJ, true><<<dim3(gx, gy, tab.count), 256, smem, st>>>(tab, s, shortcut ? 1 : 0);
      return;
    }
  }
  cudaFuncSetAttribute(k_gemm<NB, BM, BN, SAFE, CONJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  k_gemm<NB, BM, BN, SAFE, CONJ><<<dim3(gx, gy, tab.count), 256, smem, st>>>(tab, s, shortcut ? 1 : 0);
}

template <int NB, bool SAFE, bool CONJ>
static cudaError_t run_steps(const ProbTable &tab, const EngineProblem *probs, int count,
                             bool shortcut, bool lp, uint32_t *status, cudaStream_t st) {
  int maxblk = 0;
  for (int p = 0; p < count; ++p) maxblk = std::max(maxblk, (probs[p].m + NB - 1) / NB);
  const bool tracing = trace_on();
  const bool gen = count > 0 && probs[0].V != nullptr;   // a table is all generalized or none
  bool any_oz = false;                                   // batched: tensor-core plans, one per problem
  for (int p = 0; p < count; ++p) any_oz = any_oz || probs[p].oz != nullptr;
  for (int s = 0; s < maxblk; ++s) {
    int dx = 0, rows_max = 0, cols_max = 0;
    long long tiles_big = 0, tiles_mid = 0, total_cols = 0;
    double gflops = 0, gbytes = 0, dflops = 0, dbytes = 0;
    for (int p = 0; p < count; ++p) {
      const int m = probs[p].m, n = probs[p].n, nblk = (m + NB - 1) / NB;
      if (s >= nblk || n == 0) continue;
      const int b = CONJ ? nblk - 1 - s : s;
      const int hi = m - b * NB, lo = std::max(0, hi - NB);
      const int ncols = shortcut ? n - (lo + 1) : n;
      if (ncols <= 0) continue;
      const int rows = CONJ ? m - hi : lo;
      const double K = hi - lo;
      dx = std::max(dx, ncols);
      total_cols += ncols;
      // algorithmic work: 8 real FLOPs per complex multiply-add
      dflops += (gen ? 8.0 : 4.0) * K * K * ncols;
      dbytes += 16.0 * K * K / 2 + 32.0 * K * ncols;
      if (rows > 0) {
        rows_max = std::max(rows_max, rows);
        cols_max = std::max(cols_max, ncols);
        tiles_big += (long long)((rows + 63) / 64) * ((ncols + 31) / 32);
        tiles_mid += (long long)((rows + 31) / 32) * ((ncols + 15) / 16);
        gflops += (gen ? 16.0 : 8.0) * rows * K * ncols;
        gbytes += 16.0 * rows * K + 16.0 * K * ncols + 32.0 * (double)rows * ncols;
      }
    }
    if (dx > 0) {
      void *h = tracing ? trace_start(1, dflops, dbytes, st) : nullptr;
      const cudaError_t e = launch_diag(tab, NB, SAFE, CONJ, s, shortcut ? 1 : 0, dx, total_cols,
                                        status, st, gen);
      if (e != cudaSuccess) return e;
      trace_stop(h, st);
      count_launches(1);
    }
    if (rows_max > 0 && count == 1 && probs[0].oz) {
      // Substitution step on the tensor cores (digit-plane product).
      const int m = probs[0].m, nblk = (m + NB - 1) / NB;
      const int b = CONJ ? nblk - 1 - s : s;
      const int hi = m - b * NB, lo = std::max(0, hi - NB);
      const int jstart = shortcut ? lo + 1 : 0;
      // (generalized: the X planes carry [X; -lambda X] and are sliced here)
      const cudaError_t e = ozaki_update(*probs[0].oz, b, lo, hi, probs[0].B, probs[0].ldb, jstart,
                                         probs[0].n - jstart, SAFE ? tab.p[0].pend : nullptr, status,
                                         gflops, st, tab.p[0].oz_bp != nullptr, gen ? probs[0].shifts : nullptr,
                                         probs[0].shift_stride, lp);
      if (e != cudaSuccess) return e;
    } else if (rows_max > 0 && count > 1 && any_oz) {
      // Batched substitution step on the tensor cores: every problem's panel
      // in one launch (grid slice z = problem).
      OzBatchStep bs[kMaxProbs];
      for (int p = 0; p < count; ++p) {
        const int m = probs[p].m, n = probs[p].n, nblk = (m + NB - 1) / NB;
        bs[p] = OzBatchStep{};
        if (s >= nblk || n == 0 || !probs[p].oz) continue;
        const int b = CONJ ? nblk - 1 - s : s;
        const int hi = m - b * NB, lo = std::max(0, hi - NB);
        const int jstart = shortcut ? lo + 1 : 0;
        bs[p].plan = probs[p].oz;
        bs[p].b = b; bs[p].lo = lo; bs[p].hi = hi;
        bs[p].B = probs[p].B; bs[p].ldb = probs[p].ldb;
        bs[p].jstart = jstart; bs[p].ncols = n - jstart;
        bs[p].pend = SAFE ? tab.p[p].pend : nullptr;
      }
      const cudaError_t e = ozaki_update_batched(bs, count, status, st);
      if (e != cudaSuccess) return e;
    } else if (rows_max > 0) {
      // FP64 throughput per SM is low, so the tile is chosen to give the grid
      // at least two waves of CTAs over the 152 SMs when the problem allows.
      void *h = tracing ? trace_start(0, gflops, gbytes, st) : nullptr;
      if (tiles_big >= 2 * kNumSMs)
        launch_gemm<NB, 64, 32, SAFE, CONJ>(tab, (cols_max + 31) / 32, (rows_max + 63) / 64, s, shortcut, lp, st, gen);
      else if (tiles_mid >= kNumSMs)
        launch_gemm<NB, 32, 16, SAFE, CONJ>(tab, (cols_max + 15) / 16, (rows_max + 31) / 32, s, shortcut, lp, st, gen);
      else
        launch_gemm<NB, 32, 8, SAFE, CONJ>(tab, (cols_max + 7) / 8, (rows_max + 31) / 32, s, shortcut, lp, st, gen);
      trace_stop(h, st);
      count_launches(1);
    }
  }
  return cudaGetLastError();
}

template <int NB>
static cudaError_t run_nb(const ProbTable &tab, const EngineProblem *probs, int count, bool safe,
                          bool conj, bool shortcut, bool lp, uint32_t *status, cudaStream_t st) {
  if (safe) return run_steps<NB, true, false>(tab, probs, count, shortcut, false, status, st);
  if (conj) return run_steps<NB, false, true>(tab, probs, count, shortcut, false, status, st);
  return run_steps<NB, false, false>(tab, probs, count, shortcut, lp, status, st);
}

cudaError_t engine_run(const EngineProblem *probs, int count, int nb, bool safe, bool conj,
                       bool shortcut, void *ws, uint32_t *status, cudaStream_t st, bool lp) {
  char *cur = static_cast<char *>(ws);
  bool any_oz = false;
  for (int i = 0; i < count; ++i) any_oz = any_oz || probs[i].oz != nullptr;
  if (any_oz) status = ozaki_call_status(status, st);   // one word (cleared once) for every step
  for (int base = 0; base < count; base += kMaxProbs) {
    const int cnt = std::min(kMaxProbs, count - base);
    ProbTable tab;
    tab.count = cnt;
    int maxm = 0, maxn = 0;
    for (int i = 0; i < cnt; ++i) {
      const EngineProblem &q = probs[base + i];
      Prob &P = tab.p[i];
      P = Prob{};
      P.U = q.U; P.ldu = q.ldu; P.shifts = q.shifts; P.shift_stride = q.shift_stride;
      P.B = q.B; P.ldb = q.ldb; P.scales = q.scales; P.scale_exp = q.scale_exp;
      P.m = q.m; P.n = q.n; P.nblk = (q.m + nb - 1) / nb; P.diag_z = q.diag_z;
      P.V = q.V; P.ldv = q.ldv;
      if (safe && q.m > 0 && q.n > 0) {
        P.G = carve<double>(cur, q.n);
        P.e = carve<int>(cur, q.n);
        P.pend = carve<int>(cur, q.n);
        P.E = carve<int>(cur, (size_t)P.nblk * q.n);
        P.cin = carve<double>(cur, q.m);
        P.cup = carve<double>(cur, q.m);
        P.rowsum = carve<double>(cur, q.m);
        P.cblk = carve<double>(cur, P.nblk);
        P.delta = carve<double>(cur, 1);
        if (q.V) {
          P.cinV = carve<double>(cur, q.m);
          P.cupV = carve<double>(cur, q.m);
          P.rowsumV = carve<double>(cur, q.m);
          P.cblkV = carve<double>(cur, P.nblk);
          P.deltaV = carve<double>(cur, 1);
        }
      }
      maxm = std::max(maxm, q.m);
      maxn = std::max(maxn, q.n);
    }
    if (maxm == 0 || maxn == 0) continue;
    for (int i = 0; i < cnt; ++i) {           // the diagonal step writes the X digit planes
      const EngineProblem &q = probs[base + i];
      if (q.oz && !q.V) {
        tab.p[i].oz_bp = reinterpret_cast<uint32_t *>(q.oz->bp);
        tab.p[i].oz_cexp = q.oz->cexp;
        tab.p[i].oz_kb = q.oz->KB;
      }
    }
    const int sc = shortcut ? 1 : 0;
    if (safe) {
      const bool gen = probs[base].V != nullptr;
      k_colnorms<<<dim3(maxm, 1, cnt), kColThreads, 0, st>>>(tab, nb, status, 0);
      if (gen) k_colnorms<<<dim3(maxm, 1, cnt), kColThreads, 0, st>>>(tab, nb, status, 1);
      k_zero_scan<<<dim3((maxn + 255) / 256, (maxm + 255) / 256, cnt), 256, 0, st>>>(tab, sc);
      k_rowsums<<<dim3((maxm + 7) / 8, 1, cnt), 256, 0, st>>>(tab, 0);
      if (gen) k_rowsums<<<dim3((maxm + 7) / 8, 1, cnt), 256, 0, st>>>(tab, 1);
      k_safe_finish<<<dim3(1, 1, cnt), 256, 0, st>>>(tab, nb);
      k_safe_init<<<dim3(maxn, 1, cnt), kColThreads, 0, st>>>(tab, sc, status);
      count_launches(gen ? 7 : 5);
    }
    cudaError_t err;
    switch (nb) {
      case 16: err = run_nb<16>(tab, probs + base, cnt, safe, conj, shortcut, lp, status, st); break;
      case 32: err = run_nb<32>(tab, probs + base, cnt, safe, conj, shortcut, lp, status, st); break;
      case 64: err = run_nb<64>(tab, probs + base, cnt, safe, conj, shortcut, lp, status, st); break;
      default: return cudaErrorInvalidValue;
    }
    if (err != cudaSuccess) return err;
    if (safe) {
      k_fixup<<<dim3(maxn, 1, cnt), kColThreads, 0, st>>>(tab, nb, sc);
      count_launches(1);
    }
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

cudaError_t engine_trevc_setup(const double2 *T, long long ldt, int m, double2 *Z, long long ldz,
                               cudaStream_t st) {
  if (m > 0) {
    k_trevc_setup<<<m, 256, 0, st>>>(T, ldt, m, Z, ldz);
    count_launches(1);
  }
  return cudaGetLastError();
}

// Alg. 10's set-up: lam[j] = T(j,j) / S(j,j), Z(r,j) = lam[j] S(r,j) - T(r,j)
// for r < j and zero elsewhere (the oracle's rounding: no fused operations).
__global__ void k_gtrevc_setup(const double2 *T, long long ldt, const double2 *S, long long lds, int m,
                               double2 *Z, long long ldz, double2 *lam) {
  const int j = blockIdx.y;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  const double2 lj = zdiv_rn(T[(long long)j * (ldt + 1)], S[(long long)j * (lds + 1)]);
  if (r == 0) lam[j] = lj;
  Z[r + (long long)j * ldz] = r < j ? zsub(zmul_rn(lj, S[r + (long long)j * lds]), T[r + (long long)j * ldt])
                                    : make_double2(0.0, 0.0);
}

cudaError_t engine_gtrevc_setup(const double2 *T, long long ldt, const double2 *S, long long lds, int m,
                                double2 *Z, long long ldz, double2 *lam, cudaStream_t st) {
  if (m > 0) {
    k_gtrevc_setup<<<dim3((m + 255) / 256, m), 256, 0, st>>>(T, ldt, S, lds, m, Z, ldz, lam);
    count_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace msts
