// msts_diag.cu -- the diagonal-block step of the blocked multi-shift solve:
// for every shift j, back substitution on U(I1,I1) - lambda_j I (Alg. 3), or
// in the safe variant Alg. 4 on that block followed by the column update of
// Alg. 5; forward substitution on the conjugate transpose for MSTS_CONJ_TRANS.
//
// GB300 mapping.  The FP64 unit of each SM sub-partition retires one warp
// instruction per ~64 cycles whatever the number of active lanes, and an FP64
// division costs ~10 dependent instructions.  So
//   - each shift is handled by a group of L lanes (L = 4..32, chosen per launch
//     so that enough warps exist to occupy every sub-partition); lane l of the
//     group owns rows l, l + L, l + 2L, ... of the block in registers;
//   - the reciprocals of all pivots are formed up front, in parallel over the
//     rows, so the serial chain of the substitution has no division in it;
//   - U(I1,I1) is staged once per CTA in shared memory and read by broadcast.
// All warp shuffles sit outside data-dependent branches; decisions that need
// them (the safe variant's plain/safeguarded choice) are made warp-uniform.
#include <algorithm>

#include "msts_common.cuh"
#include "msts_digits.cuh"
#include "msts_diag.h"
#include "msts_diag_util.cuh"

namespace msts {

constexpr int kDiagThreads = 128;

// 1: Alg. 4's decisions by the serial chain in every block (tuning knob; the
// closed form gives the same values)
__device__ int g_alg4_chain_d = 0;

template <int L>
__device__ __forceinline__ double gshfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src, L); }
template <int L>
__device__ __forceinline__ int gshfl_i(int v, int src) { return __shfl_sync(0xffffffffu, v, src, L); }
template <int L>
__device__ __forceinline__ double2 gshfl_z(double2 v, int src) {
  return make_double2(gshfl<L>(v.x, src), gshfl<L>(v.y, src));
}
template <int L>
__device__ __forceinline__ double gmax(double v) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o, L));
  return v;
}
template <int L>
__device__ __forceinline__ int gmax_i(int v) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o, L));
  return v;
}
template <int L>
__device__ __forceinline__ long long gmax_ll(long long v) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v = max(v, (long long)__shfl_xor_sync(0xffffffffu, v, o, L));
  return v;
}

// GEN: the generalized problem (appendix, Alg. 8/9), U' = U(I1,I1) - s_j V(I1,I1):
// pivots U(i,i) - s_j V(i,i), AXPY entries U(r,i) - s_j V(r,i) (applied as
// x_i U(r,i) - (s_j x_i) V(r,i)), and in the safe form the column bounds
// cin_U + |s_j| cin_V, C_blk(U) + |s_j| C_blk(V) and
// delta_j = max(eps (||U||_inf + |s_j| ||V||_inf), DBL_MIN).
template <int NB, int L, bool SAFE, bool CONJ, bool GEN>
__global__ void __launch_bounds__(kDiagThreads)
k_diag(const __grid_constant__ ProbTable tab, int step, int shortcut, uint32_t *status) {
  constexpr int RPL = NB / L;            // rows per lane
  constexpr int SPW = 32 / L;            // shifts per warp
  constexpr int SPC = (kDiagThreads / 32) * SPW;
  constexpr int LD = NB + 1;
  static_assert(!(GEN && CONJ), "generalized solves are upper only");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *sU = reinterpret_cast<double2 *>(smem_raw);   // U(I1,I1) column-major, LD
  double2 *sV = sU + NB * LD;                            // V(I1,I1) (GEN)
  double *sC = reinterpret_cast<double *>(sU + (GEN ? 2 : 1) * NB * LD);   // within-block column norms
  double *sCV = sC + NB;                                 // those of V (GEN)
  double2 *sInv = reinterpret_cast<double2 *>(sC + (GEN ? 2 : 1) * NB);   // 1 / p_i: [i SPC + shift]

  const Prob &P = tab.p[blockIdx.z];
  if (step >= P.nblk) return;
  const int b = CONJ ? P.nblk - 1 - step : step;
  int lo, hi;
  block_range(P, b, NB, lo, hi);
  const int nbf = hi - lo;
  const int jcta = (shortcut ? lo + 1 : 0) + blockIdx.x * SPC;
  if (jcta >= P.n) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = lane & (L - 1);
  const int gs = warp * SPW + lane / L;   // this shift within the CTA
  const int j = jcta + gs;
  const bool active = j < P.n;
  const int nbe = !active ? 0 : (shortcut ? min(hi, j) - lo : nbf);   // TREVC: rows >= j stay zero
  double2 *col = P.B + (long long)(active ? j : 0) * P.ldb + lo;

  // U(I1,I1) (and V) to shared memory by asynchronous copies: no registers
  // held, every copy in flight at once, zeros below the diagonal and past the
  // block written by the copies themselves.  No kernel of the solve writes U,
  // V or the column norms, so after the first block step these copies start
  // before the wait for the previous kernel (they overlap its last CTAs).
  auto stage_u = [&]() {
    for (int idx = threadIdx.x; idx < NB * NB; idx += kDiagThreads) {
      const int c = idx / NB, r = idx - c * NB;
      const bool in = r <= c && c < nbf;
      cp_async16(&sU[c * LD + r], in ? &P.U[(lo + r) + (long long)(lo + c) * P.ldu] : P.U, in);
      if (GEN) cp_async16(&sV[c * LD + r], in ? &P.V[(lo + r) + (long long)(lo + c) * P.ldv] : P.V, in);
    }
    if (SAFE)
      for (int k = threadIdx.x; k < NB; k += kDiagThreads) {
        sC[k] = k < nbf ? P.cin[lo + k] : 0.0;
        if (GEN) sCV[k] = k < nbf ? P.cinV[lo + k] : 0.0;
      }
  };
  if (step > 0) stage_u();
  pdl_wait();                            // B and the safe state come from the kernel before
  if (step == 0) stage_u();

  // Every other global load the step needs is issued here, so that a warp
  // waits for one round trip to memory instead of several in sequence: the
  // shift, the right-hand side, delta and (safe) the column's scale state and
  // the block's bound C_blk.
  double2 lam = active ? P.shifts[(long long)j * P.shift_stride] : make_double2(0.0, 0.0);
  double2 y[RPL], inv[RPL];
#pragma unroll
  for (int q = 0; q < RPL; ++q) y[q] = l + L * q < nbe ? col[l + L * q] : make_double2(0.0, 0.0);
  const double delta_u = SAFE ? *P.delta : 0.0, delta_v = SAFE && GEN ? *P.deltaV : 0.0;
  int e_col = 0;
  double G_col = 0.0;
  if (SAFE && active) {
    e_col = P.e[j];
    G_col = P.G[j];
  }
  const double cblk_u = SAFE ? P.cblk[b] : 0.0, cblk_v = SAFE && GEN ? P.cblkV[b] : 0.0;

  cp_async_wait_all();
  __syncthreads();

  if (CONJ) lam = zconj(lam);
  const double al = GEN ? zabs_exp(lam) : 0.0;           // |s_j|
  const double dlt = !SAFE ? 0.0 : !GEN ? delta_u : fmax(__dadd_rn(delta_u, __dmul_rn(al, delta_v)), kDblMin);
  // the unperturbed pivot: U(i,i) - lambda (or - lambda V(i,i))
  auto pivot0 = [&](int i) {
    const double2 d = sU[i * LD + i];
    return GEN ? zsub(d, zmul_rn(lam, sV[i * LD + i])) : zsub(CONJ ? zconj(d) : d, lam);
  };
  auto pivot = [&](int i) {
    double2 p = pivot0(i);
    if (SAFE && zzero_words(p)) p = make_double2(dlt, 0.0);   // U(i,i) = lambda -> delta (Sec. 3)
    return p;
  };
  // bound on the off-diagonal column norm of row i's column of U'
  auto ccol = [&](int i) { return GEN ? __dadd_rn(sC[i], __dmul_rn(al, sCV[i])) : sC[i]; };

  int pex[RPL];                          // biased exponent field of max(|Re p|, |Im p|)
  bool zero_piv = false;
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int r = l + L * q;
    const bool v = r < nbe;
    const double2 p0 = pivot0(r);
    zero_piv |= v && zzero_words(p0);
    const double2 p = pivot(r);
    inv[q] = v ? zrecip(p) : make_double2(0.0, 0.0);
    sInv[r * SPC + gs] = inv[q];
    pex[q] = (int)(max(absbits(p.x), absbits(p.y)) >> 52);
  }
  __syncwarp();                          // sInv: read by the lanes of the same group
  if (zero_piv) raise_status(status, SAFE ? MSTS_STATUS_DELTA : MSTS_STATUS_ZERO_PIVOT);

  // x_i = y_i (1 / p_i) for row i = L qi + li, broadcast in the group: Re x_i
  // by the owner lane li, Im x_i by its partner li ^ 1 (zmul's two
  // multiply-adds, the same operations), half the FP64 instructions of the
  // multiply on the row's chain; the partner takes y_i from the owner and
  // 1 / p_i from shared memory.
  auto xrow = [&](int qi, int li) {
    const double yr = gshfl<L>(y[qi].x, li), yi = gshfl<L>(y[qi].y, li);
    const double2 ip = sInv[(L * qi + li) * SPC + gs];
    const bool re = l == li;
    const double m1 = __hiloint2double(__double2hiint(yi) ^ (re ? (int)0x80000000 : 0), __double2loint(yi));
    const double part = fma(yr, re ? ip.x : ip.y, m1 * (re ? ip.y : ip.x));
    return make_double2(gshfl<L>(part, li), gshfl<L>(part, li ^ 1));
  };

  // One row of the substitution: x_i = y_i / piv_i by the owner lane, broadcast
  // in the group, AXPY on the rows each lane owns.
  // Row i = L qi + li of the substitution: AXPY on the rows each lane owns.
  // The loops below unroll over the row slot qi only (so that qi is a
  // compile-time constant and y[] stays in registers) and run over li at run
  // time: the unrolled code stays small enough for the instruction cache, and
  // slots wholly on the dead side of row i still drop out at compile time.
  auto axpy = [&](int qi, int li, double2 xi) {
    const double2 cx = GEN ? zmul(lam, xi) : xi;          // s_j x_i for the V part
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      if (!CONJ) {        // rows l + L q < i
        if (q < qi || (q == qi && l < li)) {
          y[q] = zfms(y[q], xi, sU[(L * qi + li) * LD + l + L * q]);
          if (GEN) y[q] = zfma(y[q], cx, sV[(L * qi + li) * LD + l + L * q]);
        }
      } else {            // rows l + L q > i
        if (q > qi || (q == qi && l > li)) y[q] = zfms(y[q], xi, zconj(sU[(l + L * q) * LD + L * qi + li]));
      }
    }
  };
  auto substitute = [&]() {
#pragma unroll
    for (int s_ = 0; s_ < RPL; ++s_) {
      const int qi = CONJ ? s_ : RPL - 1 - s_;
#pragma unroll 1
      for (int u_ = 0; u_ < L; ++u_) {
        const int li = CONJ ? u_ : L - 1 - u_;
        const double2 xi = xrow(qi, li);   // zero for rows >= nbe
        if (l == li) y[qi] = xi;
        axpy(qi, li, xi);
      }
    }
  };

  // The digit planes of the block's X and their column exponents, for the
  // tensor-core substitution step that follows (integer work only; every lane
  // takes part in the group reduction, inactive ones with zeros).
  auto write_planes = [&](const double2 (&v)[RPL]) {
    if (P.oz_bp == nullptr || (CONJ ? P.m - hi : lo) <= 0) return;   // uniform
    int e = -(1 << 29);
#pragma unroll
    for (int q = 0; q < RPL; ++q) e = max(e, bound_exp(v[q]));
    e = gmax_i<L>(e);
    if (e < -(1 << 28)) e = 0;
    if (!active) return;
    const int jstart = shortcut ? lo + 1 : 0;
    const int c = j - jstart, ncols = P.n - jstart, kw = P.oz_kb / 2;
    if (l == 0) P.oz_cexp[c] = e;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      uint32_t w[kOzS];
      digit_pairs(v[q], e, w);
#pragma unroll
      for (int t = 0; t < kOzS; ++t) P.oz_bp[(size_t)(t * ncols + c) * kw + l + L * q] = w[t];
    }
    for (int r = NB + l; r < kw; r += L)                 // K padding beyond n_b rows
#pragma unroll
      for (int t = 0; t < kOzS; ++t) P.oz_bp[(size_t)(t * ncols + c) * kw + r] = 0u;
  };

  if (!SAFE) {
    substitute();
#pragma unroll
    for (int q = 0; q < RPL; ++q)
      if (l + L * q < nbe) col[l + L * q] = y[q];
    write_planes(y);
    return;
  }

  // ----- safe variant (upper only) ------------------------------------------
  const double OM = omega();
  // max_r |y_r| over the block: common power-of-two scale, then squares.
  auto maxabs = [&]() {
    int E = -1022;
#pragma unroll
    for (int q = 0; q < RPL; ++q) E = max(E, zexp(y[q]));
    E = gmax_i<L>(E);
    long long m2 = 0;                                  // max of the scaled squares, as bits (>= 0)
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      // y 2^-E on the exponent fields (exact: the products by 2^-E)
      const double a = dscale_exp0(y[q].x, -E), bb = dscale_exp0(y[q].y, -E);
      m2 = max(m2, __double_as_longlong(fma(a, a, bb * bb)));
    }
    return sqrt(__longlong_as_double(gmax_ll<L>(m2))) * pow2i(E);
  };

  // Alg. 4 with its decisions taken after the fact.  A rescale by a power of
  // two commutes exactly with every later operation of the substitution (as
  // long as no value is subnormal), so the block is solved once in a scaling
  // of its own, kept clear of overflow by integer bounds on the exponents and
  // rare rescales (phase A).  Alg. 4's two tests are then decided from per-row
  // quantities computed in parallel over the lanes (phase B): the block's
  // cumulative rescale exponent has a closed form (alg4_block_ka), and the
  // serial chain of G sums and rescales (phase C) runs only where that form
  // cannot decide.  The block is finally brought to Alg. 4's scaling (phase
  // D); every value is then the one the serial safeguarded loop computes.
  const double G0 = maxabs();                         // G before the first row (Alg. 4)
  // phase A: |y| < 2^Eb for every row; Kown = this block's own scaling
  int Eb = G0 == 0.0 ? -1100 : (int)(__double_as_longlong(G0) >> 52) - 1022;
  int Kown = 0;
  bool patho = false;                                 // a rescale so large that small values would underflow
  double2 ypre[RPL];                                  // each row's value at its diagonal step
  int kpre[RPL];                                      // Kown at that step
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    ypre[q] = make_double2(0.0, 0.0);
    kpre[q] = 0;
  }
#pragma unroll
  for (int s_ = 0; s_ < RPL; ++s_) {
   const int qi = RPL - 1 - s_;
#pragma unroll 1
   for (int u_ = 0; u_ < L; ++u_) {
    const int li = L - 1 - u_, i = L * qi + li;
    const int pi = gshfl_i<L>(pex[qi], li);
    patho |= i < nbe && pi == 0;                      // subnormal pivot: |p| >= 2^(pi - 1023) fails
    // |x_i| = |y_i| / |p_i| < 2^(Eb + 1024 - pi); the AXPY adds at most |x_i| C_i.
    const int eC = (int)(__double_as_longlong(ccol(i)) >> 52) - 1022;
    const int xb = Eb + 1025 - pi;
    int cand = i < nbe ? max(xb + max(eC, 0), Eb) + 1 : Eb;
    if (cand > 1010) {                                // keep clear of overflow
      const int kk = cand - 900;
      patho |= kk > 600;                              // e.g. a pivot near the bottom of the range
#pragma unroll
      for (int q = 0; q < RPL; ++q) y[q] = zscale_exp(y[q], -kk);
      Kown += kk;
      cand -= kk;
    }
    const double2 xi = xrow(qi, li);
    if (l == li) {
      ypre[qi] = y[qi];
      kpre[qi] = Kown;
      y[qi] = xi;
    }
    axpy(qi, li, xi);
    Eb = cand;
   }
  }
  int kexp = 0;
  if (!__any_sync(0xffffffffu, active && patho)) {
  // phase B: per owned row, the exponent of M_r = |y_r| / |p_r| in the
  // unscaled form, and the term a_r 2^Kown of S = G0 + sum_r a_r 2^Kown
  // (a_r = |x_r| C_r, x_r in the final own scaling) estimated in FP32
  int em[RPL];
  int em_max = kBoundNone, tmax = kBoundNone, tmin = -kBoundNone;
  float tf[RPL];
  int te[RPL];
  bool odd = false;
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    const int r = l + L * q;
    em[q] = -(1 << 28);
    tf[q] = 0.0f;
    te[q] = kBoundNone;
    if (r < nbe) {
      if (!zzero_words(ypre[q])) {
        // floor(log2 M) <= ey - ep + 1 for normal operands; Alg. 4's test
        // (M 2^(kpre - Ka) >= Omega with Ka >= 0) can only fire above it.
        const int ey = (int)(((unsigned)max(__double2hiint(ypre[q].x) & 0x7fffffff,
                                            __double2hiint(ypre[q].y) & 0x7fffffff)) >> 20);
        const int up = ey - pex[q] + 1 + kpre[q];
        if (ey != 0 && pex[q] != 0 && up < kOmegaExp) {
          em[q] = up;
        } else {
          bool ok;
          const double2 pr = pivot(r);
          const int re = ratio_exp_est(ypre[q], pr, ok);
          em[q] = (ok ? re : ratio_exp_fast(ypre[q], pr)) + kpre[q];
        }
      }
      int e;
      tf[q] = abs_prod_est(y[q], ccol(r), e, odd);
      if (tf[q] != 0.0f) {
        odd |= e < -1020;                             // a_r itself near the subnormal range
        te[q] = e + Kown;
      }
      alg4_term_exps(tf[q], te[q], tmax, tmin);
    }
    em_max = max(em_max, em[q]);
  }
  float tg = 0.0f;                                    // G0, counted once per shift
  int eg = kBoundNone;
  if (l == 0) {
    tg = dbl_lead_f(G0, eg, odd);
    alg4_term_exps(tg, eg, tmax, tmin);
  }
  em_max = gmax_i<L>(em_max);
  tmax = gmax_i<L>(tmax);
  tmin = -gmax_i<L>(-tmin);
  odd = gmax_i<L>((int)odd) != 0;
  float sp = f_scale_down(tg, eg - tmax);
#pragma unroll
  for (int q = 0; q < RPL; ++q) sp += f_scale_down(tf[q], te[q] - tmax);
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o, L);
  // phase C: Alg. 4's decisions, Ka its cumulative rescale of this block, in
  // closed form (see alg4_block_ka); a warp with a shift it cannot decide
  // runs the serial chain from the exact a_r.
  int Ka = 0;
  const bool decided = alg4_block_ka(em_max, tmax, tmin, sp, odd, Ka) && g_alg4_chain_d == 0;
  if (!__all_sync(0xffffffffu, !active || decided)) {
    Ka = 0;
    double a[RPL];                                    // a_r, exactly
#pragma unroll
    for (int q = 0; q < RPL; ++q) a[q] = l + L * q < nbe ? __dmul_rn(zabs_exp(y[q]), ccol(l + L * q)) : 0.0;
    double G = G0;
#pragma unroll
    for (int s_ = 0; s_ < RPL; ++s_) {
     const int qi = RPL - 1 - s_;
#pragma unroll 1
     for (int u_ = 0; u_ < L; ++u_) {
      const int li = L - 1 - u_, i = L * qi + li;
      const double ai = gshfl<L>(a[qi], li);
      const int emi = gshfl_i<L>(em[qi], li);
      if (i < nbe) {
        const int eM = emi - Ka;
        if (eM >= kOmegaExp) {                        // M >= Omega: rescale b first
          const int kk = eM - (kOmegaExp - 1);
          Ka += kk;
          G = dscale_exp(G, -kk);
        }
        G = __dadd_rn(G, dscale_exp(ai, Kown - Ka));
        if (ge_omega(G)) {                            // protect the AXPY
          const int kk = choose_k_exp(G);
          Ka += kk;
          G = dscale_exp(G, -kk);
        }
      }
     }
    }
  }
  // phase D: to Alg. 4's scaling
  kexp = Ka;
  if (Kown != Ka) {
#pragma unroll
    for (int q = 0; q < RPL; ++q) y[q] = zscale_exp(y[q], Kown - Ka);
  }
  } else {
    // The serial safeguarded back substitution (Alg. 4, second branch),
    // group-uniform, from the block's right-hand side.
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = l + L * q;
      y[q] = r < nbe ? col[r] : make_double2(0.0, 0.0);
    }
    double G = G0;
#pragma unroll
    for (int s_ = 0; s_ < RPL; ++s_) {
     const int qi = RPL - 1 - s_;
#pragma unroll 1
     for (int u_ = 0; u_ < L; ++u_) {
      const int li = L - 1 - u_, i = L * qi + li;
      const double2 yi = gshfl_z<L>(y[qi], li);
      int eM = -100000;
      if (i < nbe && !zzero_words(yi)) eM = ratio_exp_fast(yi, pivot(i));
      if (eM >= kOmegaExp) {                          // M >= Omega: rescale b first
        const int kk = eM - (kOmegaExp - 1);
#pragma unroll
        for (int q = 0; q < RPL; ++q) y[q] = zshift(y[q], kk);
        kexp += kk;
        G = dshift(G, kk);
      }
      // diagonal step by a division: in this path the reciprocal of a
      // subnormal pivot may have overflowed
      double2 xi = gshfl_z<L>(i < nbe ? zdiv_fast(y[qi], pivot(i)) : make_double2(0.0, 0.0), li);
      if (l == li) y[qi] = xi;
      if (i < nbe) {
        G = __dadd_rn(G, __dmul_rn(zabs_exp(xi), ccol(i)));
        if (ge_omega(G)) {                               // protect the AXPY
          const int kk = choose_k(G);
#pragma unroll
          for (int q = 0; q < RPL; ++q) y[q] = zshift(y[q], kk);
          xi = zshift(xi, kk);
          kexp += kk;
          G = dshift(G, kk);
        }
      }
      axpy(qi, li, xi);
     }
    }
  }

  // Alg. 5: t < 1 rescales the rest of the column (lazily: the substitution
  // GEMM applies it to I0 and the final fix-up to I2), then
  // G(j) += C_blk ||X(I1,j)||_inf with a whole-column rescale at Omega.
  const double N = maxabs();
  int ej = 0, pend = 0, k2 = 0;
  double Gj = 0.0;
  if (active) {
    ej = e_col;
    Gj = G_col;
    if (kexp > 0) { ej += kexp; Gj = dscale_exp0(Gj, -kexp); pend = kexp; }
    const double cb = GEN ? __dadd_rn(cblk_u, __dmul_rn(al, cblk_v)) : cblk_u;
    Gj = __dadd_rn(Gj, __dmul_rn(cb, N));
    if (Gj >= OM) {
      k2 = choose_k_exp(Gj);
      ej += k2;
      Gj = dscale_exp(Gj, -k2);
      pend += k2;
    }
  }
  double2 xo[RPL];
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    xo[q] = k2 ? zscale_exp(y[q], -k2) : y[q];
    if (active && l + L * q < nbe) col[l + L * q] = xo[q];
  }
  write_planes(xo);
  if (active && l == 0) {
    P.e[j] = ej;
    P.G[j] = Gj;
    P.pend[j] = pend;
    P.E[(long long)b * P.n + j] = ej;
    if (pend > 0) raise_status(status, MSTS_STATUS_SCALED);
  }
}

template <int NB, int L, bool SAFE, bool CONJ, bool GEN>
static cudaError_t launch(const ProbTable &tab, int step, int shortcut, int ncols_max,
                          uint32_t *status, cudaStream_t st) {
  constexpr int SPC = (kDiagThreads / 32) * (32 / L);
  constexpr size_t smem = (GEN ? 2 : 1) * ((size_t)NB * (NB + 1) * sizeof(double2) + NB * sizeof(double)) +
                          (size_t)NB * SPC * sizeof(double2);   // + the inverses of the pivots
  cudaError_t e = cudaFuncSetAttribute(k_diag<NB, L, SAFE, CONJ, GEN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_diag<NB, L, SAFE, CONJ, GEN>, dim3((ncols_max + SPC - 1) / SPC, 1, tab.count),
                    dim3(kDiagThreads), smem, st, tab, step, shortcut, status);
}

template <int NB, bool SAFE, bool CONJ, bool GEN>
static cudaError_t launch_nb(int L, const ProbTable &tab, int step, int shortcut, int ncols_max,
                             uint32_t *status, cudaStream_t st) {
  if constexpr (NB == 64) {
    if (L <= 16) return launch<64, 16, SAFE, CONJ, GEN>(tab, step, shortcut, ncols_max, status, st);
    return launch<64, 32, SAFE, CONJ, GEN>(tab, step, shortcut, ncols_max, status, st);
  } else if constexpr (NB == 32) {
    if (L <= 4) return launch<32, 4, SAFE, CONJ, GEN>(tab, step, shortcut, ncols_max, status, st);
    if (L == 8) return launch<32, 8, SAFE, CONJ, GEN>(tab, step, shortcut, ncols_max, status, st);
    if (L == 16) return launch<32, 16, SAFE, CONJ, GEN>(tab, step, shortcut, ncols_max, status, st);
    return launch<32, 32, SAFE, CONJ, GEN>(tab, step, shortcut, ncols_max, status, st);
  } else {
    if (L <= 4) return launch<16, 4, SAFE, CONJ, GEN>(tab, step, shortcut, ncols_max, status, st);
    if (L == 8) return launch<16, 8, SAFE, CONJ, GEN>(tab, step, shortcut, ncols_max, status, st);
    return launch<16, 16, SAFE, CONJ, GEN>(tab, step, shortcut, ncols_max, status, st);
  }
}

// Lanes per shift.  A warp issues its FP64 instructions at one per 64 cycles
// whether they depend on each other or not, warps on one sub-partition share
// that rate, and every warp also waits on its shuffles and memory: a launch
// lasts as long as its busiest SM, so its time is set by the lane width L (the
// FP64 instructions a shift costs) and by k, the number of 128-thread CTAs on
// the busiest SM, hardly by how many SMs are busy.  For n_b = 32 the width is
// the one with the smallest time in
// tables measured on GB300 (one launch per solve, m = n_b = 32, 304..12160
// shifts; k = 1..4, then a constant slope per further CTA, microseconds).
// Every width gives the same results bit for bit.  Other block sizes take the
// smallest width with at least 4 warps per SM.
namespace {
struct LaneCost {
  float t[4];
  float slope;
};
constexpr LaneCost kPlainCost[4] = {        // L = 4, 8, 16, 32 (plain and conjugate-transposed)
    {{42.8f, 61.5f, 88.7f, 115.9f}, 27.2f},
    {{32.4f, 43.2f, 58.6f, 75.0f}, 16.3f},
    {{26.4f, 35.6f, 43.4f, 54.7f}, 11.6f},
    {{23.7f, 30.3f, 39.5f, 45.1f}, 9.0f}};
constexpr LaneCost kSafeCost[4] = {         // the safe solve (Alg. 4 replay, Alg. 5 update)
    {{60.2f, 82.0f, 115.6f, 149.2f}, 33.6f},
    {{42.0f, 54.6f, 75.5f, 99.1f}, 24.1f},
    {{31.7f, 40.7f, 54.6f, 69.4f}, 15.7f},
    {{27.6f, 33.9f, 44.5f, 56.0f}, 12.7f}};
double lane_cost(const LaneCost &c, long long k) {
  return k <= 4 ? c.t[k - 1] : c.t[3] + (double)(k - 4) * c.slope;
}
}  // namespace

int diag_lanes(int nb, long long total_cols, bool safe) {
  if (nb == 32) {
    const LaneCost *tab = safe ? kSafeCost : kPlainCost;
    int best = 32;
    double tbest = 0.0;
    for (int i = 0, L = 4; L <= 32; ++i, L *= 2) {
      const long long ctas = (total_cols * L + kDiagThreads - 1) / kDiagThreads;
      const long long k = std::max(1LL, (ctas + 151) / 152);
      const double t = lane_cost(tab[i], k);
      if (i == 0 || t < tbest) {
        tbest = t;
        best = L;
      }
    }
    return best;
  }
  const int lmax = nb < 32 ? nb : 32;
  for (int L = nb >= 64 ? 16 : 4; L < lmax; L *= 2)
    if (total_cols * L >= 32LL * 4 * 152) return L;
  return lmax;
}

// Four-warp layout (msts_diagw.cu) or one-warp layout for n_b = 32, from
// per-launch times measured on GB300 (microseconds):
//   safe, TREVC of the 4096 workload (ncu launch list, per block step):
//     active shifts     31    543   1055   1311   2079   2591   3359   3871
//     one-warp        22.9   25.7   34.1   45.2   45.8   71.4   69.4   70.1
//     four-warp L=4   31.5   36.3   36.4   42.2   42.8   54.4   54.7   67.4
//     four-warp L=2   49.3   52.3   52.6   54.2   54.8   63.9   63.6   63.9
//   single-block solves (m = n_b = 32, CUDA events), shifts 608 / 2432 / 4864 / 9728:
//     plain one-warp 22.1 / 30.4 / 40.3 / 60.4, four-warp best 23.9 (L=4) / 29.2 (L=2)
//       / 37.5 (L=2) / 52.9 (L=1); safe one-warp 25.9 / 40.0 / 53.8 / 83.3, four-warp
//       best 33.8 (L=4) / 39.9 (L=4) / 52.9 (L=2) / 79.5 (L=1).
// Rechecked with the closed-form Alg. 4 decisions and the two-lane row multiply
// (whole-workload medians, every launch forced to one layout): TREVC 4096 per
// launch 9.06 ms, four-warp L = 4 / 2 / 1 9.25 / 10.85 / 14.99, one-warp 9.50 (the
// last block steps, ~4000 shifts, now favour L = 4: 53.4 against 56.9 us);
// pseudospectra 2000^2 at 10^4 shifts (plain solves) L = 1 / 2 / 4 506 / 497 / 523 ms,
// one-warp 516 ms.  The four-warp layout pays a named-barrier hand-off per row,
// so it wins only where enough shifts keep the FP64 pipes busy.  Rechecked after
// the chunk-pair row layout of upper four-lane solves (TREVC 4096 with the
// one-warp / four-warp switch at 600, 900, 1200, 1600 shifts: 8.78 / 8.74 /
// 8.71 / 8.73 ms; the L = 4 / 2 switch at 4500, 6000 or never: equal within
// 0.01 ms; pseudospectra 494 ms with these plain thresholds, 503-511 ms with
// four other sets): the thresholds below stay.
namespace {
int g_diag_override = 0;
}
void set_diag_override(int lanes) { g_diag_override = lanes; }

int diagw_lanes(long long total_cols, bool safe) {
  if (g_diag_override > 0) return g_diag_override;
  if (total_cols < (safe ? 1200 : 2000)) return 0;   // one-warp layout
  if (total_cols < (safe ? 4500 : 3500)) return 4;
  return total_cols < 12000 ? 2 : 1;
}

cudaError_t launch_diag(const ProbTable &tab, int nb, bool safe, bool conj, int step, int shortcut,
                        int ncols_max, long long total_cols, uint32_t *status, cudaStream_t st, bool gen) {
  if (nb == 32 && !gen && g_diag_override >= 0) {
    const int lw = diagw_lanes(total_cols, safe);
    if (lw > 0) return launch_diagw(tab, safe, conj, step, shortcut, ncols_max, lw, status, st);
  }
  const int L = diag_lanes(nb, total_cols, safe);
#define MSTS_DIAG_CASE(NBV)                                                                          \
  case NBV:                                                                                          \
    if (gen && safe) return launch_nb<NBV, true, false, true>(L, tab, step, shortcut, ncols_max, status, st); \
    if (gen) return launch_nb<NBV, false, false, true>(L, tab, step, shortcut, ncols_max, status, st);    \
    if (safe) return launch_nb<NBV, true, false, false>(L, tab, step, shortcut, ncols_max, status, st);  \
    if (conj) return launch_nb<NBV, false, true, false>(L, tab, step, shortcut, ncols_max, status, st);  \
    return launch_nb<NBV, false, false, false>(L, tab, step, shortcut, ncols_max, status, st);
  switch (nb) {
    MSTS_DIAG_CASE(16)
    MSTS_DIAG_CASE(32)
    MSTS_DIAG_CASE(64)
    default: return cudaErrorInvalidValue;
  }
#undef MSTS_DIAG_CASE
}

}  // namespace msts

extern "C" {
int msts_tune_set(int32_t knob, int32_t value) {
  if (knob == MSTS_TUNE_ALG4_CHAIN) {
    if (value != 0 && value != 1) return -2;
    if (cudaMemcpyToSymbol(msts::g_alg4_chain_d, &value, sizeof(int)) != cudaSuccess) return -3;
    return msts::set_alg4_chain_w(value) == cudaSuccess ? 0 : -3;
  }
  if (knob != MSTS_TUNE_DIAG_LANES) return -1;
  if (value != 0 && value != -1 && value != 1 && value != 2 && value != 4) return -2;
  msts::set_diag_override(value);
  return 0;
}
}  // extern "C"
