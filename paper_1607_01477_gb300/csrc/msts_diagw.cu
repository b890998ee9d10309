// msts_diagw.cu -- the diagonal-block step for n_b = 32 (standard problems,
// Alg. 3 / Alg. 4 on the shifted block U(I1,I1) - lambda_j I, and the
// forward substitution on the conjugate transpose), with each shift's rows
// spread over the four warps of a CTA.
//
// Why this layout.  FP64 arithmetic on this part issues one warp instruction
// per 64 cycles per warp, dependent or not (76 with four warps on an SM, half
// that rate each for two warps on one sub-partition): about 1.7 lane
// operations per clock per SM, whatever the number of lanes that need them.
// With one group of lanes per shift inside one warp, the per-row multiply
// x_i = y_i (1 / p_i) and the partially predicated AXPY occupy whole warp
// instructions for a few useful lanes.  Here L = 1, 2 or 4 lanes hold one
// shift (32 / L shifts per CTA) and the rows of the block are dealt out to the
// four warps: row r lives in warp r mod 4, lane (r / 4) mod L of the shift's
// group, register slot r / (4 L).  Every FP64 instruction of the AXPY then
// serves 32 / L shifts at once with no idle lane for L = 1, the per-row
// multiply is issued by one warp only, and the four warps (one per
// sub-partition) share the work of every shift.  The owner of row i publishes
// x_i in shared memory and releases a named barrier; the other warps wait on
// it.  The owner of the next row applies x_i to that row first, publishes its
// own x, and only then applies x_i to the rest of its rows (one-row
// lookahead), so the serial chain per row is one complex multiply-add and one
// complex multiply.  Solves with L = 4 deal the rows out in chunks of four
// consecutive rows instead (warp w: chunks w and 7 - w), which issues about a
// third fewer multiply-add instructions per warp; in upper solves a chunk's
// owner produces its four rows without a hand-off.
//
// Measured: the layout spends ~4x fewer FP64 instructions per shift than the
// one-warp layout, but the hand-off per row (barrier, shared-memory round trip,
// the critical multiply-adds queued behind the other warps' FP64 work) makes a
// CTA take ~24-44 us per block however few shifts it holds; it is faster only
// where the FP64 pipes are the bound, i.e. with many shifts per SM (the
// dispatch takes it from measured per-launch tables, msts_diag.cu).
//
// Every value sees the same operations in the same order as in the one-warp
// layout (msts_diag.cu): the same reciprocals, the same fused multiply-adds
// row by row, the same power-of-two rescales, the same decisions of Alg. 4
// (closed form, or the serial chain where it cannot decide); the results are
// the same bit for bit.  The right-hand sides and
// the results move between global and shared memory in coalesced column
// order.  Blocks where the replay cannot be exact (a subnormal pivot, a
// rescale beyond 2^600) take the serial safeguarded loop of Alg. 4, one
// thread per shift.
#include "msts_common.cuh"
#include "msts_diag.h"
#include "msts_diag_util.cuh"
#include "msts_digits.cuh"

namespace msts {

// 1: Alg. 4's decisions by the serial chain in every block (tuning knob; the
// closed form gives the same values)
__device__ int g_alg4_chain_w = 0;

namespace {

constexpr int kWNB = 32;                 // block size n_b
constexpr int kWWarps = 4;               // warps per CTA: row owners
constexpr int kWThreads = 32 * kWWarps;
constexpr int kWLD = kWNB + 1;           // column stride of the staged U(I1,I1), in complex entries
constexpr int kWLDY = kWNB + 1;          // column stride of the staged right-hand sides

__device__ __forceinline__ void nbar_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kWThreads) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(kWThreads) : "memory");
}
// named barrier of row i (ids 1..8; 0 is __syncthreads): every warp meets the
// barriers of the rows in the same order and never runs more than one row
// ahead of a barrier it waits on, so ids repeat safely every 8 rows.
__device__ __forceinline__ int row_bar(int i) { return 1 + (i & 7); }

template <int L>
struct WShape {
  static constexpr int SPC = 32 / L;               // shifts per CTA
  static constexpr int RPT = kWNB / (kWWarps * L); // rows per thread
};

template <int L, bool SAFE>
constexpr size_t diagw_smem() {
  constexpr int SPC = WShape<L>::SPC;
  return sizeof(double2) * ((size_t)kWNB * kWLD + (size_t)kWNB * SPC + (size_t)SPC * kWLDY +
                             (L > 1 ? (size_t)kWNB * SPC : 0)) +
         sizeof(double) * kWNB + sizeof(int) * ((size_t)kWNB * SPC + kWWarps * SPC + SPC) +
         sizeof(long long) * kWWarps * SPC + 16;
}

template <int L, bool SAFE, bool CONJ>
__global__ void __launch_bounds__(kWThreads)
k_diagw(const __grid_constant__ ProbTable tab, int step, int shortcut, uint32_t *status) {
  constexpr int SPC = WShape<L>::SPC, RPT = WShape<L>::RPT, NB = kWNB, LD = kWLD, LDY = kWLDY;
  constexpr int SLOT = kWWarps * L;      // rows per register slot (cyclic layout)
  // Upper solves with L = 4 take the chunk-pair layout: the block's rows in
  // eight chunks of four, warp w holding chunk w (slot 0) and chunk 7 - w
  // (slot 1), lane h row 4 c + h of chunk c.  Each of a warp's multiply-add
  // instructions then covers four consecutive rows, so it is issued only while
  // one of them lies above the current row: 34 slot multiply-adds per warp and
  // block against 48 in the cyclic layout (31 carry useful work), the same
  // number for every warp.
  constexpr bool CHUNK = L == 4 && !CONJ;
  // The conjugate-transposed solves with L = 4 use the same layout on the
  // cyclic layout's loop (the next row first, then the rest), the owner of a
  // chunk leaving its other slot's share of the chunk's x_i until it has
  // produced the chunk's last row.  The loop is written for chunks of L rows
  // in groups of eight (warp w: chunks 8 b + w and 8 b + 7 - w in slots 2 b,
  // 2 b + 1), but at L = 2 it measured slower than the cyclic layout on the
  // pseudospectra workload (554 ms, 537 without the deferral, against 486) for
  // a reason not found, so L = 2 stays cyclic; with L = 1 every slot is one
  // row and the cyclic layout wastes nothing.
  constexpr bool CHUNKG = L == 4 && CONJ;
  static_assert(!(SAFE && CONJ), "the safe solve is upper only");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *sU = reinterpret_cast<double2 *>(smem_raw);      // U(I1,I1), column-major, LD
  double2 *sX = sU + NB * LD;                                // x_i of every shift: [i SPC + js]
  double2 *sY = sX + NB * SPC;                               // per-shift columns: [js LDY + r]
  double2 *sInv = sY + SPC * LDY;                            // 1 / p_i (L > 1): [i SPC + js]
  double *sC = reinterpret_cast<double *>(sInv + (L > 1 ? NB * SPC : 0));   // within-block column norms
  int *sPex = reinterpret_cast<int *>(sC + NB);              // pivot exponent fields [i SPC + js]
  int *sRedI = sPex + NB * SPC;                              // [w SPC + js]
  int *sShift = sRedI + kWWarps * SPC;                       // [js]
  long long *sRedL = reinterpret_cast<long long *>(
      (reinterpret_cast<uintptr_t>(sShift + SPC) + 7) & ~uintptr_t(7));   // [w SPC + js]

  const Prob &P = tab.p[blockIdx.z];
  if (step >= P.nblk) return;
  const int b = CONJ ? P.nblk - 1 - step : step;
  int lo, hi;
  block_range(P, b, NB, lo, hi);
  const int nbf = hi - lo;
  const int jstart = shortcut ? lo + 1 : 0;
  const int jcta = jstart + blockIdx.x * SPC;
  if (jcta >= P.n) return;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int js = lane / L, h = lane % L;
  const int j = jcta + js;
  const bool active = j < P.n;
  auto nbe_of = [&](int jj) { return shortcut ? min(hi, jj) - lo : nbf; };   // TREVC: rows >= j stay zero
  const int nbe = active ? nbe_of(j) : 0;
  // chunk held in slot q (chunk-pair layouts)
  auto chunk_of = [&](int q) { return 8 * (q >> 1) + ((q & 1) ? 7 - w : w); };
  auto row_of = [&](int q) { return (CHUNK || CHUNKG) ? L * chunk_of(q) + h : w + 4 * (h + L * q); };

  // U(I1,I1) by asynchronous 16-byte copies.  No kernel of the solve writes U
  // or the column norms, so after the first block step these copies start
  // before the wait for the previous kernel (they overlap its last CTAs).
  auto stage_u = [&]() {
    for (int idx = tid; idx < NB * NB; idx += kWThreads) {
      const int c = idx / NB, r = idx - c * NB;
      const bool in = r <= c && c < nbf;
      cp_async16(&sU[c * LD + r], in ? &P.U[(lo + r) + (long long)(lo + c) * P.ldu] : P.U, in);
    }
    if (SAFE)
      for (int k = tid; k < NB; k += kWThreads) sC[k] = k < nbf ? P.cin[lo + k] : 0.0;
  };
  if (step > 0) stage_u();
  pdl_wait();                            // B, the safe state and the planes' buffer come from the kernel before
  if (step == 0) stage_u();
  // Global loads (one round trip): the shift, delta and (safe) the column's
  // scale state and C_blk; then the block's right-hand sides by asynchronous
  // 16-byte copies in coalesced order.
  double2 lam = active ? P.shifts[(long long)j * P.shift_stride] : make_double2(0.0, 0.0);
  const double dlt = SAFE ? *P.delta : 0.0;
  int e_col = 0;
  double G_col = 0.0;
  if (SAFE && active) {
    e_col = P.e[j];
    G_col = P.G[j];
  }
  const double cblk = SAFE ? P.cblk[b] : 0.0;
  for (int idx = tid; idx < SPC * NB; idx += kWThreads) {
    const int c = idx / NB, r = idx - c * NB, jj = jcta + c;
    const bool in = jj < P.n && r < nbe_of(jj);
    cp_async16(&sY[c * LDY + r], in ? &P.B[(long long)jj * P.ldb + lo + r] : P.B, in);
  }
  cp_async_wait_all();
  __syncthreads();

  if (CONJ) lam = zconj(lam);
  auto pivot0 = [&](int i) {
    const double2 d = sU[i * LD + i];
    return zsub(CONJ ? zconj(d) : d, lam);
  };
  auto pivot = [&](int i) {
    double2 p = pivot0(i);
    if (SAFE && zzero_words(p)) p = make_double2(dlt, 0.0);   // U(i,i) = lambda -> delta (Sec. 3)
    return p;
  };

  double2 y[RPT], inv[RPT];
  int pex[RPT];
  bool zero_piv = false;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int r = row_of(q);
    const bool v = r < nbe;
    y[q] = sY[js * LDY + r];
    const double2 p0 = pivot0(r);
    zero_piv |= v && zzero_words(p0);
    const double2 p = pivot(r);
    inv[q] = v ? zrecip(p) : make_double2(0.0, 0.0);
    if (L > 1) sInv[r * SPC + js] = inv[q];
    pex[q] = (int)(max(absbits(p.x), absbits(p.y)) >> 52);
    if (SAFE) sPex[r * SPC + js] = pex[q];
  }
  __syncwarp();                          // sInv: a row's inverse is read in its own warp
  if (zero_piv) raise_status(status, SAFE ? MSTS_STATUS_DELTA : MSTS_STATUS_ZERO_PIVOT);

  // max_r |y_r| over the shift's block rows (all four warps), as in the
  // one-warp layout: common power-of-two scale, then the largest square.
  auto maxabs = [&]() {
    int E = -1022;
#pragma unroll
    for (int q = 0; q < RPT; ++q) E = max(E, zexp(y[q]));
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o, L));
    __syncthreads();
    if (h == 0) sRedI[w * SPC + js] = E;
    __syncthreads();
#pragma unroll
    for (int v = 0; v < kWWarps; ++v) E = max(E, sRedI[v * SPC + js]);
    long long m2 = 0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      // y 2^-E on the exponent fields (exact: the products by 2^-E)
      const double a = dscale_exp0(y[q].x, -E), bb = dscale_exp0(y[q].y, -E);
      m2 = max(m2, __double_as_longlong(fma(a, a, bb * bb)));
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) m2 = max(m2, (long long)__shfl_xor_sync(0xffffffffu, m2, o, L));
    if (h == 0) sRedL[w * SPC + js] = m2;
    __syncthreads();
#pragma unroll
    for (int v = 0; v < kWWarps; ++v) m2 = max(m2, sRedL[v * SPC + js]);
    return sqrt(__longlong_as_double(m2)) * pow2i(E);
  };

  // ----- the substitution -----------------------------------------------------
  // Safe variant, phase A: the block is solved in a power-of-two scaling of
  // its own, kept clear of overflow by integer bounds on the exponents (every
  // thread of a shift runs the same bound chain); rescales apply to all rows.
  double G0 = 0.0;
  int Eb = 0, Kown = 0;
  bool patho = false;
  int kpre[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) kpre[q] = 0;
  if (SAFE) {
    G0 = maxabs();
    Eb = G0 == 0.0 ? -1100 : (int)(__double_as_longlong(G0) >> 52) - 1022;
  }
  // Alg. 4's bound chain for row i: returns the rescale exponent taken there.
  auto chain = [&](int i) -> int {
    const int pi = sPex[i * SPC + js];
    patho |= i < nbe && pi == 0;         // subnormal pivot: |p| >= 2^(pi - 1023) fails
    const int eC = (int)(__double_as_longlong(sC[i]) >> 52) - 1022;
    const int xb = Eb + 1025 - pi;
    int cand = i < nbe ? max(xb + max(eC, 0), Eb) + 1 : Eb;
    int kk = 0;
    if (cand > 1010) {                   // keep clear of overflow
      kk = cand - 900;
      patho |= kk > 600;                 // e.g. a pivot near the bottom of the range
      Kown += kk;
      cand -= kk;
    }
    Eb = cand;
    return kk;
  };
  auto rescale_slot = [&](int q, int kk) { y[q] = zscale_exp(y[q], -kk); };

  // the AXPY of x_i into the rows of slot q (qs: slot of row i)
  auto axpy_slot = [&](int q, int qs, int i, double2 x) {
    const int r = row_of(q);
    if (!CONJ) {
      if (q < qs || (q == qs && r < i)) y[q] = zfms(y[q], x, sU[i * LD + r]);
    } else {
      if (q > qs || (q == qs && r > i)) y[q] = zfms(y[q], x, zconj(sU[r * LD + i]));
    }
  };
  // Row i (slot qn of its owner) by its owner warp: x_i = y_i / p_i, published.
  auto produce = [&](int qn, int i, int kk) {
    const int hi_ = (CHUNK || CHUNKG) ? (i & (L - 1)) : (i >> 2) & (L - 1);
    if (SAFE && kk) {
#pragma unroll
      for (int q = 0; q < RPT; ++q)
        if (q == qn) rescale_slot(q, kk);
    }
    double2 yq = y[0], iq = inv[0];
#pragma unroll
    for (int q = 1; q < RPT; ++q)
      if (q == qn) { yq = y[q]; iq = inv[q]; }
    double2 x;
    if (L > 1) {
      // x_i = y_i (1 / p_i): Re x_i by the owner lane, Im x_i by its partner
      // (zmul's two multiply-adds, the same operations), half the FP64
      // instructions of the multiply on the row's chain
      const double yr = __shfl_sync(0xffffffffu, yq.x, hi_, L), yi = __shfl_sync(0xffffffffu, yq.y, hi_, L);
      const double2 ip = sInv[i * SPC + js];
      const bool re = h == hi_;
      const double m1 = __hiloint2double(__double2hiint(yi) ^ (re ? (int)0x80000000 : 0), __double2loint(yi));
      const double part = fma(yr, re ? ip.x : ip.y, m1 * (re ? ip.y : ip.x));
      x = make_double2(__shfl_sync(0xffffffffu, part, hi_, L), __shfl_sync(0xffffffffu, part, hi_ ^ 1, L));
    } else {
      x = zmul(yq, iq);
    }
    if (h == hi_) {
      if (SAFE) sY[js * LDY + i] = yq;   // the row's value at its diagonal step (for the replay)
      sX[i * SPC + js] = x;
#pragma unroll
      for (int q = 0; q < RPT; ++q)
        if (q == qn) {
          y[q] = x;
          if (SAFE) kpre[q] = Kown;
        }
    }
    __threadfence_block();
    nbar_arrive(row_bar(i));
    return x;
  };

  // chain state: kk_cur is the rescale of the current row, kk_nxt of the next
  if constexpr (CHUNK) {
    // The chunk-pair layout.  Chunk c is owned by warp 7 - c (c >= 4, its slot
    // 1) or warp c (c < 4, its slot 0); the owner produces the chunk's rows one
    // after another without a hand-off, the first of them while the previous
    // chunk's last x arrives (one-row lookahead as in the cyclic layout).
    // While a warp owns a chunk c >= 4, its slot 0 (rows below the chunk)
    // takes the chunk's x_i and rescales only after the chunk's last row is
    // produced, in the same order (the multiply-adds of a row stay off the
    // chain of the next row).  Every row sees the operations of the serial
    // substitution in its order, as in the cyclic layout.
    auto axpy_rows = [&](int q, int i, double2 x) {
      const int r = row_of(q);
      if (r < i) y[q] = zfms(y[q], x, sU[i * LD + r]);
    };
    auto rescale_all = [&](int kk) {
#pragma unroll
      for (int q = 0; q < RPT; ++q) rescale_slot(q, kk);
    };
    int kk_cur = SAFE ? chain(NB - 1) : 0;
    double2 xown = make_double2(0.0, 0.0);
    bool rescaled_ahead = false;
    if (w == 0) {                        // owner of chunk 7: row 31 in its slot 1
      if (SAFE && kk_cur) rescale_all(kk_cur);
      xown = produce(1, NB - 1, 0);
      rescaled_ahead = true;
    }
#pragma unroll 1
    for (int c = 7; c >= 4; --c) {
      const bool own = w == 7 - c;
      int dk[3] = {0, 0, 0};             // the owner's deferred rescales of slot 0
#pragma unroll
      for (int k = 3; k >= 0; --k) {
        const int i = 4 * c + k;
        const int kk_nxt = SAFE ? chain(i - 1) : 0;
        if (SAFE && kk_cur && !rescaled_ahead) rescale_all(kk_cur);
        double2 x;
        if (own) {
          x = xown;
        } else {
          nbar_sync(row_bar(i));
          x = sX[i * SPC + js];
        }
        rescaled_ahead = false;
        if (own) {
          if (k > 0) {
            axpy_rows(1, i, x);
            xown = produce(1, i - 1, kk_nxt);
            dk[k - 1] = kk_nxt;          // slot 0: x_i from sX, then this rescale
            rescaled_ahead = true;
          } else {
            __syncwarp();                // the chunk's x_i, stored by this warp's lanes
#pragma unroll
            for (int d = 2; d >= 0; --d) {
              axpy_rows(0, 4 * c + d + 1, sX[(4 * c + d + 1) * SPC + js]);
              if (SAFE && dk[d]) rescale_slot(0, dk[d]);
            }
            axpy_rows(0, i, x);
            if (c == 4) {                // chunk 3 is this warp's too: row 15 in slot 0
              xown = produce(0, i - 1, kk_nxt);
              if (SAFE && kk_nxt) rescale_slot(1, kk_nxt);
              rescaled_ahead = true;
            }
          }
        } else if (k == 0 && w == 8 - c) {   // next chunk's owner: row 4 c - 1 in slot 1
          axpy_rows(1, i, x);
          xown = produce(1, i - 1, kk_nxt);
          axpy_rows(0, i, x);
          if (SAFE && kk_nxt) rescale_slot(0, kk_nxt);
          rescaled_ahead = true;
        } else {
          axpy_rows(0, i, x);            // chunk w lies below chunk c
          if (w > 7 - c) axpy_rows(1, i, x);   // so does chunk 7 - w
        }
        kk_cur = kk_nxt;
      }
    }
#pragma unroll 1
    for (int c = 3; c >= 0; --c) {
      const bool own = w == c;
#pragma unroll
      for (int k = 3; k >= 0; --k) {
        const int i = 4 * c + k;
        const bool last = i == 0;
        const int kk_nxt = (SAFE && !last) ? chain(i - 1) : 0;
        if (SAFE && kk_cur && !rescaled_ahead) rescale_all(kk_cur);
        double2 x;
        if (own) {
          x = xown;
        } else {
          nbar_sync(row_bar(i));
          x = sX[i * SPC + js];
        }
        rescaled_ahead = false;
        if ((own && k > 0) || (!own && k == 0 && w == c - 1)) {   // the next row is this warp's
          axpy_rows(0, i, x);
          xown = produce(0, i - 1, kk_nxt);
          if (SAFE && kk_nxt) rescale_slot(1, kk_nxt);
          rescaled_ahead = true;
        } else if (w < c) {
          axpy_rows(0, i, x);            // slot 1 (chunk 7 - w >= 4) lies above
        }
        kk_cur = kk_nxt;
      }
    }
  } else if constexpr (CHUNKG) {
    // chunk c's owner and the slot that holds it there
    auto owner_of = [](int c) { const int t = c & 7; return t < 4 ? t : 7 - t; };
    auto slot_of = [](int c) { return 2 * (c >> 3) + ((c & 7) >= 4 ? 1 : 0); };
    // slot q still has rows on the unsolved side of row i
    auto pending = [&](int q, int i) {
      const int r0 = L * chunk_of(q);
      return CONJ ? r0 + L - 1 > i : r0 < i;
    };
    auto axpy_rows = [&](int q, int i, double2 x) {
      const int r = row_of(q);
      if (!CONJ) {
        if (r < i) y[q] = zfms(y[q], x, sU[i * LD + r]);
      } else {
        if (r > i) y[q] = zfms(y[q], x, zconj(sU[r * LD + i]));
      }
    };
    static_assert(!SAFE || L == 2, "safe solves are upper, and upper L = 4 takes the loop above");
    const int i0 = CONJ ? 0 : NB - 1;
    int kk_cur = SAFE ? chain(i0) : 0;
    int dk = 0;                          // safe, L = 2: the rescale after the deferred x_i
    double2 xown = make_double2(0.0, 0.0);
    bool rescaled_ahead = false;
    if (w == owner_of(i0 / L)) {         // prologue: the first row's owner
      if (SAFE && kk_cur) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) rescale_slot(q, kk_cur);
      }
      xown = produce(slot_of(i0 / L), i0, 0);
      rescaled_ahead = true;
    }
#pragma unroll 1
    for (int n = 0; n < NB; ++n) {
      const int i = CONJ ? n : NB - 1 - n;
      const bool last = n == NB - 1;
      const int inext = CONJ ? i + 1 : i - 1;
      const int kk_nxt = (SAFE && !last) ? chain(inext) : 0;
      if (SAFE && kk_cur && !rescaled_ahead) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) rescale_slot(q, kk_cur);
      }
      const int kc = CONJ ? L - 1 - (i & (L - 1)) : (i & (L - 1));   // rows after i in its chunk
      const bool own = w == owner_of(i / L);
      double2 x;
      if (own) {
        x = xown;
      } else {
        nbar_sync(row_bar(i));
        x = sX[i * SPC + js];
      }
      rescaled_ahead = false;
      if (own && kc > 0) {
        // the chunk's next row is this warp's: its slot, publish; the other
        // slots take x_i (and the rescale after it) after the chunk's last row
        const int qn = slot_of(i / L);
#pragma unroll
        for (int q = 0; q < RPT; ++q)
          if (q == qn) axpy_rows(q, i, x);
        xown = produce(qn, inext, kk_nxt);
        if (SAFE) dk = kk_nxt;
        rescaled_ahead = true;
        kk_cur = kk_nxt;
        continue;
      }
      if (own && L > 1) {                // the chunk's last row: the deferred share, in order
        __syncwarp();                    // the chunk's x_i, stored by this warp's lanes
        const int qo = slot_of(i / L);
#pragma unroll
        for (int d = L - 1; d >= 1; --d) {
          const int rd = CONJ ? i - d : i + d;
          const double2 xd = sX[rd * SPC + js];
#pragma unroll
          for (int q = 0; q < RPT; ++q)
            if (q != qo) {
              if (pending(q, rd)) axpy_rows(q, rd, xd);
              if (SAFE && dk) rescale_slot(q, dk);
            }
        }
      }
      if (!last && w == owner_of(inext / L)) {
        // next row's owner: that row's slot first, publish it, then the rest
        const int qn = slot_of(inext / L);
#pragma unroll
        for (int q = 0; q < RPT; ++q)
          if (q == qn) axpy_rows(q, i, x);
        xown = produce(qn, inext, kk_nxt);
#pragma unroll
        for (int q = 0; q < RPT; ++q)
          if (q != qn) {
            if (pending(q, i)) axpy_rows(q, i, x);
            if (SAFE && kk_nxt) rescale_slot(q, kk_nxt);
          }
        rescaled_ahead = true;
      } else {
#pragma unroll
        for (int q = 0; q < RPT; ++q)
          if (pending(q, i)) axpy_rows(q, i, x);
      }
      kk_cur = kk_nxt;
    }
  } else {
    const int i0 = CONJ ? 0 : NB - 1;
    int kk_cur = SAFE ? chain(i0) : 0;
    double2 xown = make_double2(0.0, 0.0);
    if (w == (i0 & 3)) {                 // prologue: the first row's owner
      if (SAFE && kk_cur) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) rescale_slot(q, kk_cur);
      }
      xown = produce(CONJ ? 0 : RPT - 1, i0, 0);
    }
    bool rescaled_ahead = w == (i0 & 3);  // this warp applied kk_cur to all its rows already
#pragma unroll
    for (int s_ = 0; s_ < RPT; ++s_) {
      const int qs = CONJ ? s_ : RPT - 1 - s_;
#pragma unroll 1
      for (int u_ = 0; u_ < SLOT; ++u_) {
        const int k = CONJ ? u_ : SLOT - 1 - u_;
        const int i = SLOT * qs + k;
        const bool last = CONJ ? i == NB - 1 : i == 0;
        const int inext = CONJ ? i + 1 : i - 1;
        const int kk_nxt = (SAFE && !last) ? chain(inext) : 0;
        if (SAFE && kk_cur && !rescaled_ahead) {
#pragma unroll
          for (int q = 0; q < RPT; ++q) rescale_slot(q, kk_cur);
        }
        double2 x;
        if (w == (i & 3)) {
          x = xown;
        } else {
          nbar_sync(row_bar(i));
          x = sX[i * SPC + js];
        }
        rescaled_ahead = false;
        if (!last && w == (inext & 3)) {
          // next row's owner: that row first, publish it, then the rest
          const bool same = CONJ ? k < SLOT - 1 : k > 0;
          if (same) {
#pragma unroll
            for (int q = 0; q < RPT; ++q)
              if (q == qs) axpy_slot(q, qs, i, x);
            xown = produce(qs, inext, kk_nxt);
          } else {
            constexpr int dq = CONJ ? 1 : -1;
            const int qn = qs + dq;          // compile-time after unrolling
            if (qn >= 0 && qn < RPT) {
#pragma unroll
              for (int q = 0; q < RPT; ++q)
                if (q == qn) axpy_slot(q, qs, i, x);
              xown = produce(qn, inext, kk_nxt);
            }
          }
          const int qn = same ? qs : qs + (CONJ ? 1 : -1);
#pragma unroll
          for (int q = 0; q < RPT; ++q)
            if (q != qn) {
              axpy_slot(q, qs, i, x);
              if (SAFE && kk_nxt) rescale_slot(q, kk_nxt);
            }
          rescaled_ahead = true;
        } else {
#pragma unroll
          for (int q = 0; q < RPT; ++q) axpy_slot(q, qs, i, x);
        }
        kk_cur = kk_nxt;
      }
    }
  }
  __syncthreads();                       // every x_i read; sX and sY free for reuse

  int kexp = 0;
  if (SAFE) {
    double *sA = reinterpret_cast<double *>(sX);                       // a_i = |x_i| C_i   [i SPC + js]
    int *sEm = reinterpret_cast<int *>(sA + NB * SPC);                 // exponent of M_i   [i SPC + js]
    auto ccol = [&](int i) { return sC[i]; };
    const bool any_patho = __syncthreads_or(active && patho);
    if (!any_patho) {
      // phase B: per owned row, the exponent of M_r = |y_r| / |p_r| in the
      // unscaled form, and the term a_r 2^Kown of S = G0 + sum_r a_r 2^Kown
      // (a_r = |x_r| C_r, x_r in the final own scaling) estimated in FP32
      int em_max = kBoundNone, tmax = kBoundNone, tmin = -kBoundNone;
      float tf[RPT];
      int te[RPT];
      bool odd = false;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = row_of(q);
        int em = -(1 << 28);
        tf[q] = 0.0f;
        te[q] = kBoundNone;
        if (r < nbe) {
          const double2 yp = sY[js * LDY + r];
          if (!zzero_words(yp)) {
            // floor(log2 M) <= ey - ep + 1 for normal operands; Alg. 4's test
            // (M 2^(kpre - Ka) >= Omega with Ka >= 0) can only fire above it.
            const int ey = (int)(((unsigned)max(__double2hiint(yp.x) & 0x7fffffff,
                                                __double2hiint(yp.y) & 0x7fffffff)) >> 20);
            const int up = ey - pex[q] + 1 + kpre[q];
            if (ey != 0 && pex[q] != 0 && up < kOmegaExp) {
              em = up;
            } else {
              bool ok;
              const double2 pr = pivot(r);
              const int re = ratio_exp_est(yp, pr, ok);
              em = (ok ? re : ratio_exp_fast(yp, pr)) + kpre[q];
            }
          }
          int e;
          tf[q] = abs_prod_est(y[q], ccol(r), e, odd);
          if (tf[q] != 0.0f) {
            odd |= e < -1020;                   // a_r itself near the subnormal range
            te[q] = e + Kown;
          }
          alg4_term_exps(tf[q], te[q], tmax, tmin);
        }
        sEm[r * SPC + js] = em;                 // for the chain, if it has to run
        em_max = max(em_max, em);
      }
      float tg = 0.0f;                          // G0, counted once per shift
      int eg = kBoundNone;
      if (w == 0 && h == 0) {
        tg = dbl_lead_f(G0, eg, odd);
        alg4_term_exps(tg, eg, tmax, tmin);
      }
      // the shift's maxima and minimum: its L lanes, then its four warps
      int *sR = reinterpret_cast<int *>(sA);   // [k][w][js], k = em_max, tmax, tmin, odd
      float *sRf = reinterpret_cast<float *>(sR + 4 * kWWarps * SPC);
#pragma unroll
      for (int o = L / 2; o > 0; o >>= 1) {
        em_max = max(em_max, __shfl_xor_sync(0xffffffffu, em_max, o, L));
        tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o, L));
        tmin = min(tmin, __shfl_xor_sync(0xffffffffu, tmin, o, L));
        odd |= __shfl_xor_sync(0xffffffffu, (int)odd, o, L) != 0;
      }
      if (h == 0) {
        sR[(0 * kWWarps + w) * SPC + js] = em_max;
        sR[(1 * kWWarps + w) * SPC + js] = tmax;
        sR[(2 * kWWarps + w) * SPC + js] = tmin;
        sR[(3 * kWWarps + w) * SPC + js] = (int)odd;
      }
      __syncthreads();
#pragma unroll
      for (int v = 0; v < kWWarps; ++v) {
        em_max = max(em_max, sR[(0 * kWWarps + v) * SPC + js]);
        tmax = max(tmax, sR[(1 * kWWarps + v) * SPC + js]);
        tmin = min(tmin, sR[(2 * kWWarps + v) * SPC + js]);
        odd |= sR[(3 * kWWarps + v) * SPC + js] != 0;
      }
      // the FP32 sum of the terms scaled by 2^-tmax
      float sp = f_scale_down(tg, eg - tmax);
#pragma unroll
      for (int q = 0; q < RPT; ++q) sp += f_scale_down(tf[q], te[q] - tmax);
#pragma unroll
      for (int o = L / 2; o > 0; o >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o, L);
      if (h == 0) sRf[w * SPC + js] = sp;
      __syncthreads();
      const float ssum = (sRf[0 * SPC + js] + sRf[1 * SPC + js]) + (sRf[2 * SPC + js] + sRf[3 * SPC + js]);
      int Kest = 0;
      const bool decided = alg4_block_ka(em_max, tmax, tmin, ssum, odd, Kest) && g_alg4_chain_w == 0;
      kexp = Kest;
      if (__syncthreads_or(active && !decided)) {
        // the chain itself, from the exact a_r (the whole CTA)
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          const int r = row_of(q);
          sA[r * SPC + js] = r < nbe ? __dmul_rn(zabs_exp(y[q]), ccol(r)) : 0.0;
        }
        __syncthreads();
        // phase C: Alg. 4's decisions; Ka = its cumulative rescale of this
        // block.  One warp runs the chain of each shift (its 32 dependent FP64
        // additions would otherwise be issued by all four) and shares Ka.
        if (w == 0) {
          int Ka = 0;
          double G = G0;
#pragma unroll 4
          for (int u_ = 0; u_ < NB; ++u_) {
            const int i = NB - 1 - u_;
            if (i < nbe) {
              const double ai = sA[i * SPC + js];
              const int eM = sEm[i * SPC + js] - Ka;
              if (eM >= kOmegaExp) {           // M >= Omega: rescale b first
                const int kk = eM - (kOmegaExp - 1);
                Ka += kk;
                G = dscale_exp(G, -kk);
              }
              G = __dadd_rn(G, dscale_exp(ai, Kown - Ka));
              if (ge_omega(G)) {               // protect the AXPY
                const int kk = choose_k_exp(G);
                Ka += kk;
                G = dscale_exp(G, -kk);
              }
            }
          }
          if (h == 0) sShift[js] = Ka;
        }
        __syncthreads();
        kexp = sShift[js];
      }
      // phase D: to Alg. 4's scaling
      const int Ka = kexp;
      if (Kown != Ka) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) y[q] = zscale_exp(y[q], Kown - Ka);
      }
    } else {
      // The serial safeguarded back substitution (Alg. 4, second branch) from
      // the block's right-hand side, one thread per shift, the shift's rows in
      // shared memory; the same operations in the same order as the one-warp
      // layout's serial path.
      if (w == 0 && h == 0) {
        double2 *ys = sY + js * LDY;
        for (int r = 0; r < NB; ++r) ys[r] = r < nbe ? P.B[(long long)j * P.ldb + lo + r] : make_double2(0.0, 0.0);
        double G = G0;
        for (int u_ = 0; u_ < NB; ++u_) {
          const int i = NB - 1 - u_;
          const double2 yi = ys[i];
          int eM = -100000;
          if (i < nbe && !zzero_words(yi)) eM = ratio_exp_fast(yi, pivot(i));
          if (eM >= kOmegaExp) {             // M >= Omega: rescale b first
            const int kk = eM - (kOmegaExp - 1);
            for (int r = 0; r < NB; ++r) ys[r] = zshift(ys[r], kk);
            kexp += kk;
            G = dshift(G, kk);
          }
          // diagonal step by a division: the reciprocal of a subnormal pivot may overflow
          double2 xi = i < nbe ? zdiv_fast(ys[i], pivot(i)) : make_double2(0.0, 0.0);
          ys[i] = xi;
          if (i < nbe) {
            G = __dadd_rn(G, __dmul_rn(zabs_exp(xi), ccol(i)));
            if (ge_omega(G)) {               // protect the AXPY
              const int kk = choose_k(G);
              for (int r = 0; r < NB; ++r) ys[r] = zshift(ys[r], kk);
              xi = zshift(xi, kk);
              kexp += kk;
              G = dshift(G, kk);
            }
          }
          for (int r = 0; r < i; ++r) ys[r] = zfms(ys[r], xi, sU[i * LD + r]);
        }
        sShift[js] = kexp;
      }
      __syncthreads();
      kexp = sShift[js];
#pragma unroll
      for (int q = 0; q < RPT; ++q) y[q] = sY[js * LDY + row_of(q)];
    }
  }

  // Alg. 5: t < 1 rescales the rest of the column (lazily: the substitution
  // step applies it to I0 and the final fix-up to I2), then
  // G(j) += C_blk ||X(I1,j)||_inf with a whole-column rescale at Omega.
  int ej = 0, pend = 0, k2 = 0;
  double Gj = 0.0;
  if (SAFE) {
    const double N = maxabs();
    if (active) {
      ej = e_col;
      Gj = G_col;
      if (kexp > 0) { ej += kexp; Gj = dscale_exp0(Gj, -kexp); pend = kexp; }
      Gj = __dadd_rn(Gj, __dmul_rn(cblk, N));
      if (Gj >= omega()) {
        k2 = choose_k_exp(Gj);
        ej += k2;
        Gj = dscale_exp(Gj, -k2);
        pend += k2;
      }
    }
  }

  // results through shared memory: coalesced column stores, and the digit
  // planes of X(I1,:) with one exponent per column for the tensor-core step
  __syncthreads();                       // sY free (replay / serial path done)
  int e = -(1 << 29);
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const double2 xo = (SAFE && k2) ? zscale_exp(y[q], -k2) : y[q];
    sY[js * LDY + row_of(q)] = xo;
    e = max(e, bound_exp(xo));
  }
  const bool planes = P.oz_bp != nullptr && (CONJ ? P.m - hi : lo) > 0;
  if (planes) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o, L));
    if (h == 0) sRedI[w * SPC + js] = e;
  }
  if (SAFE && active && w == 0 && h == 0) {
    P.e[j] = ej;
    P.G[j] = Gj;
    P.pend[j] = pend;
    P.E[(long long)b * P.n + j] = ej;
    if (pend > 0) raise_status(status, MSTS_STATUS_SCALED);
  }
  __syncthreads();
  for (int idx = tid; idx < SPC * NB; idx += kWThreads) {
    const int c = idx / NB, r = idx - c * NB, jj = jcta + c;
    if (jj < P.n && r < nbe_of(jj)) P.B[(long long)jj * P.ldb + lo + r] = sY[c * LDY + r];
  }
  if (planes) {
    if (tid < SPC) {
      int ec = sRedI[tid];
#pragma unroll
      for (int v = 1; v < kWWarps; ++v) ec = max(ec, sRedI[v * SPC + tid]);
      sShift[tid] = ec < -(1 << 28) ? 0 : ec;
    }
    __syncthreads();
    const int ncols = P.n - jstart, kw = P.oz_kb / 2;
    for (int idx = tid; idx < SPC * kw; idx += kWThreads) {
      const int c = idx / kw, r = idx - c * kw, jj = jcta + c;
      if (jj >= P.n) continue;
      const int cc = jj - jstart;
      if (r == 0) P.oz_cexp[cc] = sShift[c];
      uint32_t wd[kOzS];
      if (r < NB) {
        digit_pairs(sY[c * LDY + r], sShift[c], wd);
      } else {
#pragma unroll
        for (int t = 0; t < kOzS; ++t) wd[t] = 0u;   // K padding beyond n_b rows
      }
#pragma unroll
      for (int t = 0; t < kOzS; ++t) P.oz_bp[(size_t)(t * ncols + cc) * kw + r] = wd[t];
    }
  }
}

template <int L, bool SAFE, bool CONJ>
cudaError_t launch_w(const ProbTable &tab, int step, int shortcut, int ncols_max, uint32_t *status,
                     cudaStream_t st) {
  constexpr size_t smem = diagw_smem<L, SAFE>();
  constexpr int SPC = WShape<L>::SPC;
  cudaError_t e = cudaFuncSetAttribute(k_diagw<L, SAFE, CONJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_diagw<L, SAFE, CONJ>, dim3((ncols_max + SPC - 1) / SPC, 1, tab.count), dim3(kWThreads),
                    smem, st, tab, step, shortcut, status);
}

template <bool SAFE, bool CONJ>
cudaError_t launch_wl(int L, const ProbTable &tab, int step, int shortcut, int ncols_max, uint32_t *status,
                      cudaStream_t st) {
  if (L >= 4) return launch_w<4, SAFE, CONJ>(tab, step, shortcut, ncols_max, status, st);
  if (L == 2) return launch_w<2, SAFE, CONJ>(tab, step, shortcut, ncols_max, status, st);
  return launch_w<1, SAFE, CONJ>(tab, step, shortcut, ncols_max, status, st);
}

}  // namespace

cudaError_t set_alg4_chain_w(int on) { return cudaMemcpyToSymbol(g_alg4_chain_w, &on, sizeof(int)); }

cudaError_t launch_diagw(const ProbTable &tab, bool safe, bool conj, int step, int shortcut, int ncols_max,
                         int lanes, uint32_t *status, cudaStream_t st) {
  if (safe) return launch_wl<true, false>(lanes, tab, step, shortcut, ncols_max, status, st);
  if (conj) return launch_wl<false, true>(lanes, tab, step, shortcut, ncols_max, status, st);
  return launch_wl<false, false>(lanes, tab, step, shortcut, ncols_max, status, st);
}

}  // namespace msts
