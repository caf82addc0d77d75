// One warp's block SVT of a narrow block (min(m, n) <= 16, max(m, n) <= 32),
// the whole block in registers -- eq:bsvt under the Sec. 9 shift.  Used by
// the per-scale warp kernel (k_block_warp.cu) and by the nested-scale
// kernel (k_nested.cu).
//   Steps:
//   gather R_b(Shift_s(A)), A = A1 + A2, as C (mm x nn, the block or its
//   transpose: SVT(B^T) = SVT(B)^T); lane (h, c) holds column c of C at the
//   rows of parity h, so that one load instruction reads two 64-byte row
//   segments;
//   skip when an upper bound of sigma_max^2 is <= tau^2 (Sec. 8): ||C||_F^2,
//   then Gershgorin on G = C^T C (formed by shuffles), then a certificate
//   that c0 I - G is positive definite (Cholesky in registers, lane c holding
//   row c) with c0 below tau^2 by the factorisation's rounding margin;
//   otherwise the SVD by one-sided Jacobi (Hestenes): columns p, q of C V
//   are rotated until every pair is orthogonal to working precision, with
//   the round-robin pair order of the block's columns (nn rounded up to
//   even: nn - 1 rounds of nn / 2 disjoint pairs per sweep); the singular
//   values are the column norms of C V (no Gram
//   matrix, so no squared condition number) and the right singular vectors
//   are the columns of V;
//   Z' = (C V) diag(f) V^T with f_j = max(1 - tau / sigma_j, 0) (eq:svt),
//   scattered through Shift_{-s}, and the fused dual update W' = 2 Z' - A
//   of eq:admm.
// Nothing but the inputs and outputs touches global memory.
#pragma once

#include <float.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace msllr {
namespace {

// the second half of A from global memory (none: zero)
struct A2Global {
  const float* p;
  __device__ __forceinline__ float operator()(size_t off, int, int) const {
    return p ? __ldg(p + off) : 0.f;
  }
};

constexpr int kWT = 32;
constexpr int kWarps = kWT / 32;
constexpr float kRotTol = 2e-6f;    // rotate columns p, q while |c_p . c_q| > tol ||c_p|| ||c_q||
constexpr float kTinyCol = 1e-13f;  // squared norm of a numerically zero column, relative to ||C||_F^2
constexpr int kMaxSweeps = 12;
constexpr unsigned kFull = 0xffffffffu;

// Block b of the scale by the calling warp.  RPL: rows of C per lane
// (mm <= 2 RPL); NP: columns in the rotation order when fixed at compile
// time (16 for blocks 15 or 16 wide), 0 to take it from the block.  `vs` is
// the warp's 16 x 17 shared scratch (V, for the rebuild); `a2(off, row,
// col)` gives the second half of A at global offset off, block element
// (row, col) in the block's own orientation (A2Global: a.A2 itself).
template <int RPL, bool ST, int NP, class SRC>
__device__ __forceinline__ void warp_block_svt(const ScaleLaunch& a, int b, float (*vs)[17],
                                               const SRC& a2) {
  const int lane = threadIdx.x & 31;
  const int h = lane >> 4, c = lane & 15;
  PHASE_INIT();
  const BlockGeom g = block_geom_t<ST>(a, b);
  const int mm = g.mm(), nn = g.nn();
  const bool tr = g.transposed();
  const bool col = c < nn;

  // gather (all loads in flight at once: predicated, the two halves of A
  // added after the last load); ||C||_F^2
  float x[RPL];
  float fro = 0.f;
  {
    float y[RPL];
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      const int r = h + 2 * i;
      const bool in = col && r < mm;
      const int rr = in ? r : 0, cc = in ? c : 0;
      const size_t off = tr ? g.offset(cc, rr) : g.offset(rr, cc);
      x[i] = in ? __ldg(a.A1 + off) : 0.f;
      y[i] = in ? (tr ? a2(off, cc, rr) : a2(off, rr, cc)) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      x[i] += y[i];
      fro = fmaf(x[i], x[i], fro);
    }
  }
  fro = warp_sum(fro);
  PHASE(0, 0);
  const float thr = a.tau * a.tau;
  bool skipped = a.skip_bound && fro <= thr;
  float fl = 0.f;  // flops of the steps run
  if (a.skip_bound && !skipped) {
    // G = C^T C: lane (h, c) forms row c of G from its rows of C and the
    // other columns' values at the same rows (shuffles), then adds the other
    // half's partial sums
    float gr[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) gr[j] = 0.f;
#pragma unroll
    for (int i = 0; i < RPL; ++i)
#pragma unroll
      for (int j = 0; j < 16; ++j) gr[j] = fmaf(x[i], __shfl_sync(kFull, x[i], (h << 4) | j), gr[j]);
    float rs = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      gr[j] += __shfl_xor_sync(kFull, gr[j], 16);
      rs += fabsf(gr[j]);
    }
    // Gershgorin: lambda_max(G) <= max_c sum_j |G_cj| (Sec. 8)
    const float gbound = fminf(fro, warp_max(rs));
    fl += (float)(2 * mm * nn * nn + 2 * nn * nn);
    if (gbound <= thr) {
      skipped = true;
    } else {
      // certified lambda_max(G) < tau^2 by the Cholesky factorisation of
      // c0 I - G, c0 below tau^2 by the backward-error margin of the
      // factorisation (Golub & Van Loan, Sec. 4.2.7); lane c holds row c
      const int n8 = (nn + 7) & ~7;
      const float c0 = thr - (float)(n8 * n8) * FLT_EPSILON * (thr + gbound);
      bool pd = c0 > 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) gr[j] = (j == c ? c0 : 0.f) - gr[j];
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        if (kk < nn && pd) {
          const float d = __shfl_sync(kFull, gr[kk], kk);
          pd = d > 0.f;
          const float l = gr[kk] * rsqrtf(d > 0.f ? d : 1.f);  // L(c, kk) for c > kk
#pragma unroll
          for (int j = kk + 1; j < 16; ++j)
            if (j < nn) gr[j] = fmaf(-l, __shfl_sync(kFull, l, j), gr[j]);
        }
      }
      fl += (float)(nn * nn * nn) / 3.f;
      skipped = pd;
    }
  }

  PHASE(0, 1);
  float z[RPL];
#pragma unroll
  for (int i = 0; i < RPL; ++i) z[i] = 0.f;
  int k = 0;
  int sweeps = 0;
  if (!skipped) {
    // one-sided Jacobi: y = C V, V = I at the start
    float y[RPL], v[8];
#pragma unroll
    for (int i = 0; i < RPL; ++i) y[i] = x[i];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = (h + 2 * i == c) ? 1.f : 0.f;
    const float inv_fro = 1.f / fro;
    const int np = NP ? NP : (nn + 1) & ~1;  // columns in the rotation order (nn rounded up to even)
    for (; sweeps < kMaxSweeps;) {
      ++sweeps;
      // squared norm of this lane's column of C V: recomputed every sweep,
      // carried through the sweep's rotations by a' = a -/+ t ga
      float al = 0.f;
#pragma unroll
      for (int i = 0; i < RPL; ++i) al = fmaf(y[i], y[i], al);
      al += __shfl_xor_sync(kFull, al, 16);
      bool rotated = false;
#pragma unroll 1
      for (int rd = 0; rd < np - 1; ++rd) {
        // round-robin partner among the np (even) columns: column np - 1
        // stays, the others turn (p + q = 2 rd mod (np - 1)); lanes past np
        // are their own partners and never rotate
        int o = 2 * rd - c;  // in (-(np - 1), 2 (np - 1)): one correction reduces it
        if (o < 0) o += np - 1;
        else if (o >= np - 1) o -= np - 1;
        if (c == rd) o = np - 1;
        if (c == np - 1) o = rd;
        if (c >= np) o = c;
        const int src = (h << 4) | o;
        const float be = __shfl_sync(kFull, al, src);
        float yo[RPL];
        float g0 = 0.f, g1 = 0.f;
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          yo[i] = __shfl_sync(kFull, y[i], src);
          if (i & 1) g1 = fmaf(y[i], yo[i], g1);
          else g0 = fmaf(y[i], yo[i], g0);
        }
        float ga = g0 + g1;
        ga += __shfl_xor_sync(kFull, ga, 16);
        // the rotation that zeroes the off-diagonal of the 2 x 2 Gram matrix
        // [[a_lo, ga], [ga, a_hi]] of columns lo < hi (Golub & Van Loan,
        // Alg. 8.5.1): both lanes of the pair evaluate it in that order, so
        // they get the same (c, s), and apply
        //   c_lo' = c c_lo - s c_hi,   c_hi' = s c_lo + c c_hi
        // (t needs no full accuracy: any (c, s) with c^2 + s^2 = 1 is a
        // rotation; c comes from rsqrt with one Newton step)
        const bool lo = c < o;
        const float a_lo = lo ? al : be, a_hi = lo ? be : al;
        const float gn = ga * inv_fro;
        float cr = 1.f, sr = 0.f, t = 0.f;
        // (a column at the rounding level of ||C||_F is numerically zero:
        // no rotation, else an exactly rank-deficient block never settles)
        if (o != c && fminf(a_lo, a_hi) > kTinyCol * fro &&
            gn * gn > (kRotTol * kRotTol) * ((a_lo * inv_fro) * (a_hi * inv_fro))) {
          // the angle with tan 2 phi = 2 ga / (a_hi - a_lo), |phi| <= pi / 4,
          // by half angles: cos 2 phi = |D| / q, sin 2 phi = 2 ga sign(D) / q,
          // q = sqrt(D^2 + 4 ga^2); c = sqrt((1 + cos 2 phi) / 2) >= 1 / sqrt(2),
          // s = sin 2 phi / (2 c); two rsqrt, each with one Newton step
          const float dn = (a_hi - a_lo) * inv_fro;
          const float q2 = fmaf(dn, dn, 4.f * gn * gn);
          float rq = rsqrtf(q2);
          rq = rq * fmaf(-0.5f * q2 * rq, rq, 1.5f);
          const float hh = fmaf(0.5f * fabsf(dn), rq, 0.5f);
          float rh = rsqrtf(hh);
          rh = rh * fmaf(-0.5f * hh * rh, rh, 1.5f);
          cr = hh * rh;
          sr = copysignf(1.f, dn) * gn * rq * rh;
          t = sr * rh;  // tan phi = s / c
          rotated = true;
        }
        const float so = lo ? -sr : sr;  // weight of the partner column
        al = lo ? fmaf(-t, ga, al) : fmaf(t, ga, al);
#pragma unroll
        for (int i = 0; i < RPL; ++i) y[i] = fmaf(so, yo[i], cr * y[i]);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float vo = __shfl_sync(kFull, v[i], src);
          v[i] = fmaf(so, vo, cr * v[i]);
        }
      }
      if (!__any_sync(kFull, rotated)) break;
    }
    PHASE(0, 2);
    if (threadIdx.x == 0) PHASE_ADD(0, 5, sweeps);
    // singular values: the column norms of C V
    float al = 0.f;
#pragma unroll
    for (int i = 0; i < RPL; ++i) al = fmaf(y[i], y[i], al);
    al += __shfl_xor_sync(kFull, al, 16);
    const float sig = sqrtf(al);
    const float f = (col && sig > a.tau) ? 1.f - a.tau / sig : 0.f;
    const unsigned act = __ballot_sync(kFull, f > 0.f) & 0xffffu;
    k = __popc(act);
    if (k > 0) {
      if (a.nuc_acc) {
        double t = (lane < 16 && f > 0.f) ? (double)(sig - a.tau) : 0.0;
        t = warp_sum_d(t);
        if (lane == 0) atomicAdd(a.nuc_acc, t);
      }
      // Z' = sum over kept j of f_j (C V)_j V_j^T; lane (h, c) needs V(c, j),
      // which another lane holds: V goes through shared memory
#pragma unroll
      for (int i = 0; i < 8; ++i) vs[h + 2 * i][c] = v[i];
      __syncwarp();
      unsigned rest = act;
      while (rest) {
        const int j = __ffs(rest) - 1;
        rest &= rest - 1;
        const float w = __shfl_sync(kFull, f, j) * vs[c][j];
        const int sj = (h << 4) | j;
#pragma unroll
        for (int i = 0; i < RPL; ++i) z[i] = fmaf(__shfl_sync(kFull, y[i], sj), w, z[i]);
      }
    }
  }
  // scatter Z' and W' = 2 Z' - A through Shift_{-s}
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const int r = h + 2 * i;
    if (col && r < mm) {
      const size_t off = tr ? g.offset(c, r) : g.offset(r, c);
      a.Zout[off] = z[i];
      if (a.Wout) a.Wout[off] = 2.f * z[i] - x[i];
    }
  }
  PHASE(0, 3);
  if (lane == 0) {
    if (a.rank_out) a.rank_out[b] = k;
    if (a.cnt) {
      if (skipped) atomicAdd(a.cnt, 1ull);
      if (k == 0) atomicAdd(a.cnt + 1, 1ull);
      if (!skipped) atomicAdd(a.cnt + 3, 1ull);
      // per sweep np - 1 rounds of np / 2 column pairs: norms and inner
      // product (6 mm), the two columns of C V and of V rotated (6 mm + 96);
      // the rebuild 2 mm nn per kept pair
      const int npr = (nn + 1) & ~1;
      const double fj = (double)sweeps * (npr - 1) * (npr / 2) * (12.0 * mm + 96.0) + 2.0 * mm * nn * k;
      if (fl > 0.f || fj > 0.0) atomicAdd(a.cnt + 5, (unsigned long long)(fj + fl));
    }
  }
}

}  // namespace
}  // namespace msllr
