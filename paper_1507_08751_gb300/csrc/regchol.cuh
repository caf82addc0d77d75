// Certified test "lambda_max(X) < c" for a symmetric X of order n <= NMAX:
// c I - X is positive definite iff its Cholesky factorisation exists
// (Golub & Van Loan, Sec. 4.2).  Used for the zero-rank test of a block
// (X = G, c just below tau^2) and for the deflated certificate of the
// Lanczos path (X = P G P).
//
// The matrix lives in registers for the whole factorisation.  It is padded
// to n8 = roundup(n, 8) with an identity block (positive definiteness is
// unchanged) and cut into 4x4 tiles of the lower triangle.  Columns 0..7 are
// formed straight into the first panel strip; every other tile belongs to
// one thread for the whole run, the tiles ordered by column, last column
// first, and dealt round-robin to the threads, so the tiles still active at
// any panel are a prefix of that order and the trailing updates stay
// balanced to one tile per thread.
//
// Per panel of 8 columns (right-looking, Sec. 4.2.9 of the same book):
//   1. the owners of the panel's tiles write them to a column-major strip
//      in shared memory (double-buffered),
//   2. every warp factors the 8x8 diagonal block (all get the same answer,
//      so no barrier is needed before 3): in every thread's registers for
//      small CTAs, by shuffles across 8 lanes where registers are scarce,
//   3. each row below solves for its 8 factor entries (one thread per row),
//   4. every thread subtracts the rank-8 product from its active tiles.
// Two CTA barriers per panel; no shared-memory traffic for the trailing
// matrix itself.
//
// Rounding: a successful factorisation of the computed c I - X is exact for
// c I - X + E with ||E||_2 <= n8^2 eps ||c I - X||_2 (Cholesky backward
// error, Golub & Van Loan Sec. 4.2.7, for any order of the inner-product
// sums), so callers take c below the wanted bound by that margin.
#pragma once

#include <float.h>

#include "common.cuh"

namespace msllr {

// shared scratch (floats) of regchol_pd: two 8 x n8 strips and one packed
// 8 x 8 factor per warp
__host__ __device__ constexpr int regchol_scratch_floats(int nmax, int nt) {
  return 16 * nmax + (nt / 32) * 36;
}

__device__ __forceinline__ int regchol_tri_row(int e) {
  int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
  while (((i + 1) * (i + 2)) / 2 <= e) ++i;
  while ((i * (i + 1)) / 2 > e) --i;
  return i;
}

// Returns true iff c I - X is numerically positive definite, where
//   X(r, q) = src.at(r, q) - [U What^T + What U^T](r, q)   (r >= q)
// with U, What (n8 x ku, column-major, leading dimension n8, rows >= n zero)
// in shared memory, or ku = 0.  With frob = true the shift is
//   c = c0 - n8^2 eps (c0 + ||X||_F)
// (the Frobenius norm bounds ||X||_2 for the rounding margin), else c = c0.
// Returns false when c <= 0.  `scr` holds regchol_scratch_floats(NMAX, NT)
// floats (16-byte aligned); `red` is block_sum scratch.  src is not
// modified.  All threads of the CTA must call; the answer is uniform.
template <int NT, int NMAX, class SX, bool REGF = (NT <= 128)>
__device__ bool regchol_pd(SX src, int n, float c0, bool frob, const float* U, const float* Wh,
                           int ku, float* scr, float* red, int slot = -1) {
  static_assert(NMAX % 8 == 0 && NT % 32 == 0, "shape");
  constexpr int NB = NMAX / 4;
  constexpr int TMAX = NB >= 3 ? (NB - 2) * (NB - 1) / 2 : 1;
  constexpr int SL = (TMAX + NT - 1) / NT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n8 = (n + 7) & ~7, nb = n8 >> 2;
  const int ntile = nb >= 3 ? (nb - 2) * (nb - 1) / 2 : 0;
  float* S = scr;                   // strips: S[(buf * 8 + u) * n8 + r]
  float* Lw = S + 16 * n8 + warp * 36;  // this warp's copy of the diagonal factor

  float v[SL][16];
  int ta[SL], tb[SL];
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int idx = s * NT + tid;
    ta[s] = tb[s] = -1;
    if (idx < ntile) {
      const int i = regchol_tri_row(idx);
      tb[s] = nb - 1 - i;
      ta[s] = tb[s] + (idx - (i * (i + 1)) / 2);
    }
  }

  // -X into the tiles and into the first strip
  float fro = 0.f;
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    if (tb[s] < 0) continue;
    const int r0 = 4 * ta[s], q0 = 4 * tb[s];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = r0 + i, q = q0 + j;
        v[s][i * 4 + j] = (r < n && q <= r) ? -src.at(r, q) : 0.f;
      }
    if (ku > 0) {
      for (int u = 0; u < ku; ++u) {
        const float4 ur = *reinterpret_cast<const float4*>(U + u * n8 + r0);
        const float4 wr = *reinterpret_cast<const float4*>(Wh + u * n8 + r0);
        const float4 uc = *reinterpret_cast<const float4*>(U + u * n8 + q0);
        const float4 wc = *reinterpret_cast<const float4*>(Wh + u * n8 + q0);
        const float urv[4] = {ur.x, ur.y, ur.z, ur.w}, wrv[4] = {wr.x, wr.y, wr.z, wr.w};
        const float ucv[4] = {uc.x, uc.y, uc.z, uc.w}, wcv[4] = {wc.x, wc.y, wc.z, wc.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j)
            v[s][i * 4 + j] = fmaf(urv[i], wcv[j], fmaf(wrv[i], ucv[j], v[s][i * 4 + j]));
      }
    }
    if (frob) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float x = v[s][i * 4 + j];
          const float w = (ta[s] != tb[s] || i > j) ? 2.f : (i == j ? 1.f : 0.f);
          fro = fmaf(w * x, x, fro);
        }
    }
  }
  for (int e = tid; e < 8 * n8; e += NT) {
    const int u = e / n8, r = e - u * n8;
    float x = 0.f;
    if (r < n && u <= r) {
      x = -src.at(r, u);
      for (int q = 0; q < ku; ++q)
        x = fmaf(U[q * n8 + r], Wh[q * n8 + u], fmaf(Wh[q * n8 + r], U[q * n8 + u], x));
    }
    S[e] = x;
    fro = fmaf(r == u ? x : 2.f * x, x, fro);
  }
  float c = c0;
  if (frob) {
    // the relative rounding of the sum of squares is far below the margin
    const float fx = sqrtf(block_sum<NT>(fro, red)) * 1.0001f;
    c = c0 - (float)n8 * (float)n8 * FLT_EPSILON * (c0 + fx);
  }
  if (!(c > 0.f)) return false;
  __syncthreads();
  PHASE_INIT();
  if (tid < 8) S[tid * n8 + tid] += c;
#pragma unroll
  for (int s = 0; s < SL; ++s)
    if (tb[s] >= 0 && ta[s] == tb[s]) {
      v[s][0] += c;
      v[s][5] += c;
      v[s][10] += c;
      v[s][15] += c;
    }

  for (int p = 0; 8 * p < n8; ++p) {
    const int j0 = 8 * p;
    float* Sb = S + (p & 1) * 8 * n8;
    if (p > 0) {
#pragma unroll
      for (int s = 0; s < SL; ++s)
        if (tb[s] == 2 * p || tb[s] == 2 * p + 1) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            *reinterpret_cast<float4*>(Sb + (4 * tb[s] + j - j0) * n8 + 4 * ta[s]) =
                make_float4(v[s][j], v[s][4 + j], v[s][8 + j], v[s][12 + j]);
        }
    }
    __syncthreads();
    // 8x8 diagonal block into this warp's packed copy Lw (lower triangle,
    // the diagonal replaced by the reciprocal pivots).  Every warp factors
    // it; rsqrt (a few ulp) instead of sqrt and a division keeps the chain
    // of 8 dependent pivots short, and its error stays far inside the
    // backward-error margin.
    bool ok = true;
    if constexpr (REGF) {
      // every thread holds the whole block (broadcast loads): no shuffles
      float L[36];
#pragma unroll
      for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int u = 0; u <= t; ++u) L[t * (t + 1) / 2 + u] = Sb[u * n8 + j0 + t];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float dj = L[j * (j + 1) / 2 + j];
        ok = ok && (dj > 0.f);
        const float inv = rsqrtf(dj > 0.f ? dj : 1.f);
        L[j * (j + 1) / 2 + j] = inv;
#pragma unroll
        for (int i = j + 1; i < 8; ++i) L[i * (i + 1) / 2 + j] *= inv;
#pragma unroll
        for (int i = j + 1; i < 8; ++i)
#pragma unroll
          for (int t = j + 1; t <= i; ++t)
            L[i * (i + 1) / 2 + t] = fmaf(-L[i * (i + 1) / 2 + j], L[t * (t + 1) / 2 + j],
                                          L[i * (i + 1) / 2 + t]);
      }
      if (!ok) return false;
      if (lane == 0) {
#pragma unroll
        for (int e = 0; e < 36; ++e) Lw[e] = L[e];
      }
    } else {
      // lane l < 8 holds row l (fewer registers, shuffles on the chain)
      float row[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) row[t] = (lane < 8 && t <= lane) ? Sb[t * n8 + j0 + lane] : 0.f;
      float myinv = 1.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float dj = __shfl_sync(0xffffffffu, row[j], j);
        ok = ok && (dj > 0.f);
        const float inv = rsqrtf(dj > 0.f ? dj : 1.f);
        if (lane == j) myinv = inv;
        if (lane > j) row[j] *= inv;
#pragma unroll
        for (int t = j + 1; t < 8; ++t) {
          const float ltj = __shfl_sync(0xffffffffu, row[j], t);
          if (lane >= t) row[t] = fmaf(-row[j], ltj, row[t]);
        }
      }
      if (!ok) return false;
      if (lane < 8) {
        const int base = lane * (lane + 1) / 2;
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (t < lane) Lw[base + t] = row[t];
        Lw[base + lane] = myinv;
      }
    }
    __syncwarp();
    // rows below the block: L21 = A21 L11^{-T}
    for (int r = j0 + 8 + tid; r < n8; r += NT) {
      float x[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        float acc = Sb[t * n8 + r];
#pragma unroll
        for (int u = 0; u < t; ++u) acc = fmaf(-x[u], Lw[t * (t + 1) / 2 + u], acc);
        x[t] = acc * Lw[t * (t + 1) / 2 + t];
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) Sb[t * n8 + r] = x[t];
    }
    __syncthreads();
    // trailing rank-8 update of the active tiles (column >= j0 + 8)
    const int bmin = 2 * p + 2;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      if (tb[s] < bmin) continue;
      const float* pr = Sb + 4 * ta[s];
      const float* pc = Sb + 4 * tb[s];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 a4 = *reinterpret_cast<const float4*>(pr + u * n8);
        const float4 b4 = *reinterpret_cast<const float4*>(pc + u * n8);
        const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) v[s][i * 4 + j] = fmaf(-av[i], bv[j], v[s][i * 4 + j]);
      }
    }
  }
  PHASE(slot, 15);
  return true;
}

}  // namespace msllr
