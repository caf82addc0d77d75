// Certified top eigenpairs of a block's Gram matrix G = C^T C without a full
// tridiagonalisation, for the block SVT (eq:svt): SVT needs only the
// eigenpairs with lambda > tau^2.
//
//  1. Lanczos with full reorthogonalisation (Golub & Van Loan, Sec. 10.1)
//     builds an orthonormal Q_J and the tridiagonal T_J = Q_J^T G Q_J.  The
//     start vector is either pseudo-random or the sum of the previous
//     iteration's Ritz vectors (warm start).  On breakdown the process is
//     continued from a random vector orthogonal to Q_J.
//  2. Ritz pairs of T_J above 0.95 tau^2: Sturm-count multisection and
//     inverse iteration on T_J (symeig.cuh), U = Q_J Y.
//  3. Explicit residuals: W = G U, B = U^T W, rho = ||W - U diag(B)||_F.
//  4. Certificate: with P = I - U U^T, every eigenvalue of G lies within
//     2 rho of an eigenvalue of diag(B) (+) (P G P restricted to range P)
//     (Weyl, block form in the basis [U, U_perp]).  If the Cholesky of
//     (tau^2 - 2 rho - margins) I - P G P succeeds, no eigenvalue of G
//     outside span(U) exceeds tau^2, so the eigenpairs above tau^2 are the
//     Ritz pairs above tau^2 (up to pairs within 2 rho of tau^2, whose
//     thresholded contribution is below rho / tau).
// If any step fails (too many pairs, no convergence, certificate refused),
// the caller falls back to the Householder path.
#pragma once

#include <float.h>

#include <type_traits>

#include "common.cuh"
#include "regchol.cuh"
#include "symeig.cuh"

namespace msllr {

constexpr int kLzMaxJ = 32;  // Lanczos steps
constexpr int kLzMaxK = 8;   // Ritz pairs kept (above 0.95 tau^2)

// FP32 flops of the eigen-solve steps, each counted at its algorithmic cost
// (a multiply-add is 2 flops); the kernels add them up per block so that the
// ALU roofline follows the steps that actually ran.
__device__ __forceinline__ double fl_symv(int n) { return 2.0 * n * n; }
__device__ __forceinline__ double fl_chol(int n) { return (double)n * n * n / 3.0; }
// J Lanczos steps (matrix-vector product plus two Gram-Schmidt passes over
// j + 1 vectors), U = Q_J Y, W = G U for 8 vectors, B = U^T W
__device__ __forceinline__ double fl_lanczos(int n, int J, int ku) {
  return 2.0 * n * n * J + 4.0 * n * J * (J + 1) + 2.0 * n * J * ku + 16.0 * n * n + 16.0 * n * ku;
}
// the rank-2k deflation G - U What^T - What U^T on the lower triangle
__device__ __forceinline__ double fl_deflate(int n, int ku) { return 2.0 * ku * n * n; }
// Householder tridiagonalisation, back-transformation of k eigenvectors
__device__ __forceinline__ double fl_householder(int n, int k) {
  return 4.0 * n * n * n / 3.0 + 2.0 * n * n * k;
}

// leading dimension of the Lanczos basis in shared memory: padded for the
// thread-per-coefficient projection of small blocks
template <int NMAX>
__host__ __device__ constexpr int lz_ldq(int n) {
  return NMAX <= 64 ? n + 1 : n;
}

// shared scratch (floats) of the certificate step of lanczos_candidates
__host__ __device__ constexpr int lz_cert_floats(int nmax, int nt) {
  return 16 * nmax + regchol_scratch_floats(nmax, nt);
}

// Shared-memory scratch of the Lanczos path.
struct LzScratch {
  float* x;      // [n] current Lanczos vector q_j
  float* w;      // [n] G q_j, then the next residual
  float* alpha;  // [kLzMaxJ]
  float* beta;   // [kLzMaxJ]
  float* h;      // [2 * kLzMaxJ + 8] projection coefficients (two passes)
  float* ty;     // [jcap * kLzMaxK] eigenvectors of T_J (row i, column q)
  float* lu;     // [4 * jcap * kLzMaxK] inverse-iteration LU factors
  unsigned* piv; // [2 * kLzMaxK] pivot bits
  float* Bm;     // [kLzMaxK * kLzMaxK] U^T G U
  int jcap;      // row capacity of ty / lu (>= Lanczos steps)
};

// floats of LzScratch for a given n capacity and J capacity
__host__ __device__ constexpr int lz_scratch_floats(int nmax, int jcap) {
  return 2 * nmax + 2 * kLzMaxJ + (2 * kLzMaxJ + 8) + jcap * kLzMaxK + 4 * jcap * kLzMaxK +
         2 * kLzMaxK + kLzMaxK * kLzMaxK;
}

template <int NT>
__device__ void lz_bind(LzScratch& z, float* base, int nmax, int jcap) {
  z.x = base;
  z.w = z.x + nmax;
  z.alpha = z.w + nmax;
  z.beta = z.alpha + kLzMaxJ;
  z.h = z.beta + kLzMaxJ;
  z.ty = z.h + 2 * kLzMaxJ + 8;
  z.lu = z.ty + jcap * kLzMaxK;
  z.piv = reinterpret_cast<unsigned*>(z.lu + 4 * jcap * kLzMaxK);
  z.Bm = reinterpret_cast<float*>(z.piv + 2 * kLzMaxK);
  z.jcap = jcap;
}

__device__ __forceinline__ float lz_hash(uint32_t seed, int i) {
  uint32_t h = seed * 0x9E3779B9u + (uint32_t)i * 0x85EBCA6Bu + 0x27D4EB2Fu;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (float)(h >> 8) * (2.f / 16777216.f) - 1.f;
}

// y = G x with TPR threads per row (G symmetric in lower storage, n <= NMAX,
// x and y shared, y must not alias x).  Each thread walks its part of row r
// in two ranges, G(r, c) for c <= r and G(c, r) above, so every element of
// the row is read once and the only reduction is a shuffle inside the TPR
// lanes of the row.  Ends with a CTA barrier.
template <int NT, int NMAX, bool ABS = false, class S>
__device__ void symv_rows(S G, int n, const float* x, float* y) {
  constexpr int TPR = (NT / NMAX >= 2) ? 2 : 1;
  const int tid = threadIdx.x, p = tid % TPR;
  if constexpr (std::is_same<S, LowerPacked>::value && NT == 512) {
    // packed storage: warp w takes rows 32 (w & 7) + lane and half (w >> 3)
    // of the columns.  All lanes of a warp walk the same column c, so the
    // loads T(r) + c (c <= r) and T(c) + r (c > r), T(i) = i (i + 1) / 2,
    // hit distinct banks, and x[c] is a broadcast.  Left of the warp's row
    // band the row part is contiguous, right of it the column part advances
    // by c + 1; only the 32 columns of the band need both forms.
    const float* g = G.g;
    const int lane = tid & 31, warp = tid >> 5;
    const int b0 = 32 * (warp & 7), half = warp >> 3;
    const int r = b0 + lane;
    const int cs = (n + 1) >> 1;
    const int c_lo = half ? cs : 0, c_hi = half ? n : cs;
    float acc = 0.f;
    if (b0 < n) {
      const int rr = r < n ? r : n - 1;  // lanes past n compute a dummy row
      const int tr = (rr * (rr + 1)) / 2;
      // four accumulators, so that four loads and FMAs are in flight
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      int c = c_lo;
      const int e1 = min(c_hi, b0);
      for (; c + 3 < e1; c += 4) {
        a0 = fmaf(ABS ? fabsf(g[tr + c]) : g[tr + c], x[c], a0);
        a1 = fmaf(ABS ? fabsf(g[tr + c + 1]) : g[tr + c + 1], x[c + 1], a1);
        a2 = fmaf(ABS ? fabsf(g[tr + c + 2]) : g[tr + c + 2], x[c + 2], a2);
        a3 = fmaf(ABS ? fabsf(g[tr + c + 3]) : g[tr + c + 3], x[c + 3], a3);
      }
      for (; c < e1; ++c) a0 = fmaf(ABS ? fabsf(g[tr + c]) : g[tr + c], x[c], a0);
      const int e2 = min(c_hi, b0 + 32);
      for (; c < e2; ++c) {
        const int idx = c <= rr ? tr + c : (c * (c + 1)) / 2 + rr;
        a1 = fmaf(ABS ? fabsf(g[idx]) : g[idx], x[c], a1);
      }
      int idx = (c * (c + 1)) / 2 + rr;
      for (; c + 3 < c_hi; c += 4) {
        const int i1 = idx + c + 1;
        const int i2 = i1 + c + 2;
        const int i3 = i2 + c + 3;
        a0 = fmaf(ABS ? fabsf(g[idx]) : g[idx], x[c], a0);
        a1 = fmaf(ABS ? fabsf(g[i1]) : g[i1], x[c + 1], a1);
        a2 = fmaf(ABS ? fabsf(g[i2]) : g[i2], x[c + 2], a2);
        a3 = fmaf(ABS ? fabsf(g[i3]) : g[i3], x[c + 3], a3);
        idx = i3 + c + 4;
      }
      for (; c < c_hi; ++c) {
        a0 = fmaf(ABS ? fabsf(g[idx]) : g[idx], x[c], a0);
        idx += c + 1;
      }
      acc = (a0 + a1) + (a2 + a3);
    }
    if (half && r < n) y[r] = acc;
    __syncthreads();
    if (!half && r < n) y[r] += acc;
  } else {
    // the row loop is uniform across the CTA so that every lane reaches the
    // shuffle below
    for (int r0 = 0; r0 < n; r0 += NT / TPR) {
      const int r = r0 + tid / TPR;
      float a0 = 0.f, a1 = 0.f;
      if (r < n) {
        int c = p;
        for (; c + TPR <= r; c += 2 * TPR) {
          const float g0 = G.at(r, c), g1 = G.at(r, c + TPR);
          a0 = fmaf(ABS ? fabsf(g0) : g0, x[c], a0);
          a1 = fmaf(ABS ? fabsf(g1) : g1, x[c + TPR], a1);
        }
        if (c <= r) {
          const float g = G.at(r, c);
          a0 = fmaf(ABS ? fabsf(g) : g, x[c], a0);
          c += TPR;
        }
        for (; c + TPR < n; c += 2 * TPR) {
          const float g0 = G.at(c, r), g1 = G.at(c + TPR, r);
          a0 = fmaf(ABS ? fabsf(g0) : g0, x[c], a0);
          a1 = fmaf(ABS ? fabsf(g1) : g1, x[c + TPR], a1);
        }
        if (c < n) {
          const float g = G.at(c, r);
          a0 = fmaf(ABS ? fabsf(g) : g, x[c], a0);
        }
      }
      float acc = a0 + a1;
      if constexpr (TPR == 2) acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (p == 0 && r < n) y[r] = acc;
    }
  }
  __syncthreads();
}

// Y = G X for 8 vectors at once (X, Y shared, n x 8 row-major, 16-byte
// aligned): every element of G is read once per row walk for all 8
// products.  Same row split as symv_rows; ends with a CTA barrier.
template <int NT, int NMAX, class S>
__device__ void symm_rows8(S G, int n, const float* X, float* Yo) {
  constexpr int TPR = (NT / NMAX >= 2) ? 2 : 1;
  const int tid = threadIdx.x, p = tid % TPR;
  for (int r0 = 0; r0 < n; r0 += NT / TPR) {
    const int r = r0 + tid / TPR;
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.f;
    if (r < n) {
      for (int c = p; c < n; c += TPR) {
        const float g = c <= r ? G.at(r, c) : G.at(c, r);
        const float4 x0 = *reinterpret_cast<const float4*>(X + c * 8);
        const float4 x1 = *reinterpret_cast<const float4*>(X + c * 8 + 4);
        acc[0] = fmaf(g, x0.x, acc[0]);
        acc[1] = fmaf(g, x0.y, acc[1]);
        acc[2] = fmaf(g, x0.z, acc[2]);
        acc[3] = fmaf(g, x0.w, acc[3]);
        acc[4] = fmaf(g, x1.x, acc[4]);
        acc[5] = fmaf(g, x1.y, acc[5]);
        acc[6] = fmaf(g, x1.z, acc[6]);
        acc[7] = fmaf(g, x1.w, acc[7]);
      }
    }
    if constexpr (TPR == 2) {
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 1);
    }
    if (p == 0 && r < n) {
      *reinterpret_cast<float4*>(Yo + r * 8) = make_float4(acc[0], acc[1], acc[2], acc[3]);
      *reinterpret_cast<float4*>(Yo + r * 8 + 4) = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
  }
  __syncthreads();
}

// w <- (I - Q Q^T) w twice (classical Gram-Schmidt, two passes) over Q's
// columns 0..nq-1 (column i at Q + i*ldq, shared).  h1 and h2 receive the
// two passes' coefficients; returns ||w||^2 after the second pass.  Small
// n: one thread per coefficient with four partial sums (ldq = n + 1 keeps
// the threads on distinct banks); large n: one warp per coefficient.
template <int NT, int NMAX>
__device__ float lz_project(float* w, const float* Q, int ldq, int n, int nq, float* h1,
                            float* h2, float* red) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float part = 0.f;
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    float* h = pass == 0 ? h1 : h2;
    if constexpr (NMAX <= 64) {
      for (int i = tid; i < nq; i += NT) {
        const float* qi = Q + i * ldq;
        float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
        int e = 0;
        for (; e + 3 < n; e += 4) {
          d0 = fmaf(qi[e], w[e], d0);
          d1 = fmaf(qi[e + 1], w[e + 1], d1);
          d2 = fmaf(qi[e + 2], w[e + 2], d2);
          d3 = fmaf(qi[e + 3], w[e + 3], d3);
        }
        for (; e < n; ++e) d0 = fmaf(qi[e], w[e], d0);
        h[i] = (d0 + d1) + (d2 + d3);
      }
    } else {
      for (int i = warp; i < nq; i += NW) {
        float d = 0.f;
        for (int e = lane; e < n; e += 32) d = fmaf(Q[i * ldq + e], w[e], d);
        d = warp_sum(d);
        if (lane == 0) h[i] = d;
      }
    }
    __syncthreads();
    for (int e = tid; e < n; e += NT) {
      float v = w[e];
      for (int i = 0; i < nq; ++i) v = fmaf(-h[i], Q[i * ldq + e], v);
      w[e] = v;
      if (pass == 1) part = fmaf(v, v, part);
    }
    __syncthreads();
  }
  return block_sum<NT>(part, red);
}

// Inverse iteration on T (s.d, s.e, size J) for the k shifts s.shf[0..k),
// one thread per target, LU factors in shared memory; eigenvectors into ty
// (row i, column q, stride kLzMaxK), orthonormalised inside clusters.
template <int NT>
__device__ void lz_tri_vectors(int J, int k, float tnorm, EigScratch& s, LzScratch& z) {
  const int tid = threadIdx.x;
  const float tiny = FLT_EPSILON * tnorm;
  constexpr int ST = kLzMaxK;
  float* dd = z.lu;
  float* du = dd + z.jcap * ST;
  float* du2 = du + z.jcap * ST;
  float* dl = du2 + z.jcap * ST;
  for (int pass = 0; pass < 2; ++pass) {
    if (tid < k) {
      const int q = tid;
      if (pass == 0) {
        const float shift = s.shf[q];
        for (int i = 0; i < J; ++i) dd[i * ST + q] = s.d[i] - shift;
        for (int i = 0; i < J - 1; ++i) {
          du[i * ST + q] = s.e[i];
          dl[i * ST + q] = s.e[i];
          du2[i * ST + q] = 0.f;
        }
        unsigned bits[2] = {0u, 0u};
        for (int i = 0; i < J - 1; ++i) {
          const float di = dd[i * ST + q], li = dl[i * ST + q];
          if (fabsf(di) >= fabsf(li)) {
            const float dv = (di == 0.f) ? tiny : di;
            dd[i * ST + q] = dv;
            const float f = li / dv;
            dl[i * ST + q] = f;
            dd[(i + 1) * ST + q] -= f * du[i * ST + q];
          } else {
            const float f = di / li;
            dd[i * ST + q] = li;
            dl[i * ST + q] = f;
            const float t = du[i * ST + q];
            du[i * ST + q] = dd[(i + 1) * ST + q];
            dd[(i + 1) * ST + q] = t - f * dd[(i + 1) * ST + q];
            if (i < J - 2) {
              du2[i * ST + q] = du[(i + 1) * ST + q];
              du[(i + 1) * ST + q] = -f * du[(i + 1) * ST + q];
            }
            bits[i >> 5] |= 1u << (i & 31);
          }
        }
        for (int i = 0; i < J; ++i) {
          const float v = dd[i * ST + q];
          if (fabsf(v) < tiny) dd[i * ST + q] = v < 0.f ? -tiny : tiny;
        }
        z.piv[2 * q] = bits[0];
        z.piv[2 * q + 1] = bits[1];
        for (int i = 0; i < J; ++i) z.ty[i * ST + q] = tiny * lz_hash(977u + q, i);
      } else {
        for (int i = 0; i < J; ++i) z.ty[i * ST + q] *= tiny;
      }
      // solve (T - shift I) y = y
      const unsigned b0 = z.piv[2 * q], b1 = z.piv[2 * q + 1];
      float* y = z.ty + q;
      for (int i = 0; i < J - 1; ++i) {
        const float a = y[i * ST], b = y[(i + 1) * ST];
        const bool pv = (i < 32) ? ((b0 >> i) & 1u) : ((b1 >> (i - 32)) & 1u);
        if (pv) {
          y[i * ST] = b;
          y[(i + 1) * ST] = a - dl[i * ST + q] * b;
        } else {
          y[(i + 1) * ST] = b - dl[i * ST + q] * a;
        }
      }
      y[(J - 1) * ST] /= dd[(J - 1) * ST + q];
      if (J > 1)
        y[(J - 2) * ST] = (y[(J - 2) * ST] - du[(J - 2) * ST + q] * y[(J - 1) * ST]) / dd[(J - 2) * ST + q];
      for (int i = J - 3; i >= 0; --i)
        y[i * ST] = (y[i * ST] - du[i * ST + q] * y[(i + 1) * ST] - du2[i * ST + q] * y[(i + 2) * ST]) /
                    dd[i * ST + q];
      normalize_column(y, ST, J);
    }
    __syncthreads();
    cluster_mgs<NT>(z.ty, ST, J, k, s.clus, s.red);
    __syncthreads();
  }
}

// Ritz values of T_J above thr (descending) into s.lam and their vectors
// into z.ty.  Returns the count (a count above kLzMaxK means "too many").
template <int NT>
__device__ int lz_ritz(int J, float thr, EigScratch& s, LzScratch& z, float* tnorm_out) {
  const int tid = threadIdx.x;
  for (int i = tid; i < J; i += NT) {
    s.d[i] = z.alpha[i];
    s.e[i] = (i < J - 1) ? z.beta[i] : 0.f;
  }
  __syncthreads();
  float tn = 0.f;
  const int k = top_eigenvalues<NT>(J, thr, s, &tn);
  *tnorm_out = tn;
  if (k == 0 || k > kLzMaxK) return k;
  lz_tri_vectors<NT>(J, k, tn, s, z);
  return k;
}

// Gershgorin bound max_i sum_j |A_ij| of a symmetric matrix in lower storage:
// the row sums are |A| times a vector of ones.
template <int NT, int NMAX, class S>
__device__ float gershgorin_lower(S A, int n, float* ones, float* sums, float* red) {
  for (int e = threadIdx.x; e < n; e += NT) ones[e] = 1.f;
  __syncthreads();
  symv_rows<NT, NMAX, true>(A, n, ones, sums);
  float m = 0.f;
  for (int e = threadIdx.x; e < n; e += NT) m = fmaxf(m, sums[e]);
  return block_max<NT>(m, red);
}

// The whole Lanczos + certificate path.
//  Gs  G in lower storage, read only (the Lanczos operator).
//  Q   shared scratch of jmax * lz_ldq<NMAX>(n) floats (column j at
//      Q + j * lz_ldq<NMAX>(n)), jmax <= n.
//  U   receives the kept Ritz vectors (kLzMaxK * n floats, column-major,
//      any memory).
//  warm / kwarm: previous Ritz vectors (column-major n x kwarm) or kwarm = 0.
//  gbound: an upper bound of ||G||_2.
//  panel: lz_cert_floats(NMAX, NT) floats of 16-byte aligned shared
//      scratch for the certificate (may alias Q and the symv scratch).
// Steps 1-3 and the set-up of step 4.  On success returns k >= 0 (pairs
// above thr) with s.lam[0..k), the vectors in U's columns 0..k-1 (U holds
// ku >= k kept pairs, *ku_out = ku), U and What = W - U sym(B) / 2 staged at
// panel and panel + 8 n8 (n8 = roundup(n, 8)) and the certificate shift
// in *c0_out (and, if J_out is given, the Lanczos steps run in *J_out):
// the pairs are certified iff
//   regchol_pd<NT, NMAX>(G, n, *c0_out, true, panel, panel + 8 n8, ku,
//                        panel + 16 n8, red)
// holds (one call site per kernel keeps the code size and the register
// allocation of that routine in one place).  Returns -1 when the caller
// must fall back.  G is never modified.
template <int NT, int NMAX, class SG>
__device__ int lanczos_candidates(SG Gs, int n, float thr, float gbound, float* Q, int jmax,
                                  float* U, const float* warm, int kwarm,
                                  uint32_t seed, EigScratch& s, LzScratch& z, float* panel,
                                  int* ku_out, float* c0_out, int slot = -1,
                                  int* J_out = nullptr) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  PHASE_INIT();
  const float thr_keep = 0.95f * thr;  // pairs kept in U (deflated)

  // start vector
  float part = 0.f;
  for (int e = tid; e < n; e += NT) {
    float v = 0.f;
    for (int i = 0; i < kwarm; ++i) v += warm[(size_t)i * n + e] * (1.f + 0.25f * i);
    v += 1e-3f * lz_hash(seed, e);
    z.x[e] = v;
    part = fmaf(v, v, part);
  }
  const float inrm = 1.f / sqrtf(block_sum<NT>(part, s.red));
  const int ldq = lz_ldq<NMAX>(n);
  for (int e = tid; e < n; e += NT) Q[e] = z.x[e] * inrm;
  __syncthreads();
  const int jmin = min(jmax, kwarm > 0 ? kwarm + 3 : 8);
  int J = 0, k = -1;
  float tn = 0.f;
  uint32_t restart = 1;
  PHASE(slot, 6);
  for (int j = 0; j < jmax; ++j) {
    // w = G q_j, then w <- w - Q_j Q_j^T w twice: alpha_j is the q_j
    // coefficient of the two passes, beta_j = ||w|| (full reorthogonalisation)
    symv_rows<NT, NMAX>(Gs, n, Q + (size_t)j * ldq, z.w);
    PHASE(slot, 7);
    float b = sqrtf(lz_project<NT, NMAX>(z.w, Q, ldq, n, j + 1, z.h, z.h + kLzMaxJ, s.red));
    const float a = z.h[j] + z.h[kLzMaxJ + j];
    PHASE(slot, 9);
    if (tid == 0) {
      z.alpha[j] = a;
      z.beta[j] = b;
    }
    J = j + 1;
    if (J == n) break;  // Q spans everything: T_J is similar to G
    if (J < jmax) {
      if (!(b > 1e-5f * gbound)) {
        // breakdown: an invariant subspace was found; continue from a random
        // direction orthogonal to it
        for (int e = tid; e < n; e += NT) z.w[e] = lz_hash(seed + 7919u * restart, e);
        ++restart;
        __syncthreads();
        const float bn = sqrtf(lz_project<NT, NMAX>(z.w, Q, ldq, n, j + 1, z.h, z.h + kLzMaxJ, s.red));
        if (!(bn > 0.f)) break;
        if (tid == 0) z.beta[j] = 0.f;
        b = bn;
      }
      const float ib = 1.f / b;
      for (int e = tid; e < n; e += NT) Q[(size_t)(j + 1) * ldq + e] = z.w[e] * ib;
      __syncthreads();
    }
    PHASE(slot, 10);
    if (J >= jmin && ((J - jmin) % 4 == 0 || J == jmax)) {
      // converged when every kept Ritz pair has |beta_J * y_{J-1}| small
      k = lz_ritz<NT>(J, thr_keep, s, z, &tn);
      PHASE(slot, 11);
      if (k > kLzMaxK) {
      if (J_out) *J_out = J;
      return -1;
    }
      bool conv = true;
      const float bJ = z.beta[J - 1];
      for (int q = 0; q < k; ++q)
        if (fabsf(bJ * z.ty[(J - 1) * kLzMaxK + q]) > 1e-5f * fmaxf(s.lam[0], thr)) conv = false;
      if (conv) break;
      k = -1;
    }
  }
  if (k < 0) {
    k = lz_ritz<NT>(J, thr_keep, s, z, &tn);
    if (k > kLzMaxK) {
      if (J_out) *J_out = J;
      return -1;
    }
  }
  const int ku = k;
  // U = Q_J Y (n x ku) into the caller's U and, row-major n x 8 with zero
  // columns beyond ku, into X8 (shared; Q may alias the panel, so the values
  // wait in registers for the barrier)
  static_assert(8 * NMAX <= 4 * NT, "staging split");
  float* X8 = panel + 16 * NMAX;
  float* Y8 = panel + 24 * NMAX;
  float uv[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = tid + i * NT, r = e >> 3, q = e & 7;
    float v = 0.f;
    if (r < n && q < ku)
      for (int jj = 0; jj < J; ++jj) v = fmaf(Q[jj * ldq + r], z.ty[jj * kLzMaxK + q], v);
    uv[i] = v;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = tid + i * NT, r = e >> 3, q = e & 7;
    if (r < n) {
      X8[e] = uv[i];
      if (q < ku) U[(size_t)q * n + r] = uv[i];
    }
  }
  __syncthreads();
  PHASE(slot, 12);
  // W = G U (all columns in one pass over G), B = U^T W, rho
  symm_rows8<NT, NMAX>(Gs, n, X8, Y8);
  for (int pr = warp; pr < ku; pr += NW) {
    float d[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q] = 0.f;
    for (int r = lane; r < n; r += 32) {
      const float x = X8[r * 8 + pr];
      const float4 y0 = *reinterpret_cast<const float4*>(Y8 + r * 8);
      const float4 y1 = *reinterpret_cast<const float4*>(Y8 + r * 8 + 4);
      d[0] = fmaf(x, y0.x, d[0]);
      d[1] = fmaf(x, y0.y, d[1]);
      d[2] = fmaf(x, y0.z, d[2]);
      d[3] = fmaf(x, y0.w, d[3]);
      d[4] = fmaf(x, y1.x, d[4]);
      d[5] = fmaf(x, y1.y, d[5]);
      d[6] = fmaf(x, y1.z, d[6]);
      d[7] = fmaf(x, y1.w, d[7]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float t = warp_sum(d[q]);
      if (lane == 0 && q < ku) z.Bm[pr * kLzMaxK + q] = t;
    }
  }
  __syncthreads();
  part = 0.f;
  for (int e = tid; e < 8 * n; e += NT) {
    const int q = e & 7;
    if (q < ku) {
      const float rr = Y8[e] - z.Bm[q * kLzMaxK + q] * X8[e];
      part = fmaf(rr, rr, part);
    }
  }
  const float rho = sqrtf(block_sum<NT>(part, s.red));
  PHASE(slot, 13);
  // kept pairs: Rayleigh quotients, count above thr; pairs above thr first
  int kk = 0;
  for (int q = 0; q < ku; ++q) {
    const float th = z.Bm[q * kLzMaxK + q];
    kk += th > thr;
    if (q > 0 && th > thr && !(z.Bm[(q - 1) * kLzMaxK + (q - 1)] > thr)) {
      if (J_out) *J_out = J;
      return -1;
    }
  }
  const float c0 = thr - 2.f * rho - 8.f * (float)(ku + 1) * FLT_EPSILON * gbound;
  if (!(c0 > 0.f)) {
      if (J_out) *J_out = J;
      return -1;
    }
  __syncthreads();
  if (tid < ku) s.lam[tid] = z.Bm[tid * kLzMaxK + tid];
  // P G P = G - U What^T - What U^T with What = W - U sym(B) / 2, staged in
  // shared memory for the register Cholesky of (c I - P G P)
  const int n8 = (n + 7) & ~7;
  float* U8 = panel;
  float* W8 = panel + 8 * n8;
  for (int e = tid; e < ku * n8; e += NT) {
    const int q = e / n8, r = e - q * n8;
    float u = 0.f, w = 0.f;
    if (r < n) {
      u = X8[r * 8 + q];
      w = Y8[r * 8 + q];
      for (int p = 0; p < ku; ++p)
        w = fmaf(-0.25f * (z.Bm[p * kLzMaxK + q] + z.Bm[q * kLzMaxK + p]), X8[r * 8 + p], w);
    }
    U8[e] = u;
    W8[e] = w;
  }
  __syncthreads();
  PHASE(slot, 11);
  *ku_out = ku;
  *c0_out = c0;
  if (J_out) *J_out = J;
  return kk;
}

}  // namespace msllr
