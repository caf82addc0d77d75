// CTA-cooperative symmetric eigen-solver used by the block SVT (eq:svt).
//
// SVT_tau(C) = C V diag(f) V^T with f_j = max(1 - tau / sqrt(lambda_j), 0),
// where (lambda_j, v_j) are the eigenpairs of the Gram matrix G = C^T C.
// Only eigenpairs with lambda_j > tau^2 contribute, so the solver
//   1. reduces G to a symmetric tridiagonal T = Q^T G Q by Householder
//      reflections (lower storage, full or packed),
//   2. counts the eigenvalues above tau^2 exactly by a Sturm sequence on T
//      (this count is the certified rank of the thresholded block: 0 means
//      the block's SVT is zero),
//   3. finds those k eigenvalues by parallel multisection on Sturm counts,
//   4. finds their eigenvectors by two steps of inverse iteration on T with
//      a pivoted tridiagonal LU (one thread per eigenvector), modified
//      Gram-Schmidt inside clusters of close eigenvalues,
//   5. maps them back through the reflections (v = Q y).
// The textbook steps are Golub & Van Loan, Matrix Computations, Sec. 8.3
// (tridiagonalisation), Sec. 8.4 (Sturm bisection), Sec. 8.2/7.6 (inverse
// iteration); written here from those definitions.
#pragma once

#include <float.h>

#include "common.cuh"

namespace msllr {

// Lower-triangle accessors: at(i, k) is valid for i >= k.
struct LowerFull {
  float* g;
  int ld;
  __device__ __forceinline__ float& at(int i, int k) const { return g[i * ld + k]; }
};
struct LowerPacked {
  float* g;
  __device__ __forceinline__ float& at(int i, int k) const { return g[((i * (i + 1)) >> 1) + k]; }
};

// Shared-memory scratch of the solver.  Arrays marked [n] hold NMAX floats,
// those marked [NT] hold NT entries.
struct EigScratch {
  float* d;     // [n] diagonal of T
  float* e;     // [n] sub-diagonal of T
  float* e2;    // [n] e^2
  float* beta;  // [n] Householder scalars
  float* vbuf;  // [n]
  float* pbuf;  // [n]
  float* lam;   // [n] eigenvalues above the threshold, descending
  float* shf;   // [n] inverse-iteration shifts (lam, separated)
  int* clus;    // [n] first index of each eigenvalue's cluster
  float* lo;    // [NT]
  float* hi;    // [NT]
  float* xs;    // [NT]
  int* cnt;     // [NT]
  float* red;   // [64]
};

// ---------------------------------------------------------------------------
// 1. Householder tridiagonalisation of the symmetric matrix in the lower
// triangle of G (n x n).  On exit d/e hold T, beta[j] and column j of G
// (rows j+1..n-1) hold the reflection H_j = I - beta_j v_j v_j^T, and
// G = H_0 ... H_{n-3} T H_{n-3} ... H_0.
// ---------------------------------------------------------------------------
template <int NT, class S>
__device__ void tridiagonalize(S G, int n, EigScratch& s) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // Entries of a column below max(FLT_MIN, 2^-40 max_i |G_ii|) are treated as
  // already zero: dropping them perturbs G far below FP32 rounding, and their
  // reciprocal would overflow (denormal residues).
  float gdiag = 0.f;
  for (int i = tid; i < n; i += NT) gdiag = fmaxf(gdiag, fabsf(G.at(i, i)));
  gdiag = block_max<NT>(gdiag, s.red);
  if constexpr (NT == 32) __syncwarp();
  const float negligible = fmaxf(FLT_MIN, gdiag * 9.094947e-13f);
  for (int j = 0; j < n - 2; ++j) {
    const int len = n - j - 1;
    // The reflector is scale invariant, so the column is scaled by its
    // largest magnitude first: this keeps |x|^2 away from underflow (denormal
    // residues) and overflow.
    float amax = 0.f;
    for (int i = tid; i < len; i += NT) {
      const float x = G.at(j + 1 + i, j);
      s.vbuf[i] = x;
      amax = fmaxf(amax, fabsf(x));
    }
    amax = block_max<NT>(amax, s.red);
    if constexpr (NT == 32) __syncwarp();
    const float inv = amax > negligible ? 1.f / amax : 0.f;
    float part = 0.f;
    for (int i = tid + 1; i < len; i += NT) {
      const float x = s.vbuf[i] * inv;
      part = fmaf(x, x, part);
    }
    const float sigma = block_sum<NT>(part, s.red);
    if constexpr (NT == 32) __syncwarp();
    const float x0 = s.vbuf[0];
    const float dj = G.at(j, j);
    if (sigma == 0.f) {
      // the column is already a multiple of e_1 (to working precision)
      __syncthreads();
      if (tid == 0) {
        s.d[j] = dj;
        s.e[j] = x0;
        s.beta[j] = 0.f;
      }
      __syncthreads();
      continue;
    }
    const float x0s = x0 * inv;
    const float xnorm = sqrtf(x0s * x0s + sigma);
    const float alpha = (x0s >= 0.f) ? -xnorm : xnorm;
    const float v0 = x0s - alpha;
    const float b = 2.f / (v0 * v0 + sigma);
    __syncthreads();
    // scaled reflector v = (x / amax) - alpha e_1, H = I - b v v^T
    for (int i = tid + 1; i < len; i += NT) {
      const float x = s.vbuf[i] * inv;
      s.vbuf[i] = x;
      G.at(j + 1 + i, j) = x;
    }
    if (tid == 0) {
      s.vbuf[0] = v0;
      G.at(j + 1, j) = v0;
      s.d[j] = dj;
      s.e[j] = alpha * amax;
      s.beta[j] = b;
    }
    __syncthreads();
    // p = b * A v on the trailing block A = G[j+1:, j+1:]: one thread per
    // row when the block is narrow enough, else one warp per row
    if (len <= NT) {
      const int r = tid;
      if (r < len) {
        const int R = j + 1 + r;
        float a0 = 0.f, a1 = 0.f;
        int c = 0;
        for (; c + 1 <= r; c += 2) {
          a0 = fmaf(G.at(R, j + 1 + c), s.vbuf[c], a0);
          a1 = fmaf(G.at(R, j + 2 + c), s.vbuf[c + 1], a1);
        }
        for (; c < len; ++c) {
          const int Cc = j + 1 + c;
          a0 = fmaf(c <= r ? G.at(R, Cc) : G.at(Cc, R), s.vbuf[c], a0);
        }
        s.pbuf[r] = b * (a0 + a1);
      }
    } else {
      for (int r = warp; r < len; r += NW) {
        const int R = j + 1 + r;
        float acc = 0.f;
        for (int c = lane; c < len; c += 32) {
          const int Cc = j + 1 + c;
          const float a = (c <= r) ? G.at(R, Cc) : G.at(Cc, R);
          acc = fmaf(a, s.vbuf[c], acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) s.pbuf[r] = b * acc;
      }
    }
    __syncthreads();
    float kp = 0.f;
    for (int i = tid; i < len; i += NT) kp = fmaf(s.vbuf[i], s.pbuf[i], kp);
    const float K = 0.5f * b * block_sum<NT>(kp, s.red);
    if constexpr (NT == 32) __syncwarp();
    for (int i = tid; i < len; i += NT) s.pbuf[i] = fmaf(-K, s.vbuf[i], s.pbuf[i]);
    __syncthreads();
    // A <- A - v w^T - w v^T (lower triangle)
    if (len <= NT) {
      const int r = tid;
      if (r < len) {
        const int R = j + 1 + r;
        const float vr = s.vbuf[r], wr = s.pbuf[r];
        for (int c = 0; c <= r; ++c) {
          float& g = G.at(R, j + 1 + c);
          g = g - vr * s.pbuf[c] - wr * s.vbuf[c];
        }
      }
    } else {
      for (int r = warp; r < len; r += NW) {
        const int R = j + 1 + r;
        const float vr = s.vbuf[r], wr = s.pbuf[r];
        for (int c = lane; c <= r; c += 32) {
          float& g = G.at(R, j + 1 + c);
          g = g - vr * s.pbuf[c] - wr * s.vbuf[c];
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      s.d[n - 2] = G.at(n - 2, n - 2);
      s.d[n - 1] = G.at(n - 1, n - 1);
      s.e[n - 2] = G.at(n - 1, n - 2);
    } else if (n == 1) {
      s.d[0] = G.at(0, 0);
    }
  }
  __syncthreads();
}

// Number of eigenvalues of T (d, e2 = e^2) strictly below x (Sturm count via
// the LDL^T pivots of T - xI; tiny pivots are replaced by -pivmin).
__device__ __forceinline__ int sturm_below(const float* d, const float* e2, int n, float x,
                                           float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int c = q < 0.f;
  for (int i = 1; i < n; ++i) {
    // approximate division: a few-ulp error per pivot only perturbs T by a
    // few ulps, within the backward error the Sturm count tolerates
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// ---------------------------------------------------------------------------
// 2-3. Certified count k of eigenvalues of T above `thr` and their values
// (descending) by multisection.  Requires n <= NT.  Returns k; also returns
// the infinity norm of T in *tnorm.
// ---------------------------------------------------------------------------
template <int NT>
__device__ int top_eigenvalues(int n, float thr, EigScratch& s, float* tnorm) {
  const int tid = threadIdx.x;
  float gup = -FLT_MAX, tn = 0.f, e2m = 0.f;
  for (int i = tid; i < n; i += NT) {
    const float ea = (i < n - 1) ? fabsf(s.e[i]) : 0.f;
    const float eb = (i > 0) ? fabsf(s.e[i - 1]) : 0.f;
    if (i < n - 1) s.e2[i] = s.e[i] * s.e[i];
    gup = fmaxf(gup, s.d[i] + ea + eb);
    tn = fmaxf(tn, fabsf(s.d[i]) + ea + eb);
    e2m = fmaxf(e2m, ea * ea);
  }
  gup = block_max<NT>(gup, s.red);
  tn = block_max<NT>(tn, s.red);
  e2m = block_max<NT>(e2m, s.red);
  if constexpr (NT == 32) __syncwarp();
  *tnorm = tn;
  const float pivmin = FLT_MIN * fmaxf(1.f, e2m);
  const int k = n - sturm_below(s.d, s.e2, n, thr, pivmin);
  if (k <= 0) return 0;
  const float top = gup + 4.f * FLT_EPSILON * fmaxf(fabsf(gup), tn) + pivmin;
  if (tid < k) {
    s.lo[tid] = thr;
    s.hi[tid] = top;
  }
  __syncthreads();
  // one warp (32 points per round) per target when there are enough warps,
  // otherwise NT / k threads per target with a serial scan by the leader
  const int g = (NT / k >= 32) ? 32 : NT / k;
  const int q = tid / g, mb = tid - q * g;
  const int target = n - 1 - q;  // ascending index of the eigenvalue sought
  const float tol = 2.f * FLT_EPSILON * tn;
  for (int round = 0; round < 64; ++round) {
    bool active = false;
    float x = 0.f;
    int cntx = 0;
    if (q < k) {
      const float lo = s.lo[q], hi = s.hi[q];
      if (hi - lo > fmaxf(tol, 2.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)))) {
        active = true;
        x = lo + (hi - lo) * ((float)(mb + 1) / (float)(g + 1));
        cntx = sturm_below(s.d, s.e2, n, x, pivmin);
        if (g < 32) {
          s.xs[tid] = x;
          s.cnt[tid] = cntx;
        }
      }
    }
    if (!__syncthreads_or(active)) break;
    if (g == 32) {
      if (q < k) {
        // counts grow with x: the first point above the target brackets it
        const unsigned above = __ballot_sync(0xffffffffu, active && cntx > target);
        const float lo = s.lo[q], hi = s.hi[q];
        if (active) {
          float nlo = lo, nhi = hi;
          if (above == 0u) {
            nlo = __shfl_sync(0xffffffffu, x, 31);
          } else {
            const int f = __ffs(above) - 1;
            nhi = __shfl_sync(0xffffffffu, x, f);
            if (f > 0) nlo = __shfl_sync(0xffffffffu, x, f - 1);
          }
          if (nlo > nhi) nlo = nhi;
          __syncwarp();
          if (mb == 0) {
            s.lo[q] = nlo;
            s.hi[q] = nhi;
          }
        }
      }
    } else if (active && mb == 0) {
      float lo = s.lo[q], hi = s.hi[q];
      for (int j = 0; j < g; ++j) {
        const float xj = s.xs[tid + j];
        if (s.cnt[tid + j] <= target) lo = fmaxf(lo, xj);
        else hi = fminf(hi, xj);
      }
      if (lo > hi) lo = hi;
      s.lo[q] = lo;
      s.hi[q] = hi;
    }
    __syncthreads();
  }
  if (tid < k) s.lam[tid] = 0.5f * (s.lo[tid] + s.hi[tid]);
  __syncthreads();
  if (tid == 0) {
    // inverse-iteration shifts kept apart, clusters of close eigenvalues
    const float pertol = 10.f * FLT_EPSILON * tn;
    const float ortol = 1e-3f * tn;
    s.shf[0] = s.lam[0];
    s.clus[0] = 0;
    for (int j = 1; j < k; ++j) {
      s.shf[j] = fminf(s.lam[j], s.shf[j - 1] - pertol);
      s.clus[j] = (s.lam[j - 1] - s.lam[j] <= ortol) ? s.clus[j - 1] : j;
    }
  }
  __syncthreads();
  return k;
}

// Pivoted LU of the tridiagonal T - shift I (thread-local), the LAPACK
// gttrf elimination order: row interchange when the sub-diagonal entry is
// larger than the pivot.  Tiny pivots are replaced by +-tiny.
template <int NMAX>
struct TriLU {
  float dd[NMAX], du[NMAX], du2[NMAX], dl[NMAX];
  uint32_t piv[(NMAX + 31) / 32];

  __device__ void factor(const float* d, const float* e, int n, float shift, float tiny) {
    for (int i = 0; i < n; ++i) dd[i] = d[i] - shift;
    for (int i = 0; i < (NMAX + 31) / 32; ++i) piv[i] = 0u;
    for (int i = 0; i < n - 1; ++i) {
      du[i] = e[i];
      dl[i] = e[i];
      du2[i] = 0.f;
    }
    for (int i = 0; i < n - 1; ++i) {
      if (fabsf(dd[i]) >= fabsf(dl[i])) {
        if (dd[i] == 0.f) dd[i] = tiny;
        const float f = dl[i] / dd[i];
        dl[i] = f;
        dd[i + 1] -= f * du[i];
      } else {
        const float f = dd[i] / dl[i];
        dd[i] = dl[i];
        dl[i] = f;
        const float t = du[i];
        du[i] = dd[i + 1];
        dd[i + 1] = t - f * dd[i + 1];
        if (i < n - 2) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du[i + 1];
        }
        piv[i >> 5] |= 1u << (i & 31);
      }
    }
    for (int i = 0; i < n; ++i)
      if (fabsf(dd[i]) < tiny) dd[i] = dd[i] < 0.f ? -tiny : tiny;
  }

  // Solve (T - shift I) x = y in place; y[i] lives at y[i * ldy].
  __device__ void solve(float* y, int ldy, int n) const {
    for (int i = 0; i < n - 1; ++i) {
      const float a = y[i * ldy], b = y[(i + 1) * ldy];
      if (piv[i >> 5] & (1u << (i & 31))) {
        y[i * ldy] = b;
        y[(i + 1) * ldy] = a - dl[i] * b;
      } else {
        y[(i + 1) * ldy] = b - dl[i] * a;
      }
    }
    y[(n - 1) * ldy] /= dd[n - 1];
    if (n > 1) y[(n - 2) * ldy] = (y[(n - 2) * ldy] - du[n - 2] * y[(n - 1) * ldy]) / dd[n - 2];
    for (int i = n - 3; i >= 0; --i)
      y[i * ldy] = (y[i * ldy] - du[i] * y[(i + 1) * ldy] - du2[i] * y[(i + 2) * ldy]) / dd[i];
  }
};

__device__ __forceinline__ void normalize_column(float* y, int ldy, int n) {
  float ss = 0.f;
  for (int i = 0; i < n; ++i) ss = fmaf(y[i * ldy], y[i * ldy], ss);
  const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
  for (int i = 0; i < n; ++i) y[i * ldy] *= inv;
}

// Modified Gram-Schmidt of the columns of Y (n x k, row stride ldy) inside
// each cluster; thread t owns rows t, t+NT, ... so no extra barriers needed.
template <int NT>
__device__ void cluster_mgs(float* Y, int ldy, int n, int k, const int* clus, float* red) {
  const int tid = threadIdx.x;
  for (int q = 0; q < k; ++q) {
    const int c0 = clus[q];
    if (c0 == q) continue;
    for (int i = c0; i < q; ++i) {
      float part = 0.f;
      for (int r = tid; r < n; r += NT) part = fmaf(Y[r * ldy + i], Y[r * ldy + q], part);
      const float dot = block_sum<NT>(part, red);
      for (int r = tid; r < n; r += NT) Y[r * ldy + q] = fmaf(-dot, Y[r * ldy + i], Y[r * ldy + q]);
    }
    float part = 0.f;
    for (int r = tid; r < n; r += NT) part = fmaf(Y[r * ldy + q], Y[r * ldy + q], part);
    const float nrm2 = block_sum<NT>(part, red);
    const float inv = nrm2 > 0.f ? rsqrtf(nrm2) : 0.f;
    for (int r = tid; r < n; r += NT) Y[r * ldy + q] *= inv;
  }
}

// ---------------------------------------------------------------------------
// 4-5. Eigenvectors of G for the k eigenvalues found by top_eigenvalues:
// columns 0..k-1 of Y (n x k, row stride ldy) receive orthonormal v_j.
// ---------------------------------------------------------------------------
template <int NT, int NMAX, class S>
__device__ void top_eigenvectors(S G, int n, int k, float tnorm, EigScratch& s, float* Y,
                                 int ldy, int slot = 0) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  PHASE_INIT();
  constexpr int NW = NT / 32;
  TriLU<NMAX> lu;
  const float tiny = FLT_EPSILON * tnorm;
  if (tid < k) {
    lu.factor(s.d, s.e, n, s.shf[tid], tiny);
    // deterministic pseudo-random start vector of size ~eps*|T|
    uint32_t h = 0x9E3779B9u * (uint32_t)(tid + 1);
    for (int i = 0; i < n; ++i) {
      h ^= h << 13;
      h ^= h >> 17;
      h ^= h << 5;
      Y[i * ldy + tid] = tiny * ((float)(h >> 8) * (2.f / 16777216.f) - 1.f + 1e-3f);
    }
    lu.solve(Y + tid, ldy, n);
    normalize_column(Y + tid, ldy, n);
  }
  __syncthreads();
  PHASE(slot, 8);
  cluster_mgs<NT>(Y, ldy, n, k, s.clus, s.red);
  __syncthreads();
  PHASE(slot, 9);
  if (tid < k) {
    for (int i = 0; i < n; ++i) Y[i * ldy + tid] *= tiny;
    lu.solve(Y + tid, ldy, n);
    normalize_column(Y + tid, ldy, n);
  }
  __syncthreads();
  PHASE(slot, 10);
  cluster_mgs<NT>(Y, ldy, n, k, s.clus, s.red);
  __syncthreads();
  PHASE(slot, 11);
  // back-transform v = H_0 (H_1 (... H_{n-3} y)), one warp per vector
  for (int q = warp; q < k; q += NW) {
    for (int j = n - 3; j >= 0; --j) {
      const float b = s.beta[j];
      if (b == 0.f) continue;
      float dot = 0.f;
      for (int i = j + 1 + lane; i < n; i += 32) dot = fmaf(G.at(i, j), Y[i * ldy + q], dot);
      dot = warp_sum(dot) * b;
      for (int i = j + 1 + lane; i < n; i += 32) Y[i * ldy + q] = fmaf(-dot, G.at(i, j), Y[i * ldy + q]);
      __syncwarp();
    }
  }
  __syncthreads();
  PHASE(slot, 12);
}

}  // namespace msllr
