// Block SVT (eq:svt, eq:bsvt) for blocks wider than 256 (256 < min(m, n) <=
// MSLLR_MAX_BLOCK_WIDTH), e.g. the full-matrix scale of a 1024 x 1024 job or
// the 1024 x 1024 blocks of an 8192 x 8192 one.  A block of that width does
// not fit one CTA, so every phase is spread over many CTAs and the blocks of
// a scale go through each launch together:
//   1. Gram: G_b = C_b^T C_b, 64x64 tiles of the lower triangle split over
//      row chunks; the partial sums are added in a fixed order and G_b is
//      stored as a full square (both triangles);
//   2. subspace iteration on G_b with a basis of kP = 32 columns kept from
//      the previous call (warm start): W = G V over row tiles, then one CTA
//      per block orthonormalises W + mu V by shifted CholQR followed by two
//      plain CholQR passes (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa,
//      SIAM J. Sci. Comput. 2020);
//   3. Rayleigh-Ritz on V^T G V (32 x 32, the tridiagonal solver of
//      symeig.cuh) for the pairs above tau^2, their residuals and a
//      convergence test; unconverged blocks get further rounds of steps;
//   4. certificate: lambda_max(P G P) < tau^2 with P = I - U U^T over the
//      kept Ritz vectors, proved by a tiled Cholesky factorisation of
//      c I - P G P (Golub & Van Loan Sec. 4.2), a panel launch and a
//      trailing-update launch per 64 columns; by Cauchy interlacing G then
//      has no eigenvalue above tau^2 besides the kept ones;
//   5. rebuild: Z'_b = (C_b V_f) V_f^T with V_f = U diag(sqrt(1 - tau/sigma))
//      over the pairs above tau, scattered through Shift_{-s}, with the fused
//      dual update W' = 2 Z' - A of eq:admm.
// A block whose certificate fails keeps its Ritz pairs and is counted.
#include <float.h>
#include <math.h>

#include "../../include/msllr.h"
#include "common.cuh"
#include "internal.h"
#include "symeig.cuh"

namespace msllr {

namespace {

constexpr int kHT = 64;          // Gram and Cholesky tile
constexpr int kHP = 32;          // subspace width
constexpr int kHK = 16;          // most Ritz pairs kept per block
constexpr int kHThreads = 256;   // tile kernels
constexpr int kHBlockThreads = 512;  // per-block kernels
constexpr int kHGvRows = 8;      // rows of W per CTA in W = G V

// per-block state of the wide path
struct HugeBlock {
  float trace;   // trace(G) (>= lambda_max)
  float gF;      // ||G||_F
  float c;       // certificate shift (valid when status == kHsCert)
  float theta[kHK];
  int status;    // kHs*
  int ku;        // kept Ritz pairs
  int k;         // pairs above tau
  int conv;      // Rayleigh-Ritz residual test passed
  int chol_fail; // the tiled Cholesky met a non-positive pivot
  int orth_fail; // a CholQR factorisation broke down (basis restarted)
};
enum : int { kHsSkip = 1, kHsIter = 2, kHsCert = 3, kHsNoCert = 4 };

struct HugeDims {
  int mm, nn, nblocks, T, ntiles, chunk_rows, chunks;
};

HugeDims huge_dims(int M, int N, int m, int n) {
  HugeDims d;
  d.mm = m >= n ? m : n;
  d.nn = m >= n ? n : m;
  d.nblocks = (M / m) * (N / n);
  d.T = (d.nn + kHT - 1) / kHT;
  d.ntiles = d.T * (d.T + 1) / 2;
  // row chunks: enough CTAs for two waves of 5 per SM, chunks of >= 256 rows
  d.chunk_rows = 256;
  const long long waves = 10LL * sm_count();
  while (d.chunk_rows < d.mm &&
         (long long)d.ntiles * d.nblocks * ((d.mm + 2 * d.chunk_rows - 1) / (2 * d.chunk_rows)) >= waves)
    d.chunk_rows *= 2;
  d.chunks = (d.mm + d.chunk_rows - 1) / d.chunk_rows;
  return d;
}


__device__ __forceinline__ size_t huge_off(const BlockGeom& g, int i, int c) {
  return g.transposed() ? g.offset(c, i) : g.offset(i, c);
}

__device__ __forceinline__ float huge_load(const ScaleLaunch& a, size_t off) {
  float v = a.A1[off];
  if (a.A2) v += a.A2[off];
  return v;
}

__device__ __forceinline__ void tile_of(int t, int* ta, int* tc) {
  int i = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
  while (((i + 1) * (i + 2)) / 2 <= t) ++i;
  while ((i * (i + 1)) / 2 > t) --i;
  *ta = i;
  *tc = t - (i * (i + 1)) / 2;
}

// deterministic pseudo-random value in [-1, 1)
__device__ __forceinline__ float huge_hash(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (float)(h >> 8) * (2.f / 16777216.f) - 1.f;
}

// ---------------------------------------------------------------------------
// 1. Gram partial sums: tile t of the lower triangle over one row chunk.
// ---------------------------------------------------------------------------
template <bool ST>
__global__ void __launch_bounds__(kHThreads, 4)
huge_gram_kernel(ScaleLaunch a, float* __restrict__ part, int chunk_rows, int chunks,
                 const HugeBlock* __restrict__ hb) {
  __shared__ __align__(16) float As[32][kHT + 4];
  __shared__ __align__(16) float Bs[32][kHT + 4];
  const int t = blockIdx.x, chunk = blockIdx.y, b = blockIdx.z;
  (void)hb;
  int ta, tc;
  tile_of(t, &ta, &tc);
  const BlockGeom g = block_geom_t<ST>(a, b);
  const int mm = g.mm(), nn = g.nn();
  const int a0 = ta * kHT, c0 = tc * kHT;
  const int r_begin = chunk * chunk_rows;
  const int r_end = min(mm, r_begin + chunk_rows);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
  for (int r0 = r_begin; r0 < r_end; r0 += 32) {
#pragma unroll
    for (int j = 0; j < (32 * kHT) / kHThreads; ++j) {
      const int e = tid + j * kHThreads;
      const int rr = e / kHT, cc = e - rr * kHT;
      const int i = r0 + rr;
      float va = 0.f, vb = 0.f;
      if (i < r_end) {
        if (a0 + cc < nn) va = huge_load(a, huge_off(g, i, a0 + cc));
        if (c0 + cc < nn) vb = (ta == tc) ? va : huge_load(a, huge_off(g, i, c0 + cc));
      }
      As[rr][cc] = va;
      Bs[rr][cc] = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[rr][ty * 4]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[rr][tx * 4]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
    }
    __syncthreads();
  }
  const int ntiles = gridDim.x;
  float* dst = part + (((size_t)b * chunks + chunk) * ntiles + t) * (kHT * kHT);
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) dst[(ty * 4 + x) * kHT + tx * 4 + y] = acc[x][y];
}

// Sum of the chunk partials in chunk order; G_b written as a full square,
// and per tile: the diagonal sum and the sum of squares (off-diagonal tiles
// twice), for trace(G) and ||G||_F.
__global__ void __launch_bounds__(kHThreads)
huge_gram_finish_kernel(const float* __restrict__ part, float* __restrict__ G,
                        float* __restrict__ tstat, int nn, int chunks) {
  __shared__ float red[2][kHThreads / 32];
  const int t = blockIdx.x, b = blockIdx.y, ntiles = gridDim.x;
  int ta, tc;
  tile_of(t, &ta, &tc);
  const int tid = threadIdx.x;
  float* Gb = G + (size_t)b * nn * nn;
  float dsum = 0.f, sq = 0.f;
  for (int e = tid; e < kHT * kHT; e += kHThreads) {
    const int x = e / kHT, y = e - x * kHT;
    const int i = ta * kHT + x, j = tc * kHT + y;
    float s = 0.f;
    for (int c = 0; c < chunks; ++c)
      s += part[(((size_t)b * chunks + c) * ntiles + t) * (kHT * kHT) + e];
    if (i >= nn || j >= nn) continue;
    if (ta == tc) {
      // diagonal tile: the lower half is authoritative
      if (j <= i) {
        Gb[(size_t)i * nn + j] = s;
        Gb[(size_t)j * nn + i] = s;
        sq += (i == j ? 1.f : 2.f) * s * s;
        if (i == j) dsum += s;
      }
    } else {
      Gb[(size_t)i * nn + j] = s;
      Gb[(size_t)j * nn + i] = s;
      sq += 2.f * s * s;
    }
  }
  dsum = warp_sum(dsum);
  sq = warp_sum(sq);
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = dsum;
    red[1][tid >> 5] = sq;
  }
  __syncthreads();
  if (tid == 0) {
    float d = 0.f, q = 0.f;
    for (int w = 0; w < kHThreads / 32; ++w) {
      d += red[0][w];
      q += red[1][w];
    }
    tstat[((size_t)b * ntiles + t) * 2] = d;
    tstat[((size_t)b * ntiles + t) * 2 + 1] = q;
  }
}


// Per block: trace(G) and ||G||_F from the tile sums (fixed order), the
// zero-rank shortcut trace(G) <= tau^2 (trace bounds lambda_max), state reset.
__global__ void __launch_bounds__(kHThreads)
huge_prep_kernel(const float* __restrict__ tstat, int ntiles, HugeBlock* __restrict__ hb,
                 float thr) {
  __shared__ double red[2][kHThreads / 32];
  const int b = blockIdx.x, tid = threadIdx.x;
  double d = 0.0, q = 0.0;
  for (int t = tid; t < ntiles; t += kHThreads) {
    d += (double)tstat[((size_t)b * ntiles + t) * 2];
    q += (double)tstat[((size_t)b * ntiles + t) * 2 + 1];
  }
  d = warp_sum_d(d);
  q = warp_sum_d(q);
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = d;
    red[1][tid >> 5] = q;
  }
  __syncthreads();
  if (tid == 0) {
    double dt = 0.0, qt = 0.0;
    for (int w = 0; w < kHThreads / 32; ++w) {
      dt += red[0][w];
      qt += red[1][w];
    }
    HugeBlock& h = hb[b];
    h.trace = (float)dt;
    h.gF = (float)sqrt(qt);
    h.status = (h.trace <= thr) ? kHsSkip : kHsIter;
    h.ku = 0;
    h.k = 0;
    h.conv = 0;
    h.chol_fail = 0;
    h.orth_fail = 0;
    h.c = 0.f;
  }
}

// Start basis: deterministic pseudo-random columns (any full-rank start
// serves subspace iteration), the same for every block (rows r of a block
// at V + (b nn + r) kHP), so that a block's start does not depend on its
// index.
__global__ void huge_init_basis_kernel(float* __restrict__ V, size_t total, int nn) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    V[e] = huge_hash((uint32_t)((e / kHP) % nn), (uint32_t)(e % kHP) + 0x51EDu);
}

__device__ __forceinline__ bool huge_active(const HugeBlock& h) {
  return h.status == kHsIter && !h.conv && !h.orth_fail;
}

// ---------------------------------------------------------------------------
// 2. W = G V for kHGvRows rows of one block (V, W: nn x kHP row-major): one
// output per thread, the K loop in chunks of 64 through shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kHThreads)
huge_gv_kernel(const float* __restrict__ G, const float* __restrict__ V, float* __restrict__ W,
               int nn, const HugeBlock* __restrict__ hb) {
  constexpr int KC = 64;
  static_assert(kHGvRows * kHP == kHThreads, "one output per thread");
  __shared__ float Gs[kHGvRows][KC + 1];
  __shared__ float Vs[KC][kHP];
  const int b = blockIdx.y;
  if (!huge_active(hb[b])) return;
  const int r0 = blockIdx.x * kHGvRows, tid = threadIdx.x;
  const int row = tid / kHP, col = tid % kHP;
  const float* Gb = G + (size_t)b * nn * nn;
  const float* Vb = V + (size_t)b * nn * kHP;
  float acc = 0.f;
  for (int l0 = 0; l0 < nn; l0 += KC) {
#pragma unroll
    for (int j = 0; j < (kHGvRows * KC) / kHThreads; ++j) {
      const int e = tid + j * kHThreads;
      const int rr = e / KC, cc = e % KC;
      const int gr = r0 + rr, gl = l0 + cc;
      Gs[rr][cc] = (gr < nn && gl < nn) ? Gb[(size_t)gr * nn + gl] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < (KC * kHP) / kHThreads; ++j) {
      const int e = tid + j * kHThreads;
      const int rr = e / kHP, cc = e % kHP;
      const int vl = l0 + rr;
      Vs[rr][cc] = (vl < nn) ? Vb[(size_t)vl * kHP + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 16
    for (int kk = 0; kk < KC; ++kk) acc = fmaf(Gs[row][kk], Vs[kk][col], acc);
    __syncthreads();
  }
  const int r = r0 + row;
  if (r < nn) W[(size_t)b * nn * kHP + (size_t)r * kHP + col] = acc;
}

// S = X^T Y over the nn rows of two nn x kHP row-major matrices (Y = X
// allowed), X optionally X + mu * X2.  Thread t owns entries (t/32, t%32) and
// (t/32 + 16, t%32); the row tiles pass through shared memory; the sums run
// in row order, so the result is deterministic and S(a,b) == S(b,a) when
// Y = X.  Result in Sm (kHP x (kHP+1)).  All kHBlockThreads threads call.
__device__ void huge_xty(const float* __restrict__ X, const float* __restrict__ X2, float mu,
                         const float* __restrict__ Yv, int nn, float* Xs, float* Ys, float* Sm) {
  const int tid = threadIdx.x;
  const int a0 = tid >> 5, bq = tid & 31, a1 = a0 + 16;
  float acc0 = 0.f, acc1 = 0.f;
  for (int r0 = 0; r0 < nn; r0 += 64) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = tid + j * kHBlockThreads;  // 64 x 32 tile
      const int rr = e >> 5, cc = e & 31;
      const int r = r0 + rr;
      float x = 0.f, y = 0.f;
      if (r < nn) {
        x = X[(size_t)r * kHP + cc];
        if (X2) x = fmaf(mu, X2[(size_t)r * kHP + cc], x);
        if (Yv) y = Yv[(size_t)r * kHP + cc];
      }
      Xs[rr * 33 + cc] = x;
      if (Yv) Ys[rr * 33 + cc] = y;
    }
    __syncthreads();
    const float* Yt = Yv ? Ys : Xs;
#pragma unroll 8
    for (int rr = 0; rr < 64; ++rr) {
      acc0 = fmaf(Xs[rr * 33 + a0], Yt[rr * 33 + bq], acc0);
      acc1 = fmaf(Xs[rr * 33 + a1], Yt[rr * 33 + bq], acc1);
    }
    __syncthreads();
  }
  Sm[a0 * 33 + bq] = acc0;
  Sm[a1 * 33 + bq] = acc1;
  __syncthreads();
}

// Warp 0: S + shift I = R^T R (R upper, in Rm), then Ri = R^{-1}.  Returns
// false (uniformly, after a barrier) on a non-positive or non-finite pivot.
__device__ bool huge_chol32(float* Sm, float shift, float* Rm, float* Ri, int* flag) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < 32) {
    if (lane == 0) *flag = 1;
    Sm[lane * 33 + lane] += shift;
    __syncwarp();
    bool ok = true;
    for (int j = 0; j < kHP; ++j) {
      const float d = Sm[j * 33 + j];
      if (!(d > 0.f) || !isfinite(d)) {
        ok = false;
        break;
      }
      const float r = sqrtf(d);
      const float v = lane > j ? Sm[j * 33 + lane] / r : (lane == j ? r : 0.f);
      Rm[j * 33 + lane] = v;
      __syncwarp();
      if (lane > j)
        for (int i = j + 1; i <= lane; ++i) Sm[i * 33 + lane] -= Rm[j * 33 + i] * v;
      __syncwarp();
    }
    if (!ok) {
      if (lane == 0) *flag = 0;
    } else {
      // column `lane` of R^{-1} by back substitution
      const int j = lane;
      for (int i = 0; i < kHP; ++i) Ri[i * 33 + j] = 0.f;
      Ri[j * 33 + j] = 1.f / Rm[j * 33 + j];
      for (int i = j - 1; i >= 0; --i) {
        float t = 0.f;
        for (int l = i + 1; l <= j; ++l) t = fmaf(Rm[i * 33 + l], Ri[l * 33 + j], t);
        Ri[i * 33 + j] = -t / Rm[i * 33 + i];
      }
    }
  }
  __syncthreads();
  const bool ok = *flag != 0;
  __syncthreads();
  return ok;
}

// Orthonormal basis of span(W + mu V) into V by shifted CholQR and two plain
// CholQR passes, spread over the rows: four sweeps, each a launch over
// (row chunk of kHOrthRows, block).  Sweep p (p >= 1) first sums the chunk
// partials of S from sweep p - 1 in chunk order and factors S (+ shift for
// p = 1) = R^T R in every CTA (all CTAs get the same R^{-1}); then each CTA
// maps its rows: sweep 0 X = W + mu V, sweep 1 X = (W + mu V) R^{-1},
// sweeps 2, 3 X = W R^{-1} (sweeps 1, 2 write W, sweep 3 writes V), and
// sweeps 0-2 write the partial S = X^T X of their rows.  mu = 1e-4 ||G||_F
// (a shift of G by mu I) keeps W + mu V of full rank when G is (numerically)
// of rank below kHP.  A failed factorisation marks the block (orth_fail) and
// restarts its basis.
constexpr int kHOrthRows = 32;
__global__ void __launch_bounds__(kHThreads)
huge_orth_sweep_kernel(float* __restrict__ V, float* __restrict__ W, const float* __restrict__ pin,
                       float* __restrict__ pout, int nn, int pass, HugeBlock* __restrict__ hb) {
  constexpr int NT = kHThreads, PER = kHOrthRows * kHP / NT;
  __shared__ float Xin[kHOrthRows * 33];
  __shared__ float Sm[kHP * 33];
  __shared__ float Rm[kHP * 33];
  __shared__ float Ri[kHP * 33];
  __shared__ int flag;
  const int chunk = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
  const int nchunks = gridDim.x;
  {
    const HugeBlock& h = hb[b];
    if (!huge_active(h)) return;
  }
  float* Vb = V + (size_t)b * nn * kHP;
  float* Wb = W + (size_t)b * nn * kHP;
  const int r0 = chunk * kHOrthRows;
  const float mu = 1e-4f * hb[b].gF;
  // this CTA's rows (loads in flight during the factorisation)
  float x[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int e = tid + j * NT;
    const int r = r0 + (e >> 5), cc = e & 31;
    float v = 0.f;
    if (r < nn) {
      v = Wb[(size_t)r * kHP + cc];
      if (pass <= 1) v = fmaf(mu, Vb[(size_t)r * kHP + cc], v);
    }
    x[j] = v;
  }
  bool ok = true;
  if (pass >= 1) {
    const float* pb = pin + (size_t)b * nchunks * (kHP * kHP);
    for (int e = tid; e < kHP * kHP; e += NT) {
      float t = 0.f;
      for (int c = 0; c < nchunks; ++c) t += pb[(size_t)c * (kHP * kHP) + e];
      Sm[(e >> 5) * 33 + (e & 31)] = t;
    }
    __syncthreads();
    float shift = 0.f;
    if (pass == 1) {
      float tr = 0.f;
      for (int i = 0; i < kHP; ++i) tr += Sm[i * 33 + i];
      shift = 11.f * (float)((double)nn * kHP + kHP * (kHP + 1)) * FLT_EPSILON * tr;
    }
    ok = huge_chol32(Sm, shift, Rm, Ri, &flag);
  }
  if (!ok) {
    for (int j = 0; j < PER; ++j) {
      const int e = tid + j * NT;
      const int r = r0 + (e >> 5), cc = e & 31;
      if (r < nn) Vb[(size_t)r * kHP + cc] = huge_hash((uint32_t)r + 977u * b, (uint32_t)cc + 0xB0Bu);
    }
    if (chunk == 0 && tid == 0) hb[b].orth_fail = 1;
    return;
  }
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int e = tid + j * NT;
    Xin[(e >> 5) * 33 + (e & 31)] = x[j];
  }
  __syncthreads();
  if (pass >= 1) {
    float o[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int e = tid + j * NT;
      const int rr = e >> 5, cc = e & 31;
      float t = 0.f;
#pragma unroll
      for (int a = 0; a < kHP; ++a)
        if (a <= cc) t = fmaf(Xin[rr * 33 + a], Ri[a * 33 + cc], t);
      o[j] = t;
    }
    __syncthreads();
    float* dst = pass == 3 ? Vb : Wb;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int e = tid + j * NT;
      const int rr = e >> 5, cc = e & 31;
      Xin[rr * 33 + cc] = o[j];
      if (r0 + rr < nn) dst[(size_t)(r0 + rr) * kHP + cc] = o[j];
    }
    __syncthreads();
  }
  if (pass <= 2) {
    // partial S of this chunk: thread t owns entries t, t + NT, ...
    float* pb = pout + ((size_t)b * nchunks + chunk) * (kHP * kHP);
#pragma unroll
    for (int j = 0; j < (kHP * kHP) / NT; ++j) {
      const int e = tid + j * NT;
      const int a = e >> 5, c = e & 31;
      float t = 0.f;
#pragma unroll 8
      for (int rr = 0; rr < kHOrthRows; ++rr) t = fmaf(Xin[rr * 33 + a], Xin[rr * 33 + c], t);
      pb[e] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// 3. Rayleigh-Ritz: T = V^T W (W = G V), its eigenpairs above thr_keep, the
// Ritz vectors U = V Q and G U = W Q (nn x kHK, row-major), B = U^T G U,
// residuals |G u_q - theta_q u_q| and What = G U - U sym(B) / 2 (over G U).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kHBlockThreads)
huge_rr_kernel(const float* __restrict__ V, const float* __restrict__ W, float* __restrict__ U,
               float* __restrict__ GU, int nn, float thr, HugeBlock* __restrict__ hb) {
  constexpr int NT = kHBlockThreads, NW = NT / 32;
  // the T = V^T W staging is dead once T is formed: the B partials reuse it
  __shared__ float XYs[2 * 64 * 33];
  static_assert(NW * kHK * kHK <= 2 * 64 * 33, "B partials overlay");
  float* Xs = XYs;
  float* Ys = XYs + 64 * 33;
  float (*Bred)[kHK * kHK] = reinterpret_cast<float (*)[kHK * kHK]>(XYs);
  __shared__ float Ts[kHP * 33];
  __shared__ float Ls[kHP * 33];
  __shared__ float Qs[kHP * kHK];
  __shared__ float Bm[kHK * kHK];
  __shared__ float Rred[NW][2 * kHK];
  __shared__ float ev[8 * kHP];
  __shared__ int evi[kHP];
  __shared__ float evt[3 * NT];
  __shared__ int evc[NT];
  __shared__ float red[64];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (!huge_active(hb[b])) return;
  const float* Vb = V + (size_t)b * nn * kHP;
  const float* Wb = W + (size_t)b * nn * kHP;
  float* Ub = U + (size_t)b * nn * kHK;
  float* Gb = GU + (size_t)b * nn * kHK;
  huge_xty(Vb, nullptr, 0.f, Wb, nn, Xs, Ys, Ts);
  for (int e = tid; e < kHP * kHP; e += NT) {
    const int i = e >> 5, j = e & 31;
    Ls[i * 33 + j] = 0.5f * (Ts[i * 33 + j] + Ts[j * 33 + i]);
  }
  __syncthreads();
  EigScratch s;
  s.d = ev;
  s.e = s.d + kHP;
  s.e2 = s.e + kHP;
  s.beta = s.e2 + kHP;
  s.vbuf = s.beta + kHP;
  s.pbuf = s.vbuf + kHP;
  s.lam = s.pbuf + kHP;
  s.shf = s.lam + kHP;
  s.clus = evi;
  s.lo = evt;
  s.hi = evt + NT;
  s.xs = evt + 2 * NT;
  s.cnt = evc;
  s.red = red;
  LowerFull Lacc{Ls, 33};
  tridiagonalize<NT>(Lacc, kHP, s);
  float tn = 0.f;
  // the pairs above tau^2 are the ones kept (and deflated by the certificate)
  const int kq = top_eigenvalues<NT>(kHP, thr, s, &tn);
  const int ku = kq < kHK ? kq : kHK;
  if (ku > 0) top_eigenvectors<NT, kHP>(Lacc, kHP, ku, tn, s, Qs, kHK, -1);
  __syncthreads();
  // U, G U and the warp partials of B
  float Bacc[kHK];
#pragma unroll
  for (int p = 0; p < kHK; ++p) Bacc[p] = 0.f;
  // the next row's loads are issued before the current row is used
  float vn = warp < nn ? Vb[(size_t)warp * kHP + lane] : 0.f;
  float wn = warp < nn ? Wb[(size_t)warp * kHP + lane] : 0.f;
  for (int r = warp; r < nn; r += NW) {
    const float v = vn, wv = wn;
    if (r + NW < nn) {
      vn = Vb[(size_t)(r + NW) * kHP + lane];
      wn = Wb[(size_t)(r + NW) * kHP + lane];
    }
    float u = 0.f, g = 0.f;
#pragma unroll 8
    for (int a = 0; a < kHP; ++a) {
      const float va = __shfl_sync(0xffffffffu, v, a);
      const float wa = __shfl_sync(0xffffffffu, wv, a);
      if (lane < ku) {
        const float qv = Qs[a * kHK + lane];
        u = fmaf(va, qv, u);
        g = fmaf(wa, qv, g);
      }
    }
    if (lane < ku) {
      Ub[(size_t)r * kHK + lane] = u;
      Gb[(size_t)r * kHK + lane] = g;
    }
#pragma unroll
    for (int p = 0; p < kHK; ++p) {
      const float up = __shfl_sync(0xffffffffu, u, p);
      Bacc[p] = fmaf(up, g, Bacc[p]);
    }
  }
  if (lane < kHK)
#pragma unroll
    for (int p = 0; p < kHK; ++p) Bred[warp][p * kHK + lane] = Bacc[p];
  __syncthreads();
  if (tid < kHK * kHK) {
    float t = 0.f;
    for (int w = 0; w < NW; ++w) t += Bred[w][tid];
    Bm[tid] = t;  // B(p, q) = u_p^T G u_q
  }
  __syncthreads();
  // residuals and What
  float racc = 0.f, wacc = 0.f;
  float un = 0.f, gn = 0.f;
  if (lane < ku && warp < nn) {
    un = Ub[(size_t)warp * kHK + lane];
    gn = Gb[(size_t)warp * kHK + lane];
  }
  for (int r = warp; r < nn; r += NW) {
    const float u = un, g = gn;
    if (lane < ku && r + NW < nn) {
      un = Ub[(size_t)(r + NW) * kHK + lane];
      gn = Gb[(size_t)(r + NW) * kHK + lane];
    }
    float wh = g;
#pragma unroll
    for (int p = 0; p < kHK; ++p) {
      const float up = __shfl_sync(0xffffffffu, u, p);
      if (p < ku && lane < ku)
        wh = fmaf(-0.25f * (Bm[p * kHK + lane] + Bm[lane * kHK + p]), up, wh);
    }
    if (lane < ku) {
      const float res = g - Bm[lane * kHK + lane] * u;
      racc = fmaf(res, res, racc);
      wacc = fmaf(wh, wh, wacc);
      Gb[(size_t)r * kHK + lane] = wh;
    }
  }
  if (lane < kHK) {
    Rred[warp][lane] = racc;
    Rred[warp][kHK + lane] = wacc;
  }
  __syncthreads();
  if (tid == 0) {
    HugeBlock& h = hb[b];
    float wsum = 0.f;
    float rq[kHK];
    int k = 0;
    for (int q = 0; q < ku; ++q) {
      float t = 0.f, t2 = 0.f;
      for (int w = 0; w < NW; ++w) {
        t += Rred[w][q];
        t2 += Rred[w][kHK + q];
      }
      rq[q] = sqrtf(t);
      wsum += t2;
      const float th = Bm[q * kHK + q];
      h.theta[q] = th;
      k += th > thr;
    }
    // converged: every kept pair's residual is small against tau^2, or at
    // the rounding level of G V (set by the largest eigenvalue).  Pairs just
    // above tau converge slowly; they need this accuracy all the same, since
    // the consensus step carries their error into every scale.
    int conv = 1;
    float trb = 0.f, th0 = 0.f;
    for (int q = 0; q < ku; ++q) th0 = fmaxf(th0, Bm[q * kHK + q]);
    for (int q = 0; q < ku; ++q) {
      trb += Bm[q * kHK + q];
      if (rq[q] > fmaxf(3e-4f * thr, 4e-6f * th0)) conv = 0;
    }
    // Certificate shift: lambda_max(P G P) < c proves, by Cauchy interlacing,
    // that G has at most ku eigenvalues above c (and the ku Ritz values above
    // tau^2 are lower bounds of ku eigenvalues), so exactly the kept pairs
    // lie above tau^2.  c = tau^2 less the rounding margins: the tiled
    // Cholesky of H = c I - X succeeds only if H + E is positive definite
    // with ||E||_2 <= gamma_d trace(H) (Higham, Thm. 10.3, with inner-product
    // depth d <= 2 * 64 + nn / 64 + 2), trace(H) = nn c - trace(G) + sum
    // theta; and forming X costs (2 ku + 4) eps (||G||_F + 2 sqrt(ku) ||What||_F).
    const float depth = (float)(2 * kHT + nn / kHT + 2);
    const float trh = fmaxf((float)nn * thr - (h.trace - trb), 0.f);
    const float xf = h.gF + 2.f * sqrtf((float)ku) * sqrtf(wsum);
    const float margin =
        1.1f * FLT_EPSILON * (depth * trh + (float)(2 * ku + 4) * xf);
    h.c = thr - margin;
    h.ku = ku;
    h.k = k;
    h.conv = conv;
  }
}


// ---------------------------------------------------------------------------
// 4. Certificate.  H = c I - X, X = G - U What^T - What U^T = P G P (the
// deflated Gram matrix), lower 64x64 tiles; then H = L L^T tile by tile.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kHThreads)
huge_form_kernel(const float* __restrict__ G, const float* __restrict__ U,
                 const float* __restrict__ Wh, float* __restrict__ H, int nn,
                 HugeBlock* __restrict__ hb) {
  __shared__ float Ui[kHT][kHK + 1], Wi[kHT][kHK + 1], Uj[kHT][kHK + 1], Wj[kHT][kHK + 1];
  const int t = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
  const HugeBlock& h = hb[b];
  if (h.status != kHsIter) return;
  const float c = h.c;
  if (!(c > 0.f)) {
    if (t == 0 && tid == 0) hb[b].chol_fail = 1;
    return;
  }
  const int ku = h.ku;
  int ta, tc;
  tile_of(t, &ta, &tc);
  const float* Ub = U + (size_t)b * nn * kHK;
  const float* Wb = Wh + (size_t)b * nn * kHK;
  for (int e = tid; e < kHT * kHK; e += kHThreads) {
    const int x = e / kHK, q = e - x * kHK;
    const int gi = ta * kHT + x, gj = tc * kHT + x;
    const bool qi = q < ku && gi < nn, qj = q < ku && gj < nn;
    Ui[x][q] = qi ? Ub[(size_t)gi * kHK + q] : 0.f;
    Wi[x][q] = qi ? Wb[(size_t)gi * kHK + q] : 0.f;
    Uj[x][q] = qj ? Ub[(size_t)gj * kHK + q] : 0.f;
    Wj[x][q] = qj ? Wb[(size_t)gj * kHK + q] : 0.f;
  }
  __syncthreads();
  const float* Gb = G + (size_t)b * nn * nn;
  float* Hb = H + (size_t)b * nn * nn;
  for (int e = tid; e < kHT * kHT; e += kHThreads) {
    const int x = e / kHT, y = e - x * kHT;
    const int i = ta * kHT + x, j = tc * kHT + y;
    if (i >= nn || j >= nn || j > i) continue;
    float v = Gb[(size_t)i * nn + j];
    for (int q = 0; q < ku; ++q) {
      v = fmaf(-Ui[x][q], Wj[y][q], v);
      v = fmaf(-Wi[x][q], Uj[y][q], v);
    }
    Hb[(size_t)i * nn + j] = (i == j ? c : 0.f) - v;
  }
}

// Panel j: every CTA factors the diagonal tile (j, j) in shared memory (all
// get the same factor); CTA i > 0 solves tile (j + i, j): L_ij = H_ij
// L_jj^{-T}.  A non-positive pivot marks the block.
__global__ void __launch_bounds__(kHThreads)
huge_chol_panel_kernel(float* __restrict__ H, int nn, int j, HugeBlock* __restrict__ hb) {
  __shared__ float Ld[kHT][kHT + 1];
  __shared__ float Xs[kHT][kHT + 1];
  const int b = blockIdx.y, tid = threadIdx.x;
  {
    const HugeBlock& h = hb[b];
    if (h.status != kHsIter || h.chol_fail) return;
  }
  const int i = j + blockIdx.x;
  float* Hb = H + (size_t)b * nn * nn;
  const int j0 = j * kHT, i0 = i * kHT;
  for (int e = tid; e < kHT * kHT; e += kHThreads) {
    const int x = e / kHT, y = e - x * kHT;
    const int gi = j0 + x, gj = j0 + y;
    float v;
    if (gi < nn && gj < nn) v = (y <= x) ? Hb[(size_t)gi * nn + gj] : 0.f;
    else v = (x == y) ? 1.f : 0.f;  // identity padding keeps definiteness
    Ld[x][y] = v;
  }
  __syncthreads();
  // the 64 x 64 diagonal factor, column by column (Crout form, Golub & Van
  // Loan Sec. 4.2): thread (r, part) = (tid / 4, tid mod 4) forms a quarter
  // of row r's inner product with row c, the four quarters are added by
  // shuffles inside the warp; two CTA barriers per column
  __shared__ int bad_s;
  if (tid == 0) bad_s = 0;
  const int r = tid >> 2, part = tid & 3;
  for (int c = 0; c < kHT; ++c) {
    float sdot = 0.f;
    if (r >= c)
      for (int k = part; k < c; k += 4) sdot = fmaf(Ld[r][k], Ld[c][k], sdot);
    sdot += __shfl_xor_sync(0xffffffffu, sdot, 1);
    sdot += __shfl_xor_sync(0xffffffffu, sdot, 2);
    const float t = r >= c ? Ld[r][c] - sdot : 0.f;
    if (r == c && part == 0) {
      const bool ok = t > 0.f && isfinite(t);
      if (!ok) bad_s = 1;
      Ld[c][c] = sqrtf(ok ? t : 1.f);
    }
    __syncthreads();
    if (r > c && part == 0) Ld[r][c] = t / Ld[c][c];
    __syncthreads();
  }
  const bool bad = bad_s != 0;
  if (bad) {
    if (blockIdx.x == 0 && tid == 0) hb[b].chol_fail = 1;
    return;
  }
  // the diagonal factor is needed only inside this launch (every CTA has
  // it); tile (j, j) stays as it is, so no CTA can read a half-written one
  if (i == j) return;
  for (int e = tid; e < kHT * kHT; e += kHThreads) {
    const int x = e / kHT, y = e - x * kHT;
    const int gi = i0 + x, gj = j0 + y;
    Xs[x][y] = (gi < nn && gj < nn) ? Hb[(size_t)gi * nn + gj] : 0.f;
  }
  __syncthreads();
  {
    // rows of X L^T = A: thread (x, part) = (tid / 4, tid mod 4) forms a
    // quarter of each inner product, the row's four threads (one warp) add
    // them by shuffles; no CTA barrier between columns
    const int x = tid >> 2;
    for (int c = 0; c < kHT; ++c) {
      float sdot = 0.f;
      for (int l = part; l < c; l += 4) sdot = fmaf(Xs[x][l], Ld[c][l], sdot);
      sdot += __shfl_xor_sync(0xffffffffu, sdot, 1);
      sdot += __shfl_xor_sync(0xffffffffu, sdot, 2);
      if (part == 0) Xs[x][c] = (Xs[x][c] - sdot) / Ld[c][c];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = tid; e < kHT * kHT; e += kHThreads) {
    const int x = e / kHT, y = e - x * kHT;
    const int gi = i0 + x, gj = j0 + y;
    if (gi < nn && gj < nn) Hb[(size_t)gi * nn + gj] = Xs[x][y];
  }
}

// Trailing update after panel j: H_il -= L_ij L_lj^T for j < l <= i.
__global__ void __launch_bounds__(kHThreads)
huge_chol_update_kernel(float* __restrict__ H, int nn, int j, HugeBlock* __restrict__ hb) {
  __shared__ __align__(16) float Ai[kHT][kHT + 4];
  __shared__ __align__(16) float Al[kHT][kHT + 4];
  const int b = blockIdx.y, tid = threadIdx.x;
  {
    const HugeBlock& h = hb[b];
    if (h.status != kHsIter || h.chol_fail) return;
  }
  int ta, tc;
  tile_of(blockIdx.x, &ta, &tc);
  const int i = j + 1 + ta, l = j + 1 + tc;
  float* Hb = H + (size_t)b * nn * nn;
  const int i0 = i * kHT, l0 = l * kHT, j0 = j * kHT;
  for (int e = tid; e < kHT * kHT; e += kHThreads) {
    const int x = e / kHT, kk = e - x * kHT;
    const bool kin = j0 + kk < nn;
    Ai[kk][x] = (kin && i0 + x < nn) ? Hb[(size_t)(i0 + x) * nn + j0 + kk] : 0.f;
    Al[kk][x] = (kin && l0 + x < nn) ? Hb[(size_t)(l0 + x) * nn + j0 + kk] : 0.f;
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll 8
  for (int kk = 0; kk < kHT; ++kk) {
    const float4 a4 = *reinterpret_cast<const float4*>(&Ai[kk][ty * 4]);
    const float4 b4 = *reinterpret_cast<const float4*>(&Al[kk][tx * 4]);
    const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int gi = i0 + ty * 4 + x;
    if (gi >= nn) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int gl = l0 + tx * 4 + y;
      if (gl < nn && gl <= gi) Hb[(size_t)gi * nn + gl] -= acc[x][y];
    }
  }
}


// Per block: the outcome.  V_f = U diag(sqrt(1 - tau / sqrt(theta))) over
// the pairs above tau (nn x kHK row-major, zero columns beyond k), counters
// and the nuclear-norm sum.
__global__ void __launch_bounds__(kHThreads)
huge_final_kernel(ScaleLaunch a, const float* __restrict__ U, float* __restrict__ Y, int* kout,
                  int nn, const HugeBlock* __restrict__ hb) {
  __shared__ int sel[kHK];
  __shared__ float fs[kHK];
  __shared__ int ks;
  const int b = blockIdx.x, tid = threadIdx.x;
  const HugeBlock& h = hb[b];
  const float thr = a.tau * a.tau;
  if (tid == 0) {
    int k = 0;
    if (h.status == kHsIter) {
      for (int q = 0; q < h.ku; ++q) {
        const float th = h.theta[q];
        if (th > thr) {
          sel[k] = q;
          fs[k] = sqrtf(fmaxf(1.f - a.tau / sqrtf(th), 0.f));
          ++k;
        }
      }
    }
    ks = k;
    const bool skipped = h.status == kHsSkip;
    const bool cert = skipped || (h.status == kHsIter && h.c > 0.f && !h.chol_fail);
    kout[b] = k;
    if (a.rank_out) a.rank_out[b] = k;
    if (a.cnt) {
      if (skipped) atomicAdd(a.cnt, 1ull);
      if (k == 0) atomicAdd(a.cnt + 1, 1ull);
      if (cert && !skipped) atomicAdd(a.cnt + 2, 1ull);
      if (!cert) atomicAdd(a.cnt + 4, 1ull);
    }
    if (a.nuc_acc && k > 0) {
      double t = 0.0;
      for (int q = 0; q < k; ++q)
        t += (double)fmaxf(sqrtf(h.theta[sel[q]]) - a.tau, 0.f);
      atomicAdd(a.nuc_acc, t);
    }
  }
  __syncthreads();
  const int k = ks;
  if (k == 0) return;
  const float* Ub = U + (size_t)b * nn * kHK;
  float* Yb = Y + (size_t)b * nn * kHK;
  for (int e = tid; e < nn * kHK; e += kHThreads) {
    const int r = e / kHK, c = e - r * kHK;
    Yb[e] = c < k ? Ub[(size_t)r * kHK + sel[c]] * fs[c] : 0.f;
  }
}

// ---------------------------------------------------------------------------
// 5. Z' = (C V_f) V_f^T and W' = 2 Z' - A, a warp per row of C, 4 rows per
// warp.  Rows of rank-0 blocks get Z' = 0, W' = -A.
// ---------------------------------------------------------------------------
constexpr int kHRebRows = 32;
template <bool ST>
__global__ void __launch_bounds__(kHThreads)
huge_rebuild_kernel(ScaleLaunch a, const float* __restrict__ Y, const int* __restrict__ kin) {
  const int b = blockIdx.y;
  const int k = kin[b];
  const BlockGeom g = block_geom_t<ST>(a, b);
  const int mm = g.mm(), nn = g.nn();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int RPW = kHRebRows / (kHThreads / 32);
  const float* Yb = Y + (size_t)b * nn * kHK;
  for (int rr = 0; rr < RPW; ++rr) {
    const int i = blockIdx.x * kHRebRows + warp * RPW + rr;
    if (i >= mm) break;
    float P[kHK];
#pragma unroll
    for (int q = 0; q < kHK; ++q) P[q] = 0.f;
    if (k > 0) {
      for (int c = lane; c < nn; c += 32) {
        const float av = huge_load(a, huge_off(g, i, c));
        const float4* vf = reinterpret_cast<const float4*>(Yb + (size_t)c * kHK);
#pragma unroll
        for (int t = 0; t < kHK / 4; ++t) {
          const float4 v = vf[t];
          P[4 * t] = fmaf(av, v.x, P[4 * t]);
          P[4 * t + 1] = fmaf(av, v.y, P[4 * t + 1]);
          P[4 * t + 2] = fmaf(av, v.z, P[4 * t + 2]);
          P[4 * t + 3] = fmaf(av, v.w, P[4 * t + 3]);
        }
      }
#pragma unroll
      for (int q = 0; q < kHK; ++q) P[q] = warp_sum(P[q]);
    }
    for (int c = lane; c < nn; c += 32) {
      const size_t off = huge_off(g, i, c);
      const float av = huge_load(a, off);
      float z = 0.f;
      if (k > 0) {
        const float4* vf = reinterpret_cast<const float4*>(Yb + (size_t)c * kHK);
#pragma unroll
        for (int t = 0; t < kHK / 4; ++t) {
          const float4 v = vf[t];
          z = fmaf(P[4 * t], v.x, z);
          z = fmaf(P[4 * t + 1], v.y, z);
          z = fmaf(P[4 * t + 2], v.z, z);
          z = fmaf(P[4 * t + 3], v.w, z);
        }
      }
      a.Zout[off] = z;
      if (a.Wout) a.Wout[off] = 2.f * z - av;
    }
  }
}


}  // namespace

static char* halign(char* p) { return (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255); }

size_t huge_workspace_bytes(int M, int N, int m, int n) {
  const HugeDims d = huge_dims(M, N, m, n);
  const size_t B = (size_t)d.nblocks, nn = (size_t)d.nn;
  size_t bytes = 0;
  bytes += sizeof(float) * B * d.chunks * d.ntiles * kHT * kHT;  // Gram partials
  bytes += 2 * sizeof(float) * B * nn * nn;                      // G, H
  bytes += 2 * sizeof(float) * B * d.ntiles;                     // tile sums
  bytes += 2 * sizeof(float) * B * nn * kHP;                     // V, W
  bytes += 3 * sizeof(float) * B * nn * kHK;                     // U, What, V_f
  bytes += sizeof(HugeBlock) * B + sizeof(int) * B;
  bytes += 16 * 256;
  return bytes;
}

BigWorkspace carve_huge_workspace(void* base, int M, int N, int m, int n) {
  BigWorkspace w{};
  if (!base) return w;
  const HugeDims d = huge_dims(M, N, m, n);
  const size_t B = (size_t)d.nblocks, nn = (size_t)d.nn;
  char* p = halign((char*)base);
  auto take = [&](size_t bytes) {
    char* q = p;
    p = halign(p + bytes);
    return q;
  };
  w.part = (float*)take(sizeof(float) * B * d.chunks * d.ntiles * kHT * kHT);
  w.G = (float*)take(sizeof(float) * B * nn * nn);
  w.H = (float*)take(sizeof(float) * B * nn * nn);
  w.tstat = (float*)take(2 * sizeof(float) * B * d.ntiles);
  w.V = (float*)take(sizeof(float) * B * nn * kHP);
  w.Wv = (float*)take(sizeof(float) * B * nn * kHP);
  w.U = (float*)take(sizeof(float) * B * nn * kHK);
  w.GU = (float*)take(sizeof(float) * B * nn * kHK);
  w.Y = (float*)take(sizeof(float) * B * nn * kHK);
  w.ystride = nn * kHK;
  w.hb = take(sizeof(HugeBlock) * B);
  w.k = (int*)take(sizeof(int) * B);
  return w;
}

// Start basis of every block (start of a decomposition, or a fresh call).
cudaError_t reset_huge_basis(const BigWorkspace& w, int M, int N, int m, int n, cudaStream_t st) {
  if (!w.V) return cudaSuccess;
  const HugeDims d = huge_dims(M, N, m, n);
  const size_t total = (size_t)d.nblocks * d.nn * kHP;
  const int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  huge_init_basis_kernel<<<grid, 256, 0, st>>>(w.V, total, d.nn);
  return cudaGetLastError();
}

cudaError_t launch_huge(const ScaleLaunch& s, const BigWorkspace& ws, cudaStream_t st, Prof* prof,
                        cudaEvent_t after_gram) {
  const HugeDims d = huge_dims(s.M, s.N, s.m, s.n);
  if (d.nn > MSLLR_MAX_BLOCK_WIDTH || !ws.V) return cudaErrorInvalidValue;
#define PROF_BEFORE(kind) \
  if (prof)               \
    if (cudaError_t e_ = prof->before(st, kind)) return e_;
#define PROF_AFTER() \
  if (prof)          \
    if (cudaError_t e_ = prof->after(st)) return e_;
  HugeBlock* hb = (HugeBlock*)ws.hb;
  const float thr = s.tau * s.tau;
  const int B = d.nblocks, nn = d.nn;
  PROF_BEFORE(KK_GRAM)
  if (gram_tc_eligible(s) && !gram_fp32_forced()) {
    // tensor-core Gram (k_gram_tc.cu), partial sums in the same 64 x 64 tile
    // layout and chunks, reduced below
    if (cudaError_t e_ = launch_gram_tc(s, nullptr, ws.part, d.chunks, B, d.ntiles, d.chunk_rows,
                                        1, st))
      return e_;
  } else if (s.fw || s.rows)
    huge_gram_kernel<true><<<dim3(d.ntiles, d.chunks, B), kHThreads, 0, st>>>(s, ws.part, d.chunk_rows,
                                                                      d.chunks, hb);
  else
    huge_gram_kernel<false><<<dim3(d.ntiles, d.chunks, B), kHThreads, 0, st>>>(s, ws.part, d.chunk_rows,
                                                                      d.chunks, hb);
  PROF_AFTER()
  PROF_BEFORE(KK_GRAM_REDUCE)
  huge_gram_finish_kernel<<<dim3(d.ntiles, B), kHThreads, 0, st>>>(ws.part, ws.G, ws.tstat, nn,
                                                                   d.chunks);
  PROF_AFTER()
  if (after_gram)
    if (cudaError_t e_ = cudaEventRecord(after_gram, st)) return e_;
  PROF_BEFORE(KK_MISC)
  huge_prep_kernel<<<B, kHThreads, 0, st>>>(ws.tstat, d.ntiles, hb, thr);
  PROF_AFTER()
  // subspace iteration: a first round (short when the grid does not move and
  // the basis carries over from the previous call), a second round for the
  // blocks whose Ritz residuals are still large
  const bool full = (s.m == launch_rows(s) && s.n == s.N);
  const bool warm = s.warm_start && (full || !s.shift);
  const int rounds[3] = {warm ? 2 : 6, 4, 8};
  const dim3 gv_grid((nn + kHGvRows - 1) / kHGvRows, B);
  const int orth_chunks = (nn + kHOrthRows - 1) / kHOrthRows;
  for (int r = 0; r < 3; ++r) {
    for (int st_i = 0; st_i < rounds[r]; ++st_i) {
      PROF_BEFORE(KK_SUBSPACE)
      huge_gv_kernel<<<gv_grid, kHThreads, 0, st>>>(ws.G, ws.V, ws.Wv, nn, hb);
      PROF_AFTER()
      for (int pass = 0; pass < 4; ++pass) {
        // S partials alternate between the two halves of the Gram partial
        // buffer (free once G is formed)
        float* pa = ws.part;
        float* pb = ws.part + (size_t)B * orth_chunks * (kHP * kHP);
        PROF_BEFORE(KK_SUBSPACE)
        huge_orth_sweep_kernel<<<dim3(orth_chunks, B), kHThreads, 0, st>>>(
            ws.V, ws.Wv, (pass & 1) ? pa : pb, (pass & 1) ? pb : pa, nn, pass, hb);
        PROF_AFTER()
      }
    }
    PROF_BEFORE(KK_SUBSPACE)
    huge_gv_kernel<<<gv_grid, kHThreads, 0, st>>>(ws.G, ws.V, ws.Wv, nn, hb);
    PROF_AFTER()
    PROF_BEFORE(KK_SUBSPACE)
    huge_rr_kernel<<<B, kHBlockThreads, 0, st>>>(ws.V, ws.Wv, ws.U, ws.GU, nn, thr, hb);
    PROF_AFTER()
  }
  // certificate
  PROF_BEFORE(KK_CERT)
  huge_form_kernel<<<dim3(d.ntiles, B), kHThreads, 0, st>>>(ws.G, ws.U, ws.GU, ws.H, nn, hb);
  PROF_AFTER()
  for (int j = 0; j < d.T; ++j) {
    PROF_BEFORE(KK_CERT)
    huge_chol_panel_kernel<<<dim3(d.T - j, B), kHThreads, 0, st>>>(ws.H, nn, j, hb);
    PROF_AFTER()
    const int rem = d.T - j - 1;
    if (rem > 0) {
      PROF_BEFORE(KK_CERT)
      huge_chol_update_kernel<<<dim3(rem * (rem + 1) / 2, B), kHThreads, 0, st>>>(ws.H, nn, j, hb);
      PROF_AFTER()
    }
  }
  PROF_BEFORE(KK_EIG)
  huge_final_kernel<<<B, kHThreads, 0, st>>>(s, ws.U, ws.Y, ws.k, nn, hb);
  PROF_AFTER()
  PROF_BEFORE(KK_REBUILD)
  if (s.fw || s.rows)
    huge_rebuild_kernel<true><<<dim3((d.mm + kHRebRows - 1) / kHRebRows, B), kHThreads, 0, st>>>(s, ws.Y,
                                                                                         ws.k);
  else
    huge_rebuild_kernel<false><<<dim3((d.mm + kHRebRows - 1) / kHRebRows, B), kHThreads, 0, st>>>(s, ws.Y,
                                                                                         ws.k);
  PROF_AFTER()
#undef PROF_BEFORE
#undef PROF_AFTER
  return cudaGetLastError();
}

}  // namespace msllr
