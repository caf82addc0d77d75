// Block SVT for wide blocks (64 < min(m, n) <= 256, or m*n > 8192), which
// includes the full-matrix scale of eq:bsvt.  Phases per scale:
//   1. gram_tiles: G_b = C_b^T C_b for every block, tiled 64x64 over the
//      lower triangle and split over row chunks (partial sums reduced in a
//      fixed order, so results are deterministic), stored packed;
//   2. eig_big: one CTA per block -- skip bound (Sec. 8), certified zero
//      rank or certified Lanczos eigenpairs of G_b (lanczos.cuh,
//      regchol.cuh), output V_b diag(sqrt(f));
//   3. eig_fallback: the Householder path (symeig.cuh) for the blocks step 2
//      could not certify;
//   4. rebuild: Z'_b = (C_b V_f) V_f^T, scattered through Shift_{-s}, with
//      the fused dual update W' = 2 Z' - A of eq:admm (warp per row for
//      ranks up to 8, row slabs above).
#include <math.h>
#include <stdlib.h>

#include "common.cuh"
#include "internal.h"
#include "lanczos.cuh"
#include "symeig.cuh"

namespace msllr {

cudaError_t set_phase_buffer_big(unsigned long long* p) {
  return cudaMemcpyToSymbol(g_phase_acc, &p, sizeof(p));
}

namespace {

constexpr int kTile = 64;       // Gram tile
constexpr int kChunk = 256;     // rows of C per Gram partial sum
constexpr int kGramThreads = 256;
constexpr int kEigThreads = 512;
constexpr int kEigMax = 256;
constexpr int kRebThreads = 256;
constexpr int kRebElems = 4096;  // rows-per-slab * nn
constexpr int kKC = 16;          // eigenvectors per rebuild step

struct BigDims {
  int mm, nn, nblocks, nbn, T, ntiles, chunks;
};

BigDims big_dims(int M, int N, int m, int n) {
  BigDims d;
  d.mm = m >= n ? m : n;
  d.nn = m >= n ? n : m;
  d.nbn = N / n;
  d.nblocks = (M / m) * (N / n);
  d.T = (d.nn + kTile - 1) / kTile;
  d.ntiles = d.T * (d.T + 1) / 2;
  d.chunks = (d.mm + kChunk - 1) / kChunk;
  return d;
}


// element (i, c) of C (mm x nn) -> global offset
__device__ __forceinline__ size_t c_offset(const BlockGeom& g, int i, int c) {
  return g.transposed() ? g.offset(c, i) : g.offset(i, c);
}

__device__ __forceinline__ float load_a(const ScaleLaunch& a, size_t off) {
  float v = a.A1[off];
  if (a.A2) v += a.A2[off];
  return v;
}

template <bool ST>
__global__ void __launch_bounds__(kGramThreads, 5)
gram_tiles_kernel(ScaleLaunch a, float* __restrict__ G, float* __restrict__ part, int chunks) {
  __shared__ __align__(16) float As[32][kTile + 4];
  __shared__ __align__(16) float Bs[32][kTile + 4];
  const int t = blockIdx.x, chunk = blockIdx.y, b = blockIdx.z;
  int ta = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
  while (((ta + 1) * (ta + 2)) / 2 <= t) ++ta;
  while ((ta * (ta + 1)) / 2 > t) --ta;
  const int tc = t - (ta * (ta + 1)) / 2;
  const BlockGeom g = block_geom_t<ST>(a, b);
  const int mm = g.mm(), nn = g.nn();
  const int a0 = ta * kTile, c0 = tc * kTile;
  const int r_begin = chunk * kChunk;
  const int r_end = min(mm, r_begin + kChunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
  const bool has2 = a.A2 != nullptr, dg = ta == tc;
  constexpr int kPer = (32 * kTile) / kGramThreads;
  for (int r0 = r_begin; r0 < r_end; r0 += 32) {
    // predicated loads, all in flight before the sums are formed
    float xa[kPer], ya[kPer], xb[kPer], yb[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int e = tid + j * kGramThreads;
      const int rr = e / kTile, cc = e - rr * kTile;
      const int i = r0 + rr;
      const bool in = i < r_end, ina = in && a0 + cc < nn, inb = in && !dg && c0 + cc < nn;
      const size_t oa = c_offset(g, ina ? i : r_begin, ina ? a0 + cc : 0);
      const size_t ob = c_offset(g, inb ? i : r_begin, inb ? c0 + cc : 0);
      xa[j] = ina ? __ldg(a.A1 + oa) : 0.f;
      ya[j] = (ina && has2) ? __ldg(a.A2 + oa) : 0.f;
      xb[j] = inb ? __ldg(a.A1 + ob) : 0.f;
      yb[j] = (inb && has2) ? __ldg(a.A2 + ob) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int e = tid + j * kGramThreads;
      const int rr = e / kTile, cc = e - rr * kTile;
      const float va = xa[j] + ya[j];
      As[rr][cc] = va;
      Bs[rr][cc] = dg ? va : xb[j] + yb[j];
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
  if (chunks == 1) {
    float* Gb = G + (size_t)b * nn * nn;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int i = a0 + ty * 4 + x;
      if (i >= nn) continue;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int j = c0 + tx * 4 + y;
        if (j <= i) Gb[(size_t)i * (i + 1) / 2 + j] = acc[x][y];
      }
    }
  } else {
    const int ntiles = gridDim.x;
    float* dst = part + (((size_t)b * chunks + chunk) * ntiles + t) * (kTile * kTile);
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) dst[(ty * 4 + x) * kTile + tx * 4 + y] = acc[x][y];
  }
}

__global__ void __launch_bounds__(256)
gram_reduce_kernel(const float* __restrict__ part, float* __restrict__ G, int nn, int ntiles,
                   int chunks) {
  const int t = blockIdx.x, b = blockIdx.y;
  int ta = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
  while (((ta + 1) * (ta + 2)) / 2 <= t) ++ta;
  while ((ta * (ta + 1)) / 2 > t) --ta;
  const int tc = t - (ta * (ta + 1)) / 2;
  const int per = (kTile * kTile) / gridDim.z;
  const int e0 = blockIdx.z * per;
  for (int e = e0 + threadIdx.x; e < e0 + per; e += blockDim.x) {
    const int x = e / kTile, y = e - x * kTile;
    const int i = ta * kTile + x, j = tc * kTile + y;
    if (i >= nn || j >= nn) continue;
    float s = 0.f;
    for (int c = 0; c < chunks; ++c)
      s += part[(((size_t)b * chunks + c) * ntiles + t) * (kTile * kTile) + e];
    if (j <= i) G[(size_t)b * nn * nn + (size_t)i * (i + 1) / 2 + j] = s;
  }
}

// panel region: Lanczos Q (kLzMaxJ x n), or the certificate's staging and
// Cholesky scratch, or the V_f staging
constexpr int kEigPanelFloats = (lz_cert_floats(kEigMax, kEigThreads) > kLzMaxJ * kEigMax)
                                    ? lz_cert_floats(kEigMax, kEigThreads)
                                    : kLzMaxJ * kEigMax;

size_t eig_smem_bytes(int nn) {
  return sizeof(float) * ((((size_t)nn * (nn + 1) / 2 + 3) & ~(size_t)3) + kEigPanelFloats +
                          9 * kEigMax + 4 * kEigThreads + 64 + lz_scratch_floats(kEigMax, kLzMaxJ));
}

// Up to three power steps from a pseudo-random vector: true when the
// Rayleigh quotient (a lower bound of lambda_max(G)) exceeds `thr`.  Called
// with thr = kZeroTry tau^2: a block whose quotient comes that close to
// tau^2 goes straight to the Lanczos path, because its zero-rank
// certificate would most likely fail, and a failed Cholesky costs as much
// as a successful one (the decision only routes work; the certificates
// decide the result).
constexpr float kZeroTry = 0.85f;
template <class S>
__device__ bool power_above(S G, int n, float thr, EigScratch& s, LzScratch& z, int* steps) {
  constexpr int NT = kEigThreads;
  const int tid = threadIdx.x;
  float part = 0.f;
  for (int e = tid; e < n; e += NT) {
    const float v = lz_hash(0xC0FFEEu, e) + 1.5f;
    z.x[e] = v;
    part = fmaf(v, v, part);
  }
  float nrm = sqrtf(block_sum<NT>(part, s.red));
  float rq = 0.f;
  *steps = 0;
  for (int it = 0; it < 3; ++it) {
    *steps = it + 1;
    for (int e = tid; e < n; e += NT) z.x[e] /= nrm;
    __syncthreads();
    symv_rows<NT, kEigMax>(G, n, z.x, z.w);
    float p1 = 0.f, p2 = 0.f;
    for (int e = tid; e < n; e += NT) {
      p1 = fmaf(z.x[e], z.w[e], p1);
      p2 = fmaf(z.w[e], z.w[e], p2);
    }
    rq = block_sum<NT>(p1, s.red);
    nrm = sqrtf(block_sum<NT>(p2, s.red));
    if (rq > thr || !(nrm > 0.f)) break;
    for (int e = tid; e < n; e += NT) z.x[e] = z.w[e];
    __syncthreads();
  }
  return rq > thr;
}

__global__ void __launch_bounds__(kEigThreads)
eig_big_kernel(ScaleLaunch a, const float* __restrict__ Gall, BigWorkspace ws) {
  extern __shared__ float sm[];
  constexpr int NT = kEigThreads, NMAX = kEigMax;
  const int b = blockIdx.x, tid = threadIdx.x;
  const int nn = a.m >= a.n ? a.n : a.m;
  const float* Gg = Gall + (size_t)b * nn * nn;
  float* Y = ws.Y + (size_t)b * ws.ystride;
  float* Gp = sm;
  float* panel = Gp + (((nn * (nn + 1)) / 2 + 3) & ~3);  // kEigPanelFloats, 16-byte aligned
  float* scr = panel + kEigPanelFloats;
  EigScratch s;
  s.d = scr;
  s.e = s.d + NMAX;
  s.e2 = s.e + NMAX;
  s.beta = s.e2 + NMAX;
  s.vbuf = s.beta + NMAX;
  s.pbuf = s.vbuf + NMAX;
  s.lam = s.pbuf + NMAX;
  s.shf = s.lam + NMAX;
  s.clus = reinterpret_cast<int*>(s.shf + NMAX);
  s.lo = reinterpret_cast<float*>(s.clus + NMAX);
  s.hi = s.lo + NT;
  s.xs = s.hi + NT;
  s.cnt = reinterpret_cast<int*>(s.xs + NT);
  s.red = reinterpret_cast<float*>(s.cnt + NT);
  LzScratch z;
  // Lanczos Q shares the panel region with the certificate scratch; they
  // are never live together
  float* Qs = panel;
  lz_bind<NT>(z, s.red + 64, NMAX, kLzMaxJ);
  PHASE_INIT();
  LowerPacked Gacc{Gp};
  // G arrives packed (lower triangle, row by row): a straight copy
  auto load_g = [&]() {
    const int ntri = nn * (nn + 1) / 2;
    if ((ntri & 3) == 0 && ((reinterpret_cast<uintptr_t>(Gg) & 15) == 0)) {
      const float4* src = reinterpret_cast<const float4*>(Gg);
      float4* dst = reinterpret_cast<float4*>(Gp);
      for (int e = tid; e < ntri / 4; e += NT) dst[e] = src[e];
    } else {
      for (int e = tid; e < ntri; e += NT) Gp[e] = Gg[e];
    }
    __syncthreads();
  };
  load_g();
  PHASE(3, 0);
  const float thr = a.tau * a.tau;
  // trace and Gershgorin bounds of lambda_max(G)
  float tr = 0.f;
  for (int i = tid; i < nn; i += NT) tr += Gacc.at(i, i);
  tr = block_sum<NT>(tr, s.red);
  const float rs = gershgorin_lower<NT, NMAX>(Gacc, nn, z.x, z.w, s.red);
  const float gbound = fminf(tr, rs);
  double fl = nn + fl_symv(nn);  // trace, Gershgorin row sums
  const bool full = (a.m == launch_rows(a) && a.n == a.N);
  const int kwarm = (a.warm_start && (full || !a.shift)) ? min(ws.kwarm[b], kLzMaxK) : 0;
  bool skipped = false, lanczos_ok = false;
  int k = -1, ku = 0;
  // Two certificates share one Cholesky call site: attempt 0 tests
  // lambda_max(G) < tau^2 (zero rank), attempt 1 certifies the Lanczos pairs
  // by the deflated matrix.
  const int n8 = (nn + 7) & ~7;
  float* U = Y;
  for (int attempt = 0; attempt < 2 && k < 0 && a.skip_bound; ++attempt) {
    float c0;
    int kk = 0;
    if (attempt == 0) {
      if (gbound <= thr) {
        skipped = true;
        k = 0;
        break;
      }
      if (kwarm > 0) continue;
      int psteps = 0;
      const bool above = power_above(Gacc, nn, kZeroTry * thr, s, z, &psteps);
      fl += psteps * (fl_symv(nn) + 4.0 * nn);
      if (above) continue;
      // certified lambda_max(G) < tau^2 by Cholesky of (tau^2 - margin) I - G
      c0 = thr - (float)n8 * (float)n8 * FLT_EPSILON * (thr + gbound);
      if (!(c0 > 0.f)) continue;
      PHASE(3, 6);
    } else {
      PHASE(3, 1);
      const float* warm = ws.warm + (size_t)b * kLzMaxK * nn;
      int J = 0;
      kk = lanczos_candidates<NT, NMAX>(Gacc, nn, thr, gbound, Qs,
                                                        min(nn, kLzMaxJ), U, warm, kwarm,
                                                        0x1234567u + 977u * job_block(a, b), s, z, panel, &ku,
                                                        &c0, 4, &J);
      fl += fl_lanczos(nn, J, ku);
      PHASE(3, 5);
      if (kk < 0) break;
      fl += fl_deflate(nn, ku);
    }
    fl += fl_chol(nn);
    const bool pd = regchol_pd<NT, NMAX>(Gacc, nn, c0, attempt == 1, panel, panel + 8 * n8,
                                         attempt == 1 ? ku : 0, panel + 16 * n8, s.red,
                                         3 + attempt);
    PHASE(3, 7 + attempt);
    if (pd) {
      k = kk;
      skipped = attempt == 0;
      lanczos_ok = attempt == 1;
    }
  }
  if (lanczos_ok) {
    // keep the Ritz vectors for the next call's warm start
    float* wdst = ws.warm + (size_t)b * kLzMaxK * nn;
    for (int e = tid; e < nn * ku; e += NT) wdst[e] = U[e];
    if (tid == 0) ws.kwarm[b] = ku;
    // V_f (row-major, ld nn) for the rebuild, staged through shared memory
    for (int e = tid; e < nn * k; e += NT) panel[e] = U[e];
    __syncthreads();
    for (int e = tid; e < nn * k; e += NT) {
      const int i = e / k, q = e - i * k;
      const float sig = sqrtf(s.lam[q]);
      Y[(size_t)i * nn + q] = panel[(size_t)q * nn + i] * sqrtf(fmaxf(1.f - a.tau / sig, 0.f));
    }
  }
  if (tid == 0) {
    if (a.cnt) atomicAdd(a.cnt + 5, (unsigned long long)fl);
    // k < 0: not settled here; eig_fallback_kernel takes the block
    ws.k[b] = k;
    if (k < 0) {
      if (ws.kwarm) ws.kwarm[b] = 0;
    } else {
      if (a.rank_out) a.rank_out[b] = k;
      if (a.cnt) {
        if (skipped) atomicAdd(a.cnt, 1ull);
        if (k == 0) atomicAdd(a.cnt + 1, 1ull);
        if (lanczos_ok) atomicAdd(a.cnt + 2, 1ull);
      }
      if (a.nuc_acc && k > 0) {
        double t = 0.0;
        for (int q = 0; q < k; ++q) t += (double)fmaxf(sqrtf(s.lam[q]) - a.tau, 0.f);
        atomicAdd(a.nuc_acc, t);
      }
    }
  }
}

// Householder path for the blocks eig_big_kernel left unsettled (ws.k < 0):
// tridiagonalisation, Sturm multisection and inverse iteration on the
// packed G (symeig.cuh).  Kept out of eig_big_kernel so that the common
// paths run from a smaller instruction footprint.
__device__ __forceinline__ void eig_fallback_block(const ScaleLaunch& a, const float* __restrict__ Gall,
                                                   const BigWorkspace& ws, int b) {
  extern __shared__ float sm[];
  constexpr int NT = kEigThreads, NMAX = kEigMax;
  const int tid = threadIdx.x;
  const int nn = a.m >= a.n ? a.n : a.m;
  const float* Gg = Gall + (size_t)b * nn * nn;
  float* Y = ws.Y + (size_t)b * ws.ystride;
  float* Gp = sm;
  float* scr = Gp + (((nn * (nn + 1)) / 2 + 3) & ~3);
  EigScratch s;
  s.d = scr;
  s.e = s.d + NMAX;
  s.e2 = s.e + NMAX;
  s.beta = s.e2 + NMAX;
  s.vbuf = s.beta + NMAX;
  s.pbuf = s.vbuf + NMAX;
  s.lam = s.pbuf + NMAX;
  s.shf = s.lam + NMAX;
  s.clus = reinterpret_cast<int*>(s.shf + NMAX);
  s.lo = reinterpret_cast<float*>(s.clus + NMAX);
  s.hi = s.lo + NT;
  s.xs = s.hi + NT;
  s.cnt = reinterpret_cast<int*>(s.xs + NT);
  s.red = reinterpret_cast<float*>(s.cnt + NT);
  const int ntri = nn * (nn + 1) / 2;
  for (int e = tid; e < ntri; e += NT) Gp[e] = Gg[e];
  __syncthreads();
  LowerPacked Gacc{Gp};
  const float thr = a.tau * a.tau;
  tridiagonalize<NT>(Gacc, nn, s);
  float tn = 0.f;
  const int k = top_eigenvalues<NT>(nn, thr, s, &tn);
  if (k > 0) {
    top_eigenvectors<NT, NMAX>(Gacc, nn, k, tn, s, Y, nn, -1);
    // V_f = V diag(sqrt(f)), f = 1 - tau/sigma
    for (int e = tid; e < nn * k; e += NT) {
      const int i = e / k, q = e - i * k;
      const float sig = sqrtf(s.lam[q]);
      Y[(size_t)i * nn + q] *= sqrtf(fmaxf(1.f - a.tau / sig, 0.f));
    }
  }
  if (tid == 0) {
    ws.k[b] = k;
    if (a.rank_out) a.rank_out[b] = k;
    if (a.cnt) {
      if (k == 0) atomicAdd(a.cnt + 1, 1ull);
      atomicAdd(a.cnt + 3, 1ull);
      atomicAdd(a.cnt + 6, (unsigned long long)fl_householder(nn, k));
    }
    if (a.nuc_acc && k > 0) {
      double t = 0.0;
      for (int q = 0; q < k; ++q) t += (double)fmaxf(sqrtf(s.lam[q]) - a.tau, 0.f);
      atomicAdd(a.nuc_acc, t);
    }
  }
}

// At most 32 CTAs stride over the blocks (a launch that finds nothing to do
// then holds few SMs); one CTA per block when the certified paths are off.
__global__ void __launch_bounds__(kEigThreads)
eig_fallback_kernel(ScaleLaunch a, const float* __restrict__ Gall, BigWorkspace ws, int nblocks) {
  for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
    if (ws.k[b] >= 0) continue;
    eig_fallback_block(a, Gall, ws, b);
    __syncthreads();
  }
}

size_t fallback_smem_bytes(int nn) {
  return sizeof(float) * ((((size_t)nn * (nn + 1) / 2 + 3) & ~(size_t)3) + 9 * kEigMax +
                          4 * kEigThreads + 64);
}

// Z' = (C V_f) V_f^T, W' = 2 Z' - A for blocks of rank k <= kRowK: one warp
// per row of C, a lane per 32nd column.  Row i: P = C_i V_f by lane partial
// sums and k warp reductions, Z'_i = P V_f^T; V_f (transposed) is staged once
// per CTA.  Every load of C and store of Z', W' is a warp-wide row segment.
constexpr int kRowK = 8;
constexpr int kRowsPerCta = 32;  // 8 warps x 4 rows: one wave at 4 CTAs per SM
// ST: spatio-temporal blocks; the 2-D instantiation knows fw = 0 at compile
// time, which keeps its index arithmetic in registers.
template <bool ST>
__global__ void __launch_bounds__(kRebThreads, 4)
rebuild_rows_kernel(ScaleLaunch a, const float* __restrict__ Yall, size_t ystride,
                    const int* __restrict__ kin) {
  __shared__ float Vt[kRowK * kEigMax];
  const int b = blockIdx.y;
  const int k = kin[b];
  if (k > kRowK) return;  // rebuild_kernel takes the block
  const BlockGeom g = block_geom_t<ST>(a, b);
  const int mm = g.mm(), nn = g.nn();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* Yb = Yall + (size_t)b * ystride;
  for (int i = tid; i < nn; i += kRebThreads)
    for (int q = 0; q < k; ++q) Vt[q * nn + i] = Yb[(size_t)i * nn + q];
  __syncthreads();
  constexpr int RPW = kRowsPerCta / (kRebThreads / 32);
  constexpr int CPL = kEigMax / 32;  // columns per lane
  const int row0 = blockIdx.x * kRowsPerCta + warp * RPW;
  // the next row's inputs are loaded while the current row is finished
  float nx[CPL];
#pragma unroll
  for (int t = 0; t < CPL; ++t) {
    const int c = lane + 32 * t;
    nx[t] = (row0 < mm && c < nn) ? load_a(a, c_offset(g, row0, c)) : 0.f;
  }
  for (int rr = 0; rr < RPW; ++rr) {
    const int i = row0 + rr;
    if (i >= mm) break;
    float av[CPL];
#pragma unroll
    for (int t = 0; t < CPL; ++t) {
      av[t] = nx[t];
      const int c = lane + 32 * t;
      nx[t] = (rr + 1 < RPW && i + 1 < mm && c < nn) ? load_a(a, c_offset(g, i + 1, c)) : 0.f;
    }
    float P[kRowK];
#pragma unroll
    for (int q = 0; q < kRowK; ++q) {
      P[q] = 0.f;
      if (q < k) {
#pragma unroll
        for (int t = 0; t < kEigMax / 32; ++t) {
          const int c = lane + 32 * t;
          if (c < nn) P[q] = fmaf(av[t], Vt[q * nn + c], P[q]);
        }
        P[q] = warp_sum(P[q]);
      }
    }
#pragma unroll
    for (int t = 0; t < kEigMax / 32; ++t) {
      const int c = lane + 32 * t;
      if (c < nn) {
        float z = 0.f;
#pragma unroll
        for (int q = 0; q < kRowK; ++q)
          if (q < k) z = fmaf(P[q], Vt[q * nn + c], z);
        const size_t off = c_offset(g, i, c);
        a.Zout[off] = z;
        if (a.Wout) a.Wout[off] = 2.f * z - av[t];
      }
    }
  }
}

// Z' = (C V_f) V_f^T for a slab of `rs` rows of C, W' = 2 Z' - A: blocks of
// rank above kRowK (only the Householder path produces them).  The CTAs
// stride over the (slab, block) items, so that a launch with nothing to do
// holds few SMs.
template <bool ST>
__device__ __forceinline__ void rebuild_slab(const ScaleLaunch& a, const float* __restrict__ Yall,
                                             size_t ystride, const int* __restrict__ kin, int rs,
                                             int slab, int b) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x;
  const BlockGeom g = block_geom_t<ST>(a, b);
  const int mm = g.mm(), nn = g.nn();
  const int r0 = slab * rs;
  const int rows = min(rs, mm - r0);
  const int k = kin[b];
  float* Cs = sm;                          // rows x nn
  float* Vs = Cs + rs * nn;                // kKC x (nn + 1): V_f chunk, transposed
  float* Ps = Vs + kKC * (nn + 1);         // rows x kKC
  const int ldv = nn + 1;
  const int nel = rows * nn;
#pragma unroll 4
  for (int e = tid; e < nel; e += kRebThreads) {
    const int i = e / nn, c = e - i * nn;
    Cs[e] = load_a(a, c_offset(g, r0 + i, c));
  }
  __syncthreads();
  constexpr int EL = kRebElems / kRebThreads;
  float acc[EL];
#pragma unroll
  for (int t = 0; t < EL; ++t) acc[t] = 0.f;
  const float* Yb = Yall + (size_t)b * ystride;
  for (int q0 = 0; q0 < k; q0 += kKC) {
    const int kc = min(kKC, k - q0);
    for (int e = tid; e < nn * kKC; e += kRebThreads) {
      const int i = e / kKC, j = e - i * kKC;
      Vs[j * ldv + i] = j < kc ? Yb[(size_t)i * nn + q0 + j] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < rows * kKC; e += kRebThreads) {
      const int i = e / kKC, j = e - i * kKC;
      const float* crow = Cs + i * nn;
      const float* vrow = Vs + j * ldv;
      float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
      int c = 0;
      for (; c + 3 < nn; c += 4) {
        t0 = fmaf(crow[c], vrow[c], t0);
        t1 = fmaf(crow[c + 1], vrow[c + 1], t1);
        t2 = fmaf(crow[c + 2], vrow[c + 2], t2);
        t3 = fmaf(crow[c + 3], vrow[c + 3], t3);
      }
      for (; c < nn; ++c) t0 = fmaf(crow[c], vrow[c], t0);
      Ps[e] = (t0 + t1) + (t2 + t3);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < EL; ++t) {
      const int e = tid + t * kRebThreads;
      if (e < nel) {
        const int i = e / nn, c = e - i * nn;
        float z = acc[t];
#pragma unroll
        for (int j = 0; j < kKC; ++j) z = fmaf(Ps[i * kKC + j], Vs[j * ldv + c], z);
        acc[t] = z;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < EL; ++t) {
    const int e = tid + t * kRebThreads;
    if (e < nel) {
      const int i = e / nn, c = e - i * nn;
      const size_t off = c_offset(g, r0 + i, c);
      a.Zout[off] = acc[t];
      if (a.Wout) a.Wout[off] = 2.f * acc[t] - Cs[e];
    }
  }
}

template <bool ST>
__global__ void __launch_bounds__(kRebThreads)
rebuild_kernel(ScaleLaunch a, const float* __restrict__ Yall, size_t ystride,
               const int* __restrict__ kin, int rs, int slabs, int nblocks) {
  for (int w = blockIdx.x; w < slabs * nblocks; w += gridDim.x) {
    const int b = w / slabs;
    if (kin[b] <= kRowK) continue;  // rebuild_rows_kernel took the block
    rebuild_slab<ST>(a, Yall, ystride, kin, rs, w - b * slabs, b);
    __syncthreads();
  }
}

}  // namespace

static size_t y_stride(int nn) {
  const size_t a = (size_t)nn * nn, b = (size_t)(kLzMaxJ + 2 * kLzMaxK) * nn;
  return ((a > b ? a : b) + 63) & ~(size_t)63;
}

size_t big_workspace_bytes(int M, int N, int m, int n) {
  if (choose_path(m, n) == ScalePath::Huge) return huge_workspace_bytes(M, N, m, n);
  if (choose_path(m, n) != ScalePath::Big) return 0;
  const BigDims d = big_dims(M, N, m, n);
  size_t bytes = 0;
  bytes += sizeof(float) * (size_t)d.nblocks * d.nn * d.nn;  // G
  if (d.chunks > 1) bytes += sizeof(float) * (size_t)d.nblocks * d.chunks * d.ntiles * kTile * kTile;
  bytes += sizeof(float) * (size_t)d.nblocks * y_stride(d.nn);  // Y
  bytes += sizeof(int) * (size_t)d.nblocks;                      // k
  bytes += sizeof(float) * (size_t)d.nblocks * kLzMaxK * d.nn;   // warm
  bytes += sizeof(int) * (size_t)d.nblocks;                      // kwarm
  bytes += 8 * 256;  // alignment slack for the carve below
  return bytes;
}

static char* align256(char* p) {
  return (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
}

BigWorkspace carve_big_workspace(void* base, int M, int N, int m, int n) {
  BigWorkspace w{};
  if (choose_path(m, n) == ScalePath::Huge) return carve_huge_workspace(base, M, N, m, n);
  if (!base || choose_path(m, n) != ScalePath::Big) return w;
  const BigDims d = big_dims(M, N, m, n);
  char* p = align256((char*)base);
  w.G = (float*)p;
  p = align256(p + sizeof(float) * (size_t)d.nblocks * d.nn * d.nn);
  if (d.chunks > 1) {
    w.part = (float*)p;
    p = align256(p + sizeof(float) * (size_t)d.nblocks * d.chunks * d.ntiles * kTile * kTile);
  }
  w.ystride = y_stride(d.nn);
  w.Y = (float*)p;
  p = align256(p + sizeof(float) * (size_t)d.nblocks * w.ystride);
  w.k = (int*)p;
  p = align256(p + sizeof(int) * (size_t)d.nblocks);
  w.warm = (float*)p;
  p = align256(p + sizeof(float) * (size_t)d.nblocks * kLzMaxK * d.nn);
  w.kwarm = (int*)p;
  return w;
}

cudaError_t reset_warm_start(const BigWorkspace& w, int M, int N, int m, int n, cudaStream_t st) {
  if (choose_path(m, n) == ScalePath::Huge) return reset_huge_basis(w, M, N, m, n, st);
  if (!w.kwarm) return cudaSuccess;
  const BigDims d = big_dims(M, N, m, n);
  return cudaMemsetAsync(w.kwarm, 0, sizeof(int) * (size_t)d.nblocks, st);
}

// The FP32 CUDA-core Gram instead of the tensor-core one (MSLLR_GRAM_FP32=1;
// for comparisons), read once.
bool gram_fp32_forced() {
  static const bool v = [] {
    const char* e = getenv("MSLLR_GRAM_FP32");
    return e && e[0] && e[0] != '0';
  }();
  return v;
}

cudaError_t configure_big_kernels() {
  sm_count();  // cache the SM count outside any stream capture
  gram_fp32_forced();
  if (cudaError_t e0 = configure_gram_tc()) return e0;
  cudaError_t e = cudaFuncSetAttribute(eig_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)eig_smem_bytes(kEigMax));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(eig_fallback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fallback_smem_bytes(kEigMax));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(rebuild_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           100 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(rebuild_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              100 * 1024);
}

// `after_gram` (optional) is recorded on `st` once the Gram kernels are
// enqueued, so that other streams can wait for the Gram phase to finish.
cudaError_t launch_big(const ScaleLaunch& s, const BigWorkspace& ws, cudaStream_t st, Prof* prof,
                       cudaEvent_t after_gram) {
  const BigDims d = big_dims(s.M, s.N, s.m, s.n);
  if (d.nn > kEigMax) return cudaErrorInvalidValue;
#define PROF_BEFORE(kind) \
  if (prof)               \
    if (cudaError_t e_ = prof->before(st, kind)) return e_;
#define PROF_AFTER() \
  if (prof)          \
    if (cudaError_t e_ = prof->after(st)) return e_;
  PROF_BEFORE(KK_GRAM)
  const dim3 ggrid(d.ntiles, d.chunks, d.nblocks);
  if (gram_tc_eligible(s) && !gram_fp32_forced()) {
    if (cudaError_t e_ = launch_gram_tc(s, ws.G, ws.part, d.chunks, d.nblocks, d.ntiles, kChunk,
                                        0, st))
      return e_;
  } else if (s.fw || s.rows) {
    gram_tiles_kernel<true><<<ggrid, kGramThreads, 0, st>>>(s, ws.G, ws.part, d.chunks);
  } else {
    gram_tiles_kernel<false><<<ggrid, kGramThreads, 0, st>>>(s, ws.G, ws.part, d.chunks);
  }
  PROF_AFTER()
  if (d.chunks > 1) {
    PROF_BEFORE(KK_GRAM_REDUCE)
    gram_reduce_kernel<<<dim3(d.ntiles, d.nblocks, 16), 256, 0, st>>>(ws.part, ws.G, d.nn,
                                                                      d.ntiles, d.chunks);
    PROF_AFTER()
  }
  if (after_gram)
    if (cudaError_t e_ = cudaEventRecord(after_gram, st)) return e_;
  PROF_BEFORE(KK_EIG)
  eig_big_kernel<<<d.nblocks, kEigThreads, eig_smem_bytes(d.nn), st>>>(s, ws.G, ws);
  PROF_AFTER()
  PROF_BEFORE(KK_EIG_FALLBACK)
  // up to 32 CTAs stride over the blocks: enough for scales where many
  // blocks need the Householder path (blocks of rank above 8, or with an
  // eigenvalue just below tau^2), few idle SMs where almost none do
  const int fb_grid = s.skip_bound ? (d.nblocks < 32 ? d.nblocks : 32) : d.nblocks;
  eig_fallback_kernel<<<fb_grid, kEigThreads, fallback_smem_bytes(d.nn), st>>>(s, ws.G, ws,
                                                                               d.nblocks);
  PROF_AFTER()
  const int rs = kRebElems / d.nn;
  const int slabs = (d.mm + rs - 1) / rs;
  const size_t smem = sizeof(float) * ((size_t)rs * d.nn + (size_t)(d.nn + 1) * kKC + (size_t)rs * kKC);
  PROF_BEFORE(KK_REBUILD)
  const dim3 rgrid((d.mm + kRowsPerCta - 1) / kRowsPerCta, d.nblocks);
  if (s.fw || s.rows) rebuild_rows_kernel<true><<<rgrid, kRebThreads, 0, st>>>(s, ws.Y, ws.ystride, ws.k);
  else rebuild_rows_kernel<false><<<rgrid, kRebThreads, 0, st>>>(s, ws.Y, ws.ystride, ws.k);
  PROF_AFTER()
  PROF_BEFORE(KK_REBUILD)
  const int slab_items = slabs * d.nblocks;
  const int nsm = sm_count();
  const int reb_grid = s.skip_bound ? (slab_items < nsm ? slab_items : nsm) : slab_items;
  if (s.fw || s.rows)
    rebuild_kernel<true><<<reb_grid, kRebThreads, smem, st>>>(s, ws.Y, ws.ystride, ws.k, rs, slabs,
                                                             d.nblocks);
  else
    rebuild_kernel<false><<<reb_grid, kRebThreads, smem, st>>>(s, ws.Y, ws.ystride, ws.k, rs, slabs,
                                                      d.nblocks);
  PROF_AFTER()
#undef PROF_BEFORE
#undef PROF_AFTER
  return cudaGetLastError();
}

}  // namespace msllr
