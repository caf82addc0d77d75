// One CTA's block SVT of a narrow block (min(m, n) <= 64, m*n <= 8192) --
// eq:bsvt for that block.  Used by the per-scale kernel (k_block_small.cu)
// and by the nested-scale kernel (k_nested.cu):
//   gather R_b(Shift_s(A)) into shared memory (Sec. 9 circular shift),
//   skip test on an upper bound of sigma_max (Sec. 8),
//   Gram matrix, certified rank above tau and the top eigenpairs (symeig.cuh),
//   rebuild C V diag(f) V^T, scatter through Shift_{-s}, and the fused dual
//   update W' = 2 Z' - A of eq:admm.
#pragma once

#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "lanczos.cuh"
#include "symeig.cuh"
#include "warp_block.cuh"

namespace msllr {
namespace {

// row index i of packed lower-triangle position e (e = i(i+1)/2 + j, j <= i)
__device__ __forceinline__ int tri_row(int e) {
  int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
  while (((i + 1) * (i + 2)) / 2 <= e) ++i;
  while ((i * (i + 1)) / 2 > e) --i;
  return i;
}

// Shared-memory layout of blocksvt_small_kernel (floats, 16-byte aligned
// offsets), shared by the kernel and the launcher.
//   C   mm x nn block                          [oC]
//   S   EigScratch (9 NMAX + 4 NT + 64)        [oS]
//   G   nn x (nn + 1) Gram matrix              [oG]
//   L   certificate scratch, then (widths > 16) the Lanczos basis Q, the
//       Ritz vectors U and the Lanczos scalars [oL, oQ, oU, oZ .. oEnd)
//   Y   Householder eigenvectors (nn x nn): aliases L, which is dead on
//       that path
//   P   C V diag(f) (mm x nn, rebuild only): aliases G when it fits there,
//       else appended at oEnd
template <int NT, int NMAX>
struct SmallLayout {
  static constexpr bool kLz = NMAX > 16;  // narrower blocks skip Lanczos
  static constexpr int JCAP = NMAX < kLzMaxJ ? NMAX : kLzMaxJ;
  int oC, oS, oG, oL, oQ, oU, oZ, oEnd, oP, total;
  __host__ __device__ static int al(int x) { return (x + 3) & ~3; }
  __host__ __device__ SmallLayout(int mm, int nn) {
    oC = 0;
    oS = al(mm * nn);
    oG = al(oS + 9 * NMAX + 4 * NT + 64);
    oL = al(oG + nn * (nn + 1));
    oQ = al(oL + lz_cert_floats(NMAX, NT));
    oU = kLz ? oQ + lz_ldq<NMAX>(NMAX) * JCAP : oQ;
    oZ = kLz ? oU + NMAX * kLzMaxK : oU;
    oEnd = kLz ? al(oZ + lz_scratch_floats(NMAX, JCAP)) : oQ;
    oP = mm * nn <= nn * (nn + 1) ? oG : oEnd;
    total = oP == oG ? oEnd : oEnd + mm * nn;
  }
};
static_assert(16 * 16 <= lz_cert_floats(16, 32), "Y alias (16)");
static_assert(32 * 32 <= lz_cert_floats(32, 64), "Y alias (32)");
static_assert(64 * 64 <= lz_cert_floats(64, 128) + 65 * 32 + 64 * kLzMaxK, "Y alias (64)");

// Block b of the scale by the calling CTA (NT threads, dynamic shared memory
// `sm` laid out by SmallLayout<NT, NMAX>); `a2(off, row, col)` gives the
// second half of A at global offset off, block element (row, col)
// (A2Global: a.A2 itself).
template <int NT, int NMAX, bool ST, class SRC>
__device__ __forceinline__ void small_block_svt(const ScaleLaunch& a, int b, float* sm,
                                                const SRC& a2) {
  const int tid = threadIdx.x;
  constexpr int SLOT = NT == 32 ? 0 : (NT == 64 ? 1 : 2);
  PHASE_INIT();
  const BlockGeom g = block_geom_t<ST>(a, b);
  const int mm = g.mm(), nn = g.nn();
  const int ldc = nn, ldg = nn + 1, ldy = nn;

  const SmallLayout<NT, NMAX> lay(mm, nn);
  float* C = sm + lay.oC;
  float* G = sm + lay.oG;
  float* Y = sm + lay.oL;
  float* P = sm + lay.oP;
  float* panel = sm + lay.oL;  // certificate scratch
  float* scr = sm + lay.oS;
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
  // Lanczos region: Q (lz_ldq x JCAP), U (NMAX x kLzMaxK); none for blocks
  // of width <= 16, which skip Lanczos (kAttempts == 1)
  constexpr int kAttempts = SmallLayout<NT, NMAX>::kLz ? 2 : 1;
  constexpr int JCAP = SmallLayout<NT, NMAX>::JCAP;
  float* Qs = sm + lay.oQ;
  float* Us = sm + lay.oU;
  LzScratch z;
  lz_bind<NT>(z, sm + lay.oZ, NMAX, JCAP);

  // gather A = A1 + A2 on the shifted grid; ||C||_F^2
  const int melem = a.m * a.n;
  float fro = 0.f;
#pragma unroll 8
  for (int e = tid; e < melem; e += NT) {
    const int r = e / a.n, c = e - r * a.n;
    const size_t off = g.offset(r, c);
    const float v = a.A1[off] + a2(off, r, c);
    C[g.cidx(r, c, ldc)] = v;
    fro = fmaf(v, v, fro);
  }
  fro = block_sum<NT>(fro, s.red);
  if constexpr (NT == 32) __syncwarp();
  PHASE(SLOT, 0);
  const float thr = a.tau * a.tau;
  const int n8 = (nn + 7) & ~7;
  float c_skip = 0.f;  // shift of the zero-rank Cholesky test (0: no test)
  int k = 0;
  bool skipped = false;
  float gbound = fro;  // trace(G) >= lambda_max(G)
  float fl = 0.f;      // flops of the steps run (see fl_symv in lanczos.cuh)
  if (a.skip_bound && fro <= thr) skipped = true;
  if (!skipped) {
    fl += (float)(mm * nn * (nn + 1));  // lower triangle of G
    if ((nn & 3) == 0) {
      // 4x4 register tiles of the lower triangle: per row of C one 128-bit
      // load for the tile's rows and one for its columns, 16 FMAs
      const int nt = nn >> 2, ntiles = nt * (nt + 1) / 2;
      for (int t = tid; t < ntiles; t += NT) {
        const int ta = tri_row(t), tb = t - (ta * (ta + 1)) / 2;
        float acc[4][4] = {};
        const float* ci = C + 4 * ta;
        const float* cj = C + 4 * tb;
#pragma unroll 4
        for (int r = 0; r < mm; ++r) {
          const float4 x = *reinterpret_cast<const float4*>(ci + r * ldc);
          const float4 y = *reinterpret_cast<const float4*>(cj + r * ldc);
          const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xv[u], yv[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (ta > tb || v <= u) G[(4 * ta + u) * ldg + 4 * tb + v] = acc[u][v];
      }
    } else {
      const int ntri = nn * (nn + 1) / 2;
      for (int e = tid; e < ntri; e += NT) {
        const int i = tri_row(e), j = e - (i * (i + 1)) / 2;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int r = 0;
        for (; r + 3 < mm; r += 4) {
          a0 = fmaf(C[r * ldc + i], C[r * ldc + j], a0);
          a1 = fmaf(C[(r + 1) * ldc + i], C[(r + 1) * ldc + j], a1);
          a2 = fmaf(C[(r + 2) * ldc + i], C[(r + 2) * ldc + j], a2);
          a3 = fmaf(C[(r + 3) * ldc + i], C[(r + 3) * ldc + j], a3);
        }
        for (; r < mm; ++r) a0 = fmaf(C[r * ldc + i], C[r * ldc + j], a0);
        G[i * ldg + j] = (a0 + a1) + (a2 + a3);
      }
    }
    __syncthreads();
    PHASE(SLOT, 1);
    if (a.skip_bound) {
      // Gershgorin: sigma_max^2 = lambda_max(G) <= max_i sum_j |G_ij|
      float rs = 0.f;
      for (int i = tid; i < nn; i += NT) {
        float t = 0.f;
        for (int j = 0; j <= i; ++j) t += fabsf(G[i * ldg + j]);
        for (int j = i + 1; j < nn; ++j) t += fabsf(G[j * ldg + i]);
        rs = fmaxf(rs, t);
      }
      rs = block_max<NT>(rs, s.red);
      if constexpr (NT == 32) __syncwarp();
      gbound = fminf(gbound, rs);
      fl += (float)fl_symv(nn);
      if (rs <= thr) {
        skipped = true;
      } else {
        // certified lambda_max(G) < tau^2 by Cholesky of (tau^2 - margin) I - G
        c_skip = thr - (float)(n8 * n8) * FLT_EPSILON * (thr + rs);
      }
    }
  }
  PHASE(SLOT, 2);
  // Two certificates share one Cholesky call site: attempt 0 tests
  // lambda_max(G) < tau^2 (zero rank), attempt 1 certifies the Lanczos pairs
  // by the deflated matrix (G stays intact for the fallback).
  bool lanczos_ok = false;
  // (blocks of width <= 16: the Householder path below is cheaper than
  // Lanczos for candidates that fail the zero-rank test)
  for (int attempt = 0; attempt < kAttempts && !skipped && a.skip_bound; ++attempt) {
    float c0 = c_skip;
    int kk = 0, ku = 0;
    if (attempt == 0) {
      if (!(c_skip > 0.f)) continue;
    } else if constexpr (kAttempts == 2) {
      int J = 0;
      kk = lanczos_candidates<NT, NMAX>(LowerFull{G, ldg}, nn, thr, gbound, Qs,
                                        nn < JCAP ? nn : JCAP, Us, nullptr, 0,
                                        0x51ED27u + 131u * job_block(a, b), s, z, panel, &ku, &c0,
                                        5 + SLOT, &J);
      fl += (float)fl_lanczos(nn, J, ku);
      PHASE(SLOT, 10);
      if (kk < 0) break;
      fl += (float)fl_deflate(nn, ku);
    }
    fl += (float)fl_chol(nn);
    const bool pd = regchol_pd<NT, NMAX>(LowerFull{G, ldg}, nn, c0, attempt == 1, panel,
                                         panel + 8 * n8, attempt == 1 ? ku : 0, panel + 16 * n8,
                                         s.red, attempt == 1 ? 5 + SLOT : -1);
    __syncthreads();
    PHASE(SLOT, 8 + attempt);
    if (pd) {
      skipped = attempt == 0;
      lanczos_ok = attempt == 1;
      k = kk;
    }
  }
  PHASE(SLOT, 7);
  if (!skipped && !lanczos_ok) {
    LowerFull Gacc{G, ldg};
    tridiagonalize<NT>(Gacc, nn, s);
    PHASE(SLOT, 3);
    float tn = 0.f;
    k = top_eigenvalues<NT>(nn, thr, s, &tn);
    PHASE(SLOT, 4);
    if (k > 0) top_eigenvectors<NT, NMAX>(Gacc, nn, k, tn, s, Y, ldy, SLOT);
    fl += (float)fl_householder(nn, k);
    PHASE(SLOT, 5);
  }
  const bool transposed = g.transposed();
  if (k == 0) {
    for (int e = tid; e < melem; e += NT) {
      const int r = e / a.n, c = e - r * a.n;
      const size_t off = g.offset(r, c);
      a.Zout[off] = 0.f;
      if (a.Wout) a.Wout[off] = -C[g.cidx(r, c, ldc)];
    }
    if (tid == 0) {
      if (a.rank_out) a.rank_out[b] = 0;
      if (a.cnt) {
        if (fl > 0.f) atomicAdd(a.cnt + 5, (unsigned long long)fl);
        if (skipped) atomicAdd(a.cnt, 1ull);
        atomicAdd(a.cnt + 1, 1ull);
        if (lanczos_ok) atomicAdd(a.cnt + 2, 1ull);
        else if (!skipped) atomicAdd(a.cnt + 3, 1ull);
      }
    }
    return;
  }
  // eigenvector q, entry c, at Vb[c * vsc + q * vsq]: the Ritz vectors in
  // place (column-major) or the Householder output Y (row-major)
  const float* Vb = lanczos_ok ? Us : Y;
  const int vsc = lanczos_ok ? 1 : ldy, vsq = lanczos_ok ? nn : 1;
  // f_j = 1 - tau / sigma_j for the k eigenpairs above the threshold
  if (tid < k) {
    const float sig = sqrtf(s.lam[tid]);
    s.xs[tid] = fmaxf(1.f - a.tau / sig, 0.f);
    s.lo[tid] = fmaxf(sig - a.tau, 0.f);
  }
  __syncthreads();
  // P = C V diag(f)   (mm x k, row stride nn)
  for (int e = tid; e < mm * k; e += NT) {
    const int i = e / k, q = e - i * k;
    float acc = 0.f;
    for (int c = 0; c < nn; ++c) acc = fmaf(C[i * ldc + c], Vb[c * vsc + q * vsq], acc);
    P[i * nn + q] = acc * s.xs[q];
  }
  __syncthreads();
  // Z' = P V^T, scattered through Shift_{-s}; W' = 2 Z' - A
  for (int e = tid; e < melem; e += NT) {
    const int r = e / a.n, c = e - r * a.n;
    const int i = transposed ? c : r, col = transposed ? r : c;
    float z = 0.f;
    for (int q = 0; q < k; ++q) z = fmaf(P[i * nn + q], Vb[col * vsc + q * vsq], z);
    const size_t off = g.offset(r, c);
    a.Zout[off] = z;
    if (a.Wout) a.Wout[off] = 2.f * z - C[i * ldc + col];
  }
  PHASE(SLOT, 6);
  if (tid == 0) {
    if (a.rank_out) a.rank_out[b] = k;
    if (a.cnt) {
      atomicAdd(a.cnt + 5, (unsigned long long)(fl + 4.f * (float)(mm * nn * k)));  // + rebuild
      if (lanczos_ok) atomicAdd(a.cnt + 2, 1ull);
      else atomicAdd(a.cnt + 3, 1ull);
    }
    if (a.nuc_acc) {
      double t = 0.0;
      for (int q = 0; q < k; ++q) t += (double)s.lo[q];
      atomicAdd(a.nuc_acc, t);
    }
  }
}

}  // namespace
}  // namespace msllr
