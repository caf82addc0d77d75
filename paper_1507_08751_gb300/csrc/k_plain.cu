// The plain FP32 comparator of the block SVT (eq:bsvt under the Sec. 9
// shift): one kernel launch per block, one CTA, textbook steps and nothing
// skipped --
//   G = C^T C of the gathered block (C = R_b(Shift_s(A)), or its transpose
//   for wide blocks, since SVT(B^T) = SVT(B)^T),
//   eigen-decomposition of G by the cyclic Jacobi method with the
//   round-robin (tournament) pair ordering (Golub & Van Loan, Sec. 8.5),
//   sigma_j = sqrt(lambda_j), f_j = max(1 - tau / sigma_j, 0) (eq:svt),
//   Z' = C V diag(f) V^T scattered through Shift_{-s}, W' = 2 Z' - A.
// It exists to be timed beside the optimised path (msllr_params.plain): no
// skip bound, no certificate, no batching of blocks into one launch.  Blocks
// up to 64 wide keep G, V and Q = V diag(f) V^T in shared memory; wider ones
// (up to 256) keep them in a global scratch that consecutive launches on the
// one stream reuse.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace msllr {

namespace {

constexpr int kPT = 256;          // threads of the one CTA
constexpr int kPlainSmemN = 64;   // widest block with G, V, Q in shared memory
constexpr int kStageFloats = 8192;  // rows of C staged for the rebuild
constexpr int kMaxSweeps = 24;

__device__ __forceinline__ BlockGeom plain_geom(const ScaleLaunch& a, int b) {
  BlockGeom g;
  g.M = a.M;
  g.N = a.N;
  g.ld = a.ld;
  g.m = a.m;
  g.n = a.n;
  const int nbn = a.N / a.n;
  g.p = b / nbn;
  g.q = b - g.p * nbn;
  g.sr = a.shift ? a.shift[0] % a.M : 0;
  g.sc = a.shift ? a.shift[1] % a.N : 0;
  return g;
}

// element (i, c) of C = the block (m >= n) or its transpose
__device__ __forceinline__ float plain_c(const ScaleLaunch& a, const BlockGeom& g, int i, int c) {
  const size_t off = g.transposed() ? g.offset(c, i) : g.offset(i, c);
  float v = a.A1[off];
  if (a.A2) v += a.A2[off];
  return v;
}

// Pair t of round k of the round-robin ordering of np (even) indices: index
// np - 1 stays put, the others turn one place per round, so every pair
// meets exactly once in np - 1 rounds.
__device__ __forceinline__ void rr_pair(int np, int k, int t, int* p, int* q) {
  const int r = np - 1;
  if (t == 0) {
    *p = r;
    *q = k % r;
  } else {
    *p = (k + t) % r;
    *q = (k - t + r) % r;
  }
}

__device__ __forceinline__ float cta_sum(float v, float* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  for (int i = 0; i < kPT / 32; ++i) t += red[i];
  __syncthreads();
  return t;
}

template <bool SMEM>
__global__ void __launch_bounds__(kPT) plain_block_kernel(ScaleLaunch a, int b, float* gscr) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x;
  const BlockGeom g = plain_geom(a, b);
  const int mm = g.mm(), nn = g.nn();
  const int nn2 = nn * nn;
  float* G = SMEM ? sm : gscr;
  float* V = G + nn2;
  float* Q = V + nn2;
  float* red = SMEM ? Q + nn2 : sm;  // 8 floats
  float* cs = red + 8;               // rotation (c, s) per pair, then f_j
  float* stage = cs + 2 * (nn + 2);  // staged rows of C

  // 1. G = C^T C (both triangles), V = I
  for (int e = tid; e < nn2; e += kPT) {
    const int i = e / nn, j = e - i * nn;
    V[e] = i == j ? 1.f : 0.f;
    if (j > i) continue;
    float acc = 0.f;
    for (int r = 0; r < mm; ++r) acc = fmaf(plain_c(a, g, r, i), plain_c(a, g, r, j), acc);
    G[i * nn + j] = acc;
    G[j * nn + i] = acc;
  }
  __syncthreads();

  // 2. cyclic Jacobi: sweeps of np - 1 rounds of disjoint rotations (an odd
  // width pairs the last index with a dummy that no rotation touches) until
  // the off-diagonal part is below 1e-6 of ||G||_F, or a sweep has stopped
  // reducing it (rounding level reached)
  const int np = (nn + 1) & ~1, npairs = np / 2;
  float off_prev = 0.f;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    float off = 0.f, tot = 0.f;
    for (int e = tid; e < nn2; e += kPT) {
      const float v = G[e];
      tot = fmaf(v, v, tot);
      if (e / nn != e % nn) off = fmaf(v, v, off);
    }
    off = cta_sum(off, red);
    tot = cta_sum(tot, red);
    if (!(off > 1e-12f * tot)) break;
    if (sweep > 0 && !(off < 0.9f * off_prev)) break;
    off_prev = off;
    for (int k = 0; k < np - 1; ++k) {
      // rotation of each pair (Golub & Van Loan, Alg. 8.5.1, sym.schur2)
      for (int t = tid; t < npairs; t += kPT) {
        int p, q;
        rr_pair(np, k, t, &p, &q);
        float c = 1.f, s = 0.f;
        if (p < nn && q < nn) {
          const float apq = G[p * nn + q];
          if (apq != 0.f) {
            const float theta = (G[q * nn + q] - G[p * nn + p]) / (2.f * apq);
            const float tt = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(1.f + theta * theta));
            c = 1.f / sqrtf(1.f + tt * tt);
            s = tt * c;
          }
        }
        cs[2 * t] = c;
        cs[2 * t + 1] = s;
      }
      __syncthreads();
      // rows p, q  <-  J^T G
      for (int e = tid; e < npairs * nn; e += kPT) {
        const int t = e / nn, j = e - t * nn;
        int p, q;
        rr_pair(np, k, t, &p, &q);
        if (p >= nn || q >= nn) continue;
        const float c = cs[2 * t], s = cs[2 * t + 1];
        const float gp = G[p * nn + j], gq = G[q * nn + j];
        G[p * nn + j] = c * gp - s * gq;
        G[q * nn + j] = s * gp + c * gq;
      }
      __syncthreads();
      // columns p, q  <-  G J, and V J
      for (int e = tid; e < npairs * nn; e += kPT) {
        const int t = e / nn, i = e - t * nn;
        int p, q;
        rr_pair(np, k, t, &p, &q);
        if (p >= nn || q >= nn) continue;
        const float c = cs[2 * t], s = cs[2 * t + 1];
        const float gp = G[i * nn + p], gq = G[i * nn + q];
        G[i * nn + p] = c * gp - s * gq;
        G[i * nn + q] = s * gp + c * gq;
        const float vp = V[i * nn + p], vq = V[i * nn + q];
        V[i * nn + p] = c * vp - s * vq;
        V[i * nn + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }

  // 3. soft threshold of the singular values sigma_j = sqrt(lambda_j)
  float* f = cs;
  for (int j = tid; j < nn; j += kPT) {
    const float sig = sqrtf(fmaxf(G[j * nn + j], 0.f));
    f[j] = sig > a.tau ? 1.f - a.tau / sig : 0.f;
  }
  __syncthreads();
  if (tid == 0) {
    int k = 0;
    double nuc = 0.0;
    for (int j = 0; j < nn; ++j)
      if (f[j] > 0.f) {
        ++k;
        nuc += (double)(sqrtf(fmaxf(G[j * nn + j], 0.f)) - a.tau);
      }
    if (a.rank_out) a.rank_out[b] = k;
    if (a.nuc_acc && k > 0) atomicAdd(a.nuc_acc, nuc);
    if (a.cnt && k == 0) atomicAdd(a.cnt + 1, 1ull);
  }
  // 4. Q = V diag(f) V^T
  for (int e = tid; e < nn2; e += kPT) {
    const int c = e / nn, d = e - c * nn;
    float acc = 0.f;
    for (int j = 0; j < nn; ++j)
      if (f[j] > 0.f) acc = fmaf(V[c * nn + j] * f[j], V[d * nn + j], acc);
    Q[e] = acc;
  }
  __syncthreads();

  // 5. Z' = C Q row slab by row slab (C staged, so that the in-place write of
  // Z' never overtakes a read of A), W' = 2 Z' - A
  const int rs = kStageFloats / nn;
  for (int r0 = 0; r0 < mm; r0 += rs) {
    const int rows = min(rs, mm - r0);
    for (int e = tid; e < rows * nn; e += kPT) {
      const int i = e / nn, c = e - i * nn;
      stage[e] = plain_c(a, g, r0 + i, c);
    }
    __syncthreads();
    for (int e = tid; e < rows * nn; e += kPT) {
      const int i = e / nn, c = e - i * nn;
      float z = 0.f;
      for (int d = 0; d < nn; ++d) z = fmaf(stage[i * nn + d], Q[d * nn + c], z);
      const size_t off = g.transposed() ? g.offset(c, r0 + i) : g.offset(r0 + i, c);
      a.Zout[off] = z;
      if (a.Wout) a.Wout[off] = 2.f * z - stage[e];
    }
    __syncthreads();
  }
}

size_t plain_smem_bytes(int nn) {
  const size_t small = nn <= kPlainSmemN ? 3 * (size_t)nn * nn : 0;
  return sizeof(float) * (small + 8 + 2 * ((size_t)nn + 2) + kStageFloats);
}

}  // namespace

size_t plain_scratch_bytes(int m, int n) {
  const int nn = m < n ? m : n;
  return nn > kPlainSmemN ? sizeof(float) * 3 * (size_t)nn * nn : 0;
}

cudaError_t configure_plain_kernels() {
  cudaError_t e = cudaFuncSetAttribute(plain_block_kernel<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)plain_smem_bytes(kPlainSmemN));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(plain_block_kernel<false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)plain_smem_bytes(256));
}

cudaError_t launch_soft1x1(const ScaleLaunch& s, cudaStream_t st, Prof* prof);
cudaError_t launch_noise(const ScaleLaunch& s, cudaStream_t st, Prof* prof);

cudaError_t launch_plain(const ScaleLaunch& s, float* scratch, cudaStream_t st, Prof* prof) {
  switch (choose_path(s.m, s.n)) {
    case ScalePath::Elementwise:
      return launch_soft1x1(s, st, prof);
    case ScalePath::Noise:
      return launch_noise(s, st, prof);
    case ScalePath::Huge:
      return cudaErrorInvalidValue;
    default:
      break;
  }
  const int nn = s.m < s.n ? s.m : s.n;
  const int nblocks = (s.M / s.m) * (s.N / s.n);
  const bool in_smem = nn <= kPlainSmemN;
  if (!in_smem && !scratch) return cudaErrorInvalidValue;
  const size_t smem = plain_smem_bytes(nn);
  for (int b = 0; b < nblocks; ++b) {
    if (prof)
      if (cudaError_t e = prof->before(st, KK_FUSED)) return e;
    if (in_smem) plain_block_kernel<true><<<1, kPT, smem, st>>>(s, b, nullptr);
    else plain_block_kernel<false><<<1, kPT, smem, st>>>(s, b, scratch);
    if (prof)
      if (cudaError_t e = prof->after(st)) return e;
  }
  return cudaGetLastError();
}

}  // namespace msllr
