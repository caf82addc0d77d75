// The plain FP32 comparator of the block SVT (eq:bsvt under the Sec. 9
// shift): the blocks one after another, each by its own launches, with
// textbook steps and nothing skipped --
//   G = C^T C of the gathered block (C = R_b(Shift_s(A)), or its transpose
//   for wide blocks, since SVT(B^T) = SVT(B)^T),
//   eigen-decomposition of G by the cyclic Jacobi method with the
//   round-robin (tournament) pair ordering (Golub & Van Loan, Sec. 8.5),
//   sigma_j = sqrt(lambda_j), f_j = max(1 - tau / sigma_j, 0) (eq:svt),
//   Z' = C V diag(f) V^T scattered through Shift_{-s}, W' = 2 Z' - A.
// It exists to be timed beside the optimised path (msllr_params.plain): no
// skip bound, no certificate, no batching of blocks into one launch.  Per
// block three launches: the Gram matrix (a grid of 16 x 16 tiles), the
// Jacobi eigen-solve (one CTA; G and V in shared memory up to 64 wide, else
// in a global scratch that the launches on the one stream reuse) and the
// rebuild (a grid of row slabs).
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace msllr {

namespace {

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

// sum over the CTA (NT threads; red holds NT / 32 floats)
template <int NT>
__device__ __forceinline__ float cta_sum(float v, float* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  for (int i = 0; i < NT / 32; ++i) t += red[i];
  __syncthreads();
  return t;
}

// Launch 1 of a block: G = C^T C, one 16 x 16 tile of G per CTA, the rows
// of C streamed through shared memory 16 at a time.
__global__ void __launch_bounds__(256) plain_gram_kernel(ScaleLaunch a, int b, float* G) {
  __shared__ float ci[16][17], cj[16][17];
  const BlockGeom g = plain_geom(a, b);
  const int mm = g.mm(), nn = g.nn();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = 16 * blockIdx.y, j0 = 16 * blockIdx.x;
  float acc = 0.f;
  for (int r0 = 0; r0 < mm; r0 += 16) {
    const int r = r0 + ty;
    ci[ty][tx] = (r < mm && i0 + tx < nn) ? plain_c(a, g, r, i0 + tx) : 0.f;
    cj[ty][tx] = (r < mm && j0 + tx < nn) ? plain_c(a, g, r, j0 + tx) : 0.f;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t) acc = fmaf(ci[t][ty], cj[t][tx], acc);
    __syncthreads();
  }
  if (i0 + ty < nn && j0 + tx < nn) G[(i0 + ty) * nn + j0 + tx] = acc;
}

// Launch 2 of a block, one CTA: the eigen-decomposition G = V diag(lambda)
// V^T by the cyclic Jacobi method, then Q = V diag(f) V^T with
// f_j = max(1 - tau / sqrt(lambda_j), 0).  G, V in shared memory for blocks
// up to 64 wide (NT = 256 threads), else in the global scratch (NT = 1024).
template <bool SMEM, int NT>
__global__ void __launch_bounds__(NT) plain_jacobi_kernel(ScaleLaunch a, int b, float* gscr) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x;
  const int nn = a.m < a.n ? a.m : a.n;
  const int nn2 = nn * nn;
  float* G = SMEM ? sm : gscr;
  float* V = G + nn2;
  float* Q = gscr + 2 * nn2;
  float* red = SMEM ? V + nn2 : sm;  // 32 floats
  float* cs = red + 32;              // rotation (c, s) per pair, then f_j
  for (int e = tid; e < nn2; e += NT) {
    if (SMEM) G[e] = gscr[e];
    V[e] = (e / nn == e % nn) ? 1.f : 0.f;
  }
  __syncthreads();

  // cyclic Jacobi: sweeps of np - 1 rounds of disjoint rotations (an odd
  // width pairs the last index with a dummy that no rotation touches) until
  // the off-diagonal part is below 1e-6 of ||G||_F, or a sweep has stopped
  // reducing it (rounding level reached)
  const int np = (nn + 1) & ~1, npairs = np / 2;
  float off_prev = 0.f;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    float off = 0.f, tot = 0.f;
    for (int e = tid; e < nn2; e += NT) {
      const float v = G[e];
      tot = fmaf(v, v, tot);
      if (e / nn != e % nn) off = fmaf(v, v, off);
    }
    off = cta_sum<NT>(off, red);
    tot = cta_sum<NT>(tot, red);
    if (!(off > 1e-12f * tot)) break;
    if (sweep > 0 && !(off < 0.9f * off_prev)) break;
    off_prev = off;
    for (int k = 0; k < np - 1; ++k) {
      // rotation of each pair (Golub & Van Loan, Alg. 8.5.1, sym.schur2)
      for (int t = tid; t < npairs; t += NT) {
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
      for (int e = tid; e < npairs * nn; e += NT) {
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
      for (int e = tid; e < npairs * nn; e += NT) {
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

  // soft threshold of the singular values sigma_j = sqrt(lambda_j)
  float* f = cs;
  for (int j = tid; j < nn; j += NT) {
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
  // Q = V diag(f) V^T
  for (int e = tid; e < nn2; e += NT) {
    const int c = e / nn, d = e - c * nn;
    float acc = 0.f;
    for (int j = 0; j < nn; ++j)
      if (f[j] > 0.f) acc = fmaf(V[c * nn + j] * f[j], V[d * nn + j], acc);
    Q[e] = acc;
  }
  __syncthreads();
}

// Launch 3 of a block: Z' = C Q for a slab of rows per CTA (C staged, so that
// the in-place write of Z' never overtakes a read of A), W' = 2 Z' - A.
__global__ void __launch_bounds__(256) plain_rebuild_kernel(ScaleLaunch a, int b,
                                                            const float* __restrict__ Q) {
  __shared__ float stage[kStageFloats];
  const BlockGeom g = plain_geom(a, b);
  const int mm = g.mm(), nn = g.nn();
  const int rs = kStageFloats / nn;
  const int r0 = blockIdx.x * rs;
  const int rows = min(rs, mm - r0);
  for (int e = threadIdx.x; e < rows * nn; e += 256) {
    const int i = e / nn, c = e - i * nn;
    stage[e] = plain_c(a, g, r0 + i, c);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * nn; e += 256) {
    const int i = e / nn, c = e - i * nn;
    float z = 0.f;
    for (int d = 0; d < nn; ++d) z = fmaf(stage[i * nn + d], Q[d * nn + c], z);
    const size_t off = g.transposed() ? g.offset(c, r0 + i) : g.offset(r0 + i, c);
    a.Zout[off] = z;
    if (a.Wout) a.Wout[off] = 2.f * z - stage[e];
  }
}

size_t plain_smem_bytes(int nn) {
  const size_t small = nn <= kPlainSmemN ? 2 * (size_t)nn * nn : 0;
  return sizeof(float) * (small + 32 + 2 * ((size_t)nn + 2));
}

}  // namespace

size_t plain_scratch_bytes(int m, int n) {
  const int nn = m < n ? m : n;
  return sizeof(float) * 3 * (size_t)nn * nn;
}

cudaError_t configure_plain_kernels() {
  cudaError_t e = cudaFuncSetAttribute(plain_jacobi_kernel<true, 256>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)plain_smem_bytes(kPlainSmemN));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(plain_jacobi_kernel<false, 1024>,
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
  if (!scratch) return cudaErrorInvalidValue;
  const int nn = s.m < s.n ? s.m : s.n, mm = s.m < s.n ? s.n : s.m;
  const int nblocks = (s.M / s.m) * (s.N / s.n);
  const int T = (nn + 15) / 16;
  const int slabs = (mm + kStageFloats / nn - 1) / (kStageFloats / nn);
  const size_t smem = plain_smem_bytes(nn);
  for (int b = 0; b < nblocks; ++b) {
    if (prof)
      if (cudaError_t e = prof->before(st, KK_GRAM)) return e;
    plain_gram_kernel<<<dim3(T, T), 256, 0, st>>>(s, b, scratch);
    if (prof)
      if (cudaError_t e = prof->after(st)) return e;
    if (prof)
      if (cudaError_t e = prof->before(st, KK_EIG)) return e;
    if (nn <= kPlainSmemN) plain_jacobi_kernel<true, 256><<<1, 256, smem, st>>>(s, b, scratch);
    else plain_jacobi_kernel<false, 1024><<<1, 1024, smem, st>>>(s, b, scratch);
    if (prof)
      if (cudaError_t e = prof->after(st)) return e;
    if (prof)
      if (cudaError_t e = prof->before(st, KK_REBUILD)) return e;
    plain_rebuild_kernel<<<slabs, 256, 0, st>>>(s, b, scratch + 2 * (size_t)nn * nn);
    if (prof)
      if (cudaError_t e = prof->after(st)) return e;
  }
  return cudaGetLastError();
}

}  // namespace msllr
