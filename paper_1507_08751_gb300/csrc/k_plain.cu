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
// Jacobi eigen-solve (one CTA, G packed in shared memory, V and Q in a
// global scratch that the launches on the one stream reuse) and the rebuild
// (a grid of row slabs).
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace msllr {

namespace {

constexpr int kPlainSmemN = 64;   // widest block solved by a 256-thread CTA (1024 above)
constexpr int kStageFloats = 8192;  // rows of C staged for the rebuild
constexpr int kMaxSweeps = 24;

__device__ __forceinline__ BlockGeom plain_geom(const ScaleLaunch& a, int b) {
  return block_geom(a, b);
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

// packed lower-triangle index of symmetric G(i, j)
__device__ __forceinline__ int tri(int i, int j) {
  return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i;
}

// Launch 2 of a block, one CTA: the eigen-decomposition G = V diag(lambda)
// V^T by the parallel cyclic Jacobi method (Golub & Van Loan, Sec. 8.5.4):
// each round rotates np / 2 disjoint pairs at once, so the new G is
// J^T G J with J their product, applied 2 x 2 block by 2 x 2 block (block
// (P1, P2) holds rows {p1, q1} and columns {p2, q2}: B' = R1^T B R2).  G is
// kept packed (lower triangle) in shared memory, V^T row by row in the
// global scratch.  Then Q = V diag(f) V^T with f_j = max(1 - tau /
// sqrt(lambda_j), 0).
template <int NT>
__global__ void __launch_bounds__(NT) plain_jacobi_kernel(ScaleLaunch a, int b, float* gscr) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x;
  const int nn = a.m < a.n ? a.m : a.n;
  const int nn2 = nn * nn;
  const float* Gin = gscr;  // full G from the Gram launch
  float* Vt = gscr + nn2;   // V^T: row j is eigenvector j
  float* Q = gscr + 2 * nn2;
  const int ntri = nn * (nn + 1) / 2;
  float* G = sm;                              // packed lower triangle
  float* red = sm + ((ntri + 3) & ~3);        // NT / 32 floats
  float* cs = red + NT / 32;                  // (c, s) per pair, then f_j
  for (int e = tid; e < ntri; e += NT) {
    int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    while (i * (i + 1) / 2 > e) --i;
    G[e] = Gin[i * nn + (e - i * (i + 1) / 2)];
  }
  for (int e = tid; e < nn2; e += NT) Vt[e] = (e / nn == e % nn) ? 1.f : 0.f;
  __syncthreads();

  // sweeps of np - 1 rounds (an odd width pairs the last index with a dummy
  // that no rotation touches) until the off-diagonal part is below 1e-6 of
  // ||G||_F, or a sweep has stopped reducing it (rounding level reached)
  const int np = (nn + 1) & ~1, npairs = np / 2;
  const int nblk = npairs * (npairs + 1) / 2;
  float off_prev = 0.f;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    float off = 0.f, tot = 0.f;
    for (int e = tid; e < ntri; e += NT) {
      const float v = G[e];
      int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      while (i * (i + 1) / 2 > e) --i;
      const bool diag = e == i * (i + 1) / 2 + i;
      tot = fmaf(diag ? v : 2.f * v, v, tot);
      if (!diag) off = fmaf(2.f * v, v, off);
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
          const float apq = G[tri(p, q)];
          if (apq != 0.f) {
            const float theta = (G[tri(q, q)] - G[tri(p, p)]) / (2.f * apq);
            const float tt = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(1.f + theta * theta));
            c = 1.f / sqrtf(1.f + tt * tt);
            s = tt * c;
          }
        }
        cs[2 * t] = c;
        cs[2 * t + 1] = s;
      }
      __syncthreads();
      // G <- J^T G J, one 2 x 2 block (P1 >= P2) per item
      for (int e = tid; e < nblk; e += NT) {
        int P1 = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
        while ((P1 + 1) * (P1 + 2) / 2 <= e) ++P1;
        while (P1 * (P1 + 1) / 2 > e) --P1;
        const int P2 = e - P1 * (P1 + 1) / 2;
        int p1, q1, p2, q2;
        rr_pair(np, k, P1, &p1, &q1);
        rr_pair(np, k, P2, &p2, &q2);
        const float c1 = cs[2 * P1], s1 = cs[2 * P1 + 1];
        const float c2 = cs[2 * P2], s2 = cs[2 * P2 + 1];
        if (P1 == P2) {
          if (p1 >= nn || q1 >= nn) continue;
          const float gpp = G[tri(p1, p1)], gqq = G[tri(q1, q1)], gpq = G[tri(p1, q1)];
          // [c -s; s c] [gpp gpq; gpq gqq] [c s; -s c]; the off-diagonal is zeroed
          G[tri(p1, p1)] = c1 * (c1 * gpp - s1 * gpq) - s1 * (c1 * gpq - s1 * gqq);
          G[tri(q1, q1)] = s1 * (s1 * gpp + c1 * gpq) + c1 * (s1 * gpq + c1 * gqq);
          G[tri(p1, q1)] = 0.f;
        } else {
          // rows {p1, q1} x columns {p2, q2}; an index past nn (the dummy)
          // has no entries
          const bool r0 = p1 < nn, r1 = q1 < nn, k0 = p2 < nn, k1 = q2 < nn;
          const float b00 = (r0 && k0) ? G[tri(p1, p2)] : 0.f;
          const float b01 = (r0 && k1) ? G[tri(p1, q2)] : 0.f;
          const float b10 = (r1 && k0) ? G[tri(q1, p2)] : 0.f;
          const float b11 = (r1 && k1) ? G[tri(q1, q2)] : 0.f;
          // left: rows p1, q1 by R1^T
          const float t00 = c1 * b00 - s1 * b10, t01 = c1 * b01 - s1 * b11;
          const float t10 = s1 * b00 + c1 * b10, t11 = s1 * b01 + c1 * b11;
          // right: columns p2, q2 by R2
          if (r0 && k0) G[tri(p1, p2)] = c2 * t00 - s2 * t01;
          if (r0 && k1) G[tri(p1, q2)] = s2 * t00 + c2 * t01;
          if (r1 && k0) G[tri(q1, p2)] = c2 * t10 - s2 * t11;
          if (r1 && k1) G[tri(q1, q2)] = s2 * t10 + c2 * t11;
        }
      }
      // V <- V J: rows p, q of V^T
      for (int e = tid; e < npairs * nn; e += NT) {
        const int t = e / nn, i = e - t * nn;
        int p, q;
        rr_pair(np, k, t, &p, &q);
        if (p >= nn || q >= nn) continue;
        const float c = cs[2 * t], s = cs[2 * t + 1];
        const float vp = Vt[p * nn + i], vq = Vt[q * nn + i];
        Vt[p * nn + i] = c * vp - s * vq;
        Vt[q * nn + i] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }

  // soft threshold of the singular values sigma_j = sqrt(lambda_j)
  float* f = cs;
  for (int j = tid; j < nn; j += NT) {
    const float sig = sqrtf(fmaxf(G[tri(j, j)], 0.f));
    f[j] = sig > a.tau ? 1.f - a.tau / sig : 0.f;
  }
  __syncthreads();
  if (tid == 0) {
    int k = 0;
    double nuc = 0.0;
    for (int j = 0; j < nn; ++j)
      if (f[j] > 0.f) {
        ++k;
        nuc += (double)(sqrtf(fmaxf(G[tri(j, j)], 0.f)) - a.tau);
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
      if (f[j] > 0.f) acc = fmaf(Vt[j * nn + c] * f[j], Vt[j * nn + d], acc);
    Q[e] = acc;
  }
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
  const size_t ntri = ((size_t)nn * (nn + 1) / 2 + 3) & ~(size_t)3;
  return sizeof(float) * (ntri + 1024 / 32 + 2 * ((size_t)nn + 2));
}

}  // namespace

size_t plain_scratch_bytes(int m, int n) {
  const int nn = m < n ? m : n;
  return sizeof(float) * 3 * (size_t)nn * nn;
}

cudaError_t configure_plain_kernels() {
  cudaError_t e = cudaFuncSetAttribute(plain_jacobi_kernel<256>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)plain_smem_bytes(kPlainSmemN));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(plain_jacobi_kernel<1024>,
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
    if (nn <= kPlainSmemN) plain_jacobi_kernel<256><<<1, 256, smem, st>>>(s, b, scratch);
    else plain_jacobi_kernel<1024><<<1, 1024, smem, st>>>(s, b, scratch);
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
