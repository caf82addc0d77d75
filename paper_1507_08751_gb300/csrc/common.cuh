// Small device helpers shared by the msllr kernels: warp/CTA reductions and
// the cycle-spin index map of Sec. 9.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace msllr {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA; every thread gets the total.  `red` is shared scratch of
// at least NT/32 floats.  Contains two __syncthreads (all threads must call).
template <int NT>
__device__ __forceinline__ float block_sum(float v, float* red) {
  v = warp_sum(v);
  if constexpr (NT == 32) {
    return v;
  } else {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) t += red[i];
    __syncthreads();
    return t;
  }
}

template <int NT>
__device__ __forceinline__ float block_max(float v, float* red) {
  v = warp_max(v);
  if constexpr (NT == 32) {
    return v;
  } else {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    float t = red[0];
#pragma unroll
    for (int i = 1; i < NT / 32; ++i) t = fmaxf(t, red[i]);
    __syncthreads();
    return t;
  }
}

// Geometry of one block of a scale on the cycle-spun grid (Sec. 9):
// element (r, c) of shifted block (p, q) is A[(p*m + r + sr) mod M,
// (q*n + c + sc) mod N].  `C` is the block as the eigen-solver sees it:
// mm x nn with nn = min(m, n); for a wide block (m < n) C is its transpose,
// since SVT(B^T) = SVT(B)^T.
// Spatio-temporal blocks (Sec. 10.2, fw > 0): the rows of the matrix are the
// pixels of an fh x fw frame (row y fw + x for pixel (y, x)) and its columns
// the frames; block (p, q) is the bh x bw pixel patch p (patches in
// row-major order) over the frames q n .. q n + n - 1, its row r the patch
// pixel (r / bw, r mod bw), so m = bh bw.  The shift moves the video cube
// circularly by (sy, sx) = divmod(sr, fw) pixels and sc frames.
struct BlockGeom {
  int M, N, ld;     // matrix shape and row stride (elements)
  int m, n;         // block shape
  int p, q;         // block coordinates on the shifted grid
  int sr, sc;       // shift
  int fw, fh, bh, bw, sy, sx;  // spatio-temporal blocks (fw = 0: none)
  int rbase;                    // batched jobs: first row of the block's job
  __device__ __forceinline__ int mm() const { return m >= n ? m : n; }
  __device__ __forceinline__ int nn() const { return m >= n ? n : m; }
  __device__ __forceinline__ bool transposed() const { return m < n; }
  // global element offset of block element (r, c), natural orientation
  __device__ __forceinline__ size_t offset(int r, int c) const {
    int gr;
    if (fw) {
      const int pw = fw / bw, py = p / pw, px = p - py * pw;
      const int iy = r / bw, ix = r - iy * bw;
      int y = py * bh + iy + sy;
      if (y >= fh) y -= fh;
      int x = px * bw + ix + sx;
      if (x >= fw) x -= fw;
      gr = y * fw + x;
    } else {
      gr = p * m + r + sr;
      if (gr >= M) gr -= M;
    }
    int gc = q * n + c + sc;
    if (gc >= N) gc -= N;
    return (size_t)(rbase + gr) * ld + gc;
  }
  // index into the row-major mm x nn matrix C of block element (r, c)
  __device__ __forceinline__ int cidx(int r, int c, int ldc) const {
    return m >= n ? r * ldc + c : c * ldc + r;
  }
};

// Block b of the scale described by a launch (row-major block order on the
// shifted grid; with batched jobs, the jobs' block grids one above the other,
// each job shifted by its own pair and wrapped within its own rows).  The
// full-matrix scale ignores the shift: SVT commutes with row and column
// permutations.  GEN false: the caller promises a single job of 2-D blocks
// (a.fw == 0, a.rows == 0), and the compiler drops the spatio-temporal and
// batch index arithmetic from that instantiation.
template <bool GEN, class SL>
__device__ __forceinline__ BlockGeom block_geom_t(const SL& a, int b) {
  BlockGeom g;
  const int rows = (GEN && a.rows) ? a.rows : a.M;
  g.M = rows;
  g.N = a.N;
  g.ld = a.ld;
  g.m = a.m;
  g.n = a.n;
  const int nbn = a.N / a.n;
  g.p = b / nbn;
  g.q = b - g.p * nbn;
  int job = 0;
  if (GEN && a.rows) {
    const int pj = rows / a.m;
    job = g.p / pj;
    g.p -= job * pj;
  }
  g.rbase = job * rows;
  const int fw = GEN ? a.fw : 0;
  const int* sh = a.shift ? a.shift + 2 * job : nullptr;
  const bool full = (a.m == rows && a.n == a.N && !fw);
  g.sr = (sh && !full) ? (sh[0] + a.shift_add_r) % rows : 0;
  g.sc = (sh && !full) ? (sh[1] + a.shift_add_c) % a.N : 0;
  g.fw = fw;
  g.fh = fw ? rows / fw : 0;
  g.bw = fw ? a.bw : 0;
  g.bh = fw ? a.m / a.bw : 0;
  g.sy = fw ? g.sr / fw : 0;
  g.sx = fw ? g.sr - g.sy * fw : 0;
  return g;
}

template <class SL>
__device__ __forceinline__ BlockGeom block_geom(const SL& a, int b) {
  return block_geom_t<true>(a, b);
}

// Optional per-phase timing (debug aid, enabled by the MSLLR_PHASE_TIMING
// environment variable): thread 0 of every CTA adds clock64() deltas between
// phase marks to acc[(slot * 16 + phase) * 2] and counts to the next entry.
// Each translation unit holds its own pointer, set by set_phase_buffer_*().
static __device__ unsigned long long* g_phase_acc = nullptr;
#define PHASE_INIT() long long ph_t_ = (g_phase_acc && threadIdx.x == 0) ? clock64() : 0
#define PHASE(slot, p)                                                         \
  do {                                                                         \
    if (g_phase_acc && threadIdx.x == 0 && (slot) >= 0) {                      \
      const long long t_ = clock64();                                          \
      atomicAdd(&g_phase_acc[((slot) * 16 + (p)) * 2], (unsigned long long)(t_ - ph_t_)); \
      atomicAdd(&g_phase_acc[((slot) * 16 + (p)) * 2 + 1], 1ull);              \
      ph_t_ = t_;                                                              \
    }                                                                          \
  } while (0)

// adds `v` to the accumulator of (slot, phase) and counts one (debug aid)
#define PHASE_ADD(slot, p, v)                                                    \
  do {                                                                           \
    if (g_phase_acc && (slot) >= 0) {                                            \
      atomicAdd(&g_phase_acc[((slot) * 16 + (p)) * 2], (unsigned long long)(v)); \
      atomicAdd(&g_phase_acc[((slot) * 16 + (p)) * 2 + 1], 1ull);                \
    }                                                                            \
  } while (0)

}  // namespace msllr
