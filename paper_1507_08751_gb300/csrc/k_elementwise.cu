// Element-wise kernels of the ADMM (eq:admm, Sec. 7): the consensus
// residual of the X-update, the 1x1-scale soft threshold (eq:bsvt for 1x1
// blocks) and the noise-scale shrink (Sec. 2.1) with their fused dual
// updates, and the output X-update.
//
// ADMM state kept in HBM per scale: Z_i and W_i = Z_i - U_i.  With the
// consensus residual R = (1/L)(Y - sum_j W_j) (zero at unobserved entries,
// Sec. 10.4) the X-update is X_i = W_i + R, the prox input is
// A_i = X_i + U_i = Z_i + R, the dual update U_i' = A_i - Z_i' and the new
// state W_i' = Z_i' - U_i' = 2 Z_i' - A_i.
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "../../include/msllr.h"

namespace msllr {

int sm_count() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      return 152;
    }
    cache[dev] = n;
  }
  return cache[dev];
}

namespace {

constexpr int kEwThreads = 256;

int ew_grid(size_t n_items) {
  // enough CTAs for 8 resident per SM; grid-stride beyond that
  size_t g = (n_items + kEwThreads - 1) / kEwThreads;
  const size_t cap = (size_t)sm_count() * 8;
  return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

static_assert(MSLLR_MAX_SCALES == 8, "consensus dispatch covers 1..8 scales");

// Soft threshold of eq:bsvt for a 1x1 block and the fused dual update.
__device__ __forceinline__ void soft_update(float a, float tau, float& z, float& w) {
  z = copysignf(fmaxf(fabsf(a) - tau, 0.f), a);
  w = 2.f * z - a;
}

// R = (1/L)(Y - sum_j W_j), zero at unobserved entries.  With FUSE the
// 1x1 scale's block SVT runs in the same pass (the scale is element-wise,
// so the thread that forms R(i) can finish it): A = Z11(i) + R(i),
// Z11(i) = soft(A), W11(i) = 2 Z11(i) - A.  W11 is one of the W_j summed
// here; each element is read before the same thread overwrites it.
template <int LC, bool FUSE>  // the scale count, a compile-time constant so that all loads are in flight
__global__ void __launch_bounds__(kEwThreads)
consensus_kernel(const float* __restrict__ Y, const float* W, float* __restrict__ R,
                 const uint8_t* __restrict__ mask, size_t MN, float* Z11, float* W11,
                 float tau11) {
  constexpr int L = LC;
  const float invL = 1.f / (float)L;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((MN & 3) == 0) {
    const size_t n4 = MN >> 2;
    for (size_t i = i0; i < n4; i += stride) {
      float4 acc = reinterpret_cast<const float4*>(Y)[i];
      float4 w[L];
#pragma unroll
      for (int j = 0; j < L; ++j) w[j] = reinterpret_cast<const float4*>(W + (size_t)j * MN)[i];
      float4 z11;
      if (FUSE) z11 = reinterpret_cast<const float4*>(Z11)[i];
#pragma unroll
      for (int j = 0; j < L; ++j) {
        acc.x -= w[j].x;
        acc.y -= w[j].y;
        acc.z -= w[j].z;
        acc.w -= w[j].w;
      }
      acc.x *= invL;
      acc.y *= invL;
      acc.z *= invL;
      acc.w *= invL;
      if (mask) {
        const uchar4 mk = reinterpret_cast<const uchar4*>(mask)[i];
        if (!mk.x) acc.x = 0.f;
        if (!mk.y) acc.y = 0.f;
        if (!mk.z) acc.z = 0.f;
        if (!mk.w) acc.w = 0.f;
      }
      reinterpret_cast<float4*>(R)[i] = acc;
      if (FUSE) {
        float4 zo, wo;
        soft_update(z11.x + acc.x, tau11, zo.x, wo.x);
        soft_update(z11.y + acc.y, tau11, zo.y, wo.y);
        soft_update(z11.z + acc.z, tau11, zo.z, wo.z);
        soft_update(z11.w + acc.w, tau11, zo.w, wo.w);
        reinterpret_cast<float4*>(Z11)[i] = zo;
        reinterpret_cast<float4*>(W11)[i] = wo;
      }
    }
  } else {
    for (size_t i = i0; i < MN; i += stride) {
      float acc = Y[i];
      for (int j = 0; j < L; ++j) acc -= W[(size_t)j * MN + i];
      acc *= invL;
      if (mask && !mask[i]) acc = 0.f;
      R[i] = acc;
      if (FUSE) {
        float zo, wo;
        soft_update(Z11[i] + acc, tau11, zo, wo);
        Z11[i] = zo;
        W11[i] = wo;
      }
    }
  }
}

// 1x1 blocks: SVT of [a] is sign(a) max(|a| - tau, 0).  The scale is
// element-wise, so the cycle-spin shift does not change it and is not
// applied.  Optional statistics: sum |z| (the 1x1 block nuclear norm) and
// the count of zero outputs.
__global__ void __launch_bounds__(kEwThreads)
soft1x1_kernel(const float* A1, const float* __restrict__ A2, float* Zout, float* Wout, int M,
               int N, int ld, float tau, int* rank_out, double* nuc_acc,
               unsigned long long* cnt) {
  __shared__ double sred[kEwThreads / 32];
  __shared__ unsigned long long cred[kEwThreads / 32];
  const size_t MN = (size_t)M * N;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double nuc = 0.0;
  unsigned long long zeros = 0;
  const bool aligned = ((((uintptr_t)A1) | ((uintptr_t)A2) | ((uintptr_t)Zout) | ((uintptr_t)Wout)) & 15) == 0;
  if (aligned && ld == N && (MN & 3) == 0 && !rank_out) {
    const size_t n4 = MN >> 2;
    for (size_t i = i0; i < n4; i += stride) {
      float4 a = reinterpret_cast<const float4*>(A1)[i];
      if (A2) {
        const float4 b = reinterpret_cast<const float4*>(A2)[i];
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
      }
      float4 z;
      z.x = copysignf(fmaxf(fabsf(a.x) - tau, 0.f), a.x);
      z.y = copysignf(fmaxf(fabsf(a.y) - tau, 0.f), a.y);
      z.z = copysignf(fmaxf(fabsf(a.z) - tau, 0.f), a.z);
      z.w = copysignf(fmaxf(fabsf(a.w) - tau, 0.f), a.w);
      reinterpret_cast<float4*>(Zout)[i] = z;
      if (Wout) {
        float4 w;
        w.x = 2.f * z.x - a.x;
        w.y = 2.f * z.y - a.y;
        w.z = 2.f * z.z - a.z;
        w.w = 2.f * z.w - a.w;
        reinterpret_cast<float4*>(Wout)[i] = w;
      }
      if (nuc_acc) {
        nuc += (double)fabsf(z.x) + (double)fabsf(z.y) + (double)fabsf(z.z) + (double)fabsf(z.w);
        zeros += (z.x == 0.f) + (z.y == 0.f) + (z.z == 0.f) + (z.w == 0.f);
      }
    }
  } else {
    for (size_t i = i0; i < MN; i += stride) {
      const size_t r = i / (size_t)N, c = i - r * (size_t)N;
      const size_t off = r * (size_t)ld + c;
      float a = A1[off];
      if (A2) a += A2[off];
      const float z = copysignf(fmaxf(fabsf(a) - tau, 0.f), a);
      Zout[off] = z;
      if (Wout) Wout[off] = 2.f * z - a;
      if (rank_out) rank_out[i] = z != 0.f;
      if (nuc_acc) {
        nuc += (double)fabsf(z);
        zeros += (z == 0.f);
      }
    }
  }
  if (nuc_acc) {
    nuc = warp_sum_d(nuc);
    unsigned long long zz = zeros;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zz += __shfl_xor_sync(0xffffffffu, zz, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
      sred[w] = nuc;
      cred[w] = zz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      unsigned long long tz = 0;
      for (int i = 0; i < kEwThreads / 32; ++i) {
        t += sred[i];
        tz += cred[i];
      }
      atomicAdd(nuc_acc, t);
      if (cnt) atomicAdd(cnt + 1, tz);
    }
  }
}

// Sums of a CTA's per-thread FP64 values, added to *acc by thread 0.
__device__ __forceinline__ void cta_add_d(double v, double* acc, double* sred) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sred[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kEwThreads / 32; ++i) t += sred[i];
    atomicAdd(acc, t);
  }
  __syncthreads();
}

// X_i = W_i + R (the X-update of eq:admm on the final state), U_i = Z_i - W_i,
// and in FP64 sum over i of ||X_i - Z_i||^2 (primal residual) into
// pres_acc[0] and, with `dual`, sum of ||Z_i - Z_i^prev||^2 into
// pres_acc[1], where X_out holds the previous iteration's Z on entry.
__global__ void __launch_bounds__(kEwThreads)
finalize_kernel(const float* __restrict__ W, const float* __restrict__ Z,
                const float* __restrict__ R, float* X_out, float* __restrict__ U_out,
                double* pres_acc, int dual, int L, size_t MN) {
  __shared__ double sred[kEwThreads / 32];
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  double acc = 0.0, accd = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN; i += stride) {
    const float r = R[i];
    for (int j = 0; j < L; ++j) {
      const size_t o = (size_t)j * MN + i;
      const float w = W[o], z = Z[o];
      const float x = w + r;
      if (dual) {
        const double dz = (double)z - (double)X_out[o];
        accd += dz * dz;
      }
      X_out[o] = x;
      if (U_out) U_out[o] = z - w;
      const double dxz = (double)x - (double)z;
      acc += dxz * dxz;
    }
  }
  if (pres_acc) {
    cta_add_d(acc, pres_acc, sred);
    if (dual) cta_add_d(accd, pres_acc + 1, sred);
  }
}

// Stopping test of the ADMM (Boyd et al. 2011, Sec. 3.3): with (Zs, Ws) the
// state one iteration earlier, sums in FP64 of ||U - Us||^2 (the primal
// residual ||X - Z||^2 of that iteration, since U' - U = X - Z'), of
// ||Z - Zs||^2 (the dual residual / rho), of ||Z||^2 and of ||U||^2, with
// U = Z - W.
__global__ void __launch_bounds__(kEwThreads)
residual_kernel(const float* __restrict__ Z, const float* __restrict__ W,
                const float* __restrict__ Zs, const float* __restrict__ Ws, double* acc4,
                size_t n) {
  __shared__ double sred[kEwThreads / 32];
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  double du = 0.0, dz = 0.0, zz = 0.0, uu = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double z = Z[i], w = W[i], zs = Zs[i], ws = Ws[i];
    const double u = z - w, us = zs - ws;
    du += (u - us) * (u - us);
    dz += (z - zs) * (z - zs);
    zz += z * z;
    uu += u * u;
  }
  cta_add_d(du, acc4, sred);
  cta_add_d(dz, acc4 + 1, sred);
  cta_add_d(zz, acc4 + 2, sred);
  cta_add_d(uu, acc4 + 3, sred);
}

__global__ void __launch_bounds__(kEwThreads)
init_state_kernel(const float* __restrict__ Z0, const float* __restrict__ U0, float* __restrict__ Z,
                  float* __restrict__ W, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float z = Z0 ? Z0[i] : 0.f;
    const float u = U0 ? U0[i] : 0.f;
    Z[i] = z;
    W[i] = z - u;
  }
}

// Start of an iteration: publish this iteration's shift and advance.
__global__ void advance_kernel(const int* __restrict__ table, int* iter, int* cur_shift, int jobs) {
  const int k = *iter;
  for (int j = 0; j < jobs; ++j) {
    cur_shift[2 * j] = table[2 * (k * jobs + j)];
    cur_shift[2 * j + 1] = table[2 * (k * jobs + j) + 1];
  }
  *iter = k + 1;
}

__global__ void __launch_bounds__(kEwThreads)
nonfinite_kernel(const float* __restrict__ Y, int M, int N, int ld, int* flag) {
  const size_t MN = (size_t)M * N;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  int bad = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN; i += stride) {
    const size_t r = i / (size_t)N, c = i - r * (size_t)N;
    bad |= !isfinite(Y[r * (size_t)ld + c]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void __launch_bounds__(kEwThreads)
copy_dense_kernel(const float* __restrict__ src, int M, int N, int ld, float* __restrict__ dst) {
  const size_t MN = (size_t)M * N;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN; i += stride) {
    const size_t r = i / (size_t)N, c = i - r * (size_t)N;
    dst[i] = src[r * (size_t)ld + c];
  }
}

// Noise scale (Sec. 2.1): the whole matrix is one MN x 1 block, whose only
// singular value is ||A||_F, so its SVT is A max(1 - tau / ||A||_F, 0).
// Pass 1 sums ||A||^2 in FP64 (A = A1 + A2); pass 2 applies the shrink with
// the fused dual update.  The cycle-spin shift is irrelevant (a permutation
// of the entries).
__global__ void __launch_bounds__(kEwThreads)
noise_norm_kernel(const float* __restrict__ A1, const float* __restrict__ A2, int M, int N, int ld,
                  double* __restrict__ acc) {
  __shared__ double red[kEwThreads / 32];
  const size_t MN = (size_t)M * N;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  double t = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN; i += stride) {
    const size_t r = i / (size_t)N, off = r * (size_t)ld + (i - r * (size_t)N);
    float a = A1[off];
    if (A2) a += A2[off];
    t = fma((double)a, (double)a, t);
  }
  t = warp_sum_d(t);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kEwThreads / 32; ++k) s += red[k];
    atomicAdd(acc, s);
  }
}

__global__ void __launch_bounds__(kEwThreads)
noise_shrink_kernel(const float* A1, const float* __restrict__ A2, float* Zout, float* Wout, int M,
                    int N, int ld, float tau, const double* __restrict__ acc, int* rank_out,
                    double* nuc_acc, unsigned long long* cnt) {
  const double nrm = sqrt(*acc);
  const float f = nrm > (double)tau ? (float)(1.0 - (double)tau / nrm) : 0.f;
  const size_t MN = (size_t)M * N;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN; i += stride) {
    const size_t r = i / (size_t)N, off = r * (size_t)ld + (i - r * (size_t)N);
    float a = A1[off];
    if (A2) a += A2[off];
    const float z = f * a;
    Zout[off] = z;
    if (Wout) Wout[off] = 2.f * z - a;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (rank_out) rank_out[0] = f > 0.f;
    if (nuc_acc && nrm > (double)tau) atomicAdd(nuc_acc, nrm - (double)tau);
    if (cnt && !(f > 0.f)) atomicAdd(cnt + 1, 1ull);
  }
}

}  // namespace

cudaError_t launch_consensus(const float* Y, const float* W, float* R, const uint8_t* mask, int L,
                             size_t MN, cudaStream_t st, Prof* prof, float* Z11, float* W11,
                             float tau11) {
  if (prof) prof->scale = 0;
  if (prof) if (cudaError_t e = prof->before(st, KK_CONSENSUS)) return e;
  const int grid = ew_grid((MN + 3) / 4);
  const bool fuse = Z11 != nullptr;
  switch (L) {
#define MSLLR_CONSENSUS_CASE(n)                                                                 \
  case n:                                                                                       \
    if (fuse)                                                                                   \
      consensus_kernel<n, true><<<grid, kEwThreads, 0, st>>>(Y, W, R, mask, MN, Z11, W11, tau11); \
    else                                                                                        \
      consensus_kernel<n, false><<<grid, kEwThreads, 0, st>>>(Y, W, R, mask, MN, nullptr, nullptr, 0.f); \
    break;
    MSLLR_CONSENSUS_CASE(1)
    MSLLR_CONSENSUS_CASE(2)
    MSLLR_CONSENSUS_CASE(3)
    MSLLR_CONSENSUS_CASE(4)
    MSLLR_CONSENSUS_CASE(5)
    MSLLR_CONSENSUS_CASE(6)
    MSLLR_CONSENSUS_CASE(7)
    MSLLR_CONSENSUS_CASE(8)
#undef MSLLR_CONSENSUS_CASE
    default:
      return cudaErrorInvalidValue;
  }
  if (prof) if (cudaError_t e = prof->after(st)) return e;
  return cudaGetLastError();
}

cudaError_t launch_noise(const ScaleLaunch& s, cudaStream_t st, Prof* prof) {
  if (!s.norm_acc) return cudaErrorInvalidValue;
  const size_t MN = (size_t)s.M * s.N;
  if (prof) if (cudaError_t e = prof->before(st, KK_SOFT1X1)) return e;
  if (cudaError_t e = cudaMemsetAsync(s.norm_acc, 0, sizeof(double), st)) return e;
  noise_norm_kernel<<<ew_grid(MN), kEwThreads, 0, st>>>(s.A1, s.A2, s.M, s.N, s.ld, s.norm_acc);
  if (prof) if (cudaError_t e = prof->after(st)) return e;
  if (prof) if (cudaError_t e = prof->before(st, KK_SOFT1X1)) return e;
  noise_shrink_kernel<<<ew_grid(MN), kEwThreads, 0, st>>>(s.A1, s.A2, s.Zout, s.Wout, s.M, s.N,
                                                          s.ld, s.tau, s.norm_acc, s.rank_out,
                                                          s.nuc_acc, s.cnt);
  if (prof) if (cudaError_t e = prof->after(st)) return e;
  return cudaGetLastError();
}

cudaError_t launch_soft1x1(const ScaleLaunch& s, cudaStream_t st, Prof* prof) {
  const size_t MN = (size_t)s.M * s.N;
  if (prof) if (cudaError_t e = prof->before(st, KK_SOFT1X1)) return e;
  soft1x1_kernel<<<ew_grid((MN + 3) / 4), kEwThreads, 0, st>>>(
      s.A1, s.A2, s.Zout, s.Wout, s.M, s.N, s.ld, s.tau, s.rank_out, s.nuc_acc, s.cnt);
  if (prof) if (cudaError_t e = prof->after(st)) return e;
  return cudaGetLastError();
}

#define MISC_BEFORE()                                                  \
  if (prof) {                                                          \
    prof->scale = 0;                                                   \
    if (cudaError_t e_ = prof->before(st, KK_MISC)) return e_;         \
  }
#define MISC_AFTER() \
  if (prof)          \
    if (cudaError_t e_ = prof->after(st)) return e_;

cudaError_t launch_finalize(const float* W, const float* Z, const float* R, float* X_out,
                            float* U_out, double* pres_acc, bool dual, int L, size_t MN,
                            cudaStream_t st, Prof* prof) {
  MISC_BEFORE()
  finalize_kernel<<<ew_grid(MN), kEwThreads, 0, st>>>(W, Z, R, X_out, U_out, pres_acc, dual ? 1 : 0,
                                                      L, MN);
  MISC_AFTER()
  return cudaGetLastError();
}

cudaError_t launch_residual(const float* Z, const float* W, const float* Zs, const float* Ws,
                            double* acc4, size_t n, cudaStream_t st, Prof* prof) {
  MISC_BEFORE()
  residual_kernel<<<ew_grid(n), kEwThreads, 0, st>>>(Z, W, Zs, Ws, acc4, n);
  MISC_AFTER()
  return cudaGetLastError();
}

cudaError_t launch_init_state(const float* Z0, const float* U0, float* Z, float* W, int L,
                              size_t MN, cudaStream_t st, Prof* prof) {
  const size_t n = (size_t)L * MN;
  MISC_BEFORE()
  init_state_kernel<<<ew_grid(n), kEwThreads, 0, st>>>(Z0, U0, Z, W, n);
  MISC_AFTER()
  return cudaGetLastError();
}

cudaError_t launch_advance(const int* table, int* iter, int* cur_shift, int jobs, cudaStream_t st,
                           Prof* prof) {
  if (prof) prof->scale = 0;
  if (prof) if (cudaError_t e = prof->before(st, KK_ADVANCE)) return e;
  advance_kernel<<<1, 1, 0, st>>>(table, iter, cur_shift, jobs);
  if (prof) if (cudaError_t e = prof->after(st)) return e;
  return cudaGetLastError();
}

cudaError_t launch_nonfinite(const float* Y, int M, int N, int ld, int* flag, cudaStream_t st,
                             Prof* prof) {
  MISC_BEFORE()
  nonfinite_kernel<<<ew_grid((size_t)M * N), kEwThreads, 0, st>>>(Y, M, N, ld, flag);
  MISC_AFTER()
  return cudaGetLastError();
}

cudaError_t launch_copy_dense(const float* src, int M, int N, int ld, float* dst, cudaStream_t st,
                              Prof* prof) {
  MISC_BEFORE()
  copy_dense_kernel<<<ew_grid((size_t)M * N), kEwThreads, 0, st>>>(src, M, N, ld, dst);
  MISC_AFTER()
  return cudaGetLastError();
}
#undef MISC_BEFORE
#undef MISC_AFTER

// Averaged cycle spinning (Sec. 9): the Z-updates of the shifts of a scale
// are summed with weight 1/|S| into acc (the scale's W slot, free once the
// consensus step has read it), then Z = acc and W = 2 acc - A, A = Z + R.
__global__ void __launch_bounds__(kEwThreads)
spin_accum_kernel(float* __restrict__ acc, const float* __restrict__ T, float w, int first,
                  size_t MN) {
  for (size_t e = blockIdx.x * (size_t)kEwThreads + threadIdx.x; e < MN;
       e += (size_t)gridDim.x * kEwThreads)
    acc[e] = first ? w * T[e] : fmaf(w, T[e], acc[e]);
}

__global__ void __launch_bounds__(kEwThreads)
spin_finish_kernel(float* __restrict__ Z, float* __restrict__ W, const float* __restrict__ R,
                   size_t MN) {
  for (size_t e = blockIdx.x * (size_t)kEwThreads + threadIdx.x; e < MN;
       e += (size_t)gridDim.x * kEwThreads) {
    const float a = Z[e] + R[e];
    const float z = W[e];
    Z[e] = z;
    W[e] = 2.f * z - a;
  }
}

cudaError_t launch_spin_accum(float* acc, const float* T, float w, bool first, size_t MN,
                              cudaStream_t st, Prof* prof) {
  if (prof) if (cudaError_t e = prof->before(st, KK_MISC)) return e;
  spin_accum_kernel<<<ew_grid(MN), kEwThreads, 0, st>>>(acc, T, w, first ? 1 : 0, MN);
  if (prof) if (cudaError_t e = prof->after(st)) return e;
  return cudaGetLastError();
}

cudaError_t launch_spin_finish(float* Z, float* W, const float* R, size_t MN, cudaStream_t st,
                               Prof* prof) {
  if (prof) if (cudaError_t e = prof->before(st, KK_MISC)) return e;
  spin_finish_kernel<<<ew_grid(MN), kEwThreads, 0, st>>>(Z, W, R, MN);
  if (prof) if (cudaError_t e = prof->after(st)) return e;
  return cudaGetLastError();
}

}  // namespace msllr
