// Gram matrices G_b = C_b^T C_b of wide blocks (the first phase of the wide
// path of eq:svt, Sec. 8) on the 5th-generation tensor cores: tcgen05.mma
// with TF32 operands from shared memory and the FP32 accumulator in tensor
// memory (TMEM).
//
// Accuracy ("3xTF32", Ootomo & Yokota 2022): every element x of C is split
// as x = h + l, h = x with its 13 low mantissa bits cleared (exact in TF32)
// and l = x - h (exact in FP32, |l| < 2^-10 |x|).  Then
//   C^T C = H^T H + H^T L + L^T H + L^T L
// and the kernel accumulates the first three products (three MMAs per K
// step), dropping L^T L (below 2^-20 of the product) and the TF32 rounding
// of l (below 2^-21 |x|): FP32-level accuracy at tensor-core rates.
//
// Work split: one CTA per (128 x 128 tile of the lower triangle of G, chunk
// of rows of C, block); blocks up to 256 wide (two tile rows) and the wide
// path's blocks above 256 alike.  Per stage of 16 rows of C the 256 threads load the
// tile's two column ranges of A = A1 + A2 (cycle-spun gather, coalesced
// 128-byte row segments), split them and store h and l in the canonical
// K-major layout without swizzle; one thread issues the MMAs for the stage
// and commits them to the stage's mbarrier, which the threads wait on
// before they overwrite that stage (two stages, so the loads of stage s + 1
// run under the MMAs of stage s).  The epilogue reads the accumulator with
// tcgen05.ld (warp w: TMEM lanes 32 (w mod 4) .., columns 64 (w / 4) ..) and
// writes the packed lower triangle of G, or a partial sum per row chunk in
// the 64 x 64 tile layout of the FP32 Gram kernels (reduced by the same
// kernels: packed for blocks up to 256 wide, a full square above).
//
// Every wait is bounded: a wait that runs out sets the launch's error flag,
// the CTA skips its output, frees its TMEM and returns.
#include "common.cuh"
#include "internal.h"

namespace msllr {

namespace {

constexpr int kTT = 128;                      // output tile (MMA M = N = 128)
constexpr int kKS = 16;                       // rows of C per pipeline stage
constexpr int kGT = 256;                      // threads per CTA
constexpr int kT64 = 64;                      // partial-sum tile of the FP32 path
constexpr int kTileBytes = kTT * kKS * 4;     // one operand tile, h or l: 8 KB
constexpr int kStageBytes = 4 * kTileBytes;   // A h, A l, B h, B l
constexpr int kDLd = kTT + 1;                 // row stride of the staged accumulator
constexpr int kBodyBytes = (2 * kStageBytes > kTT * kDLd * 4) ? 2 * kStageBytes : kTT * kDLd * 4;
constexpr int kSmemBytes = kBodyBytes + 64;
constexpr uint32_t kTmemCols = 128;
constexpr int kWaitPolls = 1 << 20;

// Canonical K-major operand layout without swizzle: core matrices of 8 rows
// x 16 bytes (4 TF32 along K), the two K-adjacent cores of one MMA 128 bytes
// apart (leading byte offset), 8-row groups 512 bytes apart (stride byte
// offset).  Byte offset of row i (an MMA row: a column of C) and K quad q.
__device__ __forceinline__ uint32_t op_off(int i, int q) {
  return (uint32_t)((i >> 3) * 512 + q * 128 + (i & 7) * 16);
}

// tcgen05 shared-memory matrix descriptor: start address >> 4, leading and
// stride byte offsets >> 4, descriptor version 1 at bit 46, base offset 0,
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                            ((uint32_t)(kTT >> 3) << 17) | ((uint32_t)(kTT >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kWaitPolls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (i >= 32) __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(d), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

__device__ __forceinline__ size_t c_off(const BlockGeom& g, int i, int c) {
  return g.transposed() ? g.offset(c, i) : g.offset(i, c);
}

// GEN: batched jobs or spatio-temporal blocks (block_geom_t); ST:
// spatio-temporal blocks (generic gather), else 2-D blocks, whose gather
// needs one row offset per row and one column index per thread.
template <bool GEN, bool ST>
__global__ void __launch_bounds__(kGT, 3)
gram_tc_kernel(ScaleLaunch a, float* __restrict__ G, float* __restrict__ part, int chunks,
               int ntiles64, int chunk_rows, int to_part, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int t = blockIdx.x, chunk = blockIdx.y, b = blockIdx.z;
  // tile (ti, tj), ti >= tj, of the lower triangle: t = ti (ti + 1) / 2 + tj
  int ti = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while (((ti + 1) * (ti + 2)) / 2 <= t) ++ti;
  while ((ti * (ti + 1)) / 2 > t) --ti;
  const int tj = t - (ti * (ti + 1)) / 2;
  const bool diag = ti == tj;
  const BlockGeom g = block_geom_t<GEN>(a, b);
  const int mm = g.mm(), nn = g.nn();
  const int r_begin = chunk * chunk_rows;
  const int r_end = min(mm, r_begin + chunk_rows);
  const int nsteps = (r_end - r_begin + kKS - 1) / kKS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kBodyBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kBodyBytes + 32);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = smem_u32(bar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // loader: column ci of the tile, K quads q0 and q0 + 2 of every stage.
  // The loads are predicated (no branches between them) and the two halves
  // of A are added only when the stage is stored, so all of a stage's loads
  // are in flight at once.
  const int ci = tid & (kTT - 1), q0 = tid >> 7;
  const int ca = ti * kTT + ci, cb = tj * kTT + ci;
  const bool va = ca < nn, vb = !diag && cb < nn;
  const bool has2 = a.A2 != nullptr;
  float xa[8], ya[8], xb[8], yb[8];
  // 2-D blocks: global columns of the thread's two C columns (Sec. 9 shift,
  // wrapped) and the unwrapped global row of C's row 0
  int gca = g.q * g.n + (va ? ca : 0) + g.sc;
  if (gca >= g.N) gca -= g.N;
  int gcb = g.q * g.n + (vb ? cb : 0) + g.sc;
  if (gcb >= g.N) gcb -= g.N;
  const int grow0 = g.p * g.m + g.sr;
  auto load = [&](int step) {
    const int r0 = r_begin + step * kKS;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int row = r0 + 4 * (q0 + 2 * (u >> 2)) + (u & 3);
      const bool in = row < r_end;
      uint32_t oa, ob;
      if constexpr (ST) {
        oa = (uint32_t)c_off(g, in ? row : r_begin, va ? ca : 0);
        ob = (uint32_t)c_off(g, in ? row : r_begin, vb ? cb : 0);
      } else {
        int gr = grow0 + row;
        if (gr >= g.M) gr -= g.M;
        const uint32_t ro = (uint32_t)(g.rbase + gr) * (uint32_t)g.ld;
        oa = ro + (uint32_t)gca;
        ob = ro + (uint32_t)gcb;
      }
      xa[u] = (in && va) ? __ldg(a.A1 + oa) : 0.f;
      ya[u] = (in && va && has2) ? __ldg(a.A2 + oa) : 0.f;
      xb[u] = (in && vb) ? __ldg(a.A1 + ob) : 0.f;
      yb[u] = (in && vb && has2) ? __ldg(a.A2 + ob) : 0.f;
    }
  };
  auto store = [&](int buf) {
    unsigned char* st = smem + buf * kStageBytes;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t o = op_off(ci, q0 + 2 * h);
      float v[4], w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        v[e] = xa[4 * h + e] + ya[4 * h + e];
        w[e] = xb[4 * h + e] + yb[4 * h + e];
      }
      float4 hi = make_float4(tf32_hi(v[0]), tf32_hi(v[1]), tf32_hi(v[2]), tf32_hi(v[3]));
      *reinterpret_cast<float4*>(st + o) = hi;
      *reinterpret_cast<float4*>(st + kTileBytes + o) =
          make_float4(v[0] - hi.x, v[1] - hi.y, v[2] - hi.z, v[3] - hi.w);
      if (!diag) {
        hi = make_float4(tf32_hi(w[0]), tf32_hi(w[1]), tf32_hi(w[2]), tf32_hi(w[3]));
        *reinterpret_cast<float4*>(st + 2 * kTileBytes + o) = hi;
        *reinterpret_cast<float4*>(st + 3 * kTileBytes + o) =
            make_float4(w[0] - hi.x, w[1] - hi.y, w[2] - hi.z, w[3] - hi.w);
      }
    }
  };

  uint32_t phase = 0u;  // bit k: parity of the next completion of stage k's barrier
  bool ok = true;
  load(0);
  for (int s = 0; s < nsteps; ++s) {
    const int buf = s & 1;
    if (s >= 2) {
      ok = mbar_wait(bar0 + 8 * buf, (phase >> buf) & 1u) && ok;
      phase ^= 1u << buf;
    }
    store(buf);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (s + 1 < nsteps) load(s + 1);
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = sbase + buf * kStageBytes;
      const uint32_t ah = st, al = st + kTileBytes;
      const uint32_t bh = diag ? ah : st + 2 * kTileBytes;
      const uint32_t bl = diag ? al : st + 3 * kTileBytes;
#pragma unroll
      for (int kk = 0; kk < kKS / 8; ++kk) {
        const uint32_t ko = 256u * kk;  // two K-adjacent core matrices per MMA (K = 8)
        mma_tf32(tmem, smem_desc(ah + ko), smem_desc(bh + ko), (s > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(ah + ko), smem_desc(bl + ko), 1u);
        mma_tf32(tmem, smem_desc(al + ko), smem_desc(bh + ko), 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              bar0 + 8 * buf)
          : "memory");
    }
  }
  // the last commit covers every MMA issued before it
  {
    const int lb = (nsteps - 1) & 1;
    ok = mbar_wait(bar0 + 8 * lb, (phase >> lb) & 1u) && ok;
  }
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // the accumulator goes through shared memory (the operand buffers are
  // free now; row stride kTT + 1 keeps both passes free of bank conflicts),
  // so that the global writes are warp-wide row segments
  float* Ds = reinterpret_cast<float*>(smem);
  if (ok) {
    const int x = 32 * (warp & 3) + lane;  // row of the tile (TMEM lane)
    const int ycol = 64 * (warp >> 2);      // first column of this warp
    const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)ycol;
#pragma unroll
    for (int c = 0; c < 64; c += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr + (uint32_t)c));
      asm volatile("tcgen05.wait::ld.sync.aligned;"
                   : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                     "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                     "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
                   :
                   : "memory");
#pragma unroll
      for (int e = 0; e < 16; ++e) Ds[x * kDLd + ycol + c + e] = __uint_as_float(v[e]);
    }
  } else if (tid == 0 && err) {
    atomicOr(err, 1);
  }
  __syncthreads();
  if (ok) {
    if (chunks > 1 || to_part) {
      // partial sums: the valid 64 x 64 tiles of this 128 x 128 tile, row by row
      const int T64 = (nn + kT64 - 1) / kT64;
      for (int xr = warp; xr < 2 * kTT; xr += kGT / 32) {
        const int x = xr >> 1, hc = xr & 1;
        const int a64 = 2 * ti + (x >> 6), c64 = 2 * tj + hc;
        if (c64 > a64 || a64 >= T64) continue;
        float* dst = part +
                     (((size_t)b * chunks + chunk) * ntiles64 + (a64 * (a64 + 1)) / 2 + c64) *
                         (kT64 * kT64) +
                     (size_t)(x & 63) * kT64;
        dst[lane] = Ds[x * kDLd + hc * kT64 + lane];
        dst[lane + 32] = Ds[x * kDLd + hc * kT64 + lane + 32];
      }
    } else {
      // packed lower triangle: row i's columns tj 128 .. min(i, tj 128 + 127)
      for (int x = warp; x < kTT; x += kGT / 32) {
        const int i = ti * kTT + x;
        if (i >= nn) break;
        const int cnt = min(i - tj * kTT + 1, kTT);
        float* Grow = G + (size_t)b * nn * nn + (size_t)i * (i + 1) / 2 + tj * kTT;
        for (int y = lane; y < cnt; y += 32) Grow[y] = Ds[x * kDLd + y];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

}  // namespace

bool gram_tc_eligible(const ScaleLaunch& s) {
  const int nn = s.m < s.n ? s.m : s.n;
  // element offsets are 32-bit in the kernel
  return s.m >= s.n && nn > 64 && (size_t)s.M * s.ld < ((size_t)1 << 31);
}

cudaError_t configure_gram_tc() {
  cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel<false, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(gram_tc_kernel<true, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(gram_tc_kernel<true, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

cudaError_t launch_gram_tc(const ScaleLaunch& s, float* G, float* part, int chunks, int nblocks,
                           int ntiles64, int chunk_rows, int to_part, cudaStream_t st) {
  const int nn = s.m < s.n ? s.m : s.n;
  if (!gram_tc_eligible(s)) return cudaErrorInvalidValue;
  const int T = (nn + kTT - 1) / kTT;
  const dim3 grid(T * (T + 1) / 2, chunks, nblocks);
  if (s.fw)
    gram_tc_kernel<true, true><<<grid, kGT, kSmemBytes, st>>>(s, G, part, chunks, ntiles64,
                                                              chunk_rows, to_part, s.err);
  else if (s.rows)
    gram_tc_kernel<true, false><<<grid, kGT, kSmemBytes, st>>>(s, G, part, chunks, ntiles64,
                                                               chunk_rows, to_part, s.err);
  else
    gram_tc_kernel<false, false><<<grid, kGT, kSmemBytes, st>>>(s, G, part, chunks, ntiles64,
                                                                chunk_rows, to_part, s.err);
  return cudaGetLastError();
}

}  // namespace msllr
