// Fused block SVT for narrow blocks (min(m, n) <= 64, m*n <= 8192): one CTA
// per block (small_block.cuh) does the whole of eq:bsvt for that block --
//   gather R_b(Shift_s(A)) into shared memory (Sec. 9 circular shift),
//   skip test on an upper bound of sigma_max (Sec. 8),
//   Gram matrix, certified rank above tau and the top eigenpairs (symeig.cuh),
//   rebuild C V diag(f) V^T, scatter through Shift_{-s}, and the fused dual
//   update W' = 2 Z' - A of eq:admm.
// Also holds the per-scale dispatcher.
#include "small_block.cuh"

namespace msllr {

cudaError_t launch_soft1x1(const ScaleLaunch& s, cudaStream_t st, Prof* prof);
cudaError_t launch_noise(const ScaleLaunch& s, cudaStream_t st, Prof* prof);
cudaError_t launch_big(const ScaleLaunch& s, const BigWorkspace& ws, cudaStream_t st, Prof* prof,
                       cudaEvent_t after_gram);

cudaError_t set_phase_buffer_small(unsigned long long* p) {
  return cudaMemcpyToSymbol(g_phase_acc, &p, sizeof(p));
}

namespace {

template <int NT, int NMAX, bool ST>
__global__ void __launch_bounds__(NT, NT == 32 ? 24 : (NT == 128 ? 3 : 1))
blocksvt_small_kernel(ScaleLaunch a) {
  extern __shared__ float sm[];
  small_block_svt<NT, NMAX, ST>(a, (int)blockIdx.x, sm, A2Global{a.A2});
}

template <int NT, int NMAX>
size_t small_smem_bytes(int mm, int nn) {
  return sizeof(float) * (size_t)SmallLayout<NT, NMAX>(mm, nn).total;
}

template <int NT, int NMAX>
cudaError_t launch_small_t(const ScaleLaunch& s, cudaStream_t st, Prof* prof) {
  const int mm = s.m >= s.n ? s.m : s.n, nn = s.m >= s.n ? s.n : s.m;
  const size_t smem = small_smem_bytes<NT, NMAX>(mm, nn);
  const int nblocks = (s.M / s.m) * (s.N / s.n);
  if (prof) if (cudaError_t e = prof->before(st, KK_FUSED)) return e;
  if (s.fw || s.rows) blocksvt_small_kernel<NT, NMAX, true><<<nblocks, NT, smem, st>>>(s);
  else blocksvt_small_kernel<NT, NMAX, false><<<nblocks, NT, smem, st>>>(s);
  if (prof) if (cudaError_t e = prof->after(st)) return e;
  return cudaGetLastError();
}

}  // namespace

cudaError_t configure_big_kernels();

// Opt the kernels into more than 48 KB of dynamic shared memory.  Called once
// per device from msllr_create, outside any stream capture.
cudaError_t configure_kernels() {
  cudaError_t e;
  e = cudaFuncSetAttribute(blocksvt_small_kernel<32, 16, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(blocksvt_small_kernel<64, 32, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(blocksvt_small_kernel<128, 64, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(blocksvt_small_kernel<32, 16, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(blocksvt_small_kernel<64, 32, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(blocksvt_small_kernel<128, 64, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = configure_plain_kernels();
  if (e != cudaSuccess) return e;
  if (cudaError_t e2 = configure_nested()) return e2;
  return configure_big_kernels();
}

ScalePath choose_path(int m, int n) {
  if (m == 0 && n == 0) return ScalePath::Noise;
  if (m == 1 && n == 1) return ScalePath::Elementwise;
  const int nn = m < n ? m : n;
  const long long area = (long long)m * n;
  if (nn <= 64 && area <= 8192) return ScalePath::Small;
  if (nn > 256) return ScalePath::Huge;
  return ScalePath::Big;
}

cudaError_t launch_scale(const ScaleLaunch& s, const BigWorkspace& ws, cudaStream_t st,
                         Prof* prof, cudaEvent_t after_gram) {
  switch (choose_path(s.m, s.n)) {
    case ScalePath::Elementwise:
      return launch_soft1x1(s, st, prof);
    case ScalePath::Noise:
      return launch_noise(s, st, prof);
    case ScalePath::Small: {
      const int nn = s.m < s.n ? s.m : s.n;
      if (warp_path(s.m, s.n)) return launch_warp(s, st, prof);
      if (nn <= 16) return launch_small_t<32, 16>(s, st, prof);
      if (nn <= 32) return launch_small_t<64, 32>(s, st, prof);
      return launch_small_t<128, 64>(s, st, prof);
    }
    case ScalePath::Huge:
      return launch_huge(s, ws, st, prof, after_gram);
    case ScalePath::Big:
    default:
      return launch_big(s, ws, st, prof, after_gram);
  }
}

}  // namespace msllr
