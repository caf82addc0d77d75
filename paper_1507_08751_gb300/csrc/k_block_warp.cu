// Block SVT of narrow blocks (min(m, n) <= 16, max(m, n) <= 32): one warp
// per block (warp_block.cuh), one warp per CTA -- eq:bsvt under the Sec. 9
// shift.
#include "warp_block.cuh"

namespace msllr {

cudaError_t set_phase_buffer_warp(unsigned long long* p) {
  return cudaMemcpyToSymbol(g_phase_acc, &p, sizeof(p));
}

namespace {

// RPL: rows of C per lane (mm <= 2 RPL); NP: columns in the rotation order
// when fixed at compile time (16 for blocks 15 or 16 wide), 0 to take it
// from the block
template <int RPL, bool ST, int NP>
__global__ void __launch_bounds__(kWT, RPL <= 8 ? 32 : 16)
blocksvt_warp_kernel(ScaleLaunch a, int nblocks) {
  __shared__ float vsh[kWarps][16][17];  // V of each warp, for the rebuild
  const int wid = threadIdx.x >> 5;
  const int b = blockIdx.x * kWarps + wid;
  if (b >= nblocks) return;  // the whole warp leaves together
  warp_block_svt<RPL, ST, NP>(a, b, vsh[wid], A2Global{a.A2});
}

}  // namespace

bool warp_path(int m, int n) {
  const int nn = m < n ? m : n, mm = m < n ? n : m;
  return nn >= 1 && nn <= 16 && mm <= 32;
}

cudaError_t launch_warp(const ScaleLaunch& s, cudaStream_t st, Prof* prof) {
  const int mm = s.m >= s.n ? s.m : s.n;
  const int nblocks = (s.M / s.m) * (s.N / s.n);
  const int grid = (nblocks + kWarps - 1) / kWarps;
  if (prof)
    if (cudaError_t e = prof->before(st, KK_FUSED)) return e;
  const int nn = s.m < s.n ? s.m : s.n;
  const bool gen = s.fw || s.rows, w16 = nn >= 15;
  if (mm <= 16) {
    if (w16) {
      if (gen) blocksvt_warp_kernel<8, true, 16><<<grid, kWT, 0, st>>>(s, nblocks);
      else blocksvt_warp_kernel<8, false, 16><<<grid, kWT, 0, st>>>(s, nblocks);
    } else {
      if (gen) blocksvt_warp_kernel<8, true, 0><<<grid, kWT, 0, st>>>(s, nblocks);
      else blocksvt_warp_kernel<8, false, 0><<<grid, kWT, 0, st>>>(s, nblocks);
    }
  } else {
    if (w16) {
      if (gen) blocksvt_warp_kernel<16, true, 16><<<grid, kWT, 0, st>>>(s, nblocks);
      else blocksvt_warp_kernel<16, false, 16><<<grid, kWT, 0, st>>>(s, nblocks);
    } else {
      if (gen) blocksvt_warp_kernel<16, true, 0><<<grid, kWT, 0, st>>>(s, nblocks);
      else blocksvt_warp_kernel<16, false, 0><<<grid, kWT, 0, st>>>(s, nblocks);
    }
  }
  if (prof)
    if (cudaError_t e = prof->after(st)) return e;
  return cudaGetLastError();
}

}  // namespace msllr
