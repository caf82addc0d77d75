// Cross-scale tile fusion of two nested narrow scales.  Under the one shift
// per iteration that all scales share (Sec. 9), every block of a finer
// scale (e.g. 16 x 16) lies inside one block of a coarser scale (64 x 64)
// when the block sizes divide, and both prox inputs Z_i + R read the same
// residual R there.  One CTA per coarse block therefore
//   1. reads the coarse block's R once into shared memory,
//   2. solves the fine blocks inside it, a warp each in turn
//      (warp_block.cuh), their A = Z_fine + R from that tile,
//   3. solves the coarse block (small_block.cuh) with A = Z_coarse + R from
//      the same tile,
// each with the same arithmetic as its own per-scale kernel, so the outputs
// equal the separate kernels' bit for bit; R is read once instead of twice.
#include "small_block.cuh"

namespace msllr {

namespace {

constexpr int kNT = 128;  // threads: the coarse block's CTA (64-wide blocks)

// the second half of A (the residual R) from the CTA's tile of the coarse
// block: element (r0 + row, c0 + col), row stride ld
struct A2Tile {
  const float* t;
  int ld, r0, c0;
  __device__ __forceinline__ float operator()(size_t, int row, int col) const {
    return t[(r0 + row) * ld + (c0 + col)];
  }
};

// NP: the fine blocks' fixed rotation order (16 for blocks 15 or 16 wide)
template <int NP>
__global__ void __launch_bounds__(kNT, 3)
nested_kernel(ScaleLaunch fine, ScaleLaunch coarse) {
  extern __shared__ float sm[];
  const int b = blockIdx.x;
  const BlockGeom g = block_geom_t<false>(coarse, b);
  const int m = coarse.m, n = coarse.n;
  // shared memory: the coarse block's layout; until its solve starts, the
  // R tile lives in its Gram region (m (n + 1) floats) and the warps' V
  // scratch in its certificate region, both written only later
  const SmallLayout<kNT, 64> lay(m, n);
  float* Rt = sm + lay.oG;
  const int ldr = n + 1;
  float(*vs)[16][17] = reinterpret_cast<float(*)[16][17]>(sm + lay.oL);
  for (int e = threadIdx.x; e < m * n; e += kNT) {
    const int r = e / n, c = e - r * n;
    Rt[r * ldr + c] = __ldg(coarse.A2 + g.offset(r, c));
  }
  __syncthreads();
  // fine blocks (p_f, q_f) = (p pi + du, q qi + dv) of the fine grid
  const int fm = fine.m, fn = fine.n;
  const int pi = m / fm, qi = n / fn, nbn_fine = fine.N / fn;
  const int warp = threadIdx.x >> 5;
  for (int u = warp; u < pi * qi; u += kNT / 32) {
    const int du = u / qi, dv = u - du * qi;
    const int bf = (g.p * pi + du) * nbn_fine + (g.q * qi + dv);
    warp_block_svt<8, false, NP>(fine, bf, vs[warp], A2Tile{Rt, ldr, du * fm, dv * fn});
  }
  __syncthreads();
  // the coarse block: its gather reads the tile before its Gram phase
  // overwrites that region (a barrier lies between them)
  small_block_svt<kNT, 64, false>(coarse, b, sm, A2Tile{Rt, ldr, 0, 0});
}

}  // namespace

bool nested_pair(int fm, int fn, int cm, int cn) {
  if (choose_path(fm, fn) != ScalePath::Small || !warp_path(fm, fn) || fm < fn || fm > 16)
    return false;
  if (cm != cn || choose_path(cm, cn) != ScalePath::Small || warp_path(cm, cn) || cn <= 32)
    return false;
  if (cm % fm || cn % fn) return false;
  // the R tile and the warps' V scratch fit the coarse layout's regions
  const SmallLayout<kNT, 64> lay(cm, cn);
  return cm * (cn + 1) <= lay.oL - lay.oG && (kNT / 32) * 16 * 17 <= lay.oQ - lay.oL;
}

cudaError_t configure_nested() {
  const int bytes = (int)(sizeof(float) * SmallLayout<kNT, 64>(64, 64).total);
  cudaError_t e = cudaFuncSetAttribute(nested_kernel<0>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(nested_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

cudaError_t launch_nested(const ScaleLaunch& fine, const ScaleLaunch& coarse, cudaStream_t st,
                          Prof* prof) {
  if (!nested_pair(fine.m, fine.n, coarse.m, coarse.n) || fine.fw || coarse.fw || fine.rows ||
      coarse.rows || fine.shift != coarse.shift || fine.shift_add_r || fine.shift_add_c ||
      coarse.shift_add_r || coarse.shift_add_c || !coarse.A2 || fine.A2 != coarse.A2 ||
      fine.M != coarse.M || fine.N != coarse.N || fine.ld != coarse.ld ||
      (coarse.m == coarse.M && coarse.n == coarse.N))  // the full matrix ignores the shift
    return cudaErrorInvalidValue;
  const size_t smem = sizeof(float) * (size_t)SmallLayout<kNT, 64>(coarse.m, coarse.n).total;
  const int nblocks = (coarse.M / coarse.m) * (coarse.N / coarse.n);
  const int fnn = fine.m < fine.n ? fine.m : fine.n;
  if (prof)
    if (cudaError_t e = prof->before(st, KK_FUSED)) return e;
  if (fnn >= 15) nested_kernel<16><<<nblocks, kNT, smem, st>>>(fine, coarse);
  else nested_kernel<0><<<nblocks, kNT, smem, st>>>(fine, coarse);
  if (prof)
    if (cudaError_t e = prof->after(st)) return e;
  return cudaGetLastError();
}

}  // namespace msllr
