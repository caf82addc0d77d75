// msllr_blocksvt_noalloc: the block SVT entry point for callers that cannot
// allocate device memory.  Its workspace is a file-scope __device__ array
// that exists from library load to process exit on every GPU that loads the
// library; the host finds its device address once per device with
// cudaGetSymbolAddress (the array's name in host code is only a host-side
// stand-in, never a device address).  No cudaMalloc, cudaFree or allocating
// library routine is called.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "../../include/msllr.h"
#include "internal.h"

using namespace msllr;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MSLLR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch per device

// Publishes the shift into the first bytes of the scratch, so the block
// kernels read it like the shift of any other call.
// dst[0..1]: the shift; dst[2]: the device wait timeout flag, cleared
__global__ void set_shift_kernel(int* dst, int sr, int sc) {
  dst[0] = sr;
  dst[1] = sc;
  dst[2] = 0;
}

int err(int code, const char* msg) {
  set_contextless_error(msg);
  return code;
}

}  // namespace

extern "C" int msllr_blocksvt_noalloc(const float* A, float* Z, int M, int N, int ld, int bm,
                                      int bn, double tau, int shift_r, int shift_c,
                                      int* block_rank_out, void* cuda_stream) {
  if (!A || !Z || M <= 0 || N <= 0 || ld < N)
    return err(MSLLR_EINVAL, "msllr_blocksvt_noalloc: bad matrix arguments");
  if (!(tau >= 0.0) || !isfinite(tau))
    return err(MSLLR_EINVAL, "msllr_blocksvt_noalloc: tau must be finite and >= 0");
  if (bm <= 0 || bn <= 0 || bm > M || bn > N || M % bm || N % bn)
    return err(MSLLR_EINVAL, "msllr_blocksvt_noalloc: block does not divide the matrix");
  if ((bm < bn ? bm : bn) > 256)
    return err(MSLLR_EINVAL, "msllr_blocksvt_noalloc: blocks wider than 256 need msllr_blocksvt");
  if (choose_path(bm, bn) == ScalePath::Big && (long long)(M / bm) * (N / bn) > 65535)
    return err(MSLLR_EINVAL, "msllr_blocksvt_noalloc: too many wide blocks (max 65535)");
  const char* a0 = (const char*)A;
  const char* z0 = (const char*)Z;
  const size_t span = sizeof(float) * ((size_t)(M - 1) * ld + N);
  if (a0 < z0 + span && z0 < a0 + span)
    return err(MSLLR_EINVAL, "msllr_blocksvt_noalloc: A and Z overlap");
  const size_t need = 256 + big_workspace_bytes(M, N, bm, bn);
  if (need > (size_t)MSLLR_NOALLOC_SCRATCH_BYTES) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "msllr_blocksvt_noalloc: needs %zu bytes of scratch, more than the fixed %d",
             need, MSLLR_NOALLOC_SCRATCH_BYTES);
    return err(MSLLR_EINVAL, msg);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return err(MSLLR_ECUDA, "msllr_blocksvt_noalloc: no current CUDA device");
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      // one-time set-up on this device (the current one): the scratch's device
      // address and the kernels' shared-memory attributes
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return err(MSLLR_ECUDA, "msllr_blocksvt_noalloc: cudaGetSymbolAddress failed");
      }
      if (configure_kernels() != cudaSuccess) {
        cudaGetLastError();
        return err(MSLLR_ECUDA, "msllr_blocksvt_noalloc: kernel attributes");
      }
      g_scratch_ptr[dev] = p;
    }
    base = g_scratch_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int* shift = (int*)base;
  set_shift_kernel<<<1, 1, 0, st>>>(shift, ((shift_r % M) + M) % M, ((shift_c % N) + N) % N);
  ScaleLaunch s{};
  s.A1 = A;
  s.A2 = nullptr;
  s.Zout = Z;
  s.Wout = nullptr;
  s.M = M;
  s.N = N;
  s.ld = ld;
  s.m = bm;
  s.n = bn;
  s.shift = shift;
  s.tau = (float)tau;
  s.skip_bound = 1;
  s.rank_out = block_rank_out;
  s.err = shift + 2;
  const BigWorkspace w = carve_big_workspace((char*)base + 256, M, N, bm, bn);
  cudaError_t e = cudaGetLastError();
  int timed_out = 0;
  if (e == cudaSuccess) e = launch_scale(s, w, st, nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&timed_out, shift + 2, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return err(MSLLR_ECUDA, cudaGetErrorString(e));
  if (timed_out) return err(MSLLR_ECUDA, "msllr_blocksvt_noalloc: a tensor-core wait timed out");
  return MSLLR_OK;
}
