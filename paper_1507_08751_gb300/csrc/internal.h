// Internal interfaces between the host API (msllr_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

namespace msllr {

// Block-SVT launch description for one scale (eq:bsvt under the Sec. 9
// shift).  The prox input is A = A1 + A2 (A2 may be null); the kernels write
// Z' = Shift_{-s}(BlockSVT_tau(Shift_s(A))) to Zout (which may alias A1) and,
// if Wout is not null, W' = 2 Z' - A, the ADMM state Z' - U' with
// U' = A - Z' (the dual update of eq:admm).
struct ScaleLaunch {
  const float* A1;
  const float* A2;
  float* Zout;
  float* Wout;
  int M, N, ld;            // matrix shape and row stride of A1, A2, Zout, Wout
  int m, n;                // block shape
  const int* shift;        // device int[2]: current (s_r, s_c)
  int shift_add_r, shift_add_c;  // added to the shift (averaged cycle spinning)
  float tau;
  int skip_bound;
  int warm_start;          // wide blocks: start Lanczos from the previous call's Ritz
                           // vectors (only where the block grid does not move)
  int* rank_out;           // device, one int per block, or null
  double* nuc_acc;         // device, += sum over blocks of sum_j (sigma_j - tau)_+, or null
  unsigned long long* cnt; // device [4]: blocks skipped by a bound, blocks of rank 0,
                           // blocks solved by certified Lanczos, by Householder; or null
  double* norm_acc;        // device scratch double (noise scale: ||A||_F^2)
  int fw;                  // spatio-temporal blocks (Sec. 10.2): frame width of the
                           // video whose pixels are the rows (0: 2-D blocks)
  int bw;                  // their patch width (patch height m / bw, n frames)
  int rows;                // batched jobs: rows of one job (M = jobs x rows, job j
                           // at rows j rows ..; its shift at shift[2 j]); 0: one job
  int* err;                // device flag, or null: set non-zero by a kernel whose
                           // bounded wait on the tensor cores ran out
};

// rows of one job of a launch (the whole M unless jobs are batched)
__host__ __device__ __forceinline__ int launch_rows(const ScaleLaunch& s) {
  return s.rows ? s.rows : s.M;
}

// index of block b within its own job (seeds that depend on it then do not
// depend on the batch the job runs in)
__host__ __device__ __forceinline__ int job_block(const ScaleLaunch& s, int b) {
  return s.rows ? b % ((s.rows / s.m) * (s.N / s.n)) : b;
}

// Device workspace needed by the wide-block path for one scale.
struct BigWorkspace {
  float* G;      // nblocks * nn * nn; block b at b * nn * nn, lower triangle packed row by row
  float* part;   // nblocks * chunks * ntiles * 64 * 64 (when chunks > 1)
  float* Y;      // nblocks * ystride: eigenvectors / Lanczos scratch per block
  int* k;        // nblocks
  float* warm;   // nblocks * 8 * nn: previous Ritz vectors (warm start)
  int* kwarm;    // nblocks: how many of them (0 = none)
  size_t ystride;
  // blocks wider than 256 (k_block_huge.cu): G is a full square there
  float* H;      // nblocks * nn * nn: certificate matrix, factored in place
  float* tstat;  // nblocks * ntiles * 2: per-tile diagonal sums, sums of squares
  float* V;      // nblocks * nn * 32: subspace basis (kept across calls)
  float* Wv;     // nblocks * nn * 32: G V
  float* U;      // nblocks * nn * 16: Ritz vectors
  float* GU;     // nblocks * nn * 16: G U, then What
  void* hb;      // nblocks per-block states
};

// Kernel kinds, for launch counting and per-kernel CUDA-event timing.
enum KernelKind {
  KK_ADVANCE = 0,
  KK_CONSENSUS,
  KK_SOFT1X1,
  KK_FUSED,
  KK_GRAM,
  KK_GRAM_REDUCE,
  KK_EIG,
  KK_REBUILD,
  KK_MISC,
  KK_EIG_FALLBACK,
  KK_SUBSPACE,  // wide blocks over 256: G V, orthonormalisation, Rayleigh-Ritz
  KK_CERT,      // wide blocks over 256: the tiled Cholesky certificate
  KK_COUNT
};

// Launch counter and optional event timer.  With `timing` set, every kernel
// is bracketed by two events on its own stream; the host sums the elapsed
// times per (kind, scale) after the run.
struct Prof {
  bool timing = false;
  bool per_scale = false;  // time whole per-scale segments in the forked iteration
  int scale = 0;
  long long launches[KK_COUNT][8] = {};
  std::vector<cudaEvent_t> ev;
  std::vector<int> tag;
  size_t used = 0;
  cudaError_t before(cudaStream_t st, int kind) {
    launches[kind][scale]++;
    if (!timing) return cudaSuccess;
    if (2 * used + 2 > ev.size()) {
      for (int i = 0; i < 256; ++i) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ev.push_back(e);
      }
    }
    tag.push_back(kind * 8 + scale);
    return cudaEventRecord(ev[2 * used], st);
  }
  cudaError_t after(cudaStream_t st) {
    if (!timing) return cudaSuccess;
    cudaError_t r = cudaEventRecord(ev[2 * used + 1], st);
    ++used;
    return r;
  }
};

// Path selection.
// Noise: block (0, 0), Sec. 2.1; Huge: min(m, n) > 256
enum class ScalePath { Elementwise, Small, Big, Noise, Huge };
ScalePath choose_path(int m, int n);
// Bytes of BigWorkspace a scale needs (0 for the other paths).
size_t big_workspace_bytes(int M, int N, int m, int n);
BigWorkspace carve_big_workspace(void* base, int M, int N, int m, int n);
// The wide path above 256 (k_block_huge.cu).
size_t huge_workspace_bytes(int M, int N, int m, int n);
BigWorkspace carve_huge_workspace(void* base, int M, int N, int m, int n);
cudaError_t reset_huge_basis(const BigWorkspace& w, int M, int N, int m, int n, cudaStream_t st);
cudaError_t launch_huge(const ScaleLaunch& s, const BigWorkspace& ws, cudaStream_t st, Prof* prof,
                        cudaEvent_t after_gram);
// Zero the warm-start counts of a scale's workspace (start of a decomposition).
cudaError_t reset_warm_start(const BigWorkspace& w, int M, int N, int m, int n, cudaStream_t st);

// Streaming multiprocessors of the current device (queried once per device
// and cached; configure_kernels() primes the cache outside any capture).
int sm_count();

// Narrow blocks with one warp per block (k_block_warp.cu): the block shapes
// it takes (min(m, n) <= 16, max(m, n) <= 32) and its launcher.
bool warp_path(int m, int n);
cudaError_t launch_warp(const ScaleLaunch& s, cudaStream_t st, Prof* prof);

// The plain one-block-per-launch comparator (k_plain.cu): global scratch a
// scale needs (0 when the block fits shared memory), kernel attributes, and
// the per-scale launcher (one launch per block).
size_t plain_scratch_bytes(int m, int n);
cudaError_t configure_plain_kernels();
cudaError_t launch_plain(const ScaleLaunch& s, float* scratch, cudaStream_t st, Prof* prof);

// Message returned by msllr_last_error(NULL).
void set_contextless_error(const char* msg);

// Debug phase timing buffers (see PHASE in common.cuh).
cudaError_t set_phase_buffer_small(unsigned long long* p);
cudaError_t set_phase_buffer_big(unsigned long long* p);
cudaError_t set_phase_buffer_warp(unsigned long long* p);

// Set kernel attributes (dynamic shared memory opt-in) on the current device.
cudaError_t configure_kernels();

// Gram matrices of wide blocks on the tensor cores (k_gram_tc.cu): eligible
// launches (m >= n, n > 64, fewer than 2^31 elements), kernel attributes, and the launch, which
// writes G packed (chunks == 1) or the per-chunk partial sums in the 64 x 64
// tile layout of the FP32 Gram path (ntiles64 tiles per chunk).
bool gram_tc_eligible(const ScaleLaunch& s);

// Cross-scale tile fusion (k_nested.cu): whether fine blocks fm x fn (warp
// path) nest in coarse blocks cm x cn (64-wide CTA path) for one kernel, its
// attributes, and the launch of both scales' block SVTs (same shift, 2-D
// blocks, one job, the same A2 = R).
bool nested_pair(int fm, int fn, int cm, int cn);
cudaError_t configure_nested();
struct Prof;
cudaError_t launch_nested(const ScaleLaunch& fine, const ScaleLaunch& coarse, cudaStream_t st,
                          Prof* prof);
cudaError_t configure_gram_tc();
// chunk_rows: rows of C per partial sum; to_part: write the partial sums
// even for one chunk (the wide path above 256 reduces them itself)
cudaError_t launch_gram_tc(const ScaleLaunch& s, float* G, float* part, int chunks, int nblocks,
                           int ntiles64, int chunk_rows, int to_part, cudaStream_t st);
// MSLLR_GRAM_FP32=1: the FP32 CUDA-core Gram kernels instead (comparisons)
bool gram_fp32_forced();

// Launchers (all asynchronous on `st`).  Return cudaGetLastError().
cudaError_t launch_scale(const ScaleLaunch& s, const BigWorkspace& ws, cudaStream_t st,
                         Prof* prof, cudaEvent_t after_gram = nullptr);

// R = (1/L)(Y - sum_j W_j); with Z11 (and W11, tau11) given, the 1x1
// scale's soft threshold and dual update in the same pass.
cudaError_t launch_consensus(const float* Y, const float* W, float* R, const uint8_t* mask,
                             int L, size_t MN, cudaStream_t st, Prof* prof = nullptr,
                             float* Z11 = nullptr, float* W11 = nullptr, float tau11 = 0.f);
// X_out = W + R, U_out = Z - W; FP64 ||X - Z||^2 into pres_acc[0] and, with
// `dual` (X_out holding the previous Z on entry), ||Z - Z_prev||^2 into
// pres_acc[1].
cudaError_t launch_finalize(const float* W, const float* Z, const float* R, float* X_out,
                            float* U_out, double* pres_acc, bool dual, int L, size_t MN,
                            cudaStream_t st, Prof* prof = nullptr);
// Stopping-test sums against the state (Zs, Ws) of one iteration earlier:
// acc4 += (||U - Us||^2, ||Z - Zs||^2, ||Z||^2, ||U||^2), U = Z - W.
cudaError_t launch_residual(const float* Z, const float* W, const float* Zs, const float* Ws,
                            double* acc4, size_t n, cudaStream_t st, Prof* prof = nullptr);
cudaError_t launch_init_state(const float* Z0, const float* U0, float* Z, float* W, int L,
                              size_t MN, cudaStream_t st, Prof* prof = nullptr);
// the shifts of iteration *iter (one pair per job, table iters x jobs x 2)
// into cur_shift, then ++*iter
cudaError_t launch_advance(const int* table, int* iter, int* cur_shift, int jobs, cudaStream_t st,
                           Prof* prof = nullptr);
cudaError_t launch_nonfinite(const float* Y, int M, int N, int ld, int* flag, cudaStream_t st,
                             Prof* prof = nullptr);
cudaError_t launch_copy_dense(const float* src, int M, int N, int ld, float* dst, cudaStream_t st,
                              Prof* prof = nullptr);
// Averaged cycle spinning: acc = w T (first) or acc += w T; then Z = acc,
// W = 2 acc - (Z + R) (the fused dual update of eq:admm on the average).
cudaError_t launch_spin_accum(float* acc, const float* T, float w, bool first, size_t MN,
                              cudaStream_t st, Prof* prof = nullptr);
cudaError_t launch_spin_finish(float* Z, float* W, const float* R, size_t MN, cudaStream_t st,
                               Prof* prof = nullptr);

}  // namespace msllr
