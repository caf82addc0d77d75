/*
 * msllr.h -- C ABI of the GB300 multi-scale low rank decomposition library.
 *
 * Computes the multi-scale low rank decomposition of Ong & Lustig, "Beyond
 * Low Rank + Sparse: Multi-scale Low Rank Matrix Decomposition": given an
 * M x N matrix Y and a multi-scale block partition {m_i x n_i}, i = 1..L
 * (Sec. 2), solve the convex program eq:cvx
 *       minimise sum_i lambda_i ||X_i||_(i)   subject to   Y = sum_i X_i
 * by the ADMM iteration eq:admm (Sec. 7), whose Z-update is the block-wise
 * singular value threshold eq:bsvt applied under a random cycle-spin shift
 * (Sec. 9), with the masked X-update of Sec. 10.4 when a mask is given.
 *
 * Conventions for every call:
 *  - Matrices are float32, row-major.  "Device" pointers are CUDA device
 *    memory of the context's device; "host" pointers are ordinary (pinned or
 *    pageable) host memory.  The caller owns every buffer it passes; the
 *    library never frees or retains them past the call.
 *  - Work is ordered on the context's CUDA stream.  Calls are synchronous
 *    with respect to the host unless stated otherwise: when they return
 *    MSLLR_OK, every output has been written.
 *  - Every call returns an msllr_status.  On any error nothing of the
 *    outputs is guaranteed; msllr_last_error() gives a one-line message.
 *    No C++ exception ever crosses this interface.
 *  - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef MSLLR_H
#define MSLLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum msllr_status {
  MSLLR_OK = 0,
  MSLLR_EINVAL = 1,      /* bad shape, block size, parameter or pointer      */
  MSLLR_ENOMEM = 2,      /* device allocation failed or HBM budget exceeded  */
  MSLLR_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed      */
  MSLLR_ETIMEOUT = 4,    /* a bounded wait ran out                           */
  MSLLR_ENONFINITE = 5,  /* Y holds a NaN or an infinity                     */
  MSLLR_EBUSY = 6        /* the serving queue is full                        */
} msllr_status;

/* Largest number of scales per decomposition. */
#define MSLLR_MAX_SCALES 8
/* Kernel kinds reported in msllr_stats.kernel_ms / kernel_launches:
 * 0 shift advance, 1 consensus residual, 2 1x1 soft threshold, 3 fused
 * narrow-block SVT, 4 wide-block Gram tiles, 5 Gram partial-sum reduce,
 * 6 wide-block eigen-solve, 7 wide-block rebuild, 8 set-up and output
 * kernels (finiteness check, state init, X/U output), 9 wide-block
 * Householder fallback (blocks the certified paths did not settle),
 * 10 subspace iteration of blocks wider than 256 (G V, orthonormalisation,
 * Rayleigh-Ritz), 11 their tiled Cholesky certificate. */
#define MSLLR_KERNEL_KINDS 12

/* Widest block (min(m_i, n_i)) the block-SVT kernels accept; the full-matrix
 * scale obeys the same limit on min(M, N).  Blocks up to 256 wide are solved
 * by one CTA each; wider ones (e.g. the full-matrix scale of a 1024 x 1024
 * matrix) by certified subspace iteration spread over many CTAs, where a
 * block's thresholded rank is at most 16. */
#define MSLLR_MAX_BLOCK_WIDTH 8192

typedef struct msllr_ctx msllr_ctx;

/* Options of msllr_decompose.  Zero-initialise and call
 * msllr_params_default() to get the defaults listed per field. */
typedef struct msllr_params {
  int skip_bound;    /* 1 (default): certified shortcuts -- skip a block whose
                        upper bound on sigma_max is <= tau (Sec. 8: trace,
                        Gershgorin, or a Cholesky of tau^2 I - G), and for
                        wide blocks find the pairs above tau by certified
                        Lanczos before falling back to Householder.
                        0: every block takes the full Householder
                        eigen-solve (reference path).                       */
  int cycle_spin;    /* 1 (default): one random circular shift per
                        iteration shared by all scales (Sec. 9).  0: none. */
  int use_graph;     /* 1 (default): replay one captured CUDA graph per
                        iteration.  0: plain launches.                      */
  int iter_offset;   /* index of the first shift-table entry used (default
                        0); lets a run continue another one exactly.       */
  const float* Z_init; /* device, L x M x N, or NULL (default: zeros)       */
  const float* U_init; /* device, L x M x N, or NULL (default: zeros)       */
  float* U_out;        /* device, L x M x N, or NULL: final U_i             */
  int profile;         /* 1: time every kernel with CUDA events on the
                          context stream, scales one after the other (plain
                          launches, no graph), into msllr_stats.kernel_ms.
                          2: scales run concurrently as usual and each
                          scale's whole segment is timed (kind 6 for wide
                          scales, 3 for the others).  Default 0.            */
  int spin_grid;       /* averaged cycle spinning (Sec. 9).  0 or 1 (default):
                          one shift per iteration.  g > 1: every scale of
                          m x n blocks (not 1x1, not the full matrix, not the
                          noise scale) averages its Z-update over the shifts
                          s + (a m / g_r, b n / g_c), 0 <= a < g_r, 0 <= b <
                          g_c, g_r = min(g, m), g_c = min(g, n) (which must
                          divide m and n; else EINVAL), s the iteration's
                          random shift (0 with cycle_spin = 0).  g >= the
                          block size averages over every distinct shift:
                          the update then commutes with translations.  Costs
                          g_r g_c block SVTs per scale and iteration; block
                          counts in msllr_stats add up over the shifts and
                          scale_nuclear is their mean.                      */
  int plain;           /* 1: the plain FP32 comparator path, for measurement:
                          every block of every scale is solved by its own
                          kernel launch (one CTA: Gram matrix, cyclic Jacobi
                          eigen-decomposition, threshold, rebuild), with no
                          skip bound, no certificate, no CUDA graph and no
                          concurrent scales; the 1x1 and noise scales are one
                          element-wise launch each.  Blocks up to 256 wide;
                          not with spin_grid > 1 (EINVAL).  Default 0.      */
  double stop_tol;     /* > 0: stopping test of the ADMM (Boyd et al. 2011,
                          Sec. 3.3; the paper fixes none): every stop_every
                          iterations, FP64 sums give the primal residual
                          r = ||X - Z||_F and the dual residual
                          s = rho ||Z - Z_prev||_F of that iteration; once
                          r <= stop_tol ||Z||_F and s <= stop_tol rho ||U||_F
                          the run ends after one more iteration (the one
                          that collects msllr_stats), which may be before
                          `iters`.  0 (default): exactly `iters`.           */
  int stop_every;      /* iterations between stopping tests; 0 means 10.   */
  int frame_w;         /* spatio-temporal blocks (Sec. 10.2): Y is a video
                          of M = H x frame_w pixels (row y frame_w + x for
                          pixel (y, x)) by N frames.  0 (default): none.    */
  const int* st_patch_w; /* host, L values, or NULL.  st_patch_w[i] = bw > 0
                          makes scale i the bh x bw x bt partition of the
                          video cube with bh = block_m[i] / bw and
                          bt = block_n[i]: each block is the (bh bw) x bt
                          matrix of a pixel patch (pixels in row-major
                          order) over bt frames, and the iteration's shift
                          (s_r, s_c) moves the cube by (s_r div frame_w,
                          s_r mod frame_w) pixels and s_c frames.  Needs
                          frame_w > 0 with bh | H, bw | frame_w, bt | N;
                          not with spin_grid > 1.  0 or NULL: 2-D blocks.  */
  int nested;          /* cross-scale tile fusion.  1: a narrow scale whose
                          blocks nest inside the blocks of a 33-64-wide
                          square scale (e.g. 16 x 16 inside 64 x 64) is
                          solved in the same kernel: one CTA per coarse
                          block reads the residual R once into shared memory
                          and solves the fine blocks inside it, then the
                          coarse block (the shift is shared, Sec. 9).  The
                          results equal the separate kernels' bit for bit.
                          Applies to 2-D blocks of single jobs with
                          spin_grid <= 1; other scales run as usual.
                          Default 0.                                       */
} msllr_params;

/* Per-run diagnostics, taken at the last iteration; when params->profile is
 * set, the block counts (blocks_skipped .. blocks_householder,
 * blocks_uncertified) and flops are summed over all iterations instead. */
typedef struct msllr_stats {
  int iters;                                  /* iterations run (fewer than
                                                 asked when the stopping
                                                 test ended the run)          */
  int L;                                      /* scales                       */
  double objective;                           /* sum_i lambda_i ||Z_i||_(i),
                                                 blocks taken on the grid of
                                                 the last iteration's shift   */
  double primal_residual;                     /* ||X - Z||_F over all scales  */
  double scale_nuclear[MSLLR_MAX_SCALES];     /* ||Z_i||_(i) per scale        */
  long long blocks[MSLLR_MAX_SCALES];         /* blocks per scale             */
  long long blocks_skipped[MSLLR_MAX_SCALES]; /* blocks the bound skipped     */
  long long blocks_zero[MSLLR_MAX_SCALES];    /* blocks whose certified rank
                                                 above tau was 0 (incl. skip) */
  double lambda[MSLLR_MAX_SCALES];            /* lambda_i actually used       */
  long long blocks_lanczos[MSLLR_MAX_SCALES]; /* eigenpairs by certified Lanczos
                                                 (blocks up to 256 wide) or by
                                                 certified subspace iteration
                                                 (wider blocks)               */
  long long blocks_householder[MSLLR_MAX_SCALES]; /* by the Householder path   */
  long long launches;                         /* kernels launched by the call */
  /* per kernel kind (see MSLLR_KERNEL_KINDS) and scale (kinds 0, 1 and 8
   * use scale slot 0): launches, and summed device time in ms when
   * params->profile was set (else 0). */
  long long kernel_launches[MSLLR_KERNEL_KINDS][MSLLR_MAX_SCALES];
  double kernel_ms[MSLLR_KERNEL_KINDS][MSLLR_MAX_SCALES];
  /* blocks wider than 256 whose certificate (no singular value above tau
   * outside the kept Ritz pairs) failed at the last iteration; their
   * thresholded rank is taken from the Ritz pairs.  0 in normal runs. */
  long long blocks_uncertified[MSLLR_MAX_SCALES];
  /* FP32 flops of the block eigen-solve steps that ran, each step counted
   * at its algorithmic cost (a multiply-add is 2 flops): zero-rank and
   * deflated Cholesky certificates n^3/3, Lanczos and power steps,
   * Householder tridiagonalisation 4n^3/3.  `flops`: the fused narrow-block
   * kernel (its Gram and rebuild included) or the wide-block eigen kernel;
   * `flops_fallback`: the wide-block Householder fallback kernel.  Blocks up
   * to 256 wide; 0 for the other paths. */
  long long flops[MSLLR_MAX_SCALES];
  long long flops_fallback[MSLLR_MAX_SCALES];
  /* rho ||Z - Z_prev||_F over all scales at the last iteration (FP64), the
   * dual residual of the ADMM; with primal_residual it is what the
   * stopping test reads. */
  double dual_residual;
  int stopped;                                /* 1: params->stop_tol ended the
                                                 run before `iters`          */
  int serve_jobs_running;                     /* serving queue: jobs running
                                                 on the device, this one
                                                 included, when it was
                                                 admitted; 0 for direct calls */
} msllr_stats;

/* Fill *p with the defaults.  Returns MSLLR_EINVAL if p is NULL. */
int msllr_params_default(msllr_params* p);

/* Create a context on CUDA device `device`.  `hbm_budget_bytes` caps the
 * device memory the context may hold (0 = no cap).  `cuda_stream` is a
 * cudaStream_t to order work on, or NULL for a stream the context creates.
 * Errors: EINVAL (out == NULL, bad device), ECUDA. */
int msllr_create(msllr_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream);

/* Destroy a context and free everything it holds.  NULL is accepted. */
int msllr_destroy(msllr_ctx* ctx);

/* Last error message of the context, or, when ctx is NULL, of the calling
 * host thread's last failed context-less call.  Valid until the next call on
 * the same context (or, for NULL, the next context-less call of the thread). */
const char* msllr_last_error(const msllr_ctx* ctx);

/* Shift table of the random cycle spinning (Sec. 9): for k = 0..iters-1,
 * z = splitmix64(seed + (k+1) * 0x9E3779B97F4A7C15) and
 *   out[2k] = (z >> 32) mod M,  out[2k+1] = (z & 0xffffffff) mod N.
 * `out` is host memory of 2*iters int32.  Errors: EINVAL. */
int msllr_shift_table(uint64_t seed, int iters, int M, int N, int32_t* out);

/* Default regularisation eq:lambda (Sec. 4, as used in Sec. 10):
 *   lambda = sqrt(m) + sqrt(n) + sqrt(log(M N / max(m, n))).
 * For the noise scale (m = n = 0, see MSLLR_NOISE_SCALE) the block is
 * MN x 1: lambda = sqrt(M N) + 1.
 * Errors: EINVAL when the block does not fit in the matrix. */
int msllr_lambda_default(int M, int N, int m, int n, double* out);

/* Block size (m, n) = (0, 0) selects the noise scale of Sec. 2.1: the whole
 * matrix reshaped to one MN x 1 block, whose nuclear norm is the Frobenius
 * norm, so that its SVT is A max(1 - tau / ||A||_F, 0).  Accepted wherever a
 * block size is (not by msllr_blocksvt_noalloc). */
#define MSLLR_NOISE_SCALE 0

/* One block-wise singular value threshold, eq:bsvt (Sec. 7), under the
 * circular shift s = (shift_r, shift_c) of Sec. 9:
 *     Z = Shift_{-s}( BlockSVT_tau( Shift_s(A) ) ),
 * with Shift_s(A)[r, c] = A[(r + s_r) mod M, (c + s_c) mod N] and blocks of
 * bm x bn on the shifted grid.  A and Z are device pointers, M x N with row
 * stride `ld` (>= N) elements; A and Z must not overlap.  If
 * `block_rank_out` is not NULL it receives, per block in row-major block
 * order, the number of singular values above tau (device int32,
 * (M/bm)*(N/bn) entries; one for the noise scale).  Errors: EINVAL (bm, bn
 * do not divide M, N; min(bm, bn) > MSLLR_MAX_BLOCK_WIDTH; tau < 0), ECUDA. */
int msllr_blocksvt(msllr_ctx* ctx, const float* A, float* Z, int M, int N, int ld,
                   int bm, int bn, double tau, int shift_r, int shift_c,
                   int* block_rank_out);

/* Multi-scale low rank decomposition, eq:cvx by eq:admm (Sec. 7) with the
 * random cycle-spin Z-update of Sec. 9:
 *   X_i <- (Z_i - U_i) + (1/L)(Y - sum_j (Z_j - U_j))
 *   Z_i <- Shift_{-s}(BlockSVT_{lambda_i/rho}(Shift_s(X_i + U_i)))
 *   U_i <- U_i - (Z_i - X_i)
 * starting from Z_i = U_i = 0 (or params->Z_init / U_init).
 *  Y        device, M x N, row stride ld (>= N).
 *  block_m, block_n   host arrays of L block sizes; each must divide M, N;
 *           min(m_i, n_i) <= MSLLR_MAX_BLOCK_WIDTH; (0, 0) is the noise
 *           scale (MSLLR_NOISE_SCALE).
 *  lambda   host array of L values > 0, or NULL for msllr_lambda_default.
 *  rho      > 0.
 *  seed     seeds the shift table (msllr_shift_table).
 *  mask     device uint8 M x N (row stride N), nonzero = observed, or NULL.
 *           With a mask the X-update of Sec. 10.4 is used: the residual
 *           term is zero at unobserved entries and Y there is ignored.
 *  X_out    device, L x M x N (dense): the X-update of eq:admm applied to
 *           the final (Z, U), so that sum_i X_i = Y on observed entries.
 *  Z_out    device, L x M x N, or NULL.
 *  stats    host, or NULL.
 * Errors: EINVAL, ENOMEM (budget), ENONFINITE (Y has NaN/Inf), ECUDA. */
int msllr_decompose(msllr_ctx* ctx, const float* Y, int M, int N, int ld,
                    int L, const int* block_m, const int* block_n,
                    const double* lambda, double rho, int iters, uint64_t seed,
                    const uint8_t* mask, const msllr_params* params,
                    float* X_out, float* Z_out, msllr_stats* stats);

/* Batched decompositions: `batch` independent jobs of one shape (M x N, the
 * same scales, lambda and rho), each the eq:admm iteration of
 * msllr_decompose with its own cycle-spin shift sequence (seeds[j], as
 * msllr_shift_table), run together so that every kernel launch of an
 * iteration covers the blocks of all jobs (one CUDA graph per iteration for
 * the whole batch).  Job j's result equals msllr_decompose of that job alone.
 *  Y        device, the jobs stacked row-wise: batch x M rows of N, row
 *           stride ld (job j at Y + j M ld).
 *  seeds    host array of batch shift seeds.
 *  mask     device uint8 batch x M x N, or NULL.
 *  X_out    device, L x batch x M x N: for scale i the stacked jobs at
 *           X_out + i batch M N (job j at + j M N).  Z_out likewise or NULL.
 *  stats    host or NULL: block counts and the objective summed over jobs.
 * Not with the noise scale, spin_grid > 1, spatio-temporal scales or an
 * initial state (EINVAL).  Errors as msllr_decompose. */
int msllr_decompose_batch(msllr_ctx* ctx, int batch, const float* Y, int M, int N, int ld, int L,
                          const int* block_m, const int* block_n, const double* lambda, double rho,
                          int iters, const uint64_t* seeds, const uint8_t* mask,
                          const msllr_params* params, float* X_out, float* Z_out,
                          msllr_stats* stats);

/* Same as msllr_decompose, but Y, mask, X_out and Z_out are HOST pointers:
 * the library copies Y (and mask) to the device, runs, and copies the
 * results back before returning.  params->Z_init / U_init / U_out must be
 * NULL here. */
int msllr_decompose_host(msllr_ctx* ctx, const float* Y, int M, int N, int ld,
                         int L, const int* block_m, const int* block_n,
                         const double* lambda, double rho, int iters, uint64_t seed,
                         const uint8_t* mask, const msllr_params* params,
                         float* X_out, float* Z_out, msllr_stats* stats);

/* ---- serving queue ------------------------------------------------------
 * Independent decompositions submitted to one context run concurrently on
 * its device (the jobs and their sizes are those of msllr_decompose,
 * eq:admm with the Sec. 9 cycle spin; the queue itself is plumbing around
 * it).  MSLLR_SERVE_SLOTS worker threads of the library, each with a stream
 * and workspace of its own, take the queued jobs in submission order: the
 * job at the head of the queue starts as soon as a slot is free and the
 * device memory held by the running jobs plus its own footprint fits the
 * context's HBM budget (no budget: as soon as a slot is free).  A job holds
 * device memory only while it runs.  Its inputs (Y, mask, block sizes,
 * lambda, params and the arrays they point to) are copied at submission;
 * its outputs go to the caller's HOST buffers, which must stay valid until
 * msllr_poll reports the job done or msllr_wait returns.  A job's result
 * does not depend on the jobs that run beside it.  While jobs are queued
 * or running, msllr_decompose, msllr_decompose_host and msllr_blocksvt on
 * the same context return MSLLR_EBUSY.  Destroying the context lets the
 * running jobs finish and drops the queued ones. */

/* Jobs that may wait in the queue of one context. */
#define MSLLR_SERVE_QUEUE 64
/* Jobs of one context that run on the device at the same time. */
#define MSLLR_SERVE_SLOTS 4

typedef struct msllr_job {
  const float* Y;          /* host, M x N row-major with row stride ld       */
  int M, N, ld;
  int L;                   /* scales, 1..MSLLR_MAX_SCALES                     */
  const int* block_m;      /* L block heights (divide M)                      */
  const int* block_n;      /* L block widths (divide N)                       */
  const double* lambda;    /* L weights, or NULL for the eq:lambda default   */
  double rho;              /* ADMM penalty, > 0                               */
  int iters;
  uint64_t seed;           /* cycle-spin shift sequence                       */
  const uint8_t* mask;     /* host M x N (row stride N), 1 = observed, or NULL */
  const msllr_params* params;  /* or NULL; its device-state pointers must be NULL */
  float* X_out;            /* host L x M x N: the decomposition X_i           */
  float* Z_out;            /* host L x M x N block-low-rank Z_i, or NULL      */
  msllr_stats* stats;      /* host, or NULL                                   */
} msllr_job;

/* Queue a job; *job_id identifies it for msllr_poll / msllr_wait.  Checks
 * the arguments (EINVAL) and accepts the job only if its device footprint
 * (workspace plus input and output copies) alone fits the context's HBM
 * budget (ENOMEM); EBUSY when MSLLR_SERVE_QUEUE jobs are already waiting. */
int msllr_submit(msllr_ctx* ctx, const msllr_job* job, uint64_t* job_id);

/* *done = 1 once the job has finished, 0 before.  When it reports done the
 * job leaves the queue's table and the call returns the job's own status
 * (OK, or the error the decomposition returned, message in
 * msllr_last_error); EINVAL for an unknown or already collected id. */
int msllr_poll(msllr_ctx* ctx, uint64_t job_id, int* done);

/* Wait up to timeout_ms (< 0: without limit) for the job, then return its
 * status as msllr_poll does; ETIMEOUT if it has not finished by then (the
 * job stays queued and can be waited for again).  EINVAL for an unknown id,
 * and when another thread's msllr_poll or msllr_wait collected the job while
 * this call waited (a job's status is handed out once). */
int msllr_wait(msllr_ctx* ctx, uint64_t job_id, int timeout_ms);

/* Bytes of the fixed device scratch used by msllr_blocksvt_noalloc. */
#define MSLLR_NOALLOC_SCRATCH_BYTES (32 * 1024 * 1024)

/* msllr_blocksvt without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- processes whose device memory is handed out by their own
 * pool allocator and must not be claimed behind its back by a library, and
 * loops that cannot afford the device-wide synchronisation that
 * cudaMalloc/cudaFree imply.  It needs no msllr_ctx.
 *
 * Computes exactly what msllr_blocksvt computes, with the same argument
 * meaning (block sizes that divide the matrix; not the noise scale), on the
 * stream `cuda_stream` (a cudaStream_t, or NULL for the legacy default
 * stream) of the current CUDA device, and returns after that stream has
 * finished the work.  Its workspace is one fixed array of
 * MSLLR_NOALLOC_SCRATCH_BYTES in device memory that every GPU loading the
 * library holds until the process exits; a call whose workspace would not
 * fit (many or wide blocks; the 1x1 and narrow-block paths need almost
 * none) fails with MSLLR_EINVAL and a message giving the size.
 *
 * The first call on a device does a one-time set-up on that device (it
 * looks up the scratch's device address and sets kernel attributes).
 * Every call shares the one
 * scratch array and leaves its contents behind: calls that overlap on the
 * GPU (other host threads, other streams) race and must be serialised by
 * the caller.  Errors: EINVAL, ECUDA; the message is available from
 * msllr_last_error(NULL) on the calling thread. */
int msllr_blocksvt_noalloc(const float* A, float* Z, int M, int N, int ld, int bm, int bn,
                           double tau, int shift_r, int shift_c, int* block_rank_out,
                           void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MSLLR_H */
