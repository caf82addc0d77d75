// Host side of the msllr C ABI (include/msllr.h): argument checks, the
// context's device memory, the shift table, and the ADMM driver loop of
// eq:admm (Sec. 7) with the random cycle-spin Z-update (Sec. 9).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/msllr.h"
#include "internal.h"

using namespace msllr;

namespace {

// message of the last failed call made without a context, one per host
// thread (msllr_last_error(NULL) reads the calling thread's copy)
thread_local std::string g_last_error;

}  // namespace

namespace msllr {
// Error message of calls made without a context (msllr_last_error(NULL)).
void set_contextless_error(const char* msg) { g_last_error = msg; }
}  // namespace msllr

// One job of the serving queue: its inputs are copied at submission, its
// outputs point into the caller's host memory.
struct ServeJob {
  uint64_t id = 0;
  int M = 0, N = 0, L = 0;
  std::vector<float> Y;
  std::vector<uint8_t> mask;
  std::vector<int> bm, bn;
  std::vector<double> lam;
  double rho = 1.0;
  int iters = 0;
  uint64_t seed = 0;
  msllr_params p{};
  bool has_p = false;
  std::vector<int> patch_w;  // copy of p.st_patch_w
  float* X_out = nullptr;
  float* Z_out = nullptr;
  msllr_stats* stats = nullptr;
  size_t need = 0;       // device bytes the job holds while it runs
  int running_with = 0;  // jobs running (this one included) when it was admitted
  int status = MSLLR_OK;
  bool done = false;
  std::string err;
};

struct msllr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  std::string err;

  // grow-only device workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // grow-only device copies of the host API's inputs and outputs
  void* io = nullptr;
  size_t io_bytes = 0;
  // small device scalars
  int* d_small = nullptr;          // [0] iter, [1..2] cur shift, [3] nonfinite flag, [4..5] tmp shift,
                                   // [6] device wait timeout flag
  double* d_acc = nullptr;         // [0..MAX) nuc per scale, [MAX] primal residual^2
  double* d_noise = nullptr;       // [MAX] noise-scale ||A||_F^2 scratch
  unsigned long long* d_cnt = nullptr;  // [2*MAX]
  int* d_table = nullptr;
  size_t table_cap = 0;
  int* d_shift = nullptr;          // current shift, one (s_r, s_c) pair per batched job
  int shift_cap = 0;               // pairs d_shift holds

  // one stream per scale: the scales of an iteration are independent given R.
  // Wide-block scales (the longest dependency chain) get high-priority
  // streams, the others low-priority ones.
  cudaStream_t side[MSLLR_MAX_SCALES] = {};
  cudaStream_t side_hi[MSLLR_MAX_SCALES] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[MSLLR_MAX_SCALES] = {};
  cudaEvent_t ev_gate[MSLLR_MAX_SCALES] = {};

  // error message; written under err_mu (the serving worker runs concurrently)
  std::mutex err_mu;

  // serving queue: MSLLR_SERVE_SLOTS worker threads, each with a slot
  // context of its own (stream, workspace, graph), take the queued jobs in
  // submission order as device memory allows, so that admitted jobs run
  // concurrently on the device
  std::mutex q_mu;
  std::condition_variable q_cv;     // wakes the workers
  std::condition_variable done_cv;  // a job finished
  std::deque<std::shared_ptr<ServeJob>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<ServeJob>> jobs;
  uint64_t next_job = 1;
  std::vector<msllr_ctx*> slots;
  std::vector<std::thread> workers;
  size_t serve_bytes = 0;   // device bytes held by the running jobs
  int serve_running = 0;    // running jobs
  bool stop = false;
  std::atomic<int> in_flight{0};
  // a serving slot's context: its workspace and slabs are allocated and
  // freed in stream order (cudaMallocAsync / cudaFreeAsync), so that one
  // slot's allocations never wait for the other slots' work
  bool serve_child = false;

  // cached graph of one iteration
  cudaGraphExec_t graph = nullptr;
  std::vector<char> graph_key;
  long long graph_launches[KK_COUNT][8] = {};
  unsigned long long* d_phase = nullptr;  // MSLLR_PHASE_TIMING debug accumulators
};

namespace {

int fail(msllr_ctx* ctx, int code, const std::string& msg) {
  if (ctx) {
    std::lock_guard<std::mutex> lk(ctx->err_mu);
    ctx->err = msg;
  } else {
    g_last_error = msg;
  }
  return code;
}

// calls that use the context's stream and workspace directly are refused
// while serving jobs are queued or running
int busy(msllr_ctx* ctx) {
  return ctx->in_flight.load() > 0
             ? fail(ctx, MSLLR_EBUSY, "serving jobs are in flight on this context")
             : MSLLR_OK;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(ctx, MSLLR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

uint64_t splitmix64(uint64_t x) {
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void fill_shift_table(uint64_t seed, int offset, int iters, int M, int N, int32_t* out) {
  for (int k = 0; k < iters; ++k) {
    const uint64_t z = splitmix64(seed + (uint64_t)(offset + k + 1) * 0x9E3779B97F4A7C15ull);
    out[2 * k] = (int32_t)((z >> 32) % (uint64_t)M);
    out[2 * k + 1] = (int32_t)((z & 0xffffffffull) % (uint64_t)N);
  }
}

double lambda_of(int M, int N, int m, int n) {
  // the noise scale (0, 0) is one MN x 1 block
  const double bm = (m == 0 && n == 0) ? (double)M * (double)N : (double)m;
  const double bn = (m == 0 && n == 0) ? 1.0 : (double)n;
  const double mx = bm > bn ? bm : bn;
  return sqrt(bm) + sqrt(bn) + sqrt(log((double)M * (double)N / mx));
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Make sure the context workspace holds at least `bytes`.
int ensure_ws(msllr_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return MSLLR_OK;
  if (ctx->budget && bytes + ctx->io_bytes > ctx->budget)
    return fail(ctx, MSLLR_ENOMEM,
                "workspace of " + std::to_string(bytes) + " bytes exceeds the HBM budget of " +
                    std::to_string(ctx->budget));
  if (ctx->ws) {
    if (ctx->serve_child) {
      cudaFreeAsync(ctx->ws, ctx->stream);
    } else {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->ws);
    }
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
    ctx->graph_key.clear();
  }
  cudaError_t e = ctx->serve_child ? cudaMallocAsync(&ctx->ws, bytes, ctx->stream)
                                   : cudaMalloc(&ctx->ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return fail(ctx, MSLLR_ENOMEM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
  }
  ctx->ws_bytes = bytes;
  return MSLLR_OK;
}

int check_blocks(msllr_ctx* ctx, int M, int N, int m, int n) {
  if (m == 0 && n == 0) return MSLLR_OK;  // the noise scale (Sec. 2.1)
  if (m <= 0 || n <= 0 || m > M || n > N || M % m || N % n)
    return fail(ctx, MSLLR_EINVAL,
                "block " + std::to_string(m) + "x" + std::to_string(n) + " does not divide " +
                    std::to_string(M) + "x" + std::to_string(N));
  const int nn = m < n ? m : n;
  if (nn > MSLLR_MAX_BLOCK_WIDTH)
    return fail(ctx, MSLLR_EINVAL,
                "block " + std::to_string(m) + "x" + std::to_string(n) +
                    " is wider than MSLLR_MAX_BLOCK_WIDTH");
  const long long nblocks = (long long)(M / m) * (N / n);
  const ScalePath path = choose_path(m, n);
  if ((path == ScalePath::Big || path == ScalePath::Huge) && nblocks > 65535)
    return fail(ctx, MSLLR_EINVAL, "too many wide blocks in one scale (max 65535)");
  return MSLLR_OK;
}

}  // namespace

extern "C" {

int msllr_params_default(msllr_params* p) {
  if (!p) return fail(nullptr, MSLLR_EINVAL, "params is NULL");
  memset(p, 0, sizeof(*p));
  p->skip_bound = 1;
  p->cycle_spin = 1;
  p->use_graph = 1;
  p->iter_offset = 0;
  return MSLLR_OK;
}

int msllr_create(msllr_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream) {
  msllr_ctx* ctx = nullptr;
  if (!out) return fail(nullptr, MSLLR_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(nullptr, MSLLR_EINVAL, "no CUDA device " + std::to_string(device));
  }
  ctx = new msllr_ctx();
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  auto bail = [&](int code) {
    g_last_error = ctx->err;
    msllr_destroy(ctx);
    return code;
  };
  if (cudaSetDevice(device) != cudaSuccess) return bail(fail(ctx, MSLLR_ECUDA, "cudaSetDevice"));
  if (configure_kernels() != cudaSuccess) return bail(fail(ctx, MSLLR_ECUDA, "kernel attributes"));
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreate(&ctx->stream) != cudaSuccess)
      return bail(fail(ctx, MSLLR_ECUDA, "cudaStreamCreate"));
    ctx->own_stream = true;
  }
  int prio_lo = 0, prio_hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess)
    return bail(fail(ctx, MSLLR_ECUDA, "cudaDeviceGetStreamPriorityRange"));
  for (int i = 0; i < MSLLR_MAX_SCALES; ++i)
    if (cudaStreamCreateWithPriority(&ctx->side[i], cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&ctx->side_hi[i], cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_gate[i], cudaEventDisableTiming) != cudaSuccess)
      return bail(fail(ctx, MSLLR_ECUDA, "cudaStreamCreate (scale streams)"));
  if (cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(ctx, MSLLR_ECUDA, "cudaEventCreate"));
  if (getenv("MSLLR_PHASE_TIMING")) {
    if (cudaMalloc(&ctx->d_phase, 8 * 16 * 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(ctx->d_phase, 0, 8 * 16 * 2 * sizeof(unsigned long long)) != cudaSuccess ||
        set_phase_buffer_small(ctx->d_phase) != cudaSuccess ||
        set_phase_buffer_big(ctx->d_phase) != cudaSuccess ||
        set_phase_buffer_warp(ctx->d_phase) != cudaSuccess)
      return bail(fail(ctx, MSLLR_ECUDA, "phase timing buffer"));
  }
  if (cudaMalloc(&ctx->d_small, 64 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_acc, (MSLLR_MAX_SCALES + 8) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_noise, MSLLR_MAX_SCALES * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_cnt, 8 * MSLLR_MAX_SCALES * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&ctx->d_shift, 2 * sizeof(int)) != cudaSuccess)
    return bail(fail(ctx, MSLLR_ENOMEM, "cudaMalloc of context scalars"));
  ctx->shift_cap = 1;
  *out = ctx;
  return MSLLR_OK;
}

int msllr_destroy(msllr_ctx* ctx) {
  if (!ctx) return MSLLR_OK;
  if (!ctx->workers.empty()) {
    {
      std::lock_guard<std::mutex> lk(ctx->q_mu);
      ctx->stop = true;  // the running jobs complete, queued ones are dropped
    }
    ctx->q_cv.notify_all();
    for (auto& w : ctx->workers) w.join();
  }
  for (msllr_ctx* child : ctx->slots) msllr_destroy(child);
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->io) cudaFree(ctx->io);
  if (ctx->d_phase) {
    unsigned long long h[8 * 16 * 2];
    if (cudaMemcpy(h, ctx->d_phase, sizeof h, cudaMemcpyDeviceToHost) == cudaSuccess) {
      static const char* names[8] = {"small32/warp", "small64", "small128", "eig_big", "eig_lanczos",
                                     "lz32", "lz64", "lz128"};
      for (int k = 0; k < 8; ++k) {
        fprintf(stderr, "[msllr phase] %s:", names[k]);
        for (int p = 0; p < 16; ++p)
          if (h[(k * 16 + p) * 2 + 1])
            fprintf(stderr, " p%d=%.0f(x%llu)", p,
                    (double)h[(k * 16 + p) * 2] / (double)h[(k * 16 + p) * 2 + 1],
                    h[(k * 16 + p) * 2 + 1]);
        fprintf(stderr, "\n");
      }
    }
    set_phase_buffer_small(nullptr);
    set_phase_buffer_big(nullptr);
    set_phase_buffer_warp(nullptr);
    cudaFree(ctx->d_phase);
  }
  if (ctx->d_small) cudaFree(ctx->d_small);
  if (ctx->d_acc) cudaFree(ctx->d_acc);
  if (ctx->d_noise) cudaFree(ctx->d_noise);
  if (ctx->d_cnt) cudaFree(ctx->d_cnt);
  if (ctx->d_table) cudaFree(ctx->d_table);
  if (ctx->d_shift) cudaFree(ctx->d_shift);
  for (int i = 0; i < MSLLR_MAX_SCALES; ++i) {
    if (ctx->side[i]) cudaStreamDestroy(ctx->side[i]);
    if (ctx->side_hi[i]) cudaStreamDestroy(ctx->side_hi[i]);
    if (ctx->ev_join[i]) cudaEventDestroy(ctx->ev_join[i]);
    if (ctx->ev_gate[i]) cudaEventDestroy(ctx->ev_gate[i]);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return MSLLR_OK;
}

const char* msllr_last_error(const msllr_ctx* ctx) {
  if (!ctx) return g_last_error.c_str();
  // a copy per calling thread: the serving worker may set a new message
  static thread_local std::string copy;
  std::lock_guard<std::mutex> lk(const_cast<msllr_ctx*>(ctx)->err_mu);
  copy = ctx->err;
  return copy.c_str();
}

int msllr_shift_table(uint64_t seed, int iters, int M, int N, int32_t* out) {
  if (iters < 0 || M <= 0 || N <= 0 || (!out && iters > 0))
    return fail(nullptr, MSLLR_EINVAL, "msllr_shift_table: bad arguments");
  fill_shift_table(seed, 0, iters, M, N, out);
  return MSLLR_OK;
}

int msllr_lambda_default(int M, int N, int m, int n, double* out) {
  const bool noise = m == 0 && n == 0;
  if (!out || M <= 0 || N <= 0 || (!noise && (m <= 0 || n <= 0 || m > M || n > N)))
    return fail(nullptr, MSLLR_EINVAL, "msllr_lambda_default: bad arguments");
  *out = lambda_of(M, N, m, n);
  return MSLLR_OK;
}

int msllr_blocksvt(msllr_ctx* ctx, const float* A, float* Z, int M, int N, int ld, int bm, int bn,
                   double tau, int shift_r, int shift_c, int* block_rank_out) {
  if (!ctx) return fail(nullptr, MSLLR_EINVAL, "ctx is NULL");
  if (int r = busy(ctx)) return r;
  if (!A || !Z || M <= 0 || N <= 0 || ld < N)
    return fail(ctx, MSLLR_EINVAL, "msllr_blocksvt: bad matrix arguments");
  if (!(tau >= 0.0) || !isfinite(tau)) return fail(ctx, MSLLR_EINVAL, "tau must be finite and >= 0");
  if (int r = check_blocks(ctx, M, N, bm, bn)) return r;
  const char* a0 = (const char*)A;
  const char* z0 = (const char*)Z;
  const size_t span = sizeof(float) * ((size_t)(M - 1) * ld + N);
  if (a0 < z0 + span && z0 < a0 + span) return fail(ctx, MSLLR_EINVAL, "A and Z overlap");
  CK(cudaSetDevice(ctx->device));
  const size_t big = big_workspace_bytes(M, N, bm, bn);
  if (int r = ensure_ws(ctx, align_up(big) + 256)) return r;
  const int sh[2] = {((shift_r % M) + M) % M, ((shift_c % N) + N) % N};
  CK(cudaMemcpyAsync(ctx->d_small + 4, sh, sizeof(sh), cudaMemcpyHostToDevice, ctx->stream));
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
  s.shift = ctx->d_small + 4;
  s.tau = (float)tau;
  s.skip_bound = 1;
  s.rank_out = block_rank_out;
  s.norm_acc = ctx->d_noise;
  s.err = ctx->d_small + 6;
  BigWorkspace w = carve_big_workspace(ctx->ws, M, N, bm, bn);
  CK(cudaMemsetAsync(ctx->d_small + 6, 0, sizeof(int), ctx->stream));
  CK(reset_warm_start(w, M, N, bm, bn, ctx->stream));
  CK(launch_scale(s, w, ctx->stream, nullptr));
  int timed_out = 0;
  CK(cudaMemcpyAsync(&timed_out, ctx->d_small + 6, sizeof(int), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (timed_out) return fail(ctx, MSLLR_ECUDA, "a tensor-core wait timed out on the device");
  return MSLLR_OK;
}

namespace {

struct Layout {
  size_t MN;
  float* Z;
  float* W;
  float* T;  // averaged cycle spinning: one M x N Z-update per scale, or null
  float* R;
  float* Yd;
  uint8_t* mask;
  float* plain;  // scratch of the plain comparator path, or null
  float* Zs;     // stopping test: Z and W one iteration earlier, or null
  float* Ws;
  std::vector<BigWorkspace> big;
  size_t total;
};

// Offsets of every buffer inside the workspace (base may be null to size it).
Layout plan(void* base, int M, int N, int L, const int* bm, const int* bn, bool masked,
            bool spin, bool plain = false, bool snap = false) {
  Layout lay;
  lay.MN = (size_t)M * N;
  char* b = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = b ? b + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  lay.Z = (float*)take(sizeof(float) * L * lay.MN);
  lay.W = (float*)take(sizeof(float) * L * lay.MN);
  lay.R = (float*)take(sizeof(float) * lay.MN);
  lay.T = spin ? (float*)take(sizeof(float) * L * lay.MN) : nullptr;
  lay.Yd = (float*)take(sizeof(float) * lay.MN);
  lay.mask = masked ? (uint8_t*)take(lay.MN) : nullptr;
  lay.Zs = snap ? (float*)take(sizeof(float) * L * lay.MN) : nullptr;
  lay.Ws = snap ? (float*)take(sizeof(float) * L * lay.MN) : nullptr;
  lay.plain = nullptr;
  if (plain) {
    size_t need = 0;
    for (int i = 0; i < L; ++i) {
      const size_t b = plain_scratch_bytes(bm[i], bn[i]);
      need = b > need ? b : need;
    }
    if (need) lay.plain = (float*)take(need);
    lay.total = off + 256;
    return lay;  // the plain path holds no wide-block workspace
  }
  for (int i = 0; i < L; ++i) {
    const size_t bytes = big_workspace_bytes(M, N, bm[i], bn[i]);
    char* p = take(bytes);
    lay.big.push_back(b ? carve_big_workspace(p, M, N, bm[i], bn[i]) : BigWorkspace{});
  }
  lay.total = off + 256;
  return lay;
}

// Shift offsets averaged at a scale (Sec. 9, msllr_params.spin_grid); one
// zero offset where the scale is not spun.
std::vector<std::pair<int, int>> spin_offsets(int M, int N, int m, int n, int g) {
  std::vector<std::pair<int, int>> out;
  const ScalePath path = choose_path(m, n);
  const bool spun = g > 1 && (path == ScalePath::Small || path == ScalePath::Big ||
                              path == ScalePath::Huge) && !(m == M && n == N);
  if (!spun) {
    out.push_back({0, 0});
    return out;
  }
  const int gr = g < m ? g : m, gc = g < n ? g : n;
  for (int a = 0; a < gr; ++a)
    for (int b = 0; b < gc; ++b) out.push_back({a * (m / gr), b * (n / gc)});
  return out;
}

// One ADMM iteration.  M counts the rows of all batched jobs; `rows` is the
// rows of one job (0: a single job).
int enqueue_iteration(msllr_ctx* ctx, const Layout& lay, int M, int N, int L, const int* bm,
                      const int* bn, const float* taus, const msllr_params& p, bool stats,
                      Prof* prof, int rows = 0) {
  const int jobs = rows ? M / rows : 1;
  CK(launch_advance(ctx->d_table, ctx->d_small, ctx->d_shift, jobs, ctx->stream, prof));
  // the 1x1 scale is element-wise: outside the statistics iteration it runs
  // inside the consensus pass (its soft threshold needs nothing but R(i))
  int e11 = -1;
  for (int i = 0; i < L && !stats && !p.plain; ++i)
    if (bm[i] == 1 && bn[i] == 1) {
      e11 = i;
      break;
    }
  if (e11 >= 0)
    CK(launch_consensus(lay.Yd, lay.W, lay.R, lay.mask, L, lay.MN, ctx->stream, prof,
                        lay.Z + (size_t)e11 * lay.MN, lay.W + (size_t)e11 * lay.MN, taus[e11]));
  else
    CK(launch_consensus(lay.Yd, lay.W, lay.R, lay.mask, L, lay.MN, ctx->stream, prof));
  if (p.plain) {
    // the comparator: scales one after the other on the context stream, one
    // launch per block
    for (int i = 0; i < L; ++i) {
      ScaleLaunch s{};
      s.A1 = lay.Z + (size_t)i * lay.MN;
      s.A2 = lay.R;
      s.Zout = lay.Z + (size_t)i * lay.MN;
      s.Wout = lay.W + (size_t)i * lay.MN;
      s.M = M;
      s.N = N;
      s.ld = N;
      s.m = bm[i];
      s.n = bn[i];
      s.shift = p.cycle_spin ? ctx->d_shift : nullptr;
      s.rows = rows;
      s.tau = taus[i];
      s.nuc_acc = stats ? ctx->d_acc + i : nullptr;
      s.cnt = (stats || p.profile) ? ctx->d_cnt + 8 * i : nullptr;
      s.norm_acc = ctx->d_noise + i;
      s.err = ctx->d_small + 6;
      s.bw = p.st_patch_w ? p.st_patch_w[i] : 0;
      s.fw = s.bw > 0 ? p.frame_w : 0;
      prof->scale = i;
      CK(launch_plain(s, lay.plain, ctx->stream, prof));
    }
    return MSLLR_OK;
  }
  // fork: scale i > 0 runs on its own stream, scale 0 on the context stream.
  // When kernels are timed one by one (profile), everything stays on the
  // context stream so that each event pair brackets one kernel running alone.
  const bool fork = !(prof && prof->timing && !prof->per_scale);
  if (fork) CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
  // Wide-block scales are enqueued first on high-priority streams.  Their
  // eigen kernel needs whole SMs, so the other scales wait until the wide
  // scales' Gram phase is over; the eigen CTAs then claim SMs first and the
  // narrow-block kernels fill the rest.
  bool gated[MSLLR_MAX_SCALES] = {};
  // cross-scale tile fusion (params.nested): coarse scale i solves the
  // blocks of fine scale nest_of[i] in the same kernel (one read of R)
  int nest_of[MSLLR_MAX_SCALES], absorbed[MSLLR_MAX_SCALES] = {};
  for (int i = 0; i < L; ++i) nest_of[i] = -1;
  if (p.nested && !rows && p.spin_grid <= 1 && !p.st_patch_w)
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L && nest_of[i] < 0; ++j)
        if (j != i && j != e11 && i != e11 && !absorbed[j] && nest_of[j] < 0 &&
            !absorbed[i] && !(bm[i] == M && bn[i] == N) &&
            nested_pair(bm[j], bn[j], bm[i], bn[i])) {
          nest_of[i] = j;
          absorbed[j] = 1;
        }
  auto scale_launch = [&](int i, const std::vector<std::pair<int, int>>& offs) {
    ScaleLaunch s{};
    s.A1 = lay.Z + (size_t)i * lay.MN;
    s.A2 = lay.R;
    s.Zout = lay.Z + (size_t)i * lay.MN;
    s.Wout = lay.W + (size_t)i * lay.MN;
    s.M = M;
    s.N = N;
    s.ld = N;
    s.m = bm[i];
    s.n = bn[i];
    s.shift = (p.cycle_spin || offs.size() > 1) ? ctx->d_shift : nullptr;
    s.rows = rows;
    s.tau = taus[i];
    s.skip_bound = p.skip_bound;
    s.warm_start = 1;
    s.rank_out = nullptr;
    s.nuc_acc = stats ? ctx->d_acc + i : nullptr;
    // block counts: the last iteration, or every iteration of a profiled run
    s.cnt = (stats || p.profile) ? ctx->d_cnt + 8 * i : nullptr;
    s.norm_acc = ctx->d_noise + i;
    s.err = ctx->d_small + 6;
    s.bw = p.st_patch_w ? p.st_patch_w[i] : 0;
    s.fw = s.bw > 0 ? p.frame_w : 0;
    return s;
  };
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i < L; ++i) {
      const ScalePath path = choose_path(bm[i], bn[i]);
      const bool wide = path == ScalePath::Big || path == ScalePath::Huge;
      if ((pass == 0) != wide || i == e11) continue;
      cudaStream_t st = (i == 0 || !fork) ? ctx->stream : (wide ? ctx->side_hi[i] : ctx->side[i]);
      if (i > 0 && fork) CK(cudaStreamWaitEvent(st, ctx->ev_fork, 0));
      if (pass == 1 && fork)
        for (int j = 0; j < L; ++j)
          if (gated[j]) CK(cudaStreamWaitEvent(st, ctx->ev_gate[j], 0));
      const auto offs = spin_offsets(rows ? rows : M, N, bm[i], bn[i], p.spin_grid);
      const ScaleLaunch s = scale_launch(i, offs);
      prof->scale = i;
      const bool gate = fork && wide && i > 0;
      // one block SVT, or the average over the scale's shift set
      auto run_scale = [&]() -> int {
        if (absorbed[i]) return MSLLR_OK;  // solved inside its coarse scale's kernel
        if (nest_of[i] >= 0) {
          const int j = nest_of[i];
          const ScaleLaunch sf =
              scale_launch(j, spin_offsets(rows ? rows : M, N, bm[j], bn[j], p.spin_grid));
          CK(launch_nested(sf, s, st, prof));
          return MSLLR_OK;
        }
        if (offs.size() == 1) {
          CK(launch_scale(s, lay.big[i], st, prof, gate ? ctx->ev_gate[i] : nullptr));
          return MSLLR_OK;
        }
        float* acc = lay.W + (size_t)i * lay.MN;
        float* T = lay.T + (size_t)i * lay.MN;
        const float w = 1.f / (float)offs.size();
        for (size_t j = 0; j < offs.size(); ++j) {
          ScaleLaunch sj = s;
          sj.shift_add_r = offs[j].first;
          sj.shift_add_c = offs[j].second;
          sj.Zout = T;
          sj.Wout = nullptr;
          CK(launch_scale(sj, lay.big[i], st, prof, (gate && j == 0) ? ctx->ev_gate[i] : nullptr));
          CK(launch_spin_accum(acc, T, w, j == 0, lay.MN, st, prof));
        }
        CK(launch_spin_finish(lay.Z + (size_t)i * lay.MN, acc, lay.R, lay.MN, st, prof));
        return MSLLR_OK;
      };
      if (prof->per_scale) {
        // concurrent profile: one event pair around the scale's whole segment
        CK(prof->before(st, wide ? KK_EIG : KK_FUSED));
        prof->timing = false;
        if (int r = run_scale()) return r;
        prof->timing = true;
        CK(prof->after(st));
      } else {
        if (int r = run_scale()) return r;
      }
      gated[i] = gate;
      if (i > 0 && fork) CK(cudaEventRecord(ctx->ev_join[i], st));
    }
  }
  // join
  if (fork)
    for (int i = 1; i < L; ++i)
      if (i != e11) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join[i], 0));
  return MSLLR_OK;
}

// `batch` jobs of one shape M x N stacked row-wise in Y (job j at rows
// j M ..), each with its own shift sequence from seeds[j]; X_out and Z_out
// hold per scale the batch x M x N stack.
int decompose_device(msllr_ctx* ctx, const float* Y, int M, int N, int ld, int L, const int* bm,
                     const int* bn, const double* lambda, double rho, int iters,
                     const uint64_t* seeds, int batch, const uint8_t* mask,
                     const msllr_params* params, float* X_out, float* Z_out, msllr_stats* stats) {
  if (!ctx) return fail(nullptr, MSLLR_EINVAL, "ctx is NULL");
  if (!Y || !X_out || M <= 0 || N <= 0 || ld < N)
    return fail(ctx, MSLLR_EINVAL, "msllr_decompose: bad matrix arguments");
  if (batch < 1 || !seeds || (long long)M * batch > 0x7fffffffLL)
    return fail(ctx, MSLLR_EINVAL, "batch must be >= 1 with one seed per job");
  const int MT = M * batch;           // rows of the stacked jobs
  const int rows = batch > 1 ? M : 0;  // rows of one job for the kernels
  if (L <= 0 || L > MSLLR_MAX_SCALES || !bm || !bn)
    return fail(ctx, MSLLR_EINVAL, "L must be in 1..MSLLR_MAX_SCALES with block sizes given");
  if (!(rho > 0.0) || !isfinite(rho)) return fail(ctx, MSLLR_EINVAL, "rho must be > 0");
  if (iters < 0) return fail(ctx, MSLLR_EINVAL, "iters must be >= 0");
  msllr_params p;
  msllr_params_default(&p);
  if (params) p = *params;
  if (p.iter_offset < 0) return fail(ctx, MSLLR_EINVAL, "iter_offset must be >= 0");
  if (p.spin_grid < 0) return fail(ctx, MSLLR_EINVAL, "spin_grid must be >= 0");
  if (p.plain && p.spin_grid > 1)
    return fail(ctx, MSLLR_EINVAL, "the plain comparator path takes no spin_grid");
  for (int i = 0; i < L && p.st_patch_w; ++i) {
    const int bw = p.st_patch_w[i];
    if (bw == 0) continue;
    const int fw = p.frame_w;
    if (bw < 0 || fw <= 0 || M % fw || fw % bw || bm[i] <= 0 || bn[i] <= 0 || bm[i] % bw ||
        (M / fw) % (bm[i] / bw) || N % bn[i])
      return fail(ctx, MSLLR_EINVAL,
                  "spatio-temporal scale " + std::to_string(i) +
                      ": needs frame_w > 0 dividing M, bw | frame_w, bh = block_m / bw | M / frame_w, "
                      "block_n | N");
    if (p.spin_grid > 1)
      return fail(ctx, MSLLR_EINVAL, "spin_grid does not combine with spatio-temporal scales");
  }
  for (int i = 0; i < L && p.plain; ++i)
    if (choose_path(bm[i], bn[i]) == ScalePath::Huge)
      return fail(ctx, MSLLR_EINVAL, "the plain comparator path takes blocks up to 256 wide");
  if (batch > 1) {
    if (p.spin_grid > 1 || p.frame_w || p.Z_init || p.U_init)
      return fail(ctx, MSLLR_EINVAL,
                  "batched jobs take no spin_grid, spatio-temporal scales or initial state");
    for (int i = 0; i < L; ++i) {
      if (bm[i] == 0 && bn[i] == 0)
        return fail(ctx, MSLLR_EINVAL, "batched jobs take no noise scale");
      const ScalePath path = choose_path(bm[i], bn[i]);
      if ((path == ScalePath::Big || path == ScalePath::Huge) && bm[i] > 0 && bn[i] > 0 &&
          (long long)(MT / bm[i]) * (N / bn[i]) > 65535)
        return fail(ctx, MSLLR_EINVAL, "too many wide blocks over the batch (max 65535)");
    }
  }
  for (int i = 0; i < L && p.spin_grid > 1; ++i) {
    const int m = bm[i], n = bn[i];
    if (m <= 0 || n <= 0) continue;
    const int gr = p.spin_grid < m ? p.spin_grid : m, gc = p.spin_grid < n ? p.spin_grid : n;
    if (m % gr || n % gc)
      return fail(ctx, MSLLR_EINVAL, "spin_grid must divide every block size it spins");
  }
  Prof prof;
  prof.timing = p.profile != 0;
  prof.per_scale = p.profile == 2 && !p.plain;
  if (p.profile || p.plain) p.use_graph = 0;
  struct EventPool {
    Prof* pr;
    ~EventPool() {
      for (cudaEvent_t e : pr->ev) cudaEventDestroy(e);
    }
  } pool{&prof};
  double lam[MSLLR_MAX_SCALES];
  float taus[MSLLR_MAX_SCALES];
  for (int i = 0; i < L; ++i) {
    if (int r = check_blocks(ctx, M, N, bm[i], bn[i])) return r;
    lam[i] = lambda ? lambda[i] : lambda_of(M, N, bm[i], bn[i]);
    if (!(lam[i] > 0.0) || !isfinite(lam[i]))
      return fail(ctx, MSLLR_EINVAL, "lambda_" + std::to_string(i) + " must be finite and > 0");
    taus[i] = (float)(lam[i] / rho);
  }
  CK(cudaSetDevice(ctx->device));
  const bool spin = p.spin_grid > 1;
  if (!(p.stop_tol >= 0.0) || !isfinite(p.stop_tol) || p.stop_every < 0)
    return fail(ctx, MSLLR_EINVAL, "stop_tol must be finite and >= 0, stop_every >= 0");
  const bool stop_test = p.stop_tol > 0.0;
  const int every = p.stop_every > 0 ? p.stop_every : 10;
  const Layout sizing = plan(nullptr, MT, N, L, bm, bn, mask != nullptr, spin, p.plain != 0,
                             stop_test);
  if (int r = ensure_ws(ctx, sizing.total)) return r;
  const Layout lay = plan(ctx->ws, MT, N, L, bm, bn, mask != nullptr, spin, p.plain != 0,
                          stop_test);
  cudaStream_t st = ctx->stream;
  if (batch > ctx->shift_cap) {
    if (ctx->graph) {
      cudaGraphExecDestroy(ctx->graph);
      ctx->graph = nullptr;
      ctx->graph_key.clear();
    }
    if (ctx->d_shift) {
      if (ctx->serve_child) cudaFreeAsync(ctx->d_shift, st);
      else cudaFree(ctx->d_shift);
    }
    ctx->d_shift = nullptr;
    ctx->shift_cap = 0;
    if (ctx->serve_child) CK(cudaMallocAsync((void**)&ctx->d_shift, 2 * sizeof(int) * batch, st));
    else CK(cudaMalloc(&ctx->d_shift, 2 * sizeof(int) * batch));
    ctx->shift_cap = batch;
  }

  // inputs: finiteness check, dense copies
  CK(cudaMemsetAsync(ctx->d_small + 3, 0, 4 * sizeof(int), st));
  CK(launch_nonfinite(Y, MT, N, ld, ctx->d_small + 3, st, &prof));
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, ctx->d_small + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad) return fail(ctx, MSLLR_ENONFINITE, "Y contains NaN or Inf");
  if (ld == N) CK(cudaMemcpyAsync(lay.Yd, Y, sizeof(float) * lay.MN, cudaMemcpyDeviceToDevice, st));
  else CK(launch_copy_dense(Y, MT, N, ld, lay.Yd, st, &prof));
  if (mask) CK(cudaMemcpyAsync(lay.mask, mask, lay.MN, cudaMemcpyDeviceToDevice, st));

  // shift table for iterations iter_offset .. iter_offset + iters - 1, one
  // pair per job (iters x batch x 2)
  const size_t tab = 2 * (size_t)(iters > 0 ? iters : 1) * batch;
  if (tab > ctx->table_cap) {
    if (ctx->d_table) {
      if (ctx->serve_child) cudaFreeAsync(ctx->d_table, st);
      else cudaFree(ctx->d_table);
    }
    ctx->d_table = nullptr;
    ctx->table_cap = 0;
    if (ctx->graph) {
      cudaGraphExecDestroy(ctx->graph);
      ctx->graph = nullptr;
      ctx->graph_key.clear();
    }
    if (ctx->serve_child) CK(cudaMallocAsync((void**)&ctx->d_table, tab * sizeof(int), st));
    else CK(cudaMalloc(&ctx->d_table, tab * sizeof(int)));
    ctx->table_cap = tab;
  }
  std::vector<int32_t> h_table(tab, 0);
  if (p.cycle_spin) {
    std::vector<int32_t> one(2 * (size_t)(iters > 0 ? iters : 1));
    for (int j = 0; j < batch; ++j) {
      fill_shift_table(seeds[j], p.iter_offset, iters, M, N, one.data());
      for (int k = 0; k < iters; ++k) {
        h_table[2 * ((size_t)k * batch + j)] = one[2 * k];
        h_table[2 * ((size_t)k * batch + j) + 1] = one[2 * k + 1];
      }
    }
  }
  CK(cudaMemcpyAsync(ctx->d_table, h_table.data(), tab * sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(ctx->d_small, 0, sizeof(int), st));
  CK(launch_init_state(p.Z_init, p.U_init, lay.Z, lay.W, L, lay.MN, st, &prof));
  for (int i = 0; i < L && !p.plain; ++i) CK(reset_warm_start(lay.big[i], MT, N, bm[i], bn[i], st));
  CK(cudaMemsetAsync(ctx->d_acc, 0, (MSLLR_MAX_SCALES + 8) * sizeof(double), st));
  CK(cudaMemsetAsync(ctx->d_cnt, 0, 8 * MSLLR_MAX_SCALES * sizeof(unsigned long long), st));

  // iterations 0 .. iters-2 (graph replay), the last one with statistics
  const int plain_iters = iters > 0 ? iters - 1 : 0;
  if (p.use_graph && plain_iters > 0) {
    std::vector<char> key;
    auto put = [&](const void* v, size_t n) {
      key.insert(key.end(), (const char*)v, (const char*)v + n);
    };
    put(&MT, sizeof MT);
    put(&rows, sizeof rows);
    put(&N, sizeof N);
    put(&L, sizeof L);
    put(bm, sizeof(int) * L);
    put(bn, sizeof(int) * L);
    put(taus, sizeof(float) * L);
    const int flags[5] = {p.skip_bound, p.cycle_spin, mask != nullptr, p.spin_grid, p.frame_w};
    put(flags, sizeof flags);
    for (int i = 0; i < L; ++i) {
      const int bw = p.st_patch_w ? p.st_patch_w[i] : 0;
      put(&bw, sizeof bw);
    }
    void* wsp = ctx->ws;
    put(&wsp, sizeof wsp);
    if (!ctx->graph || key != ctx->graph_key) {
      if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      Prof counter;
      int r = enqueue_iteration(ctx, lay, MT, N, L, bm, bn, taus, p, false, &counter, rows);
      memcpy(ctx->graph_launches, counter.launches, sizeof counter.launches);
      cudaError_t e = cudaStreamEndCapture(st, &g);
      if (r) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      if (e != cudaSuccess)
        return fail(ctx, MSLLR_ECUDA, std::string("stream capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&ctx->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess)
        return fail(ctx, MSLLR_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      ctx->graph_key = key;
    }
  }
  // iterations 0 .. plain_iters-1: graph replays or plain launches, with the
  // stopping test every `every` iterations when asked for
  const size_t LMN = (size_t)L * lay.MN;
  int ran = 0;
  bool stopped = false;
  double* acc4 = ctx->d_acc + MSLLR_MAX_SCALES + 2;
  for (int k = 0; k < plain_iters && !stopped; ++k) {
    const bool check = stop_test && (k + 1) % every == 0;
    if (check) {
      CK(cudaMemcpyAsync(lay.Zs, lay.Z, sizeof(float) * LMN, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(lay.Ws, lay.W, sizeof(float) * LMN, cudaMemcpyDeviceToDevice, st));
    }
    if (p.use_graph) {
      CK(cudaGraphLaunch(ctx->graph, st));
      for (int a = 0; a < KK_COUNT; ++a)
        for (int b = 0; b < 8; ++b) prof.launches[a][b] += ctx->graph_launches[a][b];
    } else if (int r = enqueue_iteration(ctx, lay, MT, N, L, bm, bn, taus, p, false, &prof, rows)) {
      return r;
    }
    ++ran;
    if (check) {
      double h4[4];
      CK(cudaMemsetAsync(acc4, 0, 4 * sizeof(double), st));
      CK(launch_residual(lay.Z, lay.W, lay.Zs, lay.Ws, acc4, LMN, st, &prof));
      CK(cudaMemcpyAsync(h4, acc4, sizeof h4, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      // r = ||X - Z|| = ||U - U_prev||, s / rho = ||Z - Z_prev||
      stopped = sqrt(h4[0]) <= p.stop_tol * sqrt(h4[2]) &&
                sqrt(h4[1]) <= p.stop_tol * sqrt(h4[3]);
    }
  }
  // the last iteration collects the statistics; the output pass then reads
  // the Z it started from (copied into X_out) for the dual residual
  if (iters > 0) {
    CK(cudaMemcpyAsync(X_out, lay.Z, sizeof(float) * LMN, cudaMemcpyDeviceToDevice, st));
    if (int r = enqueue_iteration(ctx, lay, MT, N, L, bm, bn, taus, p, true, &prof, rows)) return r;
    ++ran;
  }

  // output X-update on the final state
  CK(launch_consensus(lay.Yd, lay.W, lay.R, lay.mask, L, lay.MN, st, &prof));
  CK(launch_finalize(lay.W, lay.Z, lay.R, X_out, p.U_out, ctx->d_acc + MSLLR_MAX_SCALES,
                     iters > 0, L, lay.MN, st, &prof));
  if (Z_out)
    CK(cudaMemcpyAsync(Z_out, lay.Z, sizeof(float) * L * lay.MN, cudaMemcpyDeviceToDevice, st));
  double acc[MSLLR_MAX_SCALES + 8];
  unsigned long long cnt[8 * MSLLR_MAX_SCALES];
  CK(cudaMemcpyAsync(acc, ctx->d_acc, sizeof acc, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(cnt, ctx->d_cnt, sizeof cnt, cudaMemcpyDeviceToHost, st));
  int timed_out = 0;
  CK(cudaMemcpyAsync(&timed_out, ctx->d_small + 6, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (timed_out) return fail(ctx, MSLLR_ECUDA, "a tensor-core wait timed out on the device");
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iters = iters;
    stats->L = L;
    double obj = 0.0;
    for (int i = 0; i < L; ++i) {
      // averaged cycle spinning sums the nuclear norms of all the shifts
      const double nspin = (double)spin_offsets(M, N, bm[i], bn[i], p.spin_grid).size();  // one job
      stats->scale_nuclear[i] = acc[i] / nspin;
      obj += lam[i] * acc[i] / nspin;
      stats->blocks[i] = (bm[i] == 0 && bn[i] == 0) ? 1 : (long long)(MT / bm[i]) * (N / bn[i]);
      stats->blocks_skipped[i] = (long long)cnt[8 * i];
      stats->blocks_zero[i] = (long long)cnt[8 * i + 1];
      stats->blocks_lanczos[i] = (long long)cnt[8 * i + 2];
      stats->blocks_householder[i] = (long long)cnt[8 * i + 3];
      stats->blocks_uncertified[i] = (long long)cnt[8 * i + 4];
      stats->flops[i] = (long long)cnt[8 * i + 5];
      stats->flops_fallback[i] = (long long)cnt[8 * i + 6];
      stats->lambda[i] = lam[i];
    }
    stats->objective = obj;
    stats->iters = ran;
    stats->stopped = stopped ? 1 : 0;
    stats->primal_residual = sqrt(acc[MSLLR_MAX_SCALES]);
    stats->dual_residual = rho * sqrt(acc[MSLLR_MAX_SCALES + 1]);
    long long total = 0;
    for (int a = 0; a < KK_COUNT && a < MSLLR_KERNEL_KINDS; ++a)
      for (int b = 0; b < MSLLR_MAX_SCALES; ++b) {
        stats->kernel_launches[a][b] = prof.launches[a][b];
        total += prof.launches[a][b];
      }
    stats->launches = total;
    if (prof.timing) {
      for (size_t u = 0; u < prof.used; ++u) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, prof.ev[2 * u], prof.ev[2 * u + 1]));
        const int kind = prof.tag[u] / 8, sc = prof.tag[u] % 8;
        stats->kernel_ms[kind][sc] += ms;
      }
    }
  }
  return MSLLR_OK;
}


// Runs one serving job: device slabs for its inputs and outputs, the
// decomposition, the copies back into the caller's host buffers.
int run_job(msllr_ctx* ctx, ServeJob& j) {
  const size_t MN = (size_t)j.M * j.N;
  float* dY = nullptr;
  float* dX = nullptr;
  float* dZ = nullptr;
  uint8_t* dmask = nullptr;
  cudaStream_t s = ctx->stream;
  auto cleanup = [&]() {
    if (dY) cudaFreeAsync(dY, s);
    if (dX) cudaFreeAsync(dX, s);
    if (dZ) cudaFreeAsync(dZ, s);
    if (dmask) cudaFreeAsync(dmask, s);
  };
  CK(cudaSetDevice(ctx->device));
  if (cudaMallocAsync((void**)&dY, sizeof(float) * MN, s) != cudaSuccess ||
      cudaMallocAsync((void**)&dX, sizeof(float) * j.L * MN, s) != cudaSuccess ||
      (j.Z_out && cudaMallocAsync((void**)&dZ, sizeof(float) * j.L * MN, s) != cudaSuccess) ||
      (!j.mask.empty() && cudaMallocAsync((void**)&dmask, MN, s) != cudaSuccess)) {
    cudaGetLastError();
    cleanup();
    return fail(ctx, MSLLR_ENOMEM, "serving job: device buffers");
  }
  cudaError_t e = cudaMemcpyAsync(dY, j.Y.data(), sizeof(float) * MN, cudaMemcpyHostToDevice,
                                  ctx->stream);
  if (e == cudaSuccess && dmask)
    e = cudaMemcpyAsync(dmask, j.mask.data(), MN, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) {
    cleanup();
    return fail(ctx, MSLLR_ECUDA, std::string("serving job: host to device copy: ") +
                                      cudaGetErrorString(e));
  }
  int r = decompose_device(ctx, dY, j.M, j.N, j.N, j.L, j.bm.data(), j.bn.data(),
                           j.lam.empty() ? nullptr : j.lam.data(), j.rho, j.iters, &j.seed, 1, dmask,
                           j.has_p ? &j.p : nullptr, dX, dZ, j.stats);
  if (r == MSLLR_OK) {
    e = cudaMemcpyAsync(j.X_out, dX, sizeof(float) * j.L * MN, cudaMemcpyDeviceToHost,
                        ctx->stream);
    if (e == cudaSuccess && j.Z_out)
      e = cudaMemcpyAsync(j.Z_out, dZ, sizeof(float) * j.L * MN, cudaMemcpyDeviceToHost,
                          ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
      r = fail(ctx, MSLLR_ECUDA, std::string("serving job: device to host copy: ") +
                                     cudaGetErrorString(e));
  }
  cleanup();
  // the slot keeps no memory between jobs: the admission of the next jobs
  // counts only what the running ones hold
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
    ctx->graph_key.clear();
  }
  if (ctx->ws) cudaFreeAsync(ctx->ws, s);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  if (ctx->d_table) cudaFreeAsync(ctx->d_table, s);
  ctx->d_table = nullptr;
  ctx->table_cap = 0;
  cudaStreamSynchronize(s);
  return r;
}

// A serving worker: takes the job at the head of the queue once the device
// memory held by the running jobs leaves room for it (submission order, no
// overtaking), runs it on its slot context, and repeats until the context is
// destroyed.
void serve_loop(msllr_ctx* ctx, int slot) {
  msllr_ctx* child = ctx->slots[slot];
  for (;;) {
    std::shared_ptr<ServeJob> job;
    {
      std::unique_lock<std::mutex> lk(ctx->q_mu);
      ctx->q_cv.wait(lk, [&] {
        if (ctx->stop) return true;
        if (ctx->queue.empty()) return false;
        return !ctx->budget || ctx->serve_bytes + ctx->queue.front()->need <= ctx->budget;
      });
      if (ctx->stop) return;
      job = ctx->queue.front();
      ctx->queue.pop_front();
      ctx->serve_bytes += job->need;
      job->running_with = ++ctx->serve_running;
    }
    const int r = run_job(child, *job);
    std::string msg;
    if (r != MSLLR_OK) {
      std::lock_guard<std::mutex> lk(child->err_mu);
      msg = child->err;
    } else if (job->stats) {
      job->stats->serve_jobs_running = job->running_with;
    }
    {
      std::lock_guard<std::mutex> lk(ctx->q_mu);
      job->status = r;
      job->err = msg;
      job->done = true;
      ctx->serve_bytes -= job->need;
      --ctx->serve_running;
      ctx->in_flight.fetch_sub(1);
    }
    ctx->done_cv.notify_all();
    ctx->q_cv.notify_all();  // memory came free: the head job may fit now
  }
}

// Creates the serving slots and their workers (first submission).
int start_serving(msllr_ctx* ctx) {
  for (int i = 0; i < MSLLR_SERVE_SLOTS; ++i) {
    cudaStream_t st = nullptr;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    msllr_ctx* child = nullptr;
    if (int r = msllr_create(&child, ctx->device, 0, st)) {
      cudaStreamDestroy(st);
      return fail(ctx, r, std::string("serving slot: ") + msllr_last_error(nullptr));
    }
    child->own_stream = true;
    child->serve_child = true;
    ctx->slots.push_back(child);
  }
  for (int i = 0; i < MSLLR_SERVE_SLOTS; ++i) ctx->workers.emplace_back(serve_loop, ctx, i);
  return MSLLR_OK;
}

// a finished job leaves the table and hands its status (and message) back
int collect(msllr_ctx* ctx, std::unordered_map<uint64_t, std::shared_ptr<ServeJob>>::iterator it) {
  const int st = it->second->status;
  const std::string msg = it->second->err;
  ctx->jobs.erase(it);
  return st == MSLLR_OK ? MSLLR_OK : fail(ctx, st, msg);
}

}  // namespace

int msllr_decompose(msllr_ctx* ctx, const float* Y, int M, int N, int ld, int L,
                    const int* block_m, const int* block_n, const double* lambda, double rho,
                    int iters, uint64_t seed, const uint8_t* mask, const msllr_params* params,
                    float* X_out, float* Z_out, msllr_stats* stats) {
  if (ctx)
    if (int r = busy(ctx)) return r;
  return decompose_device(ctx, Y, M, N, ld, L, block_m, block_n, lambda, rho, iters, &seed, 1, mask,
                          params, X_out, Z_out, stats);
}

int msllr_decompose_batch(msllr_ctx* ctx, int batch, const float* Y, int M, int N, int ld, int L,
                          const int* block_m, const int* block_n, const double* lambda, double rho,
                          int iters, const uint64_t* seeds, const uint8_t* mask,
                          const msllr_params* params, float* X_out, float* Z_out,
                          msllr_stats* stats) {
  if (ctx)
    if (int r = busy(ctx)) return r;
  return decompose_device(ctx, Y, M, N, ld, L, block_m, block_n, lambda, rho, iters, seeds, batch,
                          mask, params, X_out, Z_out, stats);
}

int msllr_decompose_host(msllr_ctx* ctx, const float* Y, int M, int N, int ld, int L,
                         const int* block_m, const int* block_n, const double* lambda, double rho,
                         int iters, uint64_t seed, const uint8_t* mask, const msllr_params* params,
                         float* X_out, float* Z_out, msllr_stats* stats) {
  if (!ctx) return fail(nullptr, MSLLR_EINVAL, "ctx is NULL");
  if (int r = busy(ctx)) return r;
  if (!Y || !X_out || M <= 0 || N <= 0 || ld < N || L <= 0 || L > MSLLR_MAX_SCALES)
    return fail(ctx, MSLLR_EINVAL, "msllr_decompose_host: bad arguments");
  if (params && (params->Z_init || params->U_init || params->U_out))
    return fail(ctx, MSLLR_EINVAL, "msllr_decompose_host takes no device state pointers");
  CK(cudaSetDevice(ctx->device));
  const size_t MN = (size_t)M * N;
  // device copies of Y, X, Z and the mask in the context's grow-only I/O
  // slab: after the first call of a size, no allocation per call
  const size_t bY = align_up(sizeof(float) * MN), bX = align_up(sizeof(float) * L * MN);
  const size_t need = bY + bX + (Z_out ? bX : 0) + (mask ? align_up(MN) : 0);
  if (need > ctx->io_bytes) {
    if (ctx->budget && need + ctx->ws_bytes > ctx->budget)
      return fail(ctx, MSLLR_ENOMEM, "msllr_decompose_host: device copies exceed the HBM budget");
    if (ctx->io) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->io);
      ctx->io = nullptr;
      ctx->io_bytes = 0;
    }
    if (cudaMalloc(&ctx->io, need) != cudaSuccess) {
      cudaGetLastError();
      ctx->io = nullptr;
      return fail(ctx, MSLLR_ENOMEM, "msllr_decompose_host: device buffers");
    }
    ctx->io_bytes = need;
  }
  char* io = (char*)ctx->io;
  float* dY = (float*)io;
  float* dX = (float*)(io + bY);
  float* dZ = Z_out ? (float*)(io + bY + bX) : nullptr;
  uint8_t* dmask = mask ? (uint8_t*)(io + bY + bX + (Z_out ? bX : 0)) : nullptr;
  auto cleanup = [&]() {};
  cudaError_t e = cudaMemcpy2DAsync(dY, sizeof(float) * N, Y, sizeof(float) * ld,
                                    sizeof(float) * N, M, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess && mask)
    e = cudaMemcpyAsync(dmask, mask, MN, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) {
    cleanup();
    return fail(ctx, MSLLR_ECUDA, std::string("host to device copy: ") + cudaGetErrorString(e));
  }
  int r = decompose_device(ctx, dY, M, N, N, L, block_m, block_n, lambda, rho, iters, &seed, 1, dmask,
                           params, dX, dZ, stats);
  if (r == MSLLR_OK) {
    e = cudaMemcpyAsync(X_out, dX, sizeof(float) * L * MN, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && Z_out)
      e = cudaMemcpyAsync(Z_out, dZ, sizeof(float) * L * MN, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
      r = fail(ctx, MSLLR_ECUDA, std::string("device to host copy: ") + cudaGetErrorString(e));
  }
  cleanup();
  return r;
}

int msllr_submit(msllr_ctx* ctx, const msllr_job* job, uint64_t* job_id) {
  if (!ctx) return fail(nullptr, MSLLR_EINVAL, "ctx is NULL");
  if (!job || !job_id) return fail(ctx, MSLLR_EINVAL, "msllr_submit: job and job_id are required");
  const int M = job->M, N = job->N, L = job->L;
  if (!job->Y || !job->X_out || M <= 0 || N <= 0 || job->ld < N || L <= 0 ||
      L > MSLLR_MAX_SCALES || !job->block_m || !job->block_n || job->iters < 0 ||
      !(job->rho > 0.0) || !isfinite(job->rho))
    return fail(ctx, MSLLR_EINVAL, "msllr_submit: bad job arguments");
  if (job->params && (job->params->Z_init || job->params->U_init || job->params->U_out))
    return fail(ctx, MSLLR_EINVAL, "msllr_submit: jobs take no device state pointers");
  for (int i = 0; i < L; ++i)
    if (int r = check_blocks(ctx, M, N, job->block_m[i], job->block_n[i])) return r;
  // admission: the job's workspace plus its input and output slabs must fit
  // the context's HBM budget
  const size_t MN = (size_t)M * N;
  const bool spin = job->params && job->params->spin_grid > 1;
  const bool plain = job->params && job->params->plain;
  const size_t need = plan(nullptr, M, N, L, job->block_m, job->block_n, job->mask != nullptr, spin,
                           plain).total +
                      sizeof(float) * MN * (1 + (size_t)L * (job->Z_out ? 2 : 1)) +
                      (job->mask ? MN : 0);
  const size_t need_all = need + 2 * sizeof(int) * (size_t)(job->iters > 0 ? job->iters : 1);
  if (ctx->budget && need_all > ctx->budget)
    return fail(ctx, MSLLR_ENOMEM, "msllr_submit: job needs " + std::to_string(need_all) +
                                       " bytes, above the HBM budget");
  auto j = std::make_shared<ServeJob>();
  j->M = M;
  j->N = N;
  j->L = L;
  j->Y.resize(MN);
  for (int r = 0; r < M; ++r)
    memcpy(j->Y.data() + (size_t)r * N, job->Y + (size_t)r * job->ld, sizeof(float) * N);
  if (job->mask) j->mask.assign(job->mask, job->mask + MN);
  j->bm.assign(job->block_m, job->block_m + L);
  j->bn.assign(job->block_n, job->block_n + L);
  if (job->lambda) j->lam.assign(job->lambda, job->lambda + L);
  j->rho = job->rho;
  j->iters = job->iters;
  j->seed = job->seed;
  if (job->params) {
    j->p = *job->params;
    j->has_p = true;
    if (j->p.st_patch_w) {
      j->patch_w.assign(j->p.st_patch_w, j->p.st_patch_w + L);
      j->p.st_patch_w = j->patch_w.data();
    }
  }
  j->X_out = job->X_out;
  j->Z_out = job->Z_out;
  j->stats = job->stats;
  j->need = need_all;
  {
    std::lock_guard<std::mutex> lk(ctx->q_mu);
    if ((int)ctx->queue.size() >= MSLLR_SERVE_QUEUE)
      return fail(ctx, MSLLR_EBUSY, "msllr_submit: the serving queue is full");
    if (ctx->slots.empty())
      if (int r = start_serving(ctx)) return r;
    j->id = ctx->next_job++;
    ctx->jobs[j->id] = j;
    ctx->queue.push_back(j);
    ctx->in_flight.fetch_add(1);
  }
  ctx->q_cv.notify_one();
  *job_id = j->id;
  return MSLLR_OK;
}

int msllr_poll(msllr_ctx* ctx, uint64_t job_id, int* done) {
  if (!ctx) return fail(nullptr, MSLLR_EINVAL, "ctx is NULL");
  if (!done) return fail(ctx, MSLLR_EINVAL, "msllr_poll: done is required");
  std::lock_guard<std::mutex> lk(ctx->q_mu);
  auto it = ctx->jobs.find(job_id);
  if (it == ctx->jobs.end()) return fail(ctx, MSLLR_EINVAL, "msllr_poll: unknown job id");
  *done = it->second->done ? 1 : 0;
  return *done ? collect(ctx, it) : MSLLR_OK;
}

int msllr_wait(msllr_ctx* ctx, uint64_t job_id, int timeout_ms) {
  if (!ctx) return fail(nullptr, MSLLR_EINVAL, "ctx is NULL");
  std::unique_lock<std::mutex> lk(ctx->q_mu);
  auto it = ctx->jobs.find(job_id);
  if (it == ctx->jobs.end()) return fail(ctx, MSLLR_EINVAL, "msllr_wait: unknown job id");
  std::shared_ptr<ServeJob> j = it->second;
  auto ready = [&] { return j->done; };
  if (timeout_ms < 0) {
    ctx->done_cv.wait(lk, ready);
  } else if (!ctx->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return fail(ctx, MSLLR_ETIMEOUT, "msllr_wait: job not finished within the timeout");
  }
  // another thread's msllr_poll or msllr_wait may have collected the job
  // while this one slept
  auto again = ctx->jobs.find(job_id);
  if (again == ctx->jobs.end())
    return fail(ctx, MSLLR_EINVAL, "msllr_wait: job already collected by another call");
  return collect(ctx, again);
}

}  // extern "C"
