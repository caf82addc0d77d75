"""Thin Python binding of the msllr C ABI (include/msllr.h).

Argument marshalling only: every step of the decomposition runs in the CUDA
library libmsllr.so.  Device buffers are passed as torch CUDA tensors (their
data pointers), host buffers as NumPy arrays.  If the library has not been
built, importing works but every call raises ``MsllrError`` -- there is no
CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmsllr.so")

MSLLR_OK = 0
MSLLR_EINVAL = 1
MSLLR_ENOMEM = 2
MSLLR_ECUDA = 3
MSLLR_ETIMEOUT = 4
MSLLR_ENONFINITE = 5
MSLLR_EBUSY = 6
MAX_SCALES = 8
MAX_BLOCK_WIDTH = 8192
NOISE_SCALE = (0, 0)  # block size of the noise scale (Sec. 2.1)
KERNEL_KINDS = ("advance", "consensus", "soft1x1", "fused_small", "gram", "gram_reduce",
                "eig_big", "rebuild", "misc", "eig_fallback", "subspace", "certificate")

STATUS_NAMES = {0: "MSLLR_OK", 1: "MSLLR_EINVAL", 2: "MSLLR_ENOMEM", 3: "MSLLR_ECUDA",
                4: "MSLLR_ETIMEOUT", 5: "MSLLR_ENONFINITE", 6: "MSLLR_EBUSY"}

# every symbol the header declares
EXPORTS = (
    "msllr_params_default", "msllr_create", "msllr_destroy", "msllr_last_error",
    "msllr_shift_table", "msllr_lambda_default", "msllr_blocksvt", "msllr_decompose",
    "msllr_decompose_host", "msllr_decompose_batch", "msllr_blocksvt_noalloc", "msllr_submit",
    "msllr_poll", "msllr_wait",
)
SERVE_QUEUE = 64
SERVE_SLOTS = 4
NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


class MsllrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("skip_bound", ctypes.c_int),
        ("cycle_spin", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("iter_offset", ctypes.c_int),
        ("Z_init", ctypes.c_void_p),
        ("U_init", ctypes.c_void_p),
        ("U_out", ctypes.c_void_p),
        ("profile", ctypes.c_int),
        ("spin_grid", ctypes.c_int),
        ("plain", ctypes.c_int),
        ("stop_tol", ctypes.c_double),
        ("stop_every", ctypes.c_int),
        ("frame_w", ctypes.c_int),
        ("st_patch_w", ctypes.c_void_p),
        ("nested", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("L", ctypes.c_int),
        ("objective", ctypes.c_double),
        ("primal_residual", ctypes.c_double),
        ("scale_nuclear", ctypes.c_double * MAX_SCALES),
        ("blocks", ctypes.c_longlong * MAX_SCALES),
        ("blocks_skipped", ctypes.c_longlong * MAX_SCALES),
        ("blocks_zero", ctypes.c_longlong * MAX_SCALES),
        ("lambda_", ctypes.c_double * MAX_SCALES),
        ("blocks_lanczos", ctypes.c_longlong * MAX_SCALES),
        ("blocks_householder", ctypes.c_longlong * MAX_SCALES),
        ("launches", ctypes.c_longlong),
        ("kernel_launches", (ctypes.c_longlong * MAX_SCALES) * len(KERNEL_KINDS)),
        ("kernel_ms", (ctypes.c_double * MAX_SCALES) * len(KERNEL_KINDS)),
        ("blocks_uncertified", ctypes.c_longlong * MAX_SCALES),
        ("flops", ctypes.c_longlong * MAX_SCALES),
        ("flops_fallback", ctypes.c_longlong * MAX_SCALES),
        ("dual_residual", ctypes.c_double),
        ("stopped", ctypes.c_int),
        ("serve_jobs_running", ctypes.c_int),
    ]

    def to_dict(self):
        L = self.L
        return {
            "iters": self.iters,
            "L": L,
            "objective": self.objective,
            "primal_residual": self.primal_residual,
            "scale_nuclear": list(self.scale_nuclear[:L]),
            "blocks": list(self.blocks[:L]),
            "blocks_skipped": list(self.blocks_skipped[:L]),
            "blocks_zero": list(self.blocks_zero[:L]),
            "lambda": list(self.lambda_[:L]),
            "blocks_lanczos": list(self.blocks_lanczos[:L]),
            "blocks_householder": list(self.blocks_householder[:L]),
            "launches": self.launches,
            "kernel_launches": {k: list(self.kernel_launches[i][:max(L, 1)])
                                for i, k in enumerate(KERNEL_KINDS)},
            "kernel_ms": {k: list(self.kernel_ms[i][:max(L, 1)]) for i, k in enumerate(KERNEL_KINDS)},
            "blocks_uncertified": list(self.blocks_uncertified[:L]),
            "flops": list(self.flops[:L]),
            "flops_fallback": list(self.flops_fallback[:L]),
            "dual_residual": self.dual_residual,
            "stopped": self.stopped,
            "serve_jobs_running": self.serve_jobs_running,
        }


class Job(ctypes.Structure):
    _fields_ = [
        ("Y", ctypes.c_void_p),
        ("M", ctypes.c_int),
        ("N", ctypes.c_int),
        ("ld", ctypes.c_int),
        ("L", ctypes.c_int),
        ("block_m", ctypes.c_void_p),
        ("block_n", ctypes.c_void_p),
        ("lambda_", ctypes.c_void_p),
        ("rho", ctypes.c_double),
        ("iters", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("mask", ctypes.c_void_p),
        ("params", ctypes.c_void_p),
        ("X_out", ctypes.c_void_p),
        ("Z_out", ctypes.c_void_p),
        ("stats", ctypes.c_void_p),
    ]


_lib = None


def lib():
    """Load libmsllr.so (once).  Raises MsllrError if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MsllrError(MSLLR_ECUDA, f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, ci, cd, cu64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        L.msllr_params_default.argtypes = [ctypes.POINTER(Params)]
        L.msllr_create.argtypes = [ctypes.POINTER(vp), ci, ctypes.c_size_t, vp]
        L.msllr_destroy.argtypes = [vp]
        L.msllr_last_error.argtypes = [vp]
        L.msllr_last_error.restype = ctypes.c_char_p
        L.msllr_shift_table.argtypes = [cu64, ci, ci, ci, vp]
        L.msllr_lambda_default.argtypes = [ci, ci, ci, ci, ctypes.POINTER(cd)]
        L.msllr_blocksvt.argtypes = [vp, vp, vp, ci, ci, ci, ci, ci, cd, ci, ci, vp]
        dec = [vp, vp, ci, ci, ci, ci, vp, vp, vp, cd, ci, cu64, vp, ctypes.POINTER(Params), vp, vp,
               ctypes.POINTER(Stats)]
        L.msllr_decompose.argtypes = dec
        L.msllr_decompose_host.argtypes = dec
        L.msllr_decompose_batch.argtypes = [vp, ci, vp, ci, ci, ci, ci, vp, vp, vp, cd, ci, vp, vp,
                                            ctypes.POINTER(Params), vp, vp, ctypes.POINTER(Stats)]
        L.msllr_blocksvt_noalloc.argtypes = [vp, vp, ci, ci, ci, ci, ci, cd, ci, ci, vp, vp]
        L.msllr_submit.argtypes = [vp, ctypes.POINTER(Job), ctypes.POINTER(cu64)]
        L.msllr_poll.argtypes = [vp, cu64, ctypes.POINTER(ci)]
        L.msllr_wait.argtypes = [vp, cu64, ci]
        for name in EXPORTS:
            getattr(L, name)
        _lib = L
    return _lib


def _check(code, ctx=None):
    if code != MSLLR_OK:
        msg = lib().msllr_last_error(ctx)
        raise MsllrError(code, msg.decode() if msg else "")


def _ptr(t):
    """Device pointer of a torch tensor, or None."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise MsllrError(MSLLR_EINVAL, "tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _int_array(v):
    return (ctypes.c_int * len(v))(*[int(x) for x in v])


def _scale_arrays(scales):
    """block_m, block_n and (for spatio-temporal scales, given as 3-tuples
    (bh, bw, bt) as in Sec. 10.2) the patch widths; None when all are 2-D."""
    bm = _int_array([s[0] * s[1] if len(s) == 3 else s[0] for s in scales])
    bn = _int_array([s[-1] for s in scales])
    if all(len(s) == 2 for s in scales):
        return bm, bn, None
    return bm, bn, _int_array([s[1] if len(s) == 3 else 0 for s in scales])


def _double_array(v):
    return None if v is None else (ctypes.c_double * len(v))(*[float(x) for x in v])


def msllr_shift_table(seed, iters, M, N):
    out = np.zeros((iters, 2), dtype=np.int32)
    _check(lib().msllr_shift_table(ctypes.c_uint64(seed), iters, M, N,
                                   out.ctypes.data_as(ctypes.c_void_p)))
    return out


def msllr_lambda_default(M, N, m, n):
    v = ctypes.c_double()
    _check(lib().msllr_lambda_default(M, N, m, n, ctypes.byref(v)))
    return v.value


def msllr_blocksvt_noalloc(A, Z, bm, bn, tau, shift=(0, 0), rank_out=None, N=None, stream=None):
    """Block SVT without any device allocation (no context needed): same result as
    Context.msllr_blocksvt, using the library's fixed device scratch.  Runs on `stream`
    (a cudaStream_t handle) of the current device; None means torch's current stream,
    so that the call is ordered after the kernels that produced A."""
    M, ld = A.shape[0], A.shape[1]
    N = ld if N is None else N
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    st = ctypes.c_void_p(stream) if stream else None
    _check(lib().msllr_blocksvt_noalloc(_ptr(A), _ptr(Z), M, N, ld, bm, bn, float(tau),
                                        int(shift[0]), int(shift[1]), _ptr(rank_out), st))


def msllr_params_default():
    p = Params()
    _check(lib().msllr_params_default(ctypes.byref(p)))
    return p


class Context:
    """One msllr context (msllr_create / msllr_destroy)."""

    def __init__(self, device=0, hbm_budget_bytes=0, stream=None):
        self._ctx = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else None
        _check(lib().msllr_create(ctypes.byref(self._ctx), device, hbm_budget_bytes, st))

    def close(self):
        if self._ctx:
            lib().msllr_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls ---------------------------------------------------------------
    def msllr_blocksvt(self, A, Z, bm, bn, tau, shift=(0, 0), rank_out=None, N=None):
        """Z <- Shift_{-s}(BlockSVT_tau(Shift_s(A))) on device tensors (float32, row-major).
        The matrix is A[:, :N] (N defaults to A's width, which is then the row stride)."""
        M, ld = A.shape[0], A.shape[1]
        N = ld if N is None else N
        _check(lib().msllr_blocksvt(self._ctx, _ptr(A), _ptr(Z), M, N, ld, bm, bn, float(tau),
                                    int(shift[0]), int(shift[1]), _ptr(rank_out)), self._ctx)

    def _decompose(self, fn, Yp, M, N, ld, scales, lambdas, rho, iters, seed, maskp, params, Xp,
                   Zp, frame=None):
        L = len(scales)
        bm, bn, pw = _scale_arrays(scales)
        lam = _double_array(lambdas)
        p = params if params is not None else msllr_params_default()
        if pw is not None:
            p.frame_w = int(frame[1])
            p.st_patch_w = ctypes.cast(pw, ctypes.c_void_p)
        st = Stats()
        _check(fn(self._ctx, Yp, M, N, ld, L, bm, bn, lam, float(rho), int(iters),
                  ctypes.c_uint64(seed), maskp, ctypes.byref(p), Xp, Zp, ctypes.byref(st)),
               self._ctx)
        return st.to_dict()

    def msllr_decompose(self, Y, scales, X_out, lambdas=None, rho=1.0, iters=100, seed=0,
                        mask=None, params=None, Z_out=None, frame=None):
        """Device-pointer decomposition: Y (M x N), X_out / Z_out (L x M x N) torch CUDA
        float32 tensors, mask a torch CUDA uint8 tensor or None.  A scale is (m, n), or
        (bh, bw, bt) for spatio-temporal blocks of the video whose frame is
        frame = (H, W).  Returns the stats dict."""
        M, N = Y.shape
        return self._decompose(lib().msllr_decompose, _ptr(Y), M, N, N, scales, lambdas, rho,
                               iters, seed, _ptr(mask), params, _ptr(X_out), _ptr(Z_out),
                               frame)

    def msllr_decompose_batch(self, Y, scales, X_out, seeds, lambdas=None, rho=1.0, iters=100,
                              mask=None, params=None, Z_out=None):
        """Batched jobs of one shape: Y a torch CUDA float32 tensor (batch, M, N), X_out
        (and Z_out) (L, batch, M, N), seeds one shift seed per job, mask (batch, M, N)
        uint8 or None.  Every kernel launch covers all jobs; job j's result is that of
        msllr_decompose of job j alone.  Returns the stats dict (summed over jobs)."""
        batch, M, N = Y.shape
        if len(seeds) != batch:
            raise MsllrError(MSLLR_EINVAL, "one seed per job")
        L = len(scales)
        bm, bn, pw = _scale_arrays(scales)
        if pw is not None:
            raise MsllrError(MSLLR_EINVAL, "batched jobs take no spatio-temporal scales")
        lam = _double_array(lambdas)
        sd = (ctypes.c_uint64 * batch)(*[int(x) for x in seeds])
        p = params if params is not None else msllr_params_default()
        st = Stats()
        _check(lib().msllr_decompose_batch(self._ctx, batch, _ptr(Y), M, N, N, L, bm, bn, lam,
                                           float(rho), int(iters), sd, _ptr(mask),
                                           ctypes.byref(p), _ptr(X_out), _ptr(Z_out),
                                           ctypes.byref(st)), self._ctx)
        return st.to_dict()

    def msllr_decompose_host(self, Y, scales, X_out, lambdas=None, rho=1.0, iters=100, seed=0,
                             mask=None, params=None, Z_out=None, frame=None):
        """Host-buffer decomposition: NumPy (or pinned torch CPU) arrays; copies happen
        inside the call."""
        def hp(a, dt):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                return ctypes.c_void_p(a.data_ptr())
            if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
                raise MsllrError(MSLLR_EINVAL, f"host array must be contiguous {dt}")
            return a.ctypes.data_as(ctypes.c_void_p)
        M, N = Y.shape
        return self._decompose(lib().msllr_decompose_host, hp(Y, np.float32), M, N, N, scales,
                               lambdas, rho, iters, seed, hp(mask, np.uint8), params,
                               hp(X_out, np.float32), hp(Z_out, np.float32), frame)

    # -- serving queue ---------------------------------------------------------
    def msllr_submit(self, Y, scales, X_out, lambdas=None, rho=1.0, iters=100, seed=0,
                     mask=None, params=None, Z_out=None, frame=None):
        """Queue a decomposition of the host array Y (NumPy float32); X_out (and Z_out)
        are host arrays filled when the job completes.  Returns the job id."""
        def hp(a, dt):
            if a is None:
                return None
            if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
                raise MsllrError(MSLLR_EINVAL, f"host array must be contiguous {dt}")
            return a.ctypes.data
        M, N = Y.shape
        L = len(scales)
        bm, bn, pw = _scale_arrays(scales)
        lam = _double_array(lambdas)
        p = params if params is not None else msllr_params_default()
        if pw is not None:
            p.frame_w = int(frame[1])
            p.st_patch_w = ctypes.cast(pw, ctypes.c_void_p)
        st = Stats()
        job = Job(Y=hp(Y, np.float32), M=M, N=N, ld=N, L=L,
                  block_m=ctypes.cast(bm, ctypes.c_void_p),
                  block_n=ctypes.cast(bn, ctypes.c_void_p),
                  lambda_=ctypes.cast(lam, ctypes.c_void_p) if lam is not None else None,
                  rho=float(rho), iters=int(iters), seed=int(seed), mask=hp(mask, np.uint8),
                  params=ctypes.cast(ctypes.pointer(p), ctypes.c_void_p),
                  X_out=hp(X_out, np.float32), Z_out=hp(Z_out, np.float32),
                  stats=ctypes.cast(ctypes.pointer(st), ctypes.c_void_p))
        jid = ctypes.c_uint64()
        _check(lib().msllr_submit(self._ctx, ctypes.byref(job), ctypes.byref(jid)), self._ctx)
        # the output buffers and the stats struct must outlive the job
        if not hasattr(self, "_jobs"):
            self._jobs = {}
        self._jobs[jid.value] = (X_out, Z_out, st)
        return jid.value

    def msllr_poll(self, job_id):
        """None while the job runs; its stats dict once it has finished (raises
        MsllrError if the job failed)."""
        done = ctypes.c_int()
        code = lib().msllr_poll(self._ctx, ctypes.c_uint64(job_id), ctypes.byref(done))
        keep = getattr(self, "_jobs", {})
        if done.value:
            _, _, st = keep.pop(job_id, (None, None, None))
            _check(code, self._ctx)
            return st.to_dict() if st is not None else {}
        _check(code, self._ctx)
        return None

    def msllr_wait(self, job_id, timeout_ms=-1):
        """Wait for the job; returns its stats dict (MsllrError with MSLLR_ETIMEOUT if it
        has not finished within timeout_ms)."""
        code = lib().msllr_wait(self._ctx, ctypes.c_uint64(job_id), int(timeout_ms))
        keep = getattr(self, "_jobs", {})
        if code == MSLLR_ETIMEOUT:
            _check(code, self._ctx)
        _, _, st = keep.pop(job_id, (None, None, None))
        _check(code, self._ctx)
        return st.to_dict() if st is not None else {}
