"""Plain FP64 restatement of the multi-scale low rank ADMM (Ong & Lustig).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the
benchmark's CPU baseline; never by the product path.  Every function follows
one passage of the paper and is written for a reader checking it by eye, not
for speed: no blocking, fusion or reordering beyond what the passage states.

Notation (paper Sec. 2): Y is M x N, L scales, scale i has block size
m_i x n_i, R_b extracts block b and R_b^T embeds it back, tau_i = lambda_i/rho.

Readings of passages the paper leaves open (each one is also listed in the
design notes):
  * initial state Z_i = U_i = 0 (eq:admm gives none);
  * Shift_s(X)[r, c] = X[(r + s_r) mod M, (c + s_c) mod N], circular, and one
    shift s per iteration shared by every scale (Sec. 9);
  * the shift sequence is drawn with splitmix64 (not given in the paper);
  * SVT keeps max(sigma - tau, 0), so sigma == tau contributes nothing;
  * the returned X_i is the X-update of eq:admm applied to the final (Z, U),
    so that sum_i X_i = Y holds exactly (up to rounding);
  * masked X-update (Sec. 10.4): the residual term is zero at unobserved
    entries, and Y there is ignored;
  * the noise scale of Sec. 2.1 (the whole matrix reshaped to one MN x 1
    block, whose nuclear norm is the Frobenius norm) is written as the block
    size (0, 0); its default weight is eq:lambda with m = MN, n = 1;
  * averaged cycle spinning (Sec. 9): the set S of a scale is all shifts
    modulo its block size, or a sub-lattice of it, offset by the iteration's
    random shift when that is on.
"""

from __future__ import annotations

import math

import numpy as np

_MASK64 = (1 << 64) - 1
_GOLDEN_GAMMA = 0x9E3779B97F4A7C15


# --------------------------------------------------------------------------
# Random cycle-spin shifts (Sec. 9, "random cycle spinning").
# --------------------------------------------------------------------------

def splitmix64(x: int) -> int:
    """The splitmix64 output function (Steele, Lea & Flood, OOPSLA 2014)
    applied to the 64-bit state ``x``: two xor-shift-multiply rounds and a
    final xor-shift."""
    z = x & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def shift_table(seed: int, iters: int, M: int, N: int) -> np.ndarray:
    """Shift s_k = (s_r, s_c) for iterations k = 0..iters-1 (Sec. 9: "s is
    randomly chosen from the set S", S = all circular shifts of an M x N
    matrix).  State for iteration k is seed + (k+1)*golden_gamma, i.e. the
    k-th splitmix64 draw from ``seed``; the high 32 bits pick the row shift
    and the low 32 bits the column shift."""
    out = np.zeros((iters, 2), dtype=np.int64)
    for k in range(iters):
        z = splitmix64((seed + (k + 1) * _GOLDEN_GAMMA) & _MASK64)
        out[k, 0] = (z >> 32) % M
        out[k, 1] = (z & 0xFFFFFFFF) % N
    return out


# --------------------------------------------------------------------------
# Regularisation parameters (Sec. 4, eq:lambda).
# --------------------------------------------------------------------------

def lambda_default(M: int, N: int, m: int, n: int) -> float:
    """eq:lambda as used in the experiments (Sec. 10):
    lambda_i = sqrt(m_i) + sqrt(n_i) + sqrt(log(M N / max(m_i, n_i))).
    The noise scale (0, 0) is the MN x 1 block: sqrt(MN) + 1 (Sec. 4 notes
    the sqrt(MN) scaling)."""
    if (m, n) == (0, 0):
        m, n = M * N, 1
    return math.sqrt(m) + math.sqrt(n) + math.sqrt(math.log(M * N / max(m, n)))


def lambda_area(M: int, N: int, m: int, n: int) -> float:
    """Variant of eq:lambda with the block area inside the log,
    sqrt(m) + sqrt(n) + sqrt(log(M N / (m n))), as the tiny 64x64 workload
    specifies it."""
    return math.sqrt(m) + math.sqrt(n) + math.sqrt(math.log(M * N / (m * n)))


# --------------------------------------------------------------------------
# Shift operators (Sec. 9).
# --------------------------------------------------------------------------

def shift(X: np.ndarray, s) -> np.ndarray:
    """Shift_s(X)[r, c] = X[(r + s_r) mod M, (c + s_c) mod N]."""
    M, N = X.shape
    rows = (np.arange(M) + int(s[0])) % M
    cols = (np.arange(N) + int(s[1])) % N
    return X[np.ix_(rows, cols)]


def unshift(X: np.ndarray, s) -> np.ndarray:
    """Shift_{-s}, the inverse of ``shift``: out[(r+s_r) mod M, (c+s_c) mod N] = X[r, c]."""
    M, N = X.shape
    rows = (np.arange(M) + int(s[0])) % M
    cols = (np.arange(N) + int(s[1])) % N
    out = np.empty_like(X)
    out[np.ix_(rows, cols)] = X
    return out


# --------------------------------------------------------------------------
# Singular value thresholding (Sec. 7, eq:svt and eq:bsvt).
# --------------------------------------------------------------------------

def svt(B: np.ndarray, tau: float) -> np.ndarray:
    """eq:svt: SVT_tau(B) = U max(Sigma - tau, 0) V^T from a full SVD."""
    U, s, Vh = np.linalg.svd(B, full_matrices=False)
    return (U * np.maximum(s - tau, 0.0)) @ Vh


def soft_threshold(a: np.ndarray, tau: float) -> np.ndarray:
    """The SVD of a 1x1 matrix [a] written out: sigma = |a|, u = sign(a),
    v = 1, so SVT_tau([a]) = sign(a) max(|a| - tau, 0) -- the element-wise
    soft threshold that eq:bsvt reduces to for 1x1 blocks (Sec. 7)."""
    return np.sign(a) * np.maximum(np.abs(a) - tau, 0.0)


def _blocks(A: np.ndarray, m: int, n: int) -> np.ndarray:
    """R_b for every block b of the m x n partition (Sec. 2, Fig. Rop):
    block (p, q) is A[p*m:(p+1)*m, q*n:(q+1)*n]; returns shape (nb, m, n).
    The noise scale (0, 0) is the one block R_noise(A), the whole matrix
    reshaped to MN x 1 (Sec. 2.1)."""
    M, N = A.shape
    if (m, n) == (0, 0):
        return A.reshape(1, M * N, 1)
    if M % m or N % n:
        raise ValueError(f"block {m}x{n} does not divide {M}x{N}")
    return A.reshape(M // m, m, N // n, n).transpose(0, 2, 1, 3).reshape(-1, m, n)


def _unblocks(B: np.ndarray, M: int, N: int) -> np.ndarray:
    """sum_b R_b^T(B_b): the adjoint of ``_blocks`` (blocks do not overlap)."""
    nb, m, n = B.shape
    if (nb, m, n) == (1, M * N, 1) and (M, N) != (M * N, 1):
        return B.reshape(M, N)  # the noise block R_noise^T
    return B.reshape(M // m, N // n, m, n).transpose(0, 2, 1, 3).reshape(M, N)


def block_svt(A: np.ndarray, m: int, n: int, tau: float,
              closed_form_1x1: bool = True) -> np.ndarray:
    """eq:bsvt: BlockSVT_tau(A) = sum_b R_b^T(SVT_tau(R_b(A))).

    Every block gets a full FP64 SVD (LAPACK gesdd through NumPy, batched over
    the blocks of the scale).  For 1x1 blocks the 1x1 SVD is written out
    (``soft_threshold``) unless ``closed_form_1x1`` is False."""
    M, N = A.shape
    if m == 1 and n == 1 and closed_form_1x1:
        return soft_threshold(A, tau)
    B = _blocks(A, m, n)
    U, s, Vh = np.linalg.svd(B, full_matrices=False)
    Zb = (U * np.maximum(s - tau, 0.0)[:, None, :]) @ Vh
    return _unblocks(Zb, M, N)


# --------------------------------------------------------------------------
# Spatio-temporal blocks (Sec. 10.2: the video partitions 4x4x4 and
# 16x16x16).  The M x N video matrix has one column per frame and row
# y * W + x for pixel (y, x) of an H x W frame (M = H W).  A bh x bw x bt
# block of the video cube is reshaped by R_b into a (bh bw) x bt matrix,
# pixels in row-major order within the patch (Sec. 2, the block reshape
# operator).
# --------------------------------------------------------------------------

def blocks3d(A: np.ndarray, H: int, W: int, bh: int, bw: int, bt: int, s3=(0, 0, 0)) -> np.ndarray:
    """R_b of every bh x bw x bt block of the video cube of A, after the
    circular shift s3 = (s_y, s_x, s_t) of the cube (Sec. 9 in three
    dimensions); returns shape (nb, bh*bw, bt)."""
    M, T = A.shape
    if M != H * W or H % bh or W % bw or T % bt:
        raise ValueError("spatio-temporal block does not divide the video")
    V = A.reshape(H, W, T)
    V = np.roll(V, shift=(-int(s3[0]), -int(s3[1]), -int(s3[2])), axis=(0, 1, 2))
    V = V.reshape(H // bh, bh, W // bw, bw, T // bt, bt)
    return V.transpose(0, 2, 4, 1, 3, 5).reshape(-1, bh * bw, bt)


def unblocks3d(B: np.ndarray, H: int, W: int, T: int, bh: int, bw: int, bt: int,
               s3=(0, 0, 0)) -> np.ndarray:
    """The adjoint (and inverse) of ``blocks3d``: embed every block back and
    undo the shift; returns the (H W) x T matrix."""
    V = B.reshape(H // bh, W // bw, T // bt, bh, bw, bt).transpose(0, 3, 1, 4, 2, 5)
    V = V.reshape(H, W, T)
    V = np.roll(V, shift=(int(s3[0]), int(s3[1]), int(s3[2])), axis=(0, 1, 2))
    return V.reshape(H * W, T)


def block_svt_3d(A: np.ndarray, H: int, W: int, bh: int, bw: int, bt: int, tau: float,
                 s3=(0, 0, 0)) -> np.ndarray:
    """eq:bsvt with spatio-temporal blocks: SVT of every (bh bw) x bt block
    matrix (full FP64 SVD), embedded back."""
    B = blocks3d(A, H, W, bh, bw, bt, s3)
    U, sv, Vh = np.linalg.svd(B, full_matrices=False)
    Zb = (U * np.maximum(sv - tau, 0.0)[:, None, :]) @ Vh
    return unblocks3d(Zb, H, W, A.shape[1], bh, bw, bt, s3)


def spin_set(m: int, n: int, g: int):
    """Shifts averaged by cycle spinning at a scale of m x n blocks (Sec. 9:
    S is the set of all shifts the application allows).  Shifts that differ
    by whole blocks give the same partition, so all distinct shifts are
    {0..m-1} x {0..n-1}; ``g`` >= max(m, n) takes all of them.  A smaller g
    takes the sub-lattice of steps m/g_r, n/g_c (g_r = min(g, m), g_c =
    min(g, n), which must divide m and n): invariance to shifts by multiples
    of those steps.  g <= 1 gives {(0, 0)}."""
    if g <= 1:
        return [(0, 0)]
    gr, gc = min(g, m), min(g, n)
    if m % gr or n % gc:
        raise ValueError("spin grid must divide the block size")
    return [(a * (m // gr), b * (n // gc)) for a in range(gr) for b in range(gc)]


def block_svt_spun(A: np.ndarray, m: int, n: int, tau: float, shifts) -> np.ndarray:
    """Cycle-spun BlockSVT (Sec. 9, the averaged Z-update):
        (1/|S|) sum_{s in S} Shift_{-s}(BlockSVT_tau(Shift_s(A)))."""
    out = np.zeros_like(A, dtype=np.float64)
    for s in shifts:
        out += unshift(block_svt(shift(A, s), m, n, tau), s)
    return out / len(shifts)


def block_nuclear_norm(X: np.ndarray, m: int, n: int) -> float:
    """||X||_(i) = sum_b ||R_b(X)||_* (Sec. 3)."""
    return float(np.linalg.svd(_blocks(X, m, n), compute_uv=False).sum())


def block_dual_norm(X: np.ndarray, m: int, n: int) -> float:
    """||X||*_(i) = max_b sigma_max(R_b(X)) (Sec. 3)."""
    return float(np.linalg.svd(_blocks(X, m, n), compute_uv=False).max())


# --------------------------------------------------------------------------
# ADMM (Sec. 7, eq:admm), random cycle spinning (Sec. 9), masked
# X-update (Sec. 10.4).
# --------------------------------------------------------------------------

def consensus_residual(Y, Z, U, mask=None):
    """(1/L)(Y - sum_i (Z_i - U_i)), the data-consistency term of the
    X-update in eq:admm; zero at unobserved entries (Sec. 10.4)."""
    L = Z.shape[0]
    R = (Y - (Z - U).sum(axis=0)) / L
    if mask is not None:
        R = np.where(mask, R, 0.0)
    return R


def x_update(Y, Z, U, mask=None):
    """X_i <- (Z_i - U_i) + (1/L)(Y - sum_j (Z_j - U_j))   (eq:admm, line 1);
    at unobserved entries X_i <- Z_i - U_i (Sec. 10.4)."""
    return (Z - U) + consensus_residual(Y, Z, U, mask)[None]


def shift3d(s, W: int, T: int):
    """The iteration's shift (s_r, s_c) read on the video cube: the row shift
    names a pixel, (s_y, s_x) = divmod(s_r, W), and s_c a frame shift."""
    sy, sx = divmod(int(s[0]), W)
    return (sy, sx, int(s[1]) % T)


def admm_step(Y, Z, U, scales, taus, s, mask=None, spin=None, frame=None):
    """One iteration of eq:admm with the Sec. 9 random-shift Z-update:
        X_i <- (Z_i - U_i) + (1/L)(Y - sum_j (Z_j - U_j))
        Z_i <- Shift_{-s}(BlockSVT_{tau_i}(Shift_s(X_i + U_i)))
        U_i <- U_i - (Z_i - X_i)
    ``s`` is one (s_r, s_c) pair shared by all scales, or an (L, 2) array
    with one pair per scale.  With ``spin`` (a list of shift sets, one per
    scale, from ``spin_set``) the Z-update is the averaged one of Sec. 9 over
    the shifts s + t, t in the scale's set.  A scale given as (bh, bw, bt)
    is a spatio-temporal partition of the video cube of frame ``frame`` =
    (H, W) (Sec. 10.2), shifted by ``shift3d``.  Returns (X, Z_new, U_new)."""
    X = x_update(Y, Z, U, mask)
    s = np.asarray(s).reshape(-1, 2)
    Znew = np.empty_like(Z)
    for i, sc in enumerate(scales):
        m, n = sc[0], sc[-1]
        si = s[i] if s.shape[0] > 1 else s[0]
        if len(scales[i]) == 3:
            bh, bw, bt = scales[i]
            H, W = frame
            Znew[i] = block_svt_3d(X[i] + U[i], H, W, bh, bw, bt, taus[i],
                                   shift3d(si, W, Y.shape[1]))
            continue
        if spin is not None and len(spin[i]) > 1:
            S = [(int(si[0]) + t[0], int(si[1]) + t[1]) for t in spin[i]]
            Znew[i] = block_svt_spun(X[i] + U[i], m, n, taus[i], S)
            continue
        Znew[i] = unshift(block_svt(shift(X[i] + U[i], si), m, n, taus[i]), si)
    Unew = U - (Znew - X)
    return X, Znew, Unew


def admm(Y, scales, lambdas, rho=1.0, iters=100, shifts=None, mask=None,
         Z0=None, U0=None, history=False, spin_grid=0, frame=None):
    """Solve eq:cvx (or its masked form, Sec. 10.4) by ``iters`` iterations of
    eq:admm, starting from Z = U = 0 unless (Z0, U0) are given.

    ``shifts``: None (no cycle spinning) or an array with one shift per
    iteration, shape (iters, 2) or (iters, L, 2).
    ``frame``: (H, W) when some scales are spatio-temporal (bh, bw, bt).
    ``spin_grid``: g > 1 averages every scale's Z-update over ``spin_set``
    (Sec. 9); the 1x1, full-matrix and noise scales commute with every shift
    and keep the single update.
    Returns a dict with X (the X-update applied to the final Z, U), Z, U and,
    if ``history``, per-iteration objective sum_i lambda_i ||Z_i||_(i) and
    primal residual ||X - Z||_F."""
    Y = np.asarray(Y, dtype=np.float64)
    L = len(scales)
    M, N = Y.shape
    if mask is not None:
        mask = np.asarray(mask, dtype=bool)
        Y = np.where(mask, Y, 0.0)
    taus = [lam / rho for lam in lambdas]
    Z = np.zeros((L, M, N)) if Z0 is None else np.array(Z0, dtype=np.float64)
    U = np.zeros((L, M, N)) if U0 is None else np.array(U0, dtype=np.float64)
    obj, pres = [], []
    spin = None
    if spin_grid > 1:
        spin = [[(0, 0)] if len(sc) == 3 or tuple(sc) in ((1, 1), (M, N), (0, 0))
                else spin_set(sc[0], sc[1], spin_grid) for sc in scales]
    for k in range(iters):
        s = (0, 0) if shifts is None else shifts[k]
        extra = {}
        if spin is not None:
            extra["spin"] = spin
        if frame is not None:
            extra["frame"] = frame
        X, Z, U = admm_step(Y, Z, U, scales, taus, s, mask, **extra)
        if history:
            obj.append(sum(lam * (block_nuclear_norm(Z[i], *scales[i]) if len(scales[i]) == 2
                                  else float(np.linalg.svd(blocks3d(Z[i], *frame, *scales[i]),
                                                           compute_uv=False).sum()))
                           for i, lam in enumerate(lambdas)))
            pres.append(float(np.linalg.norm(X - Z)))
    out = {"X": x_update(Y, Z, U, mask), "Z": Z, "U": U}
    if history:
        out["objective"] = np.array(obj)
        out["primal_residual"] = np.array(pres)
    return out


def relerr(X, Xref, Y) -> np.ndarray:
    """Per-component relative Frobenius error
    ||X_i - Xref_i||_F / max(||Xref_i||_F, 1e-6 ||Y||_F)."""
    X = np.asarray(X, dtype=np.float64)
    Xref = np.asarray(Xref, dtype=np.float64)
    floor = 1e-6 * np.linalg.norm(np.asarray(Y, dtype=np.float64))
    num = np.linalg.norm((X - Xref).reshape(X.shape[0], -1), axis=1)
    den = np.maximum(np.linalg.norm(Xref.reshape(Xref.shape[0], -1), axis=1), floor)
    return num / den
