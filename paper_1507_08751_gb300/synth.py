"""Seeded synthetic inputs shaped like the paper's workloads.

Shared by the tests, the benchmark and the oracle checks.  This module holds
no arithmetic of the decomposition method itself: it only draws the
multi-scale components of the model in Sec. 2 (Y = sum_i X_i with every X_i
block-wise low rank on the unshifted grid) and returns them.  All draws use
NumPy's PCG64 with the given seed.

A "rank-r block" is sum_{t<r} u_t v_t^T with u_t in R^m, v_t in R^n drawn
i.i.d. N(0, 1), placed on block b of the scale's partition.
"""

from __future__ import annotations

import numpy as np

BASE_SEED = 1507087510


def _rank_r_blocks(rng, M, N, m, n, p_active, rank):
    """Component of one block scale: each m x n block is active with
    probability p_active and then holds a rank-``rank`` Gaussian outer
    product sum."""
    X = np.zeros((M, N))
    bm, bn = M // m, N // n
    active = rng.random((bm, bn)) < p_active
    for p, q in zip(*np.nonzero(active)):
        u = rng.standard_normal((m, rank))
        v = rng.standard_normal((n, rank))
        X[p * m:(p + 1) * m, q * n:(q + 1) * n] = u @ v.T
    return X


def tiny_64(seed=BASE_SEED):
    """64 x 64 matrix, four scales 1x1 / 4x4 / 16x16 / 64x64:
    1x1: 5% nonzeros ~ N(0,1); 4x4: rank-1 blocks active w.p. 0.05;
    16x16: rank-1 blocks active w.p. 0.1; 64x64: one rank-1 global term;
    plus i.i.d. Gaussian noise of variance 1e-4 (std 1e-2).
    Returns (Y float64, components (4, 64, 64), scales)."""
    rng = np.random.default_rng(seed)
    M = N = 64
    scales = [(1, 1), (4, 4), (16, 16), (64, 64)]
    comps = np.zeros((4, M, N))
    comps[0] = (rng.random((M, N)) < 0.05) * rng.standard_normal((M, N))
    comps[1] = _rank_r_blocks(rng, M, N, 4, 4, 0.05, 1)
    comps[2] = _rank_r_blocks(rng, M, N, 16, 16, 0.1, 1)
    comps[3] = _rank_r_blocks(rng, M, N, 64, 64, 1.0, 1)
    noise = 1e-2 * rng.standard_normal((M, N))
    return comps.sum(axis=0) + noise, comps, scales


def video(seed=BASE_SEED + 1, M=16384, N=256, mid=(16, 64, 256), p_mid=0.02,
          global_rank=2, p_sparse=0.01):
    """Surveillance-video-shaped matrix: M pixels (128x128 frames flattened)
    by N frames.  Scales 1x1, the square ``mid`` blocks and the full M x N.
    1x1: a ``p_sparse`` foreground of uniform(0,1) values; each mid scale:
    rank-1 blocks active w.p. ``p_mid``; full scale: a rank-``global_rank``
    Gaussian term.  Returns (Y float32, components float64, scales)."""
    rng = np.random.default_rng(seed)
    scales = [(1, 1)] + [(b, b) for b in mid] + [(M, N)]
    comps = np.zeros((len(scales), M, N))
    comps[0] = (rng.random((M, N)) < p_sparse) * rng.random((M, N))
    for i, b in enumerate(mid, start=1):
        comps[i] = _rank_r_blocks(rng, M, N, b, b, p_mid, 1)
    comps[-1] = rng.standard_normal((M, global_rank)) @ rng.standard_normal((N, global_rank)).T
    return comps.sum(axis=0).astype(np.float32), comps, scales


def video3d(seed=BASE_SEED + 3, H=64, W=64, T=64, blocks=((4, 4, 4), (16, 16, 16)), p_active=0.05,
            p_sparse=0.01):
    """Video matrix of H x W-pixel frames by T frames (row y W + x for pixel
    (y, x)) with spatio-temporal structure at the given bh x bw x bt block
    sizes (the Sec. 10.2 partitions): each block of the video cube is active
    with probability p_active and then holds a rank-1 term (a Gaussian patch
    image times a Gaussian time course), plus a rank-1 Gaussian background
    and a p_sparse foreground of uniform(0, 1) values.
    Returns (Y float32, scales with the full matrix last, frame (H, W))."""
    rng = np.random.default_rng(seed)
    V = np.zeros((H, W, T))
    for bh, bw, bt in blocks:
        for y0 in range(0, H, bh):
            for x0 in range(0, W, bw):
                for t0 in range(0, T, bt):
                    if rng.random() < p_active:
                        patch = rng.standard_normal((bh, bw))
                        course = rng.standard_normal(bt)
                        V[y0:y0 + bh, x0:x0 + bw, t0:t0 + bt] += patch[:, :, None] * course
    Y = V.reshape(H * W, T)
    Y += np.outer(rng.standard_normal(H * W), rng.standard_normal(T))
    Y += (rng.random((H * W, T)) < p_sparse) * rng.random((H * W, T))
    scales = [(1, 1)] + [tuple(b) for b in blocks] + [(H * W, T)]
    return Y.astype(np.float32), scales, (H, W)


def dyadic_scales(M, N, L, base=4):
    """Two-sided dyadic partition of the batching/serving workloads:
    1x1, then base^k x base^k for k = 1..L-2 (clamped so that blocks divide
    the matrix), then the full M x N."""
    scales = [(1, 1)]
    k = 1
    while len(scales) < L - 1:
        b = base ** k
        if b > min(M, N) or M % b or N % b:
            break
        scales.append((b, b))
        k += 1
    scales.append((M, N))
    return scales


def job(seed, M, N, L, p_lo=0.02, p_hi=0.1, p_sparse=0.02):
    """One batching/serving job: dyadic scales, rank-1 or rank-2 blocks
    (50/50 per scale) active w.p. uniform in [p_lo, p_hi] per scale, a global
    low-rank term and ``p_sparse`` N(0,1) sparse entries.
    Returns (Y float32, scales)."""
    rng = np.random.default_rng(seed)
    scales = dyadic_scales(M, N, L)
    Y = (rng.random((M, N)) < p_sparse) * rng.standard_normal((M, N))
    for (m, n) in scales[1:-1]:
        rank = 1 if rng.random() < 0.5 else 2
        Y += _rank_r_blocks(rng, M, N, m, n, rng.uniform(p_lo, p_hi), rank)
    rank = 1 if rng.random() < 0.5 else 2
    Y += rng.standard_normal((M, rank)) @ rng.standard_normal((N, rank)).T
    return Y.astype(np.float32), scales


def ratings(seed, M, N, density=0.05):
    """Rating-matrix-like job (Sec. 10.4 shape): observed mask at ``density``,
    integer values 1..5 on observed entries, 0 elsewhere.
    Returns (Y float32, mask uint8)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((M, N)) < density
    vals = rng.integers(1, 6, size=(M, N))
    return np.where(mask, vals, 0).astype(np.float32), mask.astype(np.uint8)


def hanning_blobs(seed=BASE_SEED + 2, M=64, N=64, scales=((1, 1), (4, 4), (16, 16), (64, 64)),
                  counts=(6, 3, 2, 1), amps=(4.0, 8.0, 16.0, 32.0)):
    """The Fig. 1 style example: every component of a scale is a rank-1 outer
    product of Hanning windows spanning one block of that scale (a single
    entry for 1x1), ``counts[i]`` of them per scale on distinct random
    blocks, with amplitude ``amps[i]``.  Returns (Y, components, scales)."""
    rng = np.random.default_rng(seed)
    comps = np.zeros((len(scales), M, N))
    for i, (m, n) in enumerate(scales):
        bm, bn = M // m, N // n
        picks = rng.choice(bm * bn, size=counts[i], replace=False)
        hm = np.hanning(m + 2)[1:-1] if m > 1 else np.ones(1)
        hn = np.hanning(n + 2)[1:-1] if n > 1 else np.ones(1)
        sign = rng.choice([-1.0, 1.0], size=counts[i])
        for t, b in enumerate(picks):
            p, q = divmod(int(b), bn)
            comps[i, p * m:(p + 1) * m, q * n:(q + 1) * n] = sign[t] * amps[i] * np.outer(hm, hn)
    return comps.sum(axis=0), comps, list(scales)


def _logspread_blocks(rng, M, N, m, n, p_active, rank=2, lo=1e-2, hi=1e2):
    """Component of one block scale: each m x n block is active with
    probability p_active and then holds sum_j s_j u_j v_j^T over ``rank``
    unit vectors u_j, v_j (normalised Gaussians) with s_j log-uniform in
    [lo, hi].  Vectorised over the active blocks."""
    X = np.zeros((M, N), dtype=np.float32)
    bm, bn = M // m, N // n
    act = np.nonzero(rng.random((bm, bn)) < p_active)
    k = act[0].size
    if k == 0:
        return X
    u = rng.standard_normal((k, m, rank))
    v = rng.standard_normal((k, n, rank))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    s = 10.0 ** rng.uniform(np.log10(lo), np.log10(hi), size=(k, rank))
    blocks = np.einsum("kmr,kr,knr->kmn", u, s, v).astype(np.float32)
    view = X.reshape(bm, m, bn, n)
    view[act[0], :, act[1], :] = blocks
    return X


def precision(seed=BASE_SEED + 5, M=8192, N=8192, p_active=0.05, p_sparse=0.02):
    """The single large precision job: M x N with six scales 1x1, 8x8, 32x32,
    128x128, 1024x1024 and the full matrix.  Each block of the four middle
    scales is active with probability ``p_active`` and then rank 2 with
    singular values log-uniform in [1e-2, 1e2], so that some sit near their
    scale's threshold; the full matrix holds one such rank-2 term and the
    1x1 scale ``p_sparse`` N(0,1) entries.  Returns (Y float32, scales)."""
    rng = np.random.default_rng(seed)
    scales = [(1, 1), (8, 8), (32, 32), (128, 128), (1024, 1024), (M, N)]
    Y = ((rng.random((M, N)) < p_sparse) * rng.standard_normal((M, N))).astype(np.float32)
    for (m, n) in scales[1:-1]:
        Y += _logspread_blocks(rng, M, N, m, n, p_active)
    Y += _logspread_blocks(rng, M, N, M, N, 1.0)
    return Y, scales
