"""GPU parity of blocks wider than 256 (certified subspace iteration spread
over many CTAs) against the FP64 oracle, through the C ABI.

Same bar as the other parity tests: relative Frobenius error <= 1e-4 per
output, block ranks equal except where a singular value lies within 1e-4
(relative) of tau.  The certificate (no singular value above tau outside the
pairs found) is required where the spectrum leaves room for its rounding
margin; inside ADMM runs, where singular values crowd just below tau, an
uncertified block is allowed and the parity bar alone applies.
"""

import numpy as np
import pytest

import oracle as O
from paper_1507_08751_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_08751_gb300 import binding as B
    B.lib()
    c = B.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _lowrank_plus_noise(seed, M, N, m, n, noise=0.3):
    """Per block: rank 0-3 content of varied strength plus dense noise."""
    rng = np.random.default_rng(seed)
    A = noise * rng.standard_normal((M, N))
    for p in range(M // m):
        for q in range(N // n):
            r = int(rng.integers(0, 4))
            amp = float(rng.choice([0.0, 1.0, 3.0, 8.0]))
            if r and amp:
                u = rng.standard_normal((m, r))
                v = rng.standard_normal((n, r))
                A[p * m:(p + 1) * m, q * n:(q + 1) * n] += amp * (u @ v.T) / np.sqrt(max(m, n))
    return A.astype(np.float32)


def _block_sv(A, m, n):
    M, N = A.shape
    B = A.reshape(M // m, m, N // n, n).transpose(0, 2, 1, 3).reshape(-1, m, n)
    return np.linalg.svd(B, compute_uv=False)


def _check_blocksvt(ctx, A, m, n, tau, shift):
    M, N = A.shape
    Z = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    rank = torch.empty(((M // m) * (N // n),), dtype=torch.int32, device="cuda")
    ctx.msllr_blocksvt(dev(A), Z, m, n, tau, shift, rank_out=rank)
    torch.cuda.synchronize()
    A64 = A.astype(np.float64)
    want = O.unshift(O.block_svt(O.shift(A64, shift), m, n, tau), shift)
    got = Z.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    err = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-6 * np.linalg.norm(A64))
    assert err <= TOL, f"relative error {err:.3e}"
    svs = _block_sv(O.shift(A64, shift), m, n)
    want_rank = (svs > tau).sum(axis=1)
    near = (np.abs(svs - tau) <= 1e-4 * np.maximum(svs[:, :1], tau)).any(axis=1)
    bad = (rank.cpu().numpy() != want_rank) & ~near
    assert not bad.any(), f"{bad.sum()} blocks with a wrong rank"
    return want_rank


WIDE_CASES = [
    # (M, N, m, n, shift): full-matrix scale, shifted square blocks, wide
    # (transposed) blocks with a width that is not a multiple of 64, several
    # blocks in a row
    (1024, 1024, 1024, 1024, (0, 0)),
    (2048, 1024, 1024, 1024, (700, 300)),
    (640, 1280, 320, 640, (5, 601)),
    (512, 1536, 512, 512, (100, 1000)),
    (3000, 300, 3000, 300, (0, 0)),
]


@pytest.mark.parametrize("M,N,m,n,shift", WIDE_CASES)
def test_wide_blocksvt_matches_oracle(ctx, M, N, m, n, shift):
    A = _lowrank_plus_noise(M * 7 + N, M, N, m, n)
    sv = _block_sv(O.shift(A.astype(np.float64), shift), m, n)
    # tau between the noise edge and the low-rank content, so that block
    # ranks stay small (at most 3 here; the path keeps up to 16 pairs)
    edge = 0.3 * (np.sqrt(m) + np.sqrt(n))
    top = np.quantile(sv[:, 0], 0.4) if sv.shape[0] > 3 else 0.5 * sv[:, 0].max()
    tau = float(max(1.5 * edge, top))
    _check_blocksvt(ctx, A, m, n, tau, shift)


def test_wide_blocksvt_exactly_low_rank(ctx):
    """A rank-2 matrix without noise: the Gram matrix is singular, the basis
    update must stay well defined; tau between and below the two singular
    values, and above both (rank 0)."""
    rng = np.random.default_rng(5)
    M, N = 1024, 512
    A = (rng.standard_normal((M, 2)) * [3.0, 1.0]) @ rng.standard_normal((2, N))
    A = A.astype(np.float32)
    s = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    for tau, rk in ((0.5 * (s[0] + s[1]), 1), (0.5 * s[1], 2), (1.5 * s[0], 0)):
        got = _check_blocksvt(ctx, A, M, N, float(tau), (0, 0))
        assert got[0] == rk


def test_wide_blocksvt_rank_zero_and_shortcut(ctx):
    """Dense noise far below tau (the trace shortcut) and just below it (a
    rank-0 block proved by the certificate)."""
    rng = np.random.default_rng(6)
    A = (0.1 * rng.standard_normal((768, 512))).astype(np.float32)
    s0 = np.linalg.svd(A.astype(np.float64), compute_uv=False)[0]
    for tau in (1e3, 1.02 * s0):
        _check_blocksvt(ctx, A, 768, 512, float(tau), (0, 0))


@pytest.mark.parametrize("M,N", [(1024, 1024), (3000, 300), (512, 768)])
def test_wide_certificate_on_separated_spectrum(ctx, M, N):
    """One SVT of the full matrix (a one-scale decomposition, first
    iteration: A = Y): low-rank content well above tau and noise well below
    it, so the certificate must hold and count the block as certified."""
    A = _lowrank_plus_noise(M + 3 * N, M, N, M, N)
    s = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    edge = 0.3 * (np.sqrt(M) + np.sqrt(N))
    tau = float(max(1.5 * edge, 0.5 * s[0]))
    X = torch.empty((1, M, N), dtype=torch.float32, device="cuda")
    Z = torch.empty_like(X)
    stats = ctx.msllr_decompose(dev(A), [(M, N)], X, lambdas=[tau], rho=1.0, iters=1, seed=1,
                                Z_out=Z)
    torch.cuda.synchronize()
    assert stats["blocks_uncertified"][0] == 0
    assert stats["blocks_lanczos"][0] + stats["blocks_skipped"][0] == 1
    want = O.svt(A.astype(np.float64), tau)
    got = Z[0].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - want) <= TOL * max(np.linalg.norm(want), 1e-6 * np.linalg.norm(A))


def _run(ctx, Y32, scales, iters, seed, mask=None):
    M, N = Y32.shape
    X = torch.empty((len(scales), M, N), dtype=torch.float32, device="cuda")
    stats = ctx.msllr_decompose(dev(Y32), scales, X, rho=1.0, iters=iters, seed=seed,
                                mask=None if mask is None else dev(mask))
    torch.cuda.synchronize()
    return X.cpu().numpy(), stats


def test_decompose_with_full_scale_1024_matches_oracle(ctx):
    """A 1024 x 1024 batching-workload job with its dyadic scales 1, 4, 16,
    64, 256 and the full matrix (a 1024-wide block)."""
    Y32, scales = synth.job(1507087510 + 3, 1024, 1024, 6)
    assert scales[-1] == (1024, 1024)
    M, N = Y32.shape
    iters, seed = 20, 11
    X, stats = _run(ctx, Y32, scales, iters, seed)
    lam = [O.lambda_default(M, N, m, n) for m, n in scales]
    ref = O.admm(Y32.astype(np.float64), scales, lam, 1.0, iters,
                 shifts=O.shift_table(seed, iters, M, N))
    err = O.relerr(X, ref["X"], Y32)
    assert np.all(err <= TOL), err
    X2, _ = _run(ctx, Y32, scales, iters, seed)
    np.testing.assert_array_equal(X, X2)


def test_decompose_with_shifted_wide_blocks_matches_oracle(ctx):
    """2048 x 1024 with 512 x 512 blocks on the cycle-spun grid (no warm
    start carries over) and the 2048 x 1024 full-matrix scale."""
    rng_seed = 1507087510 + 4
    Y32, _ = synth.job(rng_seed, 2048, 1024, 6)
    scales = [(1, 1), (16, 16), (64, 64), (256, 256), (512, 512), (2048, 1024)]
    M, N = Y32.shape
    iters, seed = 8, 12
    X, stats = _run(ctx, Y32, scales, iters, seed)
    lam = [O.lambda_default(M, N, m, n) for m, n in scales]
    ref = O.admm(Y32.astype(np.float64), scales, lam, 1.0, iters,
                 shifts=O.shift_table(seed, iters, M, N))
    err = O.relerr(X, ref["X"], Y32)
    assert np.all(err <= TOL), err


def test_decompose_masked_ratings_full_scale_matches_oracle(ctx):
    """Rating-matrix-like job (Sec. 10.4): 512 x 768 at 5% observed, the
    full-matrix scale 512 wide."""
    Y32, mask = synth.ratings(1507087510 + 5, 512, 768, density=0.05)
    scales = [(1, 1), (4, 4), (16, 16), (512, 768)]
    M, N = Y32.shape
    iters, seed = 30, 13
    X, stats = _run(ctx, Y32, scales, iters, seed, mask=mask)
    lam = [O.lambda_default(M, N, m, n) for m, n in scales]
    ref = O.admm(Y32.astype(np.float64), scales, lam, 1.0, iters,
                 shifts=O.shift_table(seed, iters, M, N), mask=mask.astype(bool))
    err = O.relerr(X, ref["X"], Y32)
    assert np.all(err <= TOL), err


def test_full_matrix_svt_8192_closed_form(ctx):
    """The widest full-matrix scale (8192 x 8192): for A = U diag(s) V^T with
    orthonormal U, V the block SVT is U diag(max(s - tau, 0)) V^T exactly
    (eq:svt); the GPU result matches it, with its rank, under a shift (the
    full matrix ignores it)."""
    M = N = 8192
    rng = np.random.default_rng(81)
    U, _ = np.linalg.qr(rng.standard_normal((M, 4)))
    V, _ = np.linalg.qr(rng.standard_normal((N, 4)))
    s = np.array([80.0, 40.0, 12.0, 3.0])
    tau = 10.0
    Ud = torch.from_numpy(U).cuda()
    Vd = torch.from_numpy(V).cuda()
    A = ((Ud * torch.from_numpy(s).cuda()) @ Vd.T).float().contiguous()
    want = (Ud * torch.from_numpy(np.maximum(s - tau, 0.0)).cuda()) @ Vd.T
    Z = torch.empty_like(A)
    rank = torch.empty((1,), dtype=torch.int32, device="cuda")
    ctx.msllr_blocksvt(A, Z, M, N, tau, (123, 4567), rank_out=rank)
    torch.cuda.synchronize()
    err = (torch.linalg.norm(Z.double() - want) / torch.linalg.norm(want)).item()
    assert err <= TOL, f"relative error {err:.3e}"
    assert int(rank.item()) == 3


def test_precision_workload_8192_matches_oracle(ctx):
    """The 8192 x 8192 job with six scales (1x1, 8x8, 32x32, 128x128,
    1024x1024, the full matrix; rank-2 blocks with singular values spread
    over [1e-2, 1e2]): two cycle-spun ADMM iterations from zero against the
    FP64 oracle on the same shift table, every X_i and Z_i to 1e-4."""
    Y32, scales = synth.precision()
    M, N = Y32.shape
    lam = [O.lambda_default(M, N, m, n) for m, n in scales]
    iters, seed = 2, 29
    X = torch.empty((len(scales), M, N), dtype=torch.float32, device="cuda")
    Z = torch.empty_like(X)
    ctx.msllr_decompose(dev(Y32), scales, X, lambdas=lam, iters=iters, seed=seed, Z_out=Z)
    torch.cuda.synchronize()
    Xh, Zh = X.cpu().numpy(), Z.cpu().numpy()
    del X, Z
    ref = O.admm(Y32.astype(np.float64), scales, lam, 1.0, iters,
                 shifts=O.shift_table(seed, iters, M, N))
    ex = O.relerr(Xh, ref["X"], Y32)
    ez = O.relerr(Zh, ref["Z"], Y32)
    assert np.all(ex <= TOL), ex
    assert np.all(ez <= TOL), ez
