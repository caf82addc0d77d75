"""GPU parity of averaged cycle spinning (Sec. 9: the Z-update averaged over a
set of shifts, msllr_params.spin_grid) against the FP64 oracle, through the
C ABI; and the translation equivariance the full shift set gives."""

import numpy as np
import pytest

import oracle as O
from paper_1507_08751_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_08751_gb300 import binding as B
    B.lib()
    return B


def _run(B, ctx, Y32, scales, lam, iters, seed, spin_grid, cycle_spin=1):
    M, N = Y32.shape
    p = B.msllr_params_default()
    p.spin_grid = spin_grid
    p.cycle_spin = cycle_spin
    X = torch.empty((len(scales), M, N), dtype=torch.float32, device="cuda")
    st = ctx.msllr_decompose(torch.from_numpy(np.ascontiguousarray(Y32)).cuda(), scales, X,
                             lambdas=lam, rho=1.0, iters=iters, seed=seed, params=p)
    torch.cuda.synchronize()
    return X.cpu().numpy(), st


def test_spun_decompose_tiny_64_matches_oracle(B):
    """64x64 workload, random shift per iteration plus the average over the
    full shift set of the 4x4 scale and a 4x4 lattice of the 16x16 scale."""
    Y, comps, scales = synth.tiny_64()
    Y32 = Y.astype(np.float32)
    M, N = Y32.shape
    lam = [O.lambda_area(M, N, m, n) for m, n in scales]
    iters, seed = 30, 7
    with B.Context(0) as ctx:
        X, st = _run(B, ctx, Y32, scales, lam, iters, seed, spin_grid=4)
    ref = O.admm(Y32.astype(np.float64), scales, lam, 1.0, iters,
                 shifts=O.shift_table(seed, iters, M, N), spin_grid=4)
    err = O.relerr(X, ref["X"], Y32)
    assert np.all(err <= TOL), err
    np.testing.assert_allclose(X.sum(0), Y32, atol=1e-5 * np.abs(Y32).max())


def test_spun_decompose_wide_blocks_matches_oracle(B):
    """A wide-block scale (128x128 blocks, the one-CTA-per-block path) and a
    fused narrow scale, each averaged over a 2x2 lattice of shifts."""
    Y32, scales = synth.job(1507087510 + 9, 256, 256, 5)
    scales = [(1, 1), (16, 16), (128, 128), (256, 256)]
    M, N = Y32.shape
    lam = [O.lambda_default(M, N, m, n) for m, n in scales]
    iters, seed = 12, 8
    with B.Context(0) as ctx:
        X, st = _run(B, ctx, Y32, scales, lam, iters, seed, spin_grid=2)
    ref = O.admm(Y32.astype(np.float64), scales, lam, 1.0, iters,
                 shifts=O.shift_table(seed, iters, M, N), spin_grid=2)
    err = O.relerr(X, ref["X"], Y32)
    assert np.all(err <= TOL), err


def test_full_spin_set_is_translation_equivariant_on_gpu(B):
    """With every shift modulo the block averaged and no random shift, the
    decomposition of a translated input is the translated decomposition."""
    Y, comps, scales = synth.tiny_64()
    Y32 = Y[:32, :32].astype(np.float32)
    scales = [(1, 1), (4, 4), (8, 8), (32, 32)]
    lam = [O.lambda_default(32, 32, m, n) for m, n in scales]
    t = (5, 11)
    with B.Context(0) as ctx:
        X1, _ = _run(B, ctx, Y32, scales, lam, 20, 1, spin_grid=8, cycle_spin=0)
        X2, _ = _run(B, ctx, np.ascontiguousarray(O.shift(Y32, t)), scales, lam, 20, 1,
                     spin_grid=8, cycle_spin=0)
    for i in range(len(scales)):
        want = O.shift(X1[i].astype(np.float64), t)
        err = np.linalg.norm(X2[i] - want) / max(np.linalg.norm(want), 1e-6 * np.linalg.norm(Y32))
        assert err <= TOL, (i, err)


def test_spin_grid_must_divide_the_blocks(B):
    Y32 = np.zeros((48, 48), np.float32)
    with B.Context(0) as ctx:
        with pytest.raises(B.MsllrError) as e:
            _run(B, ctx, Y32, [(1, 1), (6, 6), (48, 48)], None, 2, 1, spin_grid=4)
        assert e.value.code == B.MSLLR_EINVAL
