"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check uses a closed form,
a brute-force search, a different LAPACK route (symmetric eigensolvers instead
of the SVD), a constructed matrix with known factors, or an optimality
certificate of the convex program (Sec. 5, Thm. opt).  The mutation tests at
the end plant plausible mistakes in the oracle (on the CPU) and check that one
of these pins catches each of them.
"""

import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import msllr_oracle as OM
from paper_1507_08751_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _nuc_eigh(B):
    """Nuclear norm through the eigenvalues of B^T B (not the SVD routine)."""
    w = np.linalg.eigvalsh(B.T @ B)
    return float(np.sqrt(np.maximum(w, 0.0)).sum())


def _sv_eigh(B):
    """Singular values, descending, through eigvalsh of the smaller Gram."""
    G = B.T @ B if B.shape[0] >= B.shape[1] else B @ B.T
    return np.sqrt(np.maximum(np.linalg.eigvalsh(G), 0.0))[::-1]


# ---------------------------------------------------------------- shifts ----

def test_splitmix64_published_sequence():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        want = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    gamma = 0x9E3779B97F4A7C15
    got = [O.splitmix64(((k + 1) * gamma) & ((1 << 64) - 1)) for k in range(3)]
    assert got == want


def test_shift_table_range_and_uniformity():
    M, N = 48, 40
    t = O.shift_table(7, 20000, M, N)
    assert t.shape == (20000, 2)
    assert t[:, 0].min() >= 0 and t[:, 0].max() < M
    assert t[:, 1].min() >= 0 and t[:, 1].max() < N
    # chi-square of the row shifts against uniform over M cells
    cnt = np.bincount(t[:, 0], minlength=M)
    exp = len(t) / M
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    assert chi2 < M + 6 * math.sqrt(2 * M)
    assert not np.array_equal(t, O.shift_table(8, 20000, M, N))


def test_shift_matches_definition_by_loops():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((5, 7))
    s = (3, 5)
    S = O.shift(X, s)
    for r in range(5):
        for c in range(7):
            assert S[r, c] == X[(r + 3) % 5, (c + 5) % 7]
    assert np.array_equal(O.unshift(S, s), X)


# ---------------------------------------------------------------- lambda ----

@pytest.mark.parametrize("m,n", [(1, 1), (4, 4), (16, 16), (8, 32)])
def test_lambda_tracks_gaussian_complexity(m, n):
    """eq:gauss: lambda_i ~ E ||G||*_(i) up to a constant; Monte Carlo of the
    block dual norm of a unit Gaussian matrix must sit within a factor 2."""
    M, N = 64, 64
    rng = np.random.default_rng(1)
    vals = []
    for _ in range(20):
        G = rng.standard_normal((M, N))
        B = G.reshape(M // m, m, N // n, n).transpose(0, 2, 1, 3).reshape(-1, m, n)
        vals.append(max(_sv_eigh(b)[0] for b in B))
    ratio = O.lambda_default(M, N, m, n) / np.mean(vals)
    assert 0.5 < ratio < 2.0


def test_lambda_endpoints_paper_text():
    """Sec. 4: for 1x1 blocks the log term is log(MN); for the full M x N
    block the first two terms are sqrt(M) + sqrt(N)."""
    M, N = 1000, 300
    assert O.lambda_default(M, N, 1, 1) == pytest.approx(2 + math.sqrt(math.log(M * N)))
    full = O.lambda_default(M, N, M, N)
    assert full - (math.sqrt(M) + math.sqrt(N)) == pytest.approx(math.sqrt(math.log(N)))


def test_lambda_area_hand_values():
    """The area form of eq:lambda that the 64x64 workload specifies,
    sqrt(m) + sqrt(n) + sqrt(log(64^2 / (m n))), at values worked by hand:
    1x1: 2 + sqrt(12 ln 2) = 4.8840538;  4x4: 4 + sqrt(8 ln 2) = 6.3548200;
    16x16: 8 + sqrt(4 ln 2) = 9.6651092;  64x64: the log term vanishes, 16.
    The paper's form (log of MN / max(m, n)) differs at 4x4 (4 + sqrt(10 ln 2)
    = 6.6327688); a max() in place of the area would give that value here."""
    want = {(1, 1): 4.8840538, (4, 4): 6.3548200, (16, 16): 9.6651092, (64, 64): 16.0}
    for (m, n), v in want.items():
        assert O.lambda_area(64, 64, m, n) == pytest.approx(v, abs=5e-7), (m, n)
    assert O.lambda_default(64, 64, 4, 4) == pytest.approx(6.6327688, abs=5e-7)
    # non-square blocks: 2x8 of a 64x64 matrix, area 16 like 4x4
    assert O.lambda_area(64, 64, 2, 8) == pytest.approx(1.4142136 + 2.8284271 + 2.3548200, abs=5e-7)


# ------------------------------------------------------------------- SVT ----

@pytest.mark.parametrize("shape", [(6, 6), (9, 4), (3, 11), (16, 16)])
def test_svt_singular_values_closed_form(shape):
    rng = np.random.default_rng(2)
    B = rng.standard_normal(shape) * 3
    sig = _sv_eigh(B)
    tau = float(np.median(sig))
    Z = O.svt(B, tau)
    # compare squared singular values (eigenvalues of Z^T Z): the square root
    # of a rounding-level eigenvalue would be ~1e-8
    got2 = np.sort(np.linalg.eigvalsh(Z.T @ Z if Z.shape[0] >= Z.shape[1] else Z @ Z.T))[::-1]
    np.testing.assert_allclose(got2, np.maximum(sig - tau, 0.0) ** 2, atol=1e-9 * sig[0] ** 2)
    # Z lives in B's top-k left and right singular subspaces (eigh route)
    k = int((sig > tau).sum())
    wl, Ul = np.linalg.eigh(B @ B.T)
    Pk = Ul[:, -k:] @ Ul[:, -k:].T
    wr, Vr = np.linalg.eigh(B.T @ B)
    Qk = Vr[:, -k:] @ Vr[:, -k:].T
    np.testing.assert_allclose(Pk @ Z @ Qk, Z, atol=1e-9)


def _nuc2x2(Z):
    """sigma_1 + sigma_2 of a 2x2 matrix: sqrt(||Z||_F^2 + 2 |det Z|)."""
    return math.sqrt((Z * Z).sum() + 2 * abs(np.linalg.det(Z)))


@pytest.mark.parametrize("n", [2, 3])
def test_svt_is_the_prox_brute_force(n):
    """eq:svt is the prox of tau||.||_*: its objective is never beaten by
    10^4 random perturbations (2x2 uses the closed-form nuclear norm)."""
    rng = np.random.default_rng(3 + n)
    nuc = _nuc2x2 if n == 2 else _nuc_eigh
    for trial in range(5):
        A = rng.standard_normal((n, n)) * 2
        tau = 0.7 + 0.5 * trial
        Z = O.svt(A, tau)
        f0 = 0.5 * ((Z - A) ** 2).sum() + tau * nuc(Z)
        for scale in (1e-1, 1e-3):
            D = rng.standard_normal((2000, n, n)) * scale
            f = [0.5 * ((Z + d - A) ** 2).sum() + tau * nuc(Z + d) for d in D]
            assert min(f) >= f0 - 1e-12


@pytest.mark.parametrize("n", [2, 3])
def test_svt_subgradient_certificate(n):
    """(A - Z)/tau lies in the subdifferential of ||.||_* at Z (Sec. 5.1):
    it equals U1 V1^T + W with ||W|| <= 1 and W orthogonal to Z's row and
    column spaces."""
    rng = np.random.default_rng(11 + n)
    for _ in range(10):
        A = rng.standard_normal((n, n)) * 2
        tau = 1.0
        Z = O.svt(A, tau)
        D = (A - Z) / tau
        wr, Vr = np.linalg.eigh(Z.T @ Z)
        k = int((_sv_eigh(A) > tau).sum())
        if k == 0:
            assert _sv_eigh(D)[0] <= 1 + 1e-9
            continue
        V1 = Vr[:, -k:]
        # align signs: U1 = Z V1 / sigma
        U1 = Z @ V1 / np.sqrt(wr[-k:])
        W = D - U1 @ V1.T
        assert _sv_eigh(W)[0] <= 1 + 1e-9
        np.testing.assert_allclose(U1.T @ W, 0, atol=1e-9)
        np.testing.assert_allclose(W @ V1, 0, atol=1e-9)


def test_block_svt_1x1_is_scalar_prox_brute_force():
    """eq:bsvt with 1x1 blocks is the element-wise soft threshold: compare
    both oracle routes (written-out 1x1 SVD and batched LAPACK SVD) with a
    dense grid minimisation of 0.5 (z - a)^2 + tau |z|."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((6, 5)) * 3
    tau = 1.3
    grid = np.linspace(-12, 12, 240001)
    want = np.array([grid[np.argmin(0.5 * (grid - a) ** 2 + tau * np.abs(grid))] for a in A.ravel()])
    for cf in (True, False):
        got = O.block_svt(A, 1, 1, tau, closed_form_1x1=cf).ravel()
        np.testing.assert_allclose(got, want, atol=2e-4)


def test_block_svt_1xN_is_group_soft_threshold():
    """Sec. 7: 1 x n blocks give the joint (group) soft threshold; check
    against a numerical minimisation of 0.5||z - a||^2 + tau ||z||_2."""
    from scipy.optimize import minimize
    rng = np.random.default_rng(5)
    A = rng.standard_normal((4, 6)) * 2
    tau = 2.0
    Z = O.block_svt(A, 1, 6, tau)
    for r in range(4):
        a = A[r]
        res = minimize(lambda z: 0.5 * ((z - a) ** 2).sum() + tau * np.sqrt((z * z).sum() + 1e-30),
                       np.zeros(6) + 0.01, method="Nelder-Mead",
                       options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 40000, "maxfev": 40000})
        np.testing.assert_allclose(Z[r], res.x, atol=1e-4)


def test_block_svt_on_constructed_block_factors():
    """A = sum_b R_b^T(U_b diag(s_b) V_b^T) with orthonormal U_b, V_b from QR:
    BlockSVT must return sum_b R_b^T(U_b diag((s_b - tau)_+) V_b^T) -- a
    closed form that needs no SVD.  Non-square blocks catch transposed
    reshapes and swapped block indices."""
    rng = np.random.default_rng(6)
    M, N, m, n = 12, 20, 4, 5
    tau = 1.5
    A = np.zeros((M, N))
    want = np.zeros((M, N))
    Sv = []
    for p in range(M // m):
        for q in range(N // n):
            U, _ = np.linalg.qr(rng.standard_normal((m, 3)))
            V, _ = np.linalg.qr(rng.standard_normal((n, 3)))
            s = rng.uniform(0, 4, 3)
            Sv.append(s)
            A[p * m:(p + 1) * m, q * n:(q + 1) * n] = (U * s) @ V.T
            want[p * m:(p + 1) * m, q * n:(q + 1) * n] = (U * np.maximum(s - tau, 0)) @ V.T
    np.testing.assert_allclose(O.block_svt(A, m, n, tau), want, atol=1e-12)
    # block norms on the same construction (Sec. 3): known singular values
    assert O.block_nuclear_norm(A, m, n) == pytest.approx(sum(s.sum() for s in Sv), rel=1e-10)
    assert O.block_dual_norm(A, m, n) == pytest.approx(max(s.max() for s in Sv), rel=1e-10)


def test_full_scale_is_plain_svt_and_permutation_equivariant():
    """The M x N scale reduces to plain SVT (eigh route here), and SVT
    commutes with row/column permutations -- so cycle-spinning the full scale
    changes nothing (SVT(P A Q) = P SVT(A) Q)."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((10, 6)) * 2
    tau = 2.0
    w, V = np.linalg.eigh(A.T @ A)
    sig = np.sqrt(np.maximum(w, 0))
    f = np.where(sig > tau, 1 - tau / np.where(sig > 0, sig, 1), 0)
    want = A @ (V * f) @ V.T
    np.testing.assert_allclose(O.block_svt(A, 10, 6, tau), want, atol=1e-10)
    s = (3, 4)
    np.testing.assert_allclose(O.unshift(O.block_svt(O.shift(A, s), 10, 6, tau), s), want, atol=1e-10)


def test_block_svt_grid_shift_equivariance():
    """Shifting by whole blocks only permutes blocks."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((16, 24))
    s = (8, 12)
    lhs = O.block_svt(O.shift(A, s), 4, 6, 1.0)
    rhs = O.shift(O.block_svt(A, 4, 6, 1.0), s)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


# ------------------------------------------------------------------ ADMM ----

def _hanning_solution(iters=1000, c=1.0):
    Y, comps, scales = synth.hanning_blobs()
    M, N = Y.shape
    lam = [O.lambda_default(M, N, m, n) for m, n in scales]
    out = O.admm(c * Y, scales, lam, 1.0, iters)
    return Y * c, comps * c, scales, lam, out


@pytest.fixture(scope="module")
def hanning():
    return _hanning_solution()


def test_admm_kkt_certificate(hanning):
    """Thm. opt (Sec. 5 appendix): at the optimum, rho U_i tends to one common
    dual Q with ||Q||*_(i) <= lambda_i, <Q, X_i> = lambda_i ||X_i||_(i), and
    the duality gap sum_i lambda_i ||X_i||_(i) - <Q, Y> vanishes."""
    Y, comps, scales, lam, out = hanning
    X, U = out["X"], out["U"]
    Q = U.mean(axis=0)
    assert np.abs(U - Q).max() < 1e-10
    prim = 0.0
    for i, (m, n) in enumerate(scales):
        assert O.block_dual_norm(Q, m, n) <= lam[i] * (1 + 1e-8)
        nuc = O.block_nuclear_norm(X[i], m, n)
        assert np.sum(Q * X[i]) == pytest.approx(lam[i] * nuc, rel=1e-8, abs=1e-8)
        prim += lam[i] * nuc
    assert (prim - np.sum(Q * Y)) / prim < 1e-10


def test_admm_exact_recovery(hanning):
    """Fig. 1 / Thm. main: incoherent multi-scale Hanning blobs are separated
    exactly into their scales."""
    Y, comps, scales, lam, out = hanning
    for i in range(len(scales)):
        assert np.linalg.norm(out["X"][i] - comps[i]) <= 1e-8 * np.linalg.norm(comps[i])


def test_admm_homogeneity(hanning):
    """eq:cvx is positively homogeneous: the optimum for 3Y is 3x that for Y."""
    Y3, comps3, scales, lam, out3 = _hanning_solution(c=3.0)
    _, _, _, _, out1 = hanning
    np.testing.assert_allclose(out3["X"], 3 * out1["X"], atol=1e-7)


def test_admm_low_rank_plus_sparse_special_case():
    """Sec. 2: scales {1x1, MxN} are low rank + sparse; the KKT gap closes."""
    rng = np.random.default_rng(9)
    M, N = 40, 30
    Lr = rng.standard_normal((M, 2)) @ rng.standard_normal((N, 2)).T
    S = (rng.random((M, N)) < 0.05) * rng.standard_normal((M, N)) * 5
    Y = Lr + S
    scales = [(1, 1), (M, N)]
    lam = [O.lambda_default(M, N, m, n) for m, n in scales]
    out = O.admm(Y, scales, lam, 1.0, 3000)
    Q = out["U"].mean(axis=0)
    assert np.abs(out["U"] - Q).max() < 1e-8
    prim = sum(lam[i] * O.block_nuclear_norm(out["X"][i], *scales[i]) for i in range(2))
    assert (prim - np.sum(Q * Y)) / prim < 1e-8
    assert np.abs(Q).max() <= lam[0] * (1 + 1e-8)
    np.testing.assert_allclose(out["X"][0], S, atol=1e-6)
    np.testing.assert_allclose(out["X"][1], Lr, atol=1e-6)


def test_admm_step_invariants_with_cycle_spinning():
    """eq:admm with random shifts: after every X-update sum_i X_i = Y, and the
    dual update satisfies U' = (X + U) - Z'.  Masked (Sec. 10.4): the sum
    holds on observed entries and X_i = Z_i - U_i elsewhere."""
    Y, comps, scales = synth.tiny_64()
    M, N = Y.shape
    lam = [O.lambda_area(M, N, m, n) for m, n in scales]
    sh = O.shift_table(5, 30, M, N)
    L = len(scales)
    rng = np.random.default_rng(10)
    mask = rng.random((M, N)) < 0.6
    for msk in (None, mask):
        Z = np.zeros((L, M, N))
        U = np.zeros((L, M, N))
        Ym = Y if msk is None else np.where(msk, Y, 0)
        for k in range(30):
            X, Zn, Un = O.admm_step(Ym, Z, U, scales, lam, sh[k], msk)
            if msk is None:
                np.testing.assert_allclose(X.sum(0), Y, atol=1e-10)
            else:
                np.testing.assert_allclose(X.sum(0)[msk], Y[msk], atol=1e-10)
                np.testing.assert_allclose(X[:, ~msk], (Z - U)[:, ~msk], atol=1e-12)
            np.testing.assert_allclose(Un, X + U - Zn, atol=1e-10)
            Z, U = Zn, Un


def test_admm_full_mask_equals_unmasked():
    Y, comps, scales = synth.tiny_64()
    M, N = Y.shape
    lam = [O.lambda_area(M, N, m, n) for m, n in scales]
    sh = O.shift_table(3, 20, M, N)
    a = O.admm(Y, scales, lam, 1.0, 20, shifts=sh)
    b = O.admm(Y, scales, lam, 1.0, 20, shifts=sh, mask=np.ones((M, N), bool))
    np.testing.assert_array_equal(a["X"], b["X"])


def test_objective_and_primal_residual_trend_down(hanning):
    """ADMM is not monotone per iteration, and from Z = 0 the objective rises
    towards the optimum; what must trend down is the distance of the
    objective sum_i lambda_i ||Z_i||_(i) to the certified optimum and the
    primal residual ||X - Z||_F: the max over the last 10% of iterations sits
    well below the value at 10%."""
    Y, comps, scales, lam, ref = hanning
    opt = sum(lam[i] * O.block_nuclear_norm(ref["X"][i], *scales[i]) for i in range(len(scales)))
    out = O.admm(Y, scales, lam, 1.0, 400, history=True)
    gap = np.abs(out["objective"] - opt)
    assert gap[-40:].max() < 1e-2 * gap[40]
    pres = out["primal_residual"]
    assert pres[-40:].max() < 1e-2 * pres[40]


def test_relerr_floor():
    """relerr uses max(||Xref_i||, 1e-6 ||Y||) so an all-zero component does
    not divide by zero."""
    Y = np.ones((4, 4))                      # ||Y||_F = 4
    Xref = np.zeros((2, 4, 4))
    Xref[1] = 2.0                            # ||Xref_1||_F = 8
    X = Xref + 1e-9                          # ||dX_i||_F = 4e-9
    r = O.relerr(X, Xref, Y)
    assert r[0] == pytest.approx(4e-9 / 4e-6)
    assert r[1] == pytest.approx(4e-9 / 8)


# ------------------------------------------------------------- mutations ----

def _mut_sign_u_update(Y, Z, U, scales, taus, s, mask=None):
    X = OM.x_update(Y, Z, U, mask)
    s = np.asarray(s).reshape(-1, 2)
    Zn = np.empty_like(Z)
    for i, (m, n) in enumerate(scales):
        Zn[i] = OM.unshift(OM.block_svt(OM.shift(X[i] + U[i], s[0]), m, n, taus[i]), s[0])
    return X, Zn, U + (Zn - X)          # planted: wrong sign


def _mut_drop_u_in_prox(Y, Z, U, scales, taus, s, mask=None):
    X = OM.x_update(Y, Z, U, mask)
    s = np.asarray(s).reshape(-1, 2)
    Zn = np.empty_like(Z)
    for i, (m, n) in enumerate(scales):
        Zn[i] = OM.unshift(OM.block_svt(OM.shift(X[i], s[0]), m, n, taus[i]), s[0])  # planted: dropped U
    return X, Zn, U - (Zn - X)


def test_planted_admm_mistakes_break_the_certificate(monkeypatch):
    for bad in (_mut_sign_u_update, _mut_drop_u_in_prox):
        monkeypatch.setattr(OM, "admm_step", bad)
        Y, comps, scales = synth.hanning_blobs()
        M, N = Y.shape
        lam = [O.lambda_default(M, N, m, n) for m, n in scales]
        with np.errstate(all="ignore"):
            out = OM.admm(Y, scales, lam, 1.0, 300)
        err = max(np.linalg.norm(out["X"][i] - comps[i]) / np.linalg.norm(comps[i]) for i in range(4))
        assert not (err < 1e-3)


def test_planted_transposed_unblock_is_caught(monkeypatch):
    def bad_unblocks(B, M, N):
        nb, m, n = B.shape
        return B.reshape(N // n, M // m, m, n).transpose(1, 2, 0, 3).reshape(M, N)
    monkeypatch.setattr(OM, "_unblocks", bad_unblocks)
    with pytest.raises(AssertionError):
        test_block_svt_on_constructed_block_factors()


def test_planted_shift_direction_is_caught(monkeypatch):
    def bad_shift(X, s):
        M, N = X.shape
        return X[np.ix_((np.arange(M) - s[0]) % M, (np.arange(N) - s[1]) % N)]
    monkeypatch.setattr(OM, "shift", bad_shift)
    monkeypatch.setattr(O, "shift", bad_shift)
    with pytest.raises(AssertionError):
        test_shift_matches_definition_by_loops()


# --------------------------------------------------------------------------
# Noise scale (Sec. 2.1): the whole matrix as one MN x 1 block
# --------------------------------------------------------------------------

def test_noise_scale_is_the_vector_shrink():
    """The SVD of an MN x 1 block has the single singular value ||A||_F with
    u = vec(A)/||A||_F and v = 1, so its SVT is A max(1 - tau/||A||_F, 0)."""
    rng = np.random.default_rng(31)
    A = rng.standard_normal((12, 5))
    nrm = np.sqrt((A * A).sum())
    for tau in (0.3 * nrm, 0.99 * nrm, 1.5 * nrm):
        Z = O.block_svt(A, 0, 0, tau)
        np.testing.assert_allclose(Z, A * max(1.0 - tau / nrm, 0.0), rtol=1e-12, atol=1e-14)
    assert O.block_nuclear_norm(A, 0, 0) == pytest.approx(nrm, rel=1e-13)
    assert O.block_dual_norm(A, 0, 0) == pytest.approx(nrm, rel=1e-13)


def test_noise_scale_prox_is_optimal_brute_force():
    """prox of tau ||.||_F: no perturbation of the returned Z lowers
    0.5 ||Z - A||^2 + tau ||Z||_F (random directions, small and large)."""
    rng = np.random.default_rng(32)
    A = rng.standard_normal((3, 2))
    tau = 0.7
    Z = O.block_svt(A, 0, 0, tau)
    f = lambda X: 0.5 * ((X - A) ** 2).sum() + tau * np.sqrt((X * X).sum())
    f0 = f(Z)
    for _ in range(2000):
        d = rng.standard_normal(A.shape) * 10.0 ** rng.uniform(-4, 0)
        assert f(Z + d) >= f0 - 1e-12


def test_noise_scale_lambda_default():
    assert O.lambda_default(64, 32, 0, 0) == pytest.approx(np.sqrt(64 * 32) + 1.0, rel=1e-15)


def test_admm_with_noise_scale_keeps_the_invariants():
    """sum_i X_i = Y and U' = X + U - Z' with a noise scale among the scales."""
    rng = np.random.default_rng(33)
    M, N = 32, 16
    Y = np.outer(rng.standard_normal(M), rng.standard_normal(N)) + 0.1 * rng.standard_normal((M, N))
    scales = [(1, 1), (8, 8), (M, N), (0, 0)]
    lam = [O.lambda_default(M, N, m, n) for m, n in scales]
    out = O.admm(Y, scales, lam, 1.0, 40, shifts=O.shift_table(7, 40, M, N))
    np.testing.assert_allclose(out["X"].sum(0), Y, atol=1e-12)
    L = len(scales)
    Z = np.zeros((L, M, N)); U = np.zeros((L, M, N))
    s = O.shift_table(7, 1, M, N)[0]
    X, Zn, Un = O.admm_step(Y, Z, U, scales, lam, s)
    np.testing.assert_allclose(Un, X + U - Zn, atol=1e-13)
    # the noise scale's first prox: Y/L shrunk by its Frobenius norm
    A = Y / L
    np.testing.assert_allclose(Zn[3], A * max(1 - lam[3] / np.linalg.norm(A), 0), atol=1e-13)


# --------------------------------------------------------------------------
# Averaged cycle spinning (Sec. 9): the Z-update averaged over a set of shifts.
# --------------------------------------------------------------------------

def _spun_by_windows(A, m, n, tau, shifts):
    """The same average written without shifting arrays: for every shift s
    and every block of the shifted grid, take the SVT of the block read
    through explicit wrapped row/column indices and add 1/|S| of it back at
    those indices."""
    M, N = A.shape
    out = np.zeros_like(A)
    for (sr, sc) in shifts:
        for p in range(M // m):
            for q in range(N // n):
                rows = [(p * m + i + sr) % M for i in range(m)]
                cols = [(q * n + j + sc) % N for j in range(n)]
                B = A[np.ix_(rows, cols)]
                U, s, Vh = np.linalg.svd(B)
                Zb = (U[:, :len(s)] * np.maximum(s - tau, 0)) @ Vh[:len(s)]
                for i, r in enumerate(rows):
                    for j, c in enumerate(cols):
                        out[r, c] += Zb[i, j] / len(shifts)
    return out


def test_spin_set_sizes_and_lattice():
    assert O.spin_set(4, 4, 0) == [(0, 0)]
    assert O.spin_set(4, 4, 1) == [(0, 0)]
    assert sorted(O.spin_set(4, 4, 2)) == [(0, 0), (0, 2), (2, 0), (2, 2)]
    assert len(O.spin_set(4, 8, 64)) == 32          # every shift modulo the block
    assert O.spin_set(1, 8, 4) == [(0, 0), (0, 2), (0, 4), (0, 6)]
    with pytest.raises(ValueError):
        O.spin_set(6, 6, 4)


def test_spun_block_svt_brute_force_windows():
    rng = np.random.default_rng(21)
    A = rng.standard_normal((8, 12))
    for (m, n, g) in ((4, 4, 4), (4, 6, 2), (2, 3, 8)):
        S = O.spin_set(m, n, g)
        S = [(s[0] + 3, s[1] + 5) for s in S]        # offset by a random shift
        tau = 0.6
        np.testing.assert_allclose(O.block_svt_spun(A, m, n, tau, S),
                                   _spun_by_windows(A, m, n, tau, S), atol=1e-12)


def test_spun_block_svt_is_translation_equivariant_over_all_shifts():
    """Averaging over every shift modulo the block makes the operator commute
    with every translation (the purpose of cycle spinning, Sec. 9)."""
    rng = np.random.default_rng(22)
    A = rng.standard_normal((12, 8))
    m, n = 4, 4
    S = O.spin_set(m, n, 4)
    f = lambda X: O.block_svt_spun(X, m, n, 0.8, S)
    for t in ((1, 0), (0, 3), (5, 7)):
        np.testing.assert_allclose(f(O.shift(A, t)), O.shift(f(A), t), atol=1e-12)
    # a single shift is not equivariant: the check has teeth
    g = lambda X: O.block_svt(X, m, n, 0.8)
    assert np.abs(g(O.shift(A, (1, 0))) - O.shift(g(A), (1, 0))).max() > 1e-3


def test_spun_block_svt_special_cases():
    rng = np.random.default_rng(23)
    A = rng.standard_normal((8, 8))
    # tau = 0: every term is the identity, so the average is A (weights 1/|S|)
    np.testing.assert_allclose(O.block_svt_spun(A, 4, 4, 0.0, O.spin_set(4, 4, 4)), A,
                               atol=1e-12)
    # one shift: the random-shift update of Sec. 9
    s = (3, 6)
    np.testing.assert_allclose(O.block_svt_spun(A, 4, 4, 0.5, [s]),
                               O.unshift(O.block_svt(O.shift(A, s), 4, 4, 0.5), s), atol=1e-12)
    # full-matrix and 1x1 blocks commute with shifts: averaging changes nothing
    np.testing.assert_allclose(O.block_svt_spun(A, 8, 8, 0.5, [(1, 2), (5, 3)]),
                               O.svt(A, 0.5), atol=1e-12)
    np.testing.assert_allclose(O.block_svt_spun(A, 1, 1, 0.5, [(1, 2), (5, 3)]),
                               O.soft_threshold(A, 0.5), atol=1e-12)


def test_spun_admm_is_translation_equivariant_and_keeps_invariants():
    """With the full shift set and no random shift the averaged ADMM commutes
    with translations of Y; sum_i X_i = Y holds at every iterate."""
    Y, comps, scales = synth.tiny_64()
    Y = Y[:32, :32].astype(np.float64)
    scales = [(1, 1), (4, 4), (8, 8), (32, 32)]
    lam = [O.lambda_default(32, 32, m, n) for m, n in scales]
    r1 = O.admm(Y, scales, lam, 1.0, 6, spin_grid=8)
    t = (5, 11)
    r2 = O.admm(O.shift(Y, t), scales, lam, 1.0, 6, spin_grid=8)
    for i in range(len(scales)):
        np.testing.assert_allclose(r2["X"][i], O.shift(r1["X"][i], t), atol=1e-9)
    np.testing.assert_allclose(r1["X"].sum(0), Y, atol=1e-10)


# --------------------------------------------------------------------------
# Spatio-temporal blocks (Sec. 10.2): bh x bw x bt video blocks reshaped to
# (bh bw) x bt matrices.
# --------------------------------------------------------------------------

def test_blocks3d_round_trip_and_shape():
    rng = np.random.default_rng(31)
    H, W, T = 8, 12, 16
    A = rng.standard_normal((H * W, T))
    for (bh, bw, bt, s3) in ((4, 4, 4, (0, 0, 0)), (2, 6, 8, (3, 5, 11)), (8, 12, 16, (1, 2, 3))):
        B = O.blocks3d(A, H, W, bh, bw, bt, s3)
        assert B.shape == ((H // bh) * (W // bw) * (T // bt), bh * bw, bt)
        np.testing.assert_array_equal(O.unblocks3d(B, H, W, T, bh, bw, bt, s3), A)


def test_block3d_by_explicit_pixel_indices():
    """Brute force: block (py, px, pt) of the shifted cube holds, at row
    i * bw + j and column k, the entry of pixel ((py bh + i + sy) mod H,
    (px bw + j + sx) mod W) in frame (pt bt + k + st) mod T."""
    rng = np.random.default_rng(32)
    H, W, T, bh, bw, bt, s3 = 6, 8, 6, 3, 4, 2, (4, 7, 5)
    A = rng.standard_normal((H * W, T))
    B = O.blocks3d(A, H, W, bh, bw, bt, s3)
    b = 0
    for py in range(H // bh):
        for px in range(W // bw):
            for pt in range(T // bt):
                for i in range(bh):
                    for j in range(bw):
                        for k in range(bt):
                            y = (py * bh + i + s3[0]) % H
                            x = (px * bw + j + s3[1]) % W
                            t = (pt * bt + k + s3[2]) % T
                            assert B[b, i * bw + j, k] == A[y * W + x, t]
                b += 1


def test_block_svt_3d_reduces_to_2d_when_blocks_span_frame_rows():
    """A bh x W x bt block covers bh whole frame rows: its rows are the
    contiguous matrix rows y0 W .. (y0 + bh) W - 1, so the spatio-temporal
    BlockSVT equals the 2-D one with (bh W) x bt blocks."""
    rng = np.random.default_rng(33)
    H, W, T = 8, 6, 12
    A = rng.standard_normal((H * W, T))
    for (bh, bt, tau) in ((2, 4, 0.7), (4, 6, 1.5), (8, 12, 3.0)):
        np.testing.assert_allclose(O.block_svt_3d(A, H, W, bh, W, bt, tau),
                                   O.block_svt(A, bh * W, bt, tau), atol=1e-12)


def test_block_svt_3d_singular_values_closed_form():
    rng = np.random.default_rng(34)
    H, W, T = 8, 8, 8
    A = rng.standard_normal((H * W, T))
    tau = 1.1
    Z = O.block_svt_3d(A, H, W, 4, 4, 4, tau, (1, 3, 2))
    sa = np.linalg.svd(O.blocks3d(A, H, W, 4, 4, 4, (1, 3, 2)), compute_uv=False)
    sz = np.linalg.svd(O.blocks3d(Z, H, W, 4, 4, 4, (1, 3, 2)), compute_uv=False)
    np.testing.assert_allclose(sz, np.maximum(sa - tau, 0.0), atol=1e-12)


def test_spatio_temporal_admm_reduces_to_2d_and_keeps_invariants():
    """ADMM with a bh x W x bt scale and shifts off is the 2-D ADMM with
    (bh W) x bt blocks; with shifts on (the row shift read as a pixel shift)
    sum_i X_i = Y holds."""
    rng = np.random.default_rng(35)
    H, W, T = 8, 4, 16
    Y = rng.standard_normal((H * W, T))
    M, N = Y.shape
    s3d = [(1, 1), (2, W, 4), (M, N)]
    s2d = [(1, 1), (2 * W, 4), (M, N)]
    lam = [O.lambda_default(M, N, 1, 1), O.lambda_default(M, N, 2 * W, 4),
           O.lambda_default(M, N, M, N)]
    r3 = O.admm(Y, s3d, lam, 1.0, 15, frame=(H, W))
    r2 = O.admm(Y, s2d, lam, 1.0, 15)
    np.testing.assert_allclose(r3["X"], r2["X"], atol=1e-12)
    sh = O.shift_table(3, 10, M, N)
    r = O.admm(Y, [(1, 1), (2, 2, 4), (4, 4, 8), (M, N)],
               [1.0, 2.0, 3.0, 6.0], 1.0, 10, shifts=sh, frame=(H, W), history=True)
    np.testing.assert_allclose(r["X"].sum(0), Y, atol=1e-10)
    assert np.all(np.isfinite(r["objective"]))
    assert O.shift3d((13, 5), W, T) == (3, 1, 5)
