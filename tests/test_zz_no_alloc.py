"""msllr_blocksvt_noalloc: the block SVT for callers that cannot allocate
device memory (processes whose device memory is handed out by their own pool
allocator, loops that cannot take cudaMalloc's device-wide
synchronisation).  It must give what msllr_blocksvt gives,
call after call, although every call reuses the same fixed device scratch.

Collected last on purpose, and self-contained: it loads the library and
makes its own reference context, so it passes alone in a fresh process and
after the other tests."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


def _matrix(seed, M, N, m, n):
    rng = np.random.default_rng(seed)
    A = 0.3 * rng.standard_normal((M, N))
    for p in range(M // m):
        for q in range(N // n):
            r = int(rng.integers(0, 3))
            if r:
                u = rng.standard_normal((m, r))
                v = rng.standard_normal((n, r))
                A[p * m:(p + 1) * m, q * n:(q + 1) * n] += 3.0 * (u @ v.T) / np.sqrt(max(m, n))
    return torch.from_numpy(A.astype(np.float32)).cuda()


@pytest.mark.parametrize("M,N,m,n,shift", [
    (512, 256, 256, 256, (300, 17)),   # wide blocks: Gram / eigen / rebuild scratch
    (2048, 256, 2048, 256, (0, 0)),    # full-matrix scale: partial Gram sums in scratch
    (256, 256, 16, 16, (5, 9)),        # narrow blocks
])
def test_noalloc_matches_blocksvt_two_calls_in_a_row(M, N, m, n, shift):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_08751_gb300 import binding as B
    B.lib()
    nb = (M // m) * (N // n)
    with B.Context(0) as ctx:
        for call in range(2):
            A = _matrix(100 * call + M + m, M, N, m, n)
            Aq = A.double().cpu().numpy()
            sv = np.linalg.svd(Aq.reshape(M // m, m, N // n, n).transpose(0, 2, 1, 3)
                               .reshape(-1, m, n), compute_uv=False)
            tau = float(np.quantile(sv[:, 0], 0.5))
            Zref = torch.empty_like(A)
            rref = torch.empty(nb, dtype=torch.int32, device="cuda")
            ctx.msllr_blocksvt(A, Zref, m, n, tau, shift, rank_out=rref)
            Z = torch.full_like(A, float("nan"))
            r = torch.full((nb,), -1, dtype=torch.int32, device="cuda")
            B.msllr_blocksvt_noalloc(A, Z, m, n, tau, shift, rank_out=r)
            torch.cuda.synchronize()
            err = (torch.linalg.norm((Z - Zref).double()) /
                   max(torch.linalg.norm(Zref.double()).item(), 1e-6 * torch.linalg.norm(A.double()).item()))
            assert err.item() <= TOL, f"call {call}: relative error {err.item():.3e}"
            assert torch.equal(r, rref), f"call {call}: block ranks differ"


def test_noalloc_rejects_workspace_beyond_the_fixed_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_08751_gb300 import binding as B
    B.lib()
    A = torch.zeros((16384, 1024), dtype=torch.float32, device="cuda")
    Z = torch.empty_like(A)
    with pytest.raises(B.MsllrError) as e:
        B.msllr_blocksvt_noalloc(A, Z, 256, 256, 1.0)
    assert e.value.code == B.MSLLR_EINVAL
    assert "scratch" in str(e.value)


def test_noalloc_takes_no_device_memory():
    """After a first call (which sets the device up and loads the kernels it
    uses), further calls leave the device's free memory exactly as it was:
    the call claims nothing beyond the library's fixed scratch."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_08751_gb300 import binding as B
    B.lib()
    M, N, m, n = 1024, 256, 256, 256
    A = _matrix(7, M, N, m, n)
    Z = torch.empty_like(A)
    r = torch.empty(((M // m) * (N // n),), dtype=torch.int32, device="cuda")
    B.msllr_blocksvt_noalloc(A, Z, m, n, 5.0, (3, 4), rank_out=r)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(3):
        B.msllr_blocksvt_noalloc(A, Z, m, n, 5.0 + call, (3 + call, 4), rank_out=r)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
