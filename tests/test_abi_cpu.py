"""CPU-side checks of the C ABI: the library builds, loads, exports every
symbol include/msllr.h declares, and its host-only calls agree with the
oracle.  No GPU work is launched here."""

import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1507_08751_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(B.LIB_PATH):
        from paper_1507_08751_gb300 import build
        build.build()
    return B.lib()


def _header_symbols():
    text = open(os.path.join(ROOT, "include", "msllr.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(msllr_\w+)\s*\(", text, re.M)))


def test_header_declares_the_binding_exports():
    assert _header_symbols() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol(built):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (msllr_\w+)$", out, re.M))
    for sym in _header_symbols():
        assert sym in exported, sym


def test_shift_table_bit_exact_against_oracle(built):
    for seed, iters, M, N in [(0, 10, 64, 64), (1507087510, 300, 16384, 256), (2**63 + 5, 50, 7, 3)]:
        np.testing.assert_array_equal(B.msllr_shift_table(seed, iters, M, N),
                                      O.shift_table(seed, iters, M, N))


def test_lambda_default_matches_eq_lambda(built):
    for M, N, m, n in [(64, 64, 1, 1), (16384, 256, 16, 16), (16384, 256, 16384, 256), (30, 50, 3, 5),
                       (16384, 256, 0, 0)]:
        assert B.msllr_lambda_default(M, N, m, n) == pytest.approx(O.lambda_default(M, N, m, n),
                                                                    rel=1e-14)
    with pytest.raises(B.MsllrError) as e:
        B.msllr_lambda_default(10, 10, 11, 1)
    assert e.value.code == B.MSLLR_EINVAL


def test_params_default(built):
    p = B.msllr_params_default()
    assert (p.skip_bound, p.cycle_spin, p.use_graph, p.iter_offset) == (1, 1, 1, 0)
    assert not p.Z_init and not p.U_init and not p.U_out
    assert p.profile == 0 and p.spin_grid == 0 and p.plain == 0
    assert p.stop_tol == 0.0 and p.stop_every == 0


def test_params_struct_matches_header_field_order():
    """The ctypes mirror lists the header's msllr_params fields in order."""
    src = open(os.path.join(ROOT, "include", "msllr.h")).read()
    body = src[src.index("typedef struct msllr_params"):src.index("} msllr_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"^\s+(?:const\s+)?\w+\*?\s+\*?(\w+);", body, re.M)
    assert names == [f[0] for f in B.Params._fields_]


def test_create_without_device_fails_loudly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(B.MsllrError) as e:
        B.Context(0)
    assert e.value.code == B.MSLLR_EINVAL


def test_stats_struct_matches_header_field_order():
    """The ctypes mirror lists the header's msllr_stats fields in order."""
    src = open(os.path.join(ROOT, "include", "msllr.h")).read()
    body = src[src.index("typedef struct msllr_stats"):src.index("} msllr_stats;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"^\s*(?:long long|int|double)\s+(\w+)", body, re.M)
    mirror = [f[0].rstrip("_") for f in B.Stats._fields_]
    assert names == mirror
