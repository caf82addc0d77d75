"""Serving queue (msllr_submit / msllr_poll / msllr_wait): queued jobs give
what a direct msllr_decompose_host call gives for the same job, the calls
report their states, and the context refuses direct calls while jobs are in
flight.  Through the C ABI (ctypes)."""

import numpy as np
import pytest

from paper_1507_08751_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1507_08751_gb300 import binding as B
    B.lib()
    return B


def _jobs():
    """Three jobs of different shapes: the 64 x 64 four-scale example, a
    1024 x 256 video-shaped matrix with its full-matrix scale, and a masked
    ratings-like job (Sec. 10.4)."""
    Y0, _, s0 = synth.tiny_64()
    Y1, _, s1 = synth.video(M=1024, N=256)
    Y2, m2 = synth.ratings(5, 128, 96, density=0.3)
    return [
        dict(Y=Y0.astype(np.float32), scales=s0, iters=60, seed=3, mask=None),
        dict(Y=Y1.astype(np.float32), scales=s1, iters=30, seed=4, mask=None),
        dict(Y=Y2, scales=[(1, 1), (4, 4), (16, 16), (128, 96)], iters=50, seed=5, mask=m2),
    ]


def test_submitted_jobs_match_direct_calls(B):
    jobs = _jobs()
    with B.Context(0) as ctx:
        outs, ids = [], []
        for j in jobs:
            M, N = j["Y"].shape
            X = np.full((len(j["scales"]), M, N), np.nan, np.float32)
            outs.append(X)
            ids.append(ctx.msllr_submit(j["Y"], j["scales"], X, iters=j["iters"], seed=j["seed"],
                                        mask=j["mask"]))
        assert len(set(ids)) == 3
        stats = [ctx.msllr_wait(i) for i in ids]
        for j, X, st in zip(jobs, outs, stats):
            M, N = j["Y"].shape
            ref = np.empty_like(X)
            ctx.msllr_decompose_host(j["Y"], j["scales"], ref, iters=j["iters"], seed=j["seed"],
                                     mask=j["mask"])
            np.testing.assert_array_equal(X, ref)
            assert st["iters"] == j["iters"] and st["L"] == len(j["scales"])


def test_poll_wait_states_and_busy_context(B):
    Y, _, scales = synth.video(M=1024, N=256)
    Y = Y.astype(np.float32)
    M, N = Y.shape
    with B.Context(0) as ctx:
        X = np.empty((len(scales), M, N), np.float32)
        jid = ctx.msllr_submit(Y, scales, X, iters=300, seed=1)
        # the job is in flight: direct calls on this context are refused
        other = np.empty_like(X)
        with pytest.raises(B.MsllrError) as e:
            ctx.msllr_decompose_host(Y, scales, other, iters=1, seed=1)
        assert e.value.code == B.MSLLR_EBUSY
        # a zero timeout either finds it finished or times out, never fails otherwise
        try:
            st = ctx.msllr_wait(jid, timeout_ms=0)
            finished = True
        except B.MsllrError as err:
            assert err.code == B.MSLLR_ETIMEOUT
            finished = False
        if not finished:
            st = ctx.msllr_wait(jid)
        assert st["iters"] == 300
        # collected: the id is gone
        with pytest.raises(B.MsllrError) as e:
            ctx.msllr_poll(jid)
        assert e.value.code == B.MSLLR_EINVAL
        # the context is free again
        ctx.msllr_decompose_host(Y, scales, other, iters=300, seed=1)
        np.testing.assert_array_equal(X, other)
        # poll until done
        X2 = np.empty_like(X)
        jid2 = ctx.msllr_submit(Y, scales, X2, iters=5, seed=2)
        for _ in range(100000):
            st = ctx.msllr_poll(jid2)
            if st is not None:
                break
        else:
            st = ctx.msllr_wait(jid2)
        assert st["iters"] == 5


def test_submit_rejects_bad_jobs(B):
    Y, _, scales = synth.tiny_64()
    Y = Y.astype(np.float32)
    with B.Context(0, hbm_budget_bytes=1 << 16) as ctx:
        X = np.empty((len(scales), 64, 64), np.float32)
        with pytest.raises(B.MsllrError) as e:
            ctx.msllr_submit(Y, scales, X, iters=5)
        assert e.value.code == B.MSLLR_ENOMEM
    with B.Context(0) as ctx:
        X = np.empty((1, 64, 64), np.float32)
        with pytest.raises(B.MsllrError) as e:
            ctx.msllr_submit(Y, [(3, 3)], X, iters=5)  # 3 does not divide 64
        assert e.value.code == B.MSLLR_EINVAL
        with pytest.raises(B.MsllrError) as e:
            ctx.msllr_wait(12345)
        assert e.value.code == B.MSLLR_EINVAL


def _need_bytes(B, Y, scales, iters):
    """The device footprint msllr_submit charges for a job (read from its
    ENOMEM message under a one-byte budget)."""
    import re
    M, N = Y.shape
    with B.Context(0, hbm_budget_bytes=1) as ctx:
        with pytest.raises(B.MsllrError) as e:
            ctx.msllr_submit(Y, scales, np.empty((len(scales), M, N), np.float32), iters=iters)
    return int(re.search(r"needs (\d+) bytes", str(e.value)).group(1))


def test_concurrent_jobs_overlap_and_match_solo_runs(B):
    """Continuous batching: four jobs of different shapes (a masked one among
    them) submitted together run at the same time on the device -- at least
    three of them see others running when they start -- and each result is
    bit for bit the result of the same job run alone."""
    Y0, _, s0 = synth.video(M=1024, N=256)
    Y1, s1 = synth.job(11, 512, 512, 5)
    Y2, m2 = synth.ratings(7, 256, 256, density=0.05)
    Y3, _, s3 = synth.tiny_64()
    jobs = [
        dict(Y=Y0.astype(np.float32), scales=s0, iters=200, seed=21, mask=None),
        dict(Y=Y1, scales=s1, iters=200, seed=22, mask=None),
        dict(Y=Y2, scales=synth.dyadic_scales(256, 256, 5), iters=200, seed=23, mask=m2),
        dict(Y=Y3.astype(np.float32), scales=s3, iters=200, seed=24, mask=None),
    ]
    with B.Context(0) as ctx:
        outs, ids = [], []
        for j in jobs:
            M, N = j["Y"].shape
            X = np.full((len(j["scales"]), M, N), np.nan, np.float32)
            outs.append(X)
            ids.append(ctx.msllr_submit(j["Y"], j["scales"], X, iters=j["iters"], seed=j["seed"],
                                        mask=j["mask"]))
        stats = [ctx.msllr_wait(i) for i in ids]
        running = [st["serve_jobs_running"] for st in stats]
        assert max(running) >= 3, running
        for j, X in zip(jobs, outs):
            ref = np.empty_like(X)
            ctx.msllr_decompose_host(j["Y"], j["scales"], ref, iters=j["iters"], seed=j["seed"],
                                     mask=j["mask"])
            np.testing.assert_array_equal(X, ref)


def test_admission_holds_jobs_to_the_hbm_budget(B):
    """With a budget that holds one job but not two, the queued jobs run one
    at a time (each sees only itself running) and still all complete with
    the solo result."""
    Y, _, scales = synth.video(M=1024, N=256)
    Y = Y.astype(np.float32)
    need = _need_bytes(B, Y, scales, 40)
    M, N = Y.shape
    with B.Context(0, hbm_budget_bytes=int(1.5 * need)) as ctx:
        outs = [np.empty((len(scales), M, N), np.float32) for _ in range(3)]
        ids = [ctx.msllr_submit(Y, scales, X, iters=40, seed=9) for X in outs]
        stats = [ctx.msllr_wait(i) for i in ids]
        assert [st["serve_jobs_running"] for st in stats] == [1, 1, 1]
        ref = np.empty_like(outs[0])
        ctx.msllr_decompose_host(Y, scales, ref, iters=40, seed=9)
        for X in outs:
            np.testing.assert_array_equal(X, ref)


def test_two_threads_waiting_on_one_job(B):
    """Two host threads wait for the same job: one collects its status, the
    other is told that the job was already collected (EINVAL), and neither
    crashes."""
    import threading
    Y, _, scales = synth.video(M=1024, N=256)
    Y = Y.astype(np.float32)
    M, N = Y.shape
    with B.Context(0) as ctx:
        X = np.empty((len(scales), M, N), np.float32)
        jid = ctx.msllr_submit(Y, scales, X, iters=100, seed=3)
        codes = []

        def waiter():
            code = B.lib().msllr_wait(ctx._ctx, jid, -1)
            codes.append(code)

        ts = [threading.Thread(target=waiter) for _ in range(2)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert sorted(codes) == [B.MSLLR_OK, B.MSLLR_EINVAL]
