"""Failure handling without a GPU fault: a bounded device wait that nothing completes gives up
with RS_ERR_TIMEOUT and leaves the context usable; device allocations made to fail on the host
(rs_inject_alloc_failures) give RS_ERR_OOM, release what the call had taken, and the next call
succeeds; serving keeps a request whose admission allocation fails queued and admits it later;
the persistent serving kernel exits after its idle limit and is relaunched by the next request."""
import ctypes
import time

import numpy as np
import pytest

from paper_2406_01821_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2406_01821_gb300 import build, rs
    build.build()
    c = rs.Context(0)
    yield c
    rs.lib().rs_inject_alloc_failures(0, 0)
    c.close()


def small_case(seed=0):
    X, y = synth.gaussian_mixture(5003, 24, 4, seed)
    b = synth.random_rulesets(synth.quantile_table(X), 4, 70, (1, 12), (1, 5), seed)
    return X, y, 4, b


def check_counts(ctx, orc, X, y, K, b, ds):
    from paper_2406_01821_gb300 import rs
    c, pc, _ = ctx.eval_hard(ds, rs.HostBatch(b), K, len(X))
    want = orc.eval_hard(X, y, K, b)
    assert np.array_equal(c, want[0]) and np.array_equal(pc, want[1])


def test_bounded_wait_gives_up_and_context_survives(ctx, orc):
    import torch
    from paper_2406_01821_gb300 import rs
    X, y, K, b = small_case(1)
    ds = ctx.dataset(X, y, K)
    try:
        stream = torch.cuda.current_stream()
        t0 = time.perf_counter()
        rc = rs.lib().rs_selftest_bounded_wait(ctx.h, 50_000_000, rs._stream_ptr(stream))
        dt = time.perf_counter() - t0
        assert rc == -4, rs.lib().rs_last_error()
        assert 0.045 <= dt < 2.0
        check_counts(ctx, orc, X, y, K, b, ds)          # the context keeps working
    finally:
        ctx.dataset_destroy(ds)


def test_injected_allocation_failures(ctx, orc):
    """Every allocation of a call fails in turn (the ones before it succeed and must be released)."""
    import torch
    from paper_2406_01821_gb300 import rs
    X, y, K, b = small_case(2)
    ds = ctx.dataset(X, y, K)
    lib = rs.lib()
    try:
        for batch, n_alloc in ((rs.HostBatch(b), 2), (rs.DeviceBatch.from_host(b), 1)):
            for skip in range(n_alloc):
                assert lib.rs_inject_alloc_failures(skip, 1) == 0
                with pytest.raises(rs.RsError) as e:
                    ctx.eval_hard(ds, batch, K, len(X))
                assert e.value.code == -3
            lib.rs_inject_alloc_failures(0, 0)
        torch.cuda.synchronize()
        check_counts(ctx, orc, X, y, K, b, ds)
        db = rs.DeviceBatch.from_host(b)
        dl = torch.ones(b.P, device="cuda")
        for skip in range(9):          # outputs, then the soft scratch arrays one by one
            lib.rs_inject_alloc_failures(skip, 1)
            with pytest.raises(rs.RsError) as e:
                ctx.soft_bwd(ds, db, 0.3, dl)
            assert e.value.code == -3
        lib.rs_inject_alloc_failures(9, 1)    # there is no tenth allocation: the call succeeds
        ctx.soft_bwd(ds, db, 0.3, dl)
        lib.rs_inject_alloc_failures(0, 0)
        ga, gb, gt, loss = ctx.soft_bwd(ds, db, 0.3, dl)
        torch.cuda.synchronize()
        ref = orc.soft(X, y, K, b, 0.3)["loss"]
        fin = np.isfinite(ref)
        assert fin.any() and np.allclose(loss.cpu().numpy()[fin], ref[fin], rtol=1e-5, atol=0)
    finally:
        lib.rs_inject_alloc_failures(0, 0)
        ctx.dataset_destroy(ds)


def test_serving_retries_admission_and_relaunches_after_idle(orc):
    from paper_2406_01821_gb300 import build, rs
    build.build()
    c = rs.Context(0, mem_budget_bytes=1 << 30)
    lib = rs.lib()
    try:
        X, y, K, b = small_case(3)
        want = orc.eval_hard(X, y, K, b)
        ds = c.dataset(X, y, K)
        lib.rs_inject_alloc_failures(0, 4)                    # the first admission attempts fail
        t = c.submit(ds, rs.HostBatch(b))
        got = c.poll(t, b.P, K, timeout_us=30_000_000)
        assert got is not None and np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        lib.rs_inject_alloc_failures(0, 0)
        n0 = c.serving_stats()["kernel_launches"]
        time.sleep(0.2)                                       # well past the kernel's idle limit
        t = c.submit(ds, rs.HostBatch(b))
        got = c.poll(t, b.P, K, timeout_us=30_000_000)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        assert c.serving_stats()["kernel_launches"] == n0 + 1
    finally:
        lib.rs_inject_alloc_failures(0, 0)
        c.close()
