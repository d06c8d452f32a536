"""Datasets under a device-memory budget (rs_set_dataset_budget): least recently used datasets not
in use are evicted and rebuilt from the host copy when next named; every count stays equal to the
oracle's, through cached graphs, asynchronous calls and serving requests that pin their dataset."""
import ctypes

import numpy as np
import pytest

from paper_2406_01821_gb300 import synth

pytestmark = pytest.mark.gpu

N, F, K = 4000, 12, 3


def _data(i):
    X, y = synth.gaussian_mixture(N, F, K, 60 + i)
    b = synth.random_rulesets(synth.quantile_table(X), K, 40, (1, 12), (1, 4), 70 + i, pair_prob=0.3)
    return X, y, b


def _budget_ctx(flags=0):
    """A context whose budget holds two of the test's (equally sized) datasets."""
    from paper_2406_01821_gb300 import build, rs
    build.build()
    ctx = rs.Context(0, flags=flags)
    ctx.set_dataset_budget(1 << 40)             # keep host copies from the first registration on
    return ctx


def test_evict_least_recently_used_and_rebuild(orc):
    from paper_2406_01821_gb300 import rs
    ctx = _budget_ctx()
    try:
        data = [_data(i) for i in range(3)]
        want = [orc.eval_hard(X, y, K, b) for X, y, b in data]
        dss = [ctx.dataset(data[0][0], data[0][1], K)]
        one = ctx.dataset_stats()["resident_bytes"]
        ctx.set_dataset_budget(2 * one + one // 2)
        dss += [ctx.dataset(X, y, K) for X, y, _ in data[1:]]
        st = ctx.dataset_stats()
        assert st["datasets"] == 3 and st["resident"] == 2 and st["evictions"] == 1     # the first
        assert st["resident_bytes"] <= 2 * one + one // 2

        def check(i):
            c, pc, _ = ctx.eval_hard(dss[i], rs.HostBatch(data[i][2]), K)
            assert np.array_equal(c, want[i][0]) and np.array_equal(pc, want[i][1].reshape(-1, K))

        check(0)                                   # rebuilt; the second is now least recent
        st = ctx.dataset_stats()
        assert st["rebuilds"] == 1 and st["evictions"] == 2 and st["resident"] == 2
        check(2)                                   # resident: nothing moves
        assert ctx.dataset_stats()["rebuilds"] == 1
        check(1)                                   # rebuilt, the first evicted again
        st = ctx.dataset_stats()
        assert st["rebuilds"] == 2 and st["evictions"] == 3
        # device batches repeat on one stream (cached and captured graphs), around an eviction
        import torch
        stream = torch.cuda.Stream()
        db = rs.DeviceBatch.from_host(data[0][2])
        for rnd in range(2):
            for _ in range(3):
                c, pc, _ = ctx.eval_hard(dss[0], db, K, stream=stream)
                stream.synchronize()
                assert np.array_equal(c.cpu().numpy(), want[0][0])
            check(1)
            check(2)                               # the first is evicted between the rounds
        assert ctx.dataset_stats()["evictions"] >= 5
        ctx.dataset_destroy(dss[0])                # whether resident or not
        st = ctx.dataset_stats()
        assert st["datasets"] == 2
    finally:
        ctx.close()


def test_async_calls_and_static_entry(orc):
    import torch
    from paper_2406_01821_gb300 import rs
    ctx = _budget_ctx(flags=rs.CTX_ASYNC)
    try:
        data = [_data(i) for i in range(3)]
        want = [orc.eval_hard(X, y, K, b) for X, y, b in data]
        dss = [ctx.dataset(data[0][0], data[0][1], K)]
        one = ctx.dataset_stats()["resident_bytes"]
        ctx.set_dataset_budget(2 * one + one // 2)
        dss.append(ctx.dataset(data[1][0], data[1][1], K))
        stream = torch.cuda.Stream()
        dbs = [rs.DeviceBatch.from_host(b) for _, _, b in data]
        outs = []
        for i in (0, 1):                           # enqueued, not waited for
            c = torch.empty(dbs[i].c().P, dtype=torch.int32, device="cuda")
            pc = torch.empty((dbs[i].c().P, K), dtype=torch.int32, device="cuda")
            ctx.eval_hard(dss[i], dbs[i], K, out=(c, pc, None), stream=stream)
            outs.append((c, pc))
        # a dataset whose queued work has not completed is not evicted (its mark is pending);
        # whichever is chosen, the queued results are exact
        dss.append(ctx.dataset(data[2][0], data[2][1], K))
        rs.check(rs.lib().rs_check(ctx.h, rs._stream_ptr(stream)))
        for i in (0, 1):
            assert np.array_equal(outs[i][0].cpu().numpy(), want[i][0])
            assert np.array_equal(outs[i][1].cpu().numpy(), want[i][1].reshape(-1, K))
        assert ctx.dataset_stats()["evictions"] <= 1
        if ctx.dataset_stats()["resident"] == 3:     # nothing was idle then: make room now
            c, _, _ = ctx.eval_hard(dss[2], rs.HostBatch(data[2][2]), K)
            ctx.set_dataset_budget(2 * one + one // 2)
        assert ctx.dataset_stats()["resident"] == 2
        for i in (2, 1):                           # synchronous uses: the first is left evicted
            c = torch.empty(dbs[i].c().P, dtype=torch.int32, device="cuda")
            ctx.eval_hard(dss[i], dbs[i], K, out=(c, None, None), stream=stream)
            rs.check(rs.lib().rs_check(ctx.h, rs._stream_ptr(stream)))
            assert np.array_equal(c.cpu().numpy(), want[i][0])
        assert ctx.dataset_stats()["resident"] == 2
        # the allocation-free entry refuses an evicted dataset (rebuilding would allocate)
        cb = dbs[0].c()
        c = torch.empty(cb.P, dtype=torch.int32, device="cuda")
        pc = torch.empty((cb.P, K), dtype=torch.int32, device="cuda")
        rc = rs.lib().rs_eval_hard_static(ctx.h, dss[0], ctypes.byref(cb), rs._ptr(c), rs._ptr(pc), None,
                                          rs._stream_ptr(stream))
        assert rc == -1                            # RS_ERR_INVALID
        ctx.eval_hard(dss[0], dbs[0], K, out=(c, pc, None), stream=stream)   # rebuilt
        rc = rs.lib().rs_eval_hard_static(ctx.h, dss[0], ctypes.byref(cb), rs._ptr(c), rs._ptr(pc), None,
                                          rs._stream_ptr(stream))
        assert rc == 0
        rs.check(rs.lib().rs_check(ctx.h, rs._stream_ptr(stream)))
        assert np.array_equal(c.cpu().numpy(), want[0][0])
    finally:
        ctx.close()


def test_serving_request_pins_its_dataset(orc):
    from paper_2406_01821_gb300 import rs
    ctx = _budget_ctx()
    try:
        data = [_data(i) for i in range(4)]
        want = [orc.eval_hard(X, y, K, b) for X, y, b in data]
        dss = [ctx.dataset(data[0][0], data[0][1], K)]
        one = ctx.dataset_stats()["resident_bytes"]
        ctx.set_dataset_budget(2 * one + one // 2)
        dss.append(ctx.dataset(data[1][0], data[1][1], K))
        ticket = ctx.submit(dss[0], rs.HostBatch(data[0][2]))   # pins the first until polled
        dss += [ctx.dataset(X, y, K) for X, y, _ in data[2:]]   # would evict the first otherwise
        for i in (2, 3, 1, 2, 3):
            c, _, _ = ctx.eval_hard(dss[i], rs.HostBatch(data[i][2]), K)
            assert np.array_equal(c, want[i][0])
        rebuilds = ctx.dataset_stats()["rebuilds"]
        c, pc, _ = ctx.poll(ticket, data[0][2].P, K, timeout_us=60_000_000)
        assert np.array_equal(c, want[0][0]) and np.array_equal(pc, want[0][1].reshape(-1, K))
        c, _, _ = ctx.eval_hard(dss[0], rs.HostBatch(data[0][2]), K)
        assert np.array_equal(c, want[0][0])
        assert ctx.dataset_stats()["rebuilds"] == rebuilds      # it was never evicted
    finally:
        ctx.close()
