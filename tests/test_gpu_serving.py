"""Serving (continuous batching): every result of a request served in a mix of concurrent requests
of uneven sizes over several resident datasets equals the result of the same request evaluated
alone with rs_eval_hard (exact integer counts); budget admission, rejection and cancellation."""
import threading

import numpy as np
import pytest

from paper_2406_01821_gb300 import synth

pytestmark = pytest.mark.gpu


def make_runs(seed, n_runs=5):
    rng = np.random.default_rng(seed)
    runs = []
    for i in range(n_runs):
        N = int(rng.integers(500, 40000))
        F = int(rng.integers(8, 257))
        K = int(rng.integers(2, 11))
        X, y = synth.gaussian_mixture(N, F, K, seed * 100 + i)
        runs.append((X, y, K, synth.quantile_table(X)))
    return runs


def test_mix_equals_alone(orc):
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    ctx = rs.Context(0, mem_budget_bytes=1 << 30)
    try:
        runs = make_runs(1)
        dss = [ctx.dataset(X, y, K) for (X, y, K, _) in runs]
        rng = np.random.default_rng(2)
        reqs = []
        for j in range(24):
            i = int(rng.integers(0, len(runs)))
            X, y, K, q = runs[i]
            P = int(np.exp(rng.uniform(np.log(16), np.log(300))))
            b = synth.random_rulesets(q, K, P, (1, 64), (1, 8), 1000 + j)
            reqs.append((i, b))
        # alone
        alone = []
        for i, b in reqs:
            c, pc, _ = ctx.eval_hard(dss[i], rs.HostBatch(b), runs[i][2])
            alone.append((c.copy(), pc.copy()))
        # mixed: submitted from several threads, polled in any order
        tickets = [None] * len(reqs)

        def submitter(idx):
            for j in idx:
                i, b = reqs[j]
                tickets[j] = ctx.submit(dss[i], rs.HostBatch(b) if j % 2 else rs.DeviceBatch.from_host(b))
        th = [threading.Thread(target=submitter, args=(list(range(k, len(reqs), 4)),)) for k in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for j in reversed(range(len(reqs))):
            i, b = reqs[j]
            out = ctx.poll(tickets[j], b.P, runs[i][2], timeout_us=60_000_000)
            assert out is not None, "request did not finish"
            assert np.array_equal(out[0], alone[j][0]), j
            assert np.array_equal(out[1], alone[j][1]), j
            assert out[2]["submit_ns"] <= out[2]["admit_ns"] <= out[2]["done_ns"]
        # and every result against the oracle
        for j, (i, b) in enumerate(reqs):
            X, y, K, _ = runs[i]
            want = orc.eval_hard(X, y, K, b)
            assert np.array_equal(alone[j][0], want[0]), j
            assert np.array_equal(alone[j][1], want[1]), j
        st = ctx.serving_stats()
        assert st["active"] == 0 and st["queued"] == 0 and st["device_bytes_in_use"] == 0
        assert st["kernel_launches"] >= 1
    finally:
        ctx.close()


def test_budget_admission_and_errors():
    from paper_2406_01821_gb300 import build, rs
    build.build()
    X, y = synth.gaussian_mixture(20000, 32, 3, 5)
    q = synth.quantile_table(X)
    big = synth.random_rulesets(q, 3, 2000, (60, 64), (8, 8), 5)          # ~1M conditions
    small = [synth.random_rulesets(q, 3, 40, (1, 10), (1, 4), 6 + j) for j in range(6)]
    # a budget that holds one small request at a time (and not the big one)
    ctx = rs.Context(0, mem_budget_bytes=4 << 20)
    try:
        ds = ctx.dataset(X, y, 3)
        with pytest.raises(rs.RsError) as ei:
            ctx.submit(ds, rs.HostBatch(big))
        assert ei.value.code == -2
        ts = [ctx.submit(ds, rs.HostBatch(b)) for b in small]
        for t, b in zip(ts, small):
            out = ctx.poll(t, b.P, 3, timeout_us=60_000_000)
            c, _, _ = ctx.eval_hard(ds, rs.HostBatch(b), 3)
            assert np.array_equal(out[0], c)
        bad = synth.random_rulesets(q, 3, 5, 2, 2, 9)
        bad.cond_f[0] = 99
        t = ctx.submit(ds, rs.HostBatch(bad))
        with pytest.raises(rs.RsError) as ei:
            ctx.poll(t, bad.P, 3, timeout_us=60_000_000)
        assert ei.value.code == -1
        # cancellation of a request still waiting for admission
        ctx2 = rs.Context(0, mem_budget_bytes=(12 << 20))
        try:
            ds2 = ctx2.dataset(X, y, 3)
            mid = synth.random_rulesets(q, 3, 600, (40, 64), (6, 8), 11)
            t1 = ctx2.submit(ds2, rs.HostBatch(mid))
            t2 = ctx2.submit(ds2, rs.HostBatch(mid))
            rc = ctx2.cancel(t2)
            if rc == 0:
                with pytest.raises(rs.RsError) as ei:
                    ctx2.poll(t2, mid.P, 3, timeout_us=60_000_000)
                assert ei.value.code == -8
            else:
                assert ctx2.poll(t2, mid.P, 3, timeout_us=60_000_000) is not None
            assert ctx2.poll(t1, mid.P, 3, timeout_us=60_000_000) is not None
        finally:
            ctx2.close()
    finally:
        ctx.close()


def test_soft_requests_in_the_mix(orc):
    """Soft-loss requests served next to hard ones: each loss equals rs_eval_soft_fwd's bit for bit
    and the float64 oracle's within the soft tolerance; hard results stay exact; kinds are kept
    apart (a soft ticket cannot be polled as hard) and a soft request needs tau > 0."""
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    ctx = rs.Context(0, mem_budget_bytes=1 << 30)
    try:
        runs = make_runs(3, n_runs=3)
        dss = [ctx.dataset(X, y, K) for (X, y, K, _) in runs]
        rng = np.random.default_rng(4)
        jobs = []
        for j in range(12):
            i = int(rng.integers(0, len(runs)))
            X, y, K, q = runs[i]
            b = synth.random_rulesets(q, K, int(rng.integers(8, 120)), (1, 16), (1, 6), 300 + j)
            soft = j % 2 == 0
            t = ctx.submit_soft(dss[i], rs.HostBatch(b), 0.1) if soft else ctx.submit(dss[i], rs.HostBatch(b))
            jobs.append((i, b, soft, t))
        for i, b, soft, t in jobs:
            X, y, K, _ = runs[i]
            if soft:
                with pytest.raises(rs.RsError):
                    ctx.poll(t, b.P, K, timeout_us=60_000_000)      # wrong kind
                loss, info = ctx.poll_soft(t, b.P, timeout_us=60_000_000)
                direct, _ = ctx.soft_fwd(dss[i], rs.DeviceBatch.from_host(b), 0.1, N=len(X), K=K)
                torch.cuda.synchronize()
                assert np.array_equal(loss.view(np.uint32), direct.cpu().numpy().view(np.uint32))
                ref = orc.soft(X, y, K, b, 0.1)
                assert np.allclose(loss, ref["loss"], rtol=1e-5, atol=0)
            else:
                c, pc, _ = ctx.poll(t, b.P, K, timeout_us=60_000_000)
                want = orc.eval_hard(X, y, K, b)
                assert np.array_equal(c, want[0]) and np.array_equal(pc, want[1])
        with pytest.raises(rs.RsError):
            ctx.submit_soft(dss[0], rs.HostBatch(jobs[0][1]), 0.0)
    finally:
        ctx.close()


def test_device_batch_copied_at_submission(orc):
    """A device batch is copied device to device before rs_submit returns: overwriting the
    caller's arrays right after the call changes nothing, for hard and soft requests."""
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    X, y = synth.gaussian_mixture(7001, 20, 3, 41)
    b = synth.random_rulesets(synth.quantile_table(X), 3, 120, (1, 20), (1, 6), 41)
    want = orc.eval_hard(X, y, 3, b)
    want_soft = orc.soft(X, y, 3, b, 0.2)["loss"]
    with rs.Context(0) as ctx:
        ds = ctx.dataset(X, y, 3)
        db = rs.DeviceBatch.from_host(b)
        th = ctx.submit(ds, db)
        ts = ctx.submit_soft(ds, db, 0.2)
        for t in db.t.values():                  # the caller reuses its memory at once
            if t is not None:
                t.zero_()
        torch.cuda.synchronize()
        c, pc, _ = ctx.poll(th, b.P, 3, timeout_us=30_000_000)
        loss, _ = ctx.poll_soft(ts, b.P, timeout_us=30_000_000)
        ctx.dataset_destroy(ds)
    assert np.array_equal(c, want[0]) and np.array_equal(pc, want[1].reshape(b.P, 3))
    fin = np.isfinite(want_soft)
    assert np.allclose(loss[fin], want_soft[fin], rtol=1e-5, atol=0)
    assert (np.isinf(loss) == ~fin).all()


def test_served_ranked_units_with_ties_equal_oracle(orc):
    """Requests large enough for the serving kernel's rank-coded units (64 or more sets, F <= 128)
    on data full of equal values (small integers, +0 and -0) with thresholds on data values and
    one ulp either side: every count equals the oracle's."""
    from paper_2406_01821_gb300 import build, rs
    build.build()
    rng = np.random.default_rng(31)
    N, F, K = 5000, 12, 3
    X = rng.integers(-3, 4, (N, F)).astype(np.float32)
    X[:, 1] = np.where(rng.random(N) < 0.5, np.float32(0.0), np.float32(-0.0))
    y = rng.integers(0, K, N).astype(np.int32)
    ctx = rs.Context(0, mem_budget_bytes=1 << 30)
    try:
        ds = ctx.dataset(X, y, K)
        tickets, batches = [], []
        for j in range(3):
            b = synth.random_rulesets(synth.quantile_table(X), K, 96, (1, 16), (1, 5), 40 + j, pair_prob=0.25)
            idx = np.flatnonzero(b.cond_g < 0)
            a = rng.choice(np.array([1.0, -1.0, 0.5, -2.0], np.float32), len(idx))
            t = (a * X[rng.integers(0, N, len(idx)), b.cond_f[idx]]).astype(np.float32)
            shift = rng.integers(-1, 2, len(idx))
            t = np.where(shift < 0, np.nextafter(t, np.float32(-np.inf)),
                         np.where(shift > 0, np.nextafter(t, np.float32(np.inf)), t)).astype(np.float32)
            b.cond_a[idx], b.cond_t[idx] = a, t
            batches.append(b)
            tickets.append(ctx.submit(ds, rs.HostBatch(b)))
        for b, tk in zip(batches, tickets):
            c, pc, _ = ctx.poll(tk, b.P, K, timeout_us=60_000_000)
            want = orc.eval_hard(X, y, K, b)
            assert np.array_equal(c, want[0])
            assert np.array_equal(pc, want[1].reshape(b.P, K))
        ctx.dataset_destroy(ds)
    finally:
        ctx.close()


def test_dataset_in_use_by_a_request_is_not_destroyed(orc):
    """A dataset that a serving request still holds (queued, running or completed but not yet
    polled, cancelled ones included) is refused by rs_dataset_destroy, which would otherwise free
    the device copy that the request's kernels read; once the request is polled it goes."""
    from paper_2406_01821_gb300 import rs
    X, y = synth.gaussian_mixture(3000, 12, 3, 7)
    b = synth.random_rulesets(synth.quantile_table(X), 3, 40, (1, 12), (1, 4), 7)
    want = orc.eval_hard(X, y, 3, b)
    ctx = rs.Context(0)
    try:
        ds = ctx.dataset(X, y, 3)
        t = ctx.submit(ds, rs.HostBatch(b))
        with pytest.raises(rs.RsError) as e:
            ctx.dataset_destroy(ds)
        assert e.value.code == -1 and "in use" in str(e.value)
        c, pc, _ = ctx.poll(t, b.P, 3, timeout_us=60_000_000)
        assert np.array_equal(c, want[0])
        ctx.dataset_destroy(ds)
        with pytest.raises(rs.RsError) as e:
            ctx.dataset_destroy(ds)
        assert e.value.code == -7                  # RS_ERR_NOT_FOUND
        # a cancelled request holds its dataset until it is polled as well
        ds2 = ctx.dataset(X, y, 3)
        t2 = ctx.submit(ds2, rs.HostBatch(b))
        if ctx.cancel(t2) == 0:
            with pytest.raises(rs.RsError):
                ctx.dataset_destroy(ds2)
            with pytest.raises(rs.RsError) as e:
                ctx.poll(t2, b.P, 3, timeout_us=60_000_000)
            assert e.value.code == -8              # RS_ERR_CANCELLED
        else:                                      # admitted before the cancel: poll it
            assert ctx.poll(t2, b.P, 3, timeout_us=60_000_000) is not None
        ctx.dataset_destroy(ds2)
    finally:
        ctx.close()
