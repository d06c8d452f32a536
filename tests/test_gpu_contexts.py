"""Context modes and concurrency of the hard evaluation, against the oracle: asynchronous contexts
(the status folded into a sticky word that rs_check reads and clears), contexts without graphs and
with profiling, malformed batches rejected on the graph path (and the replayed graph usable right
after), and several host threads calling at once on shared and separate streams."""
import copy
import threading

import numpy as np
import pytest

from paper_2406_01821_gb300 import synth

pytestmark = pytest.mark.gpu

K = 3


def case(seed, P=30):
    X, y = synth.gaussian_mixture(3001, 10, K, seed)
    b = synth.random_rulesets(synth.quantile_table(X), K, P, (1, 8), (1, 4), seed, pair_prob=0.3)
    return X, y, b


def bad_copy(b):
    """The same batch with one rule naming a class outside 0..K-1 (rejected on the device)."""
    bb = copy.deepcopy(b)
    bb.rule_class[1] = K
    return bb


def same(c, pc, want):
    if not isinstance(c, np.ndarray):
        c, pc = c.cpu().numpy(), pc.cpu().numpy()
    return np.array_equal(c, want[0]) and np.array_equal(pc, want[1])


@pytest.fixture(scope="module")
def built():
    from paper_2406_01821_gb300 import build
    build.build()


@pytest.mark.parametrize("mode", ["async", "no_graph", "profile"])
def test_context_modes_match_oracle(built, orc, mode):
    import torch
    from paper_2406_01821_gb300 import rs
    flags = {"async": rs.CTX_ASYNC, "no_graph": rs.CTX_NO_GRAPH, "profile": rs.CTX_PROFILE}[mode]
    ctx = rs.Context(0, flags=flags)
    try:
        X, y, b = case(5)
        ds = ctx.dataset(X, y, K)
        s = torch.cuda.Stream()
        want = orc.eval_hard(X, y, K, b)
        db = rs.DeviceBatch.from_host(b)
        for _ in range(3):
            c, pc, _ = ctx.eval_hard(ds, db, K, stream=s)
            hc, hpc, _ = ctx.eval_hard(ds, rs.HostBatch(b), K, stream=s)
            ctx.check_async(s)            # any mode: waits for the stream, reads the sticky word
            assert same(c, pc, want) and same(hc, hpc, want)
        if mode == "profile":
            p = ctx.profile()
            assert p["hard_launches"] == 6 and p["hard_ms"] > 0
        ctx.dataset_destroy(ds)
    finally:
        ctx.close()


@pytest.mark.parametrize("stream_kind", ["side", "legacy"])
def test_async_context_reports_rejection_at_check(built, orc, stream_kind):
    """The call itself returns at once; rs_check reports the rejection once, then the context and
    the stream go on working."""
    import torch
    from paper_2406_01821_gb300 import rs
    ctx = rs.Context(0, flags=rs.CTX_ASYNC)
    try:
        X, y, b = case(6)
        ds = ctx.dataset(X, y, K)
        s = torch.cuda.Stream() if stream_kind == "side" else None
        ctx.eval_hard(ds, rs.DeviceBatch.from_host(bad_copy(b)), K, stream=s)
        with pytest.raises(rs.RsError) as e:
            ctx.check_async(s)
        assert e.value.code == -1
        ctx.check_async(s)
        c, pc, _ = ctx.eval_hard(ds, rs.DeviceBatch.from_host(b), K, stream=s)
        ctx.check_async(s)
        assert same(c, pc, orc.eval_hard(X, y, K, b))
        ctx.dataset_destroy(ds)
    finally:
        ctx.close()


@pytest.mark.parametrize("host", [False, True])
def test_rejection_then_replay_on_graph_path(built, orc, host):
    """A malformed batch on a capturable stream is rejected; a well-formed batch with the same
    pointers and sizes right after replays the same graph, whose status word starts clean."""
    import torch
    from paper_2406_01821_gb300 import rs
    ctx = rs.Context(0)
    try:
        X, y, b = case(7)
        bad = bad_copy(b)
        ds = ctx.dataset(X, y, K)
        s = torch.cuda.Stream()
        want = orc.eval_hard(X, y, K, b)
        out = None
        if host:
            batches = [rs.HostBatch(b), rs.HostBatch(bad), rs.HostBatch(b)]
        else:
            db = rs.DeviceBatch.from_host(b)
            out = (torch.empty(b.P, dtype=torch.int32, device="cuda"),
                   torch.empty((b.P, K), dtype=torch.int32, device="cuda"), None)
            batches = [db, db, db]
        for i, batch in enumerate(batches):
            if not host:                  # rewrite the rule classes in place: same pointers
                src = bad if i == 1 else b
                db.t["rule_class"].copy_(torch.from_numpy(src.rule_class.astype(np.int32)))
            if i == 1:
                with pytest.raises(rs.RsError) as e:
                    ctx.eval_hard(ds, batch, K, out=out, stream=s)
                assert e.value.code == -1
            else:
                c, pc, _ = ctx.eval_hard(ds, batch, K, out=out, stream=s)
                s.synchronize()
                assert same(c, pc, want)
        ctx.dataset_destroy(ds)
    finally:
        ctx.close()


def test_threads_on_shared_and_separate_streams(built, orc):
    """Four host threads, two per stream, each with its own batch (sizes differ, so calls on a
    shared stream alternate between capture and replay of one cached graph)."""
    import torch
    from paper_2406_01821_gb300 import rs
    ctx = rs.Context(0)
    try:
        X, y, _ = case(8)
        ds = ctx.dataset(X, y, K)
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        batches = [synth.random_rulesets(synth.quantile_table(X), K, 10 + 9 * i, (1, 8), (1, 4), 20 + i)
                   for i in range(4)]
        wants = [orc.eval_hard(X, y, K, bb) for bb in batches]
        failures = []

        def work(i):
            try:
                hb = rs.HostBatch(batches[i])
                for _ in range(25):
                    c, pc, _ = ctx.eval_hard(ds, hb, K, stream=streams[i % 2])
                    if not same(c, pc, wants[i]):
                        failures.append(f"thread {i}: counts differ")
                        return
            except Exception as ex:       # reported below, with the thread that raised it
                failures.append(f"thread {i}: {ex!r}")

        threads = [threading.Thread(target=work, args=(i,)) for i in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=120)
        assert not any(t.is_alive() for t in threads)
        assert not failures, failures
        ctx.dataset_destroy(ds)
    finally:
        ctx.close()
