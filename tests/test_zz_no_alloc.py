"""rs_eval_hard_static: the hard evaluation for callers that cannot allocate device memory
(a host whose device memory belongs to another allocator or is reserved up front, or a loop that
must never block in an allocator). It takes its scratch from a fixed array in the library's device
image. This file is collected last on purpose, so that a failure here comes after every other test.

Checks, through the C ABI:
  - two calls in a row (a large batch, then a smaller one that reuses the array left dirty by the
    first), with counts, per-class counts and predictions, give exactly what rs_eval_hard gives
    and what the oracle gives;
  - a batch with category-membership conditions (which the evaluator runs in another form);
  - a call made while every device allocation of the library is forced to fail still succeeds:
    the entry point reaches no allocating routine;
  - an asynchronous context reports a malformed batch through rs_check, and the next call is exact;
  - host output memory and a batch beyond the array's size are refused before anything runs."""
import ctypes

import numpy as np
import pytest

from paper_2406_01821_gb300 import synth

pytestmark = pytest.mark.gpu


def _static_call(ctx, ds, db, correct, pc, stream, preds=None):
    from paper_2406_01821_gb300 import rs
    cb = db.c()
    return rs.lib().rs_eval_hard_static(ctx.h, ds, ctypes.byref(cb), rs._ptr(correct), rs._ptr(pc),
                                        rs._ptr(preds), rs._stream_ptr(stream))


def _outputs(P, K, N=None):
    import torch
    c = torch.full((P,), -7, dtype=torch.int32, device="cuda")
    pc = torch.full((P, K), -7, dtype=torch.int32, device="cuda")
    pr = torch.full((P, N), -7, dtype=torch.int32, device="cuda") if N else None
    return c, pc, pr


def test_static_scratch_matches_regular_call_twice(orc):
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    ctx = rs.Context(0)
    try:
        X, y = synth.gaussian_mixture(30001, 64, 6, 21)
        ds = ctx.dataset(X, y, 6)
        s = torch.cuda.Stream()
        batches = [synth.random_rulesets(synth.quantile_table(X), 6, 700, (1, 40), (1, 8), 21),
                   synth.random_rulesets(synth.quantile_table(X), 6, 90, (1, 10), (1, 4), 22)]
        for i, b in enumerate(batches):         # two calls in a row share the same array
            db = rs.DeviceBatch.from_host(b)
            want_c, want_pc, want_pr = ctx.eval_hard(ds, db, 6, len(X), preds=True, stream=s)
            got_c, got_pc, got_pr = _outputs(b.P, 6, len(X) if i == 1 else None)
            rc = _static_call(ctx, ds, db, got_c, got_pc, s, got_pr)
            assert rc == 0, rs.lib().rs_last_error()
            s.synchronize()
            assert torch.equal(got_c, want_c)
            assert torch.equal(got_pc, want_pc)
            oc, opc, opr = orc.eval_hard(X, y, 6, b, want_preds=(i == 1))
            assert np.array_equal(got_c.cpu().numpy(), oc)
            assert np.array_equal(got_pc.cpu().numpy(), opc.reshape(b.P, 6))
            if i == 1:
                assert torch.equal(got_pr, want_pr)
                assert np.array_equal(got_pr.cpu().numpy(), opr.reshape(b.P, len(X)))
        ctx.dataset_destroy(ds)
    finally:
        ctx.close()


def test_static_categorical_batch(orc):
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    ctx = rs.Context(0)
    try:
        X, y = synth.categorical_mixture(12007, 48, 6, 4, n_cat=12, n_codes=48)
        b = synth.random_rulesets(synth.quantile_table(X), 6, 96, (1, 40), (1, 6), 4, cat_from=36, n_codes=48)
        assert (b.cond_op == synth.IN).sum() > 50
        ds = ctx.dataset(X, y, 6)
        db = rs.DeviceBatch.from_host(b)
        s = torch.cuda.current_stream()
        for with_preds in (False, True):
            c, pc, pr = _outputs(b.P, 6, len(X) if with_preds else None)
            assert _static_call(ctx, ds, db, c, pc, s, pr) == 0, rs.lib().rs_last_error()
            torch.cuda.synchronize()
            oc, opc, opr = orc.eval_hard(X, y, 6, b, want_preds=with_preds)
            assert np.array_equal(c.cpu().numpy(), oc)
            assert np.array_equal(pc.cpu().numpy(), opc.reshape(b.P, 6))
            if with_preds:
                assert np.array_equal(pr.cpu().numpy(), opr.reshape(b.P, len(X)))
        ctx.dataset_destroy(ds)
    finally:
        ctx.close()


def test_static_call_reaches_no_allocation(orc):
    """Every device allocation the library attempts fails while the injector is armed; the static
    entry point still succeeds, so it calls no allocating routine (the regular entry point, which
    allocates stream-ordered scratch, fails with RS_ERR_OOM under the same injector)."""
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    ctx = rs.Context(0)
    lib = rs.lib()
    try:
        X, y = synth.gaussian_mixture(9001, 32, 4, 8)
        b = synth.random_rulesets(synth.quantile_table(X), 4, 200, (1, 20), (1, 6), 8)
        ds = ctx.dataset(X, y, 4)
        db = rs.DeviceBatch.from_host(b)
        s = torch.cuda.current_stream()
        c0, pc0, _ = _outputs(b.P, 4)
        assert _static_call(ctx, ds, db, c0, pc0, s) == 0       # first call: tile descriptor
        c, pc, pr = _outputs(b.P, 4, len(X))
        lib.rs_inject_alloc_failures(0, 1 << 30)
        try:
            rc = _static_call(ctx, ds, db, c, pc, s, pr)
            rc_regular = lib.rs_eval_hard(ctx.h, ds, ctypes.byref(db.c()), rs._ptr(c0), None, None,
                                          rs._stream_ptr(torch.cuda.Stream()))
        finally:
            lib.rs_inject_alloc_failures(0, 0)
        assert rc == 0, lib.rs_last_error()
        assert rc_regular == -3                                  # RS_ERR_OOM: the injector is live
        torch.cuda.synchronize()
        oc, opc, opr = orc.eval_hard(X, y, 4, b, want_preds=True)
        assert np.array_equal(c.cpu().numpy(), oc)
        assert np.array_equal(pc.cpu().numpy(), opc.reshape(b.P, 4))
        assert np.array_equal(pr.cpu().numpy(), opr.reshape(b.P, len(X)))
        ctx.dataset_destroy(ds)
    finally:
        ctx.close()


def test_static_async_context_reports_rejection(orc):
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    ctx = rs.Context(0, flags=rs.CTX_ASYNC)
    lib = rs.lib()
    try:
        X, y = synth.gaussian_mixture(5003, 16, 3, 9)
        ds = ctx.dataset(X, y, 3)
        s = torch.cuda.Stream()
        bad = synth.random_rulesets(synth.quantile_table(X), 3, 40, (1, 8), (1, 4), 9)
        bad.rule_class[3] = 7                                    # class out of range: rejected on the device
        dbad = rs.DeviceBatch.from_host(bad)
        c, pc, _ = _outputs(bad.P, 3)
        assert _static_call(ctx, ds, dbad, c, pc, s) == 0        # enqueued; the status is folded
        assert lib.rs_check(ctx.h, rs._stream_ptr(s)) == -1      # RS_ERR_INVALID, read after the work
        good = synth.random_rulesets(synth.quantile_table(X), 3, 40, (1, 8), (1, 4), 10)
        dgood = rs.DeviceBatch.from_host(good)
        c, pc, _ = _outputs(good.P, 3)
        assert _static_call(ctx, ds, dgood, c, pc, s) == 0
        assert lib.rs_check(ctx.h, rs._stream_ptr(s)) == 0
        s.synchronize()
        oc, opc, _ = orc.eval_hard(X, y, 3, good)
        assert np.array_equal(c.cpu().numpy(), oc)
        assert np.array_equal(pc.cpu().numpy(), opc.reshape(good.P, 3))
        ctx.dataset_destroy(ds)
    finally:
        ctx.close()


def test_static_refuses_host_outputs():
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    ctx = rs.Context(0)
    try:
        X, y = synth.two_class_gaussian(1000, 8, 3)
        ds = ctx.dataset(X, y, 2)
        b = synth.random_rulesets(synth.quantile_table(X), 2, 20, (1, 4), (1, 3), 3)
        db = rs.DeviceBatch.from_host(b)
        host_c = torch.zeros(b.P, dtype=torch.int32)             # CPU memory: not for the kernels
        rc = _static_call(ctx, ds, db, host_c, None, torch.cuda.current_stream())
        assert rc == -1                                           # RS_ERR_INVALID
        assert b"device memory" in rs.lib().rs_last_error()
        ctx.dataset_destroy(ds)
    finally:
        ctx.close()


def test_static_scratch_refuses_oversized_batch():
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    ctx = rs.Context(0)
    try:
        X, y = synth.two_class_gaussian(1000, 8, 3)
        ds = ctx.dataset(X, y, 2)
        b = synth.random_rulesets(synth.quantile_table(X), 2, 1200, (64, 64), (8, 8), 3)  # 614k conds
        db = rs.DeviceBatch.from_host(b)
        c = torch.zeros(b.P, dtype=torch.int32, device="cuda")
        rc = _static_call(ctx, ds, db, c, None, torch.cuda.current_stream())
        assert rc == -2                                       # RS_ERR_TOO_LARGE
        assert b"scratch" in rs.lib().rs_last_error()
        ctx.dataset_destroy(ds)
    finally:
        ctx.close()
