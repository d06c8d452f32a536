"""rs_eval_hard_static: the hard evaluation for callers that cannot allocate device memory
(a host whose device memory belongs to another allocator or is reserved up front, or a loop that
must never block in an allocator). It takes its scratch from a fixed array in the library's device
image. This file is collected last on purpose, so that a failure here comes after every other test.

Checks, through the C ABI: two calls in a row (a large batch, then a smaller one that reuses the
array left dirty by the first) give exactly what rs_eval_hard gives; a batch beyond the array's
size is refused with RS_ERR_TOO_LARGE before anything runs."""
import ctypes

import numpy as np
import pytest

from paper_2406_01821_gb300 import synth

pytestmark = pytest.mark.gpu


def _static_call(ctx, ds, db, correct, pc, stream):
    from paper_2406_01821_gb300 import rs
    cb = db.c()
    return rs.lib().rs_eval_hard_static(ctx.h, ds, ctypes.byref(cb), rs._ptr(correct), rs._ptr(pc),
                                        None, rs._stream_ptr(stream))


def test_static_scratch_matches_regular_call_twice():
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
        for b in batches:                       # two calls in a row share the same array
            db = rs.DeviceBatch.from_host(b)
            want_c, want_pc, _ = ctx.eval_hard(ds, db, 6, stream=s)
            got_c = torch.full((b.P,), -7, dtype=torch.int32, device="cuda")
            got_pc = torch.full((b.P, 6), -7, dtype=torch.int32, device="cuda")
            rc = _static_call(ctx, ds, db, got_c, got_pc, s)
            assert rc == 0, rs.lib().rs_last_error()
            s.synchronize()
            assert torch.equal(got_c, want_c)
            assert torch.equal(got_pc, want_pc)
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
