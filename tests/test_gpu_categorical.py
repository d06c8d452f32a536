"""GPU parity of categorical membership conditions (x[f] an integer code 0..63 in a 64-bit set)
against the oracle: bit-exact counts and predictions in every form that evaluates them (the
rank-coded walk, the condition-at-a-time form; configurations of other forms are redirected),
through the static entry point and serving, and the soft path (membership as an exact indicator
with zero gradient) within the soft tolerance."""
import numpy as np
import pytest

from paper_2406_01821_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_2406_01821_gb300 import build, rs
    build.build()
    c = rs.Context(0)
    yield c
    c.close()


def workload(seed, N=12007, F=48, K=6, n_cat=12, n_codes=48, P=96):
    """Gaussian mixture with 12 categorical features of 48 codes (bits above 31 in use)."""
    X, y = synth.categorical_mixture(N, F, K, seed, n_cat=n_cat, n_codes=n_codes)
    b = synth.random_rulesets(synth.quantile_table(X), K, P, (1, 40), (1, 6), seed,
                              cat_from=F - n_cat, n_codes=n_codes)
    assert (b.cond_op == synth.IN).sum() > 50
    return X, y, K, b


def run(ctx, X, y, K, b, tile=None, preds=False, host=False):
    import torch
    from paper_2406_01821_gb300 import rs
    ds = ctx.dataset(X, y, K)
    try:
        if tile is not None:
            ctx.set_tile_config(tile)
        bb = rs.HostBatch(b) if host else rs.DeviceBatch.from_host(b)
        c, pc, pr = ctx.eval_hard(ds, bb, K, len(X), per_class=True, preds=preds)
        if not host:
            torch.cuda.synchronize()
            c, pc = c.cpu().numpy(), pc.cpu().numpy()
            pr = pr.cpu().numpy() if pr is not None else None
        return c, pc, pr
    finally:
        ctx.set_tile_config(-1)
        ctx.dataset_destroy(ds)


@pytest.mark.parametrize("tile", [None, 22, 21, 0, 5, 9, 12, 17, 18, 23])
def test_counts_in_every_configuration(ctx, orc, tile):
    X, y, K, b = workload(1)
    want = orc.eval_hard(X, y, K, b)
    got = run(ctx, X, y, K, b, tile=tile)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


@pytest.mark.parametrize("host", [False, True])
def test_predictions(ctx, orc, host):
    X, y, K, b = workload(2, N=5003)
    want = orc.eval_hard(X, y, K, b, want_preds=True)
    got = run(ctx, X, y, K, b, preds=True, host=host)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


@pytest.mark.parametrize("nonfinite", [False, True])
def test_edge_values(ctx, orc, nonfinite):
    """Fractions, negatives, -0, codes 63 / 64 and huge values in the categorical columns (and
    NaN / infinities, which take the dataset off the rank-coded path)."""
    X, y, K, b = workload(3, N=4099)
    rng = np.random.default_rng(3)
    cat = X.shape[1] - 12
    vals = np.array([-0.0, 0.5, 63.0, 64.0, -1.0, 1e9, 31.0, 32.0, 2.25, 47.0], np.float32)
    if nonfinite:
        vals = np.concatenate([vals, np.array([np.nan, np.inf, -np.inf], np.float32)])
    idx = rng.random((len(X), 12)) < 0.3
    X[:, cat:][idx] = rng.choice(vals, idx.sum())
    sel = np.flatnonzero(b.cond_op == synth.IN)    # a third of the sets hold the extreme codes
    b.cond_set[sel[::3]] |= np.uint64((1 << 63) | (1 << 32) | (1 << 31) | 1)
    want = orc.eval_hard(X, y, K, b, want_preds=True)
    got = run(ctx, X, y, K, b, preds=True)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    got = run(ctx, X, y, K, b)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_static_entry_point(ctx, orc):
    import ctypes
    import torch
    from paper_2406_01821_gb300 import rs
    X, y, K, b = workload(4, N=3001)
    want = orc.eval_hard(X, y, K, b)
    ds = ctx.dataset(X, y, K)
    try:
        db = rs.DeviceBatch.from_host(b)
        c = torch.zeros(b.P, dtype=torch.int32, device="cuda")
        pc = torch.zeros(b.P * K, dtype=torch.int32, device="cuda")
        cb = db.c()
        stream = torch.cuda.current_stream()
        rs.check(rs.lib().rs_eval_hard_static(ctx.h, ds, ctypes.byref(cb), rs._ptr(c), rs._ptr(pc), None,
                                              rs._stream_ptr(stream)))
        torch.cuda.synchronize()
        assert np.array_equal(c.cpu().numpy(), want[0])
        assert np.array_equal(pc.cpu().numpy().reshape(b.P, K), want[1])
    finally:
        ctx.dataset_destroy(ds)


def test_without_sets_membership_is_rejected(ctx):
    from paper_2406_01821_gb300 import rs
    X, y, K, b = workload(5, N=999)
    b.cond_set = None                            # op 2 with no category sets: invalid batch
    ds = ctx.dataset(X, y, K)
    try:
        with pytest.raises(rs.RsError) as e:
            ctx.eval_hard(ds, rs.HostBatch(b), K, len(X))
        assert e.value.code == -1
    finally:
        ctx.dataset_destroy(ds)


@pytest.mark.parametrize("F", [48, 160])
def test_soft_forward_and_adjoint(ctx, orc, F):
    import torch
    from paper_2406_01821_gb300 import rs
    X, y, K, b = workload(6, N=3001, F=F, K=2, P=24)
    for p in range(b.P):               # every label reachable: a first rule of each class
        r0 = b.set_rule_off[p]
        b.rule_class[r0] = 0
    b.set_default[:] = 1
    dl = np.random.default_rng(6).uniform(-1, 2, b.P)
    ref = orc.soft(X, y, 2, b, 0.1, dloss=dl, want_mag=True)
    ds = ctx.dataset(X, y, 2)
    try:
        db = rs.DeviceBatch.from_host(b)
        ga, gb, gt, loss = ctx.soft_bwd(ds, db, 0.1, torch.tensor(dl.astype(np.float32), device="cuda"))
        torch.cuda.synchronize()
        got = {"loss": loss.cpu().numpy(), "grad_a": ga.cpu().numpy(), "grad_b": gb.cpu().numpy(),
               "grad_t": gt.cpu().numpy()}
    finally:
        ctx.dataset_destroy(ds)
    fin = np.isfinite(ref["loss"])
    assert fin.sum() > b.P // 2
    assert np.allclose(got["loss"][fin], ref["loss"][fin], rtol=RTOL, atol=0)
    assert np.isposinf(got["loss"][~fin]).all()
    m = b.cond_op == synth.IN
    set_of_cond = np.repeat(np.arange(b.P), np.diff(b.rule_cond_off[b.set_rule_off]))
    keep = fin[set_of_cond]
    for n in ("a", "b", "t"):
        g, r, mag = got["grad_" + n], ref["grad_" + n], ref["mag_" + n]
        assert (g[m] == 0).all()
        err = np.abs(g - r)[keep]
        assert (err <= RTOL * np.maximum(np.abs(r), mag)[keep] + 1e-30).all(), n


def test_serving(ctx, orc):
    from paper_2406_01821_gb300 import rs
    X, y, K, b = workload(7, N=6007, P=40)       # fewer sets than the rank-coded units' minimum
    want = orc.eval_hard(X, y, K, b)
    ds = ctx.dataset(X, y, K)
    try:
        t1 = ctx.submit(ds, rs.HostBatch(b))
        t2 = ctx.submit(ds, rs.DeviceBatch.from_host(b))
        for t in (t1, t2):
            c, pc, _ = ctx.poll(t, b.P, K, timeout_us=60_000_000)
            assert np.array_equal(c, want[0]) and np.array_equal(pc, want[1])
        b2 = synth.Batch(**b.arrays())
        for p in range(b2.P):
            b2.rule_class[b2.set_rule_off[p]] = 0
        b2.set_default[:] = 1
        t3 = ctx.submit_soft(ds, rs.HostBatch(b2), 0.1)
        loss, _ = ctx.poll_soft(t3, b2.P, timeout_us=60_000_000)
        ref = orc.soft(X, y, K, b2, 0.1)["loss"]
        fin = np.isfinite(ref)
        assert np.allclose(loss[fin], ref[fin], rtol=RTOL, atol=0) and np.isposinf(loss[~fin]).all()
    finally:
        ctx.dataset_destroy(ds)
    Xw, yw = synth.categorical_mixture(999, 200, 3, 8, n_cat=4)      # too wide for rank-coded units
    bw = synth.random_rulesets(synth.quantile_table(Xw), 3, 8, (1, 4), (1, 3), 8, cat_from=196)
    dsw = ctx.dataset(Xw, yw, 3)
    try:
        with pytest.raises(rs.RsError) as e:
            ctx.submit(dsw, rs.HostBatch(bw))
        assert e.value.code == -6
    finally:
        ctx.dataset_destroy(dsw)
