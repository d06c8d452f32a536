"""GPU parity of the hard evaluator against the CPU oracle: bit-exact predictions and counts.

All calls go through the C ABI (librs.so via the ctypes binding)."""
import numpy as np
import pytest

from paper_2406_01821_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    assert torch.cuda.is_available()
    c = rs.Context(0)
    yield c
    c.close()


def run_gpu(ctx, X, y, K, batch, preds=True, tile=None, host=False):
    import torch
    from paper_2406_01821_gb300 import rs
    ds = ctx.dataset(X, y, K)
    try:
        if tile is not None:
            ctx.set_tile_config(tile)
        b = rs.HostBatch(batch) if host else rs.DeviceBatch.from_host(batch)
        correct, pc, pr = ctx.eval_hard(ds, b, K, len(X), per_class=True, preds=preds)
        if not host:
            torch.cuda.synchronize()
            correct, pc = correct.cpu().numpy(), pc.cpu().numpy()
            pr = pr.cpu().numpy() if pr is not None else None
        return correct, pc, pr
    finally:
        ctx.set_tile_config(-1)
        ctx.dataset_destroy(ds)


def assert_same(got, want, preds=True):
    assert np.array_equal(got[0], want[0]), "correct counts differ"
    assert np.array_equal(got[1], want[1]), "per-class counts differ"
    if preds:
        assert np.array_equal(got[2], want[2]), "predictions differ"


def test_plain_hard_config_bit_exact(ctx, orc):
    w = synth.plain_hard(seed=0)
    got = run_gpu(ctx, w.X, w.y, w.K, w.batch)
    want = orc.eval_hard(w.X, w.y, w.K, w.batch, want_preds=True)
    assert_same(got, want)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ragged_reduced_bit_exact(ctx, orc, seed):
    """The ragged 10-class workload at reduced N (ragged tail: N not a multiple of any tile)."""
    X, y = synth.gaussian_mixture(20011, 128, 10, seed)
    b = synth.random_rulesets(synth.quantile_table(X), 10, 192, (1, 64), (1, 8), seed)
    got = run_gpu(ctx, X, y, 10, b, preds=False)
    want = orc.eval_hard(X, y, 10, b)
    assert_same(got, want, preds=False)


def test_every_tile_config_identical(ctx, orc):
    from paper_2406_01821_gb300 import rs
    X, y = synth.gaussian_mixture(3001, 48, 4, 5)
    b = synth.random_rulesets(synth.quantile_table(X), 4, 40, (1, 20), (1, 6), 5)
    want = orc.eval_hard(X, y, 4, b, want_preds=True)
    for cfg in rs.tile_configs():
        got = run_gpu(ctx, X, y, 4, b, tile=cfg["id"])
        assert_same(got, want)


# one configuration of each evaluator form: condition-at-a-time, rule-at-a-time with predicate
# conjunction, with the margin minimum, the sign-mask form for finite data, and the rank-coded
# form (16 and 32 warps) for datasets with rank tables
FORMS = [0, 9, 12, 17, 21, 22]
RANKED = [21, 22]


@pytest.mark.parametrize("tile", FORMS)
@pytest.mark.parametrize("seed", range(4))
def test_boundary_crowded_inputs(ctx, orc, seed, tile):
    rng = np.random.default_rng(seed)
    F = int(rng.integers(1, 9))
    X0 = rng.standard_normal((4096, F)).astype(np.float32)
    b = synth.random_rulesets(synth.quantile_table(X0), 3, 24, (1, 8), (1, 4), seed,
                              pair_prob=0.5 if F > 1 else 0.0)
    X = synth.boundary_samples(b, F, 2500, seed, frac=0.9, ulps=2)
    y = rng.integers(0, 3, len(X)).astype(np.int32)
    got = run_gpu(ctx, X, y, 3, b, preds=False, tile=tile)
    want = orc.eval_hard(X, y, 3, b)
    assert_same(got, want, preds=False)
    got = run_gpu(ctx, X, y, 3, b)
    want = orc.eval_hard(X, y, 3, b, want_preds=True)
    assert_same(got, want)


def special_values(rng, n):
    pool = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1e-40, -1e-40, 1.17549435e-38,
                     3.4028235e38, -3.4028235e38, 1.0, -1.0, 0.5, 2.0, 1e-30, 1e30], np.float32)
    return pool[rng.integers(0, len(pool), n)]


@pytest.mark.parametrize("tile", FORMS)
def test_special_values_in_data_and_coefficients(ctx, orc, tile):
    rng = np.random.default_rng(11)
    N, F = 1500, 4
    X = rng.standard_normal((N, F)).astype(np.float32)
    mask = rng.random((N, F)) < 0.3
    X[mask] = special_values(rng, int(mask.sum()))
    b = synth.random_rulesets(synth.quantile_table(rng.standard_normal((256, F)).astype(np.float32)),
                              2, 32, (1, 6), (1, 3), 11, pair_prob=0.4)
    for arr in (b.cond_a, b.cond_b, b.cond_t):
        m = rng.random(len(arr)) < 0.25
        arr[m] = special_values(rng, int(m.sum()))
    y = rng.integers(0, 2, N).astype(np.int32)
    got = run_gpu(ctx, X, y, 2, b, tile=tile)
    want = orc.eval_hard(X, y, 2, b, want_preds=True)
    assert_same(got, want)


@pytest.mark.parametrize("tile", FORMS)
def test_special_coefficients_finite_data(ctx, orc, tile):
    """Finite data (the sign-mask form applies) with zero, infinite, NaN and extreme
    coefficients and thresholds."""
    rng = np.random.default_rng(12)
    N, F = 2000, 5
    X = (rng.standard_normal((N, F)) * rng.choice([1e-39, 1.0, 1e30], (N, F))).astype(np.float32)
    b = synth.random_rulesets(synth.quantile_table(X), 3, 40, (1, 6), (1, 4), 12, pair_prob=0.3)
    for arr in (b.cond_a, b.cond_b, b.cond_t):
        m = rng.random(len(arr)) < 0.3
        arr[m] = special_values(rng, int(m.sum()))
    y = rng.integers(0, 3, N).astype(np.int32)
    got = run_gpu(ctx, X, y, 3, b, preds=False, tile=tile)
    want = orc.eval_hard(X, y, 3, b)
    assert_same(got, want, preds=False)


@pytest.mark.parametrize("tile", FORMS)
def test_subnormal_products(ctx, orc, tile):
    """Products that land in the subnormal range must not be flushed to zero."""
    rng = np.random.default_rng(3)
    N = 2000
    X = (rng.standard_normal((N, 2)) * 1e-20).astype(np.float32)
    rules = []
    for t in (0.0, 1e-42, -1e-42, 1e-40):
        rules.append((1, [(0, -1, synth.GT, 1e-20, 0.0, t)]))
        rules.append((1, [(1, 0, synth.LT, 3e-21, 2e-19, 0.0)]))
    b = synth.from_lists([rules[i:i + 2] for i in range(0, len(rules), 2)], [0] * (len(rules) // 2))
    y = rng.integers(0, 2, N).astype(np.int32)
    got = run_gpu(ctx, X, y, 2, b, tile=tile)
    want = orc.eval_hard(X, y, 2, b, want_preds=True)
    assert_same(got, want)


@pytest.mark.parametrize("tile", FORMS)
@pytest.mark.parametrize("N,F,K", [(1, 1, 2), (31, 3, 2), (33, 5, 3), (257, 256, 2), (700, 300, 4),
                                   (129, 7, 40)])
def test_shapes(ctx, orc, N, F, K, tile):
    rng = np.random.default_rng(N + F)
    X = rng.standard_normal((N, F)).astype(np.float32)
    y = rng.integers(0, K, N).astype(np.int32)
    b = synth.random_rulesets(synth.quantile_table(X), K, 17, (1, 9), (1, 5), N, pair_prob=0.3 if F > 1 else 0)
    got = run_gpu(ctx, X, y, K, b, preds=False, tile=tile)
    want = orc.eval_hard(X, y, K, b)
    assert_same(got, want, preds=False)
    got = run_gpu(ctx, X, y, K, b)
    want = orc.eval_hard(X, y, K, b, want_preds=True)
    assert_same(got, want)


@pytest.mark.parametrize("tile", FORMS)
def test_empty_sets_rules_and_degenerate_cases(ctx, orc, tile):
    X, y = synth.two_class_gaussian(999, 4, 2)
    sets = [
        [],                                                    # empty set -> default
        [(1, [])],                                             # empty rule fires everywhere
        [(0, [(0, -1, synth.GT, 1.0, 0.0, 0.0)]), (1, []), (0, [(1, -1, synth.LT, 1.0, 0.0, 5.0)])],
        [(1, [(0, -1, synth.GT, 1.0, 0.0, np.inf)])],          # never true
        [(1, [(2, -1, synth.LT, 0.0, 0.0, 1.0)])],             # coefficient 0
        [(0, [(3, 1, synth.GT, 1.0, 1.0, 0.0)])],              # x3 > x1
        [(1, [(2, 2, synth.LT, 1.0, 1.0, 0.0)])],              # same feature both sides
    ]
    b = synth.from_lists(sets, [0, 1, 0, 1, 0, 1, 0])
    got = run_gpu(ctx, X, y, 2, b, tile=tile)
    want = orc.eval_hard(X, y, 2, b, want_preds=True)
    assert_same(got, want)


def test_zero_sets(ctx):
    X, y = synth.two_class_gaussian(100, 3, 0)
    b = synth.from_lists([], [])
    got = run_gpu(ctx, X, y, 2, b)
    assert got[0].shape == (0,)


def test_host_batch_path_matches(ctx, orc):
    w = synth.plain_hard(seed=3)
    got = run_gpu(ctx, w.X, w.y, w.K, w.batch, host=True)
    want = orc.eval_hard(w.X, w.y, w.K, w.batch, want_preds=True)
    assert_same(got, want)


def test_repeated_calls_and_graph_replay(ctx, orc):
    """Consecutive calls of different shapes on one stream (graph update path) stay exact."""
    import torch
    from paper_2406_01821_gb300 import rs
    X, y = synth.gaussian_mixture(5000, 16, 3, 9)
    ds = ctx.dataset(X, y, 3)
    s = torch.cuda.Stream()
    try:
        for seed in range(4):
            b = synth.random_rulesets(synth.quantile_table(X), 3, 20 + 7 * seed, (1, 12), (1, 5), seed)
            with torch.cuda.stream(s):
                c, pc, _ = ctx.eval_hard(ds, rs.DeviceBatch.from_host(b), 3, stream=s)
            s.synchronize()
            want = orc.eval_hard(X, y, 3, b)
            assert np.array_equal(c.cpu().numpy(), want[0])
            assert np.array_equal(pc.cpu().numpy(), want[1])
    finally:
        ctx.dataset_destroy(ds)


@pytest.mark.parametrize("what", ["feature", "pair_feature", "class", "default", "op", "offsets"])
def test_malformed_batch_rejected(ctx, what):
    from paper_2406_01821_gb300 import rs
    X, y = synth.two_class_gaussian(300, 4, 0)
    b = synth.random_rulesets(synth.quantile_table(X), 2, 6, 3, 2, 0, pair_prob=0.5)
    if what == "feature":
        b.cond_f[3] = 4
    elif what == "pair_feature":
        b.cond_g[2] = 9
    elif what == "class":
        b.rule_class[1] = 2
    elif what == "default":
        b.set_default[0] = -1
    elif what == "op":
        b.cond_op[0] = 7
    else:
        b.rule_cond_off[2] = b.rule_cond_off[3] + 1
    ds = ctx.dataset(X, y, 2)
    try:
        with pytest.raises(rs.RsError) as ei:
            ctx.eval_hard(ds, rs.DeviceBatch.from_host(b), 2)
        assert ei.value.code == -1
    finally:
        ctx.dataset_destroy(ds)


def test_threshold_rewrite_exhaustive(ctx):
    """For every float32 x: fl(a*x) op t equals the rewritten single compare."""
    a = [1.0, -1.0, 0.7, -0.3, 1e-30, -1e-30, 3e38, 1e-45, -1e-45, 2.5, 0.0, -0.0, np.inf, np.nan,
         0.5, 1.0000001]
    t = [0.38, -2.02, 1e-44, -1e-40, 1e-44, 5.0, -np.inf, 0.0, -0.0, np.inf, 1.0, -1.0, 0.3, 0.0,
         3.4e38, -1e-38]
    op = [0, 1] * 8
    mm = ctx.selftest_threshold_rewrite(np.array(a, np.float32), np.array(t, np.float32),
                                        np.array(op, np.int8))
    assert mm == 0
    # and the '<' of every pair too
    mm = ctx.selftest_threshold_rewrite(np.array(a, np.float32), np.array(t, np.float32),
                                        1 - np.array(op, np.int8))
    assert mm == 0


def test_threshold_rewrite_exhaustive_random(ctx):
    """Random coefficients and thresholds over the whole exponent range (normal products, where the
    cut is found next to t / a, and subnormal or overflowing ones, where the binary search finds
    it): for every float32 x, fl(a*x) op t equals the rewritten single compare."""
    rng = np.random.default_rng(17)
    n = 24
    a = (rng.choice([-1.0, 1.0], n) * 10.0 ** np.concatenate([rng.uniform(-3, 3, n - 8), rng.uniform(-40, 38, 8)]))
    t = (rng.choice([-1.0, 1.0], n) * 10.0 ** np.concatenate([rng.uniform(-3, 3, n - 8), rng.uniform(-45, 38, 8)]))
    op = rng.integers(0, 2, n).astype(np.int8)
    mm = ctx.selftest_threshold_rewrite(a.astype(np.float32), t.astype(np.float32), op)
    assert mm == 0


def test_ragged_full_size_sampled(ctx, orc):
    """The full ragged workload (P=4096, N=2^20, F=128, 10 classes) in the benchmark's launch
    configuration; sampled sets are recomputed one by one by the oracle, and every set satisfies
    correct = sum_k per_class <= N."""
    import torch
    from paper_2406_01821_gb300 import rs
    w = synth.ragged_hard(seed=0)
    ds = ctx.dataset(w.X, w.y, w.K)
    try:
        db = rs.DeviceBatch.from_host(w.batch)
        correct, pc, _ = ctx.eval_hard(ds, db, w.K)
        torch.cuda.synchronize()
        correct, pc = correct.cpu().numpy(), pc.cpu().numpy()
    finally:
        ctx.dataset_destroy(ds)
    assert np.array_equal(pc.sum(axis=1), correct)
    assert (correct <= w.N).all() and (correct >= 0).all()
    sample = np.random.default_rng(0).choice(w.batch.P, 6, replace=False)
    sub = w.batch.subset(sample)
    want_c, want_pc, _ = orc.eval_hard(w.X, w.y, w.K, sub)
    assert np.array_equal(correct[sample], want_c)
    assert np.array_equal(pc[sample], want_pc)


@pytest.mark.parametrize("tile", RANKED + [17])
@pytest.mark.parametrize("seed", range(3))
def test_rank_ties_and_thresholds_at_data_values(ctx, orc, tile, seed):
    """Tiles full of equal values (small integers, +0 and -0) and thresholds placed exactly on data
    values and one ulp either side: the per-tile rank counts must treat ties exactly."""
    rng = np.random.default_rng(100 + seed)
    N, F = 3000, 6
    X = rng.integers(-3, 4, (N, F)).astype(np.float32)
    X[:, 1] = np.where(rng.random(N) < 0.5, np.float32(0.0), np.float32(-0.0))
    X[:, 2] = rng.standard_normal(N).astype(np.float32)
    b = synth.random_rulesets(synth.quantile_table(X), 3, 48, (1, 12), (1, 6), seed, pair_prob=0.25)
    thr = b.cond_g < 0
    idx = np.flatnonzero(thr)
    vals = X[rng.integers(0, N, len(idx)), b.cond_f[idx]]
    a = rng.choice(np.array([1.0, -1.0, 0.5, -2.0], np.float32), len(idx))
    t = (a * vals).astype(np.float32)
    shift = rng.integers(-1, 2, len(idx))
    t = np.where(shift < 0, np.nextafter(t, np.float32(-np.inf)),
                 np.where(shift > 0, np.nextafter(t, np.float32(np.inf)), t)).astype(np.float32)
    b.cond_a[idx], b.cond_t[idx] = a, t
    y = rng.integers(0, 3, N).astype(np.int32)
    got = run_gpu(ctx, X, y, 3, b, preds=False, tile=tile)
    want = orc.eval_hard(X, y, 3, b)
    assert_same(got, want, preds=False)


@pytest.mark.parametrize("tile", RANKED + [17])
def test_long_rules_cross_the_record_window(ctx, orc, tile):
    """Rules of 30..150 conditions (longer than the 64-record stage) mixed with short ones."""
    X, y = synth.gaussian_mixture(2000, 24, 4, 7)
    b = synth.random_rulesets(synth.quantile_table(X), 4, 30, (1, 12), (30, 150), 7, pair_prob=0.05)
    # loosen the thresholds so that long rules still fire on some samples
    thr = b.cond_g < 0
    b.cond_t[thr] = np.where(b.cond_op[thr] == synth.GT, np.float32(-2.5), np.float32(2.5)) * np.abs(b.cond_a[thr])
    got = run_gpu(ctx, X, y, 4, b, preds=False, tile=tile)
    want = orc.eval_hard(X, y, 4, b)
    assert_same(got, want, preds=False)
    assert want[0].max() > 0


@pytest.mark.parametrize("tile", RANKED)
def test_many_labels_per_tile(ctx, orc, tile):
    """40 classes over 3001 samples: most 128-sample tiles hold several labels."""
    rng = np.random.default_rng(9)
    X = rng.standard_normal((3001, 9)).astype(np.float32)
    y = rng.integers(0, 40, 3001).astype(np.int32)
    b = synth.random_rulesets(synth.quantile_table(X), 40, 64, (1, 20), (1, 5), 9, pair_prob=0.2)
    got = run_gpu(ctx, X, y, 40, b, preds=False, tile=tile)
    want = orc.eval_hard(X, y, 40, b)
    assert_same(got, want, preds=False)


def test_wide_and_nonfinite_data_fall_back_from_ranks(ctx, orc):
    """Datasets without rank tables (F > 168, or NaN/inf present) run the rank-coded
    configuration as its sign-mask / margin-minimum twin, still exact."""
    rng = np.random.default_rng(4)
    for F, poison in ((200, False), (12, True)):
        X = rng.standard_normal((1500, F)).astype(np.float32)
        if poison:
            X[rng.integers(0, 1500, 20), rng.integers(0, F, 20)] = np.nan
        y = rng.integers(0, 2, 1500).astype(np.int32)
        b = synth.random_rulesets(synth.quantile_table(np.nan_to_num(X)), 2, 24, (1, 8), (1, 4), 4)
        got = run_gpu(ctx, X, y, 2, b, preds=False, tile=22)
        want = orc.eval_hard(X, y, 2, b)
        assert_same(got, want, preds=False)


@pytest.mark.parametrize("tile", RANKED)
@pytest.mark.parametrize("K", [3, 100])
def test_walk_stops_after_last_rule_of_tile_label(ctx, orc, tile, K):
    """One-label tiles stop where no later record can change their count (K <= 64): after the
    set's last rule of the tile's label when the set defaults to another class, after its last
    rule of another class when it defaults to the tile's label; with more classes the per-class
    table is not built."""
    X, y = synth.gaussian_mixture(6000, 16, K, 3)
    b = synth.random_rulesets(synth.quantile_table(X), K, 48, (1, 40), (1, 4), 3)
    # a few sets with no rule of some classes, and sets whose only rules of a class come first
    b.rule_class[: b.set_rule_off[4]] = 0
    # sets whose last rules name their default class (the stop after the last rule of another
    # class), one of them made only of such rules
    for p in range(4, 16):
        r0, r1 = b.set_rule_off[p], b.set_rule_off[p + 1]
        b.rule_class[max(r0, r1 - 1 - p % 4):r1] = b.set_default[p]
    b.rule_class[b.set_rule_off[16]:b.set_rule_off[17]] = b.set_default[16]
    got = run_gpu(ctx, X, y, K, b, preds=False, tile=tile)
    want = orc.eval_hard(X, y, K, b)
    assert_same(got, want, preds=False)


def test_maximum_sizes(ctx, orc):
    """The widest dataset (4096 features: only the configuration reading global memory fits) with
    the most classes (4096), predictions included; the longest rule (4095 conditions) in every
    evaluator form; and one condition more is refused."""
    from paper_2406_01821_gb300 import rs
    rng = np.random.default_rng(8)
    N, F, K = 700, 4096, 4096
    X = rng.standard_normal((N, F)).astype(np.float32)
    y = rng.integers(0, K, N).astype(np.int32)
    b = synth.random_rulesets(synth.quantile_table(X), K, 12, (1, 6), (1, 4), 8, pair_prob=0.3)
    got = run_gpu(ctx, X, y, K, b)
    want = orc.eval_hard(X, y, K, b, want_preds=True)
    assert_same(got, want)

    X, y = synth.two_class_gaussian(3000, 8, 9)
    def long_rule(n):
        conds = [(j % 8, -1, synth.GT, 1.0, 0.0, -3.0 - j * 1e-3) for j in range(n)]   # nearly always true
        return [[(1, conds), (0, [(0, -1, synth.GT, 1.0, 0.0, 0.0)])]]
    b = synth.from_lists(long_rule(4095), [0])
    want = orc.eval_hard(X, y, 2, b, want_preds=True)
    assert want[0][0] > 0
    for tile in FORMS:
        assert_same(run_gpu(ctx, X, y, 2, b, preds=False, tile=tile), want, preds=False)
    b = synth.from_lists(long_rule(4096), [0])
    with pytest.raises(rs.RsError) as ei:
        run_gpu(ctx, X, y, 2, b, preds=False)
    assert ei.value.code == -2                     # RS_ERR_TOO_LARGE


def test_graph_replay_reads_current_contents(ctx, orc):
    """On a caller's stream a call shape runs directly the first time, is captured when the next
    call repeats it, and is replayed after that; every path must read the batch's current contents
    (device arrays rewritten in place, host arrays staged again) and write the current outputs, and
    count the same kernels. Then batches of other sizes and the first one again."""
    import copy
    import torch
    from paper_2406_01821_gb300 import rs
    X, y = synth.gaussian_mixture(7001, 12, 3, 31)
    K = 3
    ds = ctx.dataset(X, y, K)
    s = torch.cuda.Stream()
    rng = np.random.default_rng(31)
    b0 = synth.random_rulesets(synth.quantile_table(X), K, 40, (1, 10), (1, 4), 31, pair_prob=0.3)
    variants = [b0]
    for _ in range(3):
        bv = copy.deepcopy(b0)
        bv.cond_t = rng.permutation(bv.cond_t).astype(np.float32)
        bv.set_default = rng.integers(0, K, size=b0.P).astype(np.int32)
        variants.append(bv)
    try:
        db = rs.DeviceBatch.from_host(b0)
        out = (torch.empty(b0.P, dtype=torch.int32, device="cuda"),
               torch.empty((b0.P, K), dtype=torch.int32, device="cuda"), None)
        launches = []
        for bv in variants:                       # device arrays rewritten in place
            db.t["cond_t"].copy_(torch.from_numpy(bv.cond_t))
            db.t["set_default"].copy_(torch.from_numpy(bv.set_default))
            before = ctx.profile()["launches"]
            with torch.cuda.stream(s):
                c, pc, _ = ctx.eval_hard(ds, db, K, out=out, stream=s)
            s.synchronize()
            launches.append(ctx.profile()["launches"] - before)
            want = orc.eval_hard(X, y, K, bv)
            assert np.array_equal(c.cpu().numpy(), want[0])
            assert np.array_equal(pc.cpu().numpy(), want[1])
        assert len(set(launches)) == 1 and launches[0] > 0   # a replay counts the kernels it runs
        for bv in variants:                       # host arrays, host outputs
            c, pc, _ = ctx.eval_hard(ds, rs.HostBatch(bv), K, stream=s)
            want = orc.eval_hard(X, y, K, bv)
            assert np.array_equal(c, want[0]) and np.array_equal(pc, want[1])
        b1 = synth.random_rulesets(synth.quantile_table(X), K, 9, (1, 30), (1, 6), 32)
        for bv in (b1, variants[2], b1):          # other sizes: captured again, same entry
            c, pc, _ = ctx.eval_hard(ds, rs.HostBatch(bv), K, stream=s)
            want = orc.eval_hard(X, y, K, bv)
            assert np.array_equal(c, want[0]) and np.array_equal(pc, want[1])
    finally:
        ctx.dataset_destroy(ds)


def test_work_counters_of_the_rank_coded_walk(orc):
    """A work-counting context reports what the rank-coded evaluator walked: with conditions that
    never hold (no early exit) every record of every rule is walked on every 128-sample tile."""
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    X, y = synth.two_class_gaussian(1000, 6, 3)
    big = np.float32(X.max() + 1.0)
    never = (0, -1, synth.GT, np.float32(1.0), 0.0, big)            # x0 > max(x): never true
    pair = (1, 2, synth.GT, np.float32(0.0), np.float32(1.0), 0.0)  # 0 * x1 > x2: a pair row
    rules = [(0, [never, pair]), (1, [never, never]), (0, [pair, never])]
    b = synth.from_lists([rules], [1])
    tiles = (len(X) + 127) // 128
    with rs.Context(0, flags=rs.CTX_COUNT_WORK | rs.CTX_NO_GRAPH) as ctx:
        ds = ctx.dataset(X, y, 2)
        ctx.set_tile_config(22)
        ctx.profile(reset=True)
        c, _, _ = ctx.eval_hard(ds, rs.DeviceBatch.from_host(b), 2)
        torch.cuda.synchronize()
        p = ctx.profile(reset=True)
        ctx.dataset_destroy(ds)
    assert c.cpu().numpy().tolist() == orc.eval_hard(X, y, 2, b)[0].tolist()
    assert p["hard_set_tiles"] == tiles
    assert p["hard_records_walked"] == 6 * tiles
    assert p["hard_rule_ends_walked"] == 3 * tiles
    assert p["hard_rows_walked"] == 2 * tiles


def test_class_tail_stop_counts_records(orc):
    """The class-tail stop, counted: with three labels and a set defaulting to class 2 whose rules
    never fire, a one-label tile of label 0 walks only the first rule, label 1 the first two, and
    label 2 also the first two (every later rule names the default's class); tiles holding
    several labels walk everything."""
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    X, y = synth.gaussian_mixture(3000, 6, 3, 8)
    never = (0, -1, synth.GT, np.float32(1.0), 0.0, np.float32(X.max() + 1.0))
    b = synth.from_lists([[(0, [never]), (1, [never]), (2, [never, never])]], [2])
    ys = np.sort(y)
    ys = np.concatenate([ys, np.full((-len(ys)) % 128, -1)])
    want = 0
    for t in ys.reshape(-1, 128):
        lab = t[t >= 0]
        want += 4 if lab.min() != lab.max() else {0: 1, 1: 2, 2: 2}[int(lab[0])]
    with rs.Context(0, flags=rs.CTX_COUNT_WORK | rs.CTX_NO_GRAPH) as ctx:
        ds = ctx.dataset(X, y, 3)
        ctx.set_tile_config(22)
        ctx.profile(reset=True)
        c, pc, _ = ctx.eval_hard(ds, rs.DeviceBatch.from_host(b), 3)
        torch.cuda.synchronize()
        p = ctx.profile(reset=True)
        ctx.dataset_destroy(ds)
    ref = orc.eval_hard(X, y, 3, b)
    assert c.cpu().numpy().tolist() == ref[0].tolist()
    assert p["hard_records_walked"] == want


def test_measured_pipe_rates():
    """The pipe-rate measurement: every stream runs, the FP32 FMA rate is within the FP32 lanes'
    nominal peak (128 per SM at the maximum clock) and above half of it."""
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    with rs.Context(0) as ctx:
        r = ctx.pipe_rates()
    prop = torch.cuda.get_device_properties(0)
    nominal = prop.multi_processor_count * 128 * 2.1e9
    assert 0.5 * nominal < r["ffma"] <= 1.05 * nominal, r
    assert all(v > 0 for v in r.values()), r
