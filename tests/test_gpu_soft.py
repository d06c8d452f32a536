"""GPU parity of the soft path (sigmoid-relaxed forward and hand-written adjoint) against the
float64 oracle.

Tolerance (float32 against float64): loss within 1e-5 relative; each gradient element within
1e-5 x max(|g64|, m64), where m64 = |dloss| (1/N) sum_n |d ell_n / d theta| is the scale of the
cancelling sum over samples that float32 round-off is measured against."""
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


def soft_gpu(ctx, X, y, K, b, tau, dloss, probs=False):
    import torch
    from paper_2406_01821_gb300 import rs
    ds = ctx.dataset(X, y, K)
    try:
        db = rs.DeviceBatch.from_host(b)
        dl = torch.tensor(np.asarray(dloss, np.float32), device="cuda")
        ga, gb, gt, loss = ctx.soft_bwd(ds, db, tau, dl)
        out = {"loss": loss, "grad_a": ga, "grad_b": gb, "grad_t": gt}
        if probs:
            lf, pr = ctx.soft_fwd(ds, db, tau, N=len(X), K=K, probs=True)
            out["loss_fwd"], out["probs"] = lf, pr
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        ctx.dataset_destroy(ds)


def check_against_oracle(got, ref):
    assert np.allclose(got["loss"], ref["loss"], rtol=RTOL, atol=0), \
        np.max(np.abs(got["loss"] / ref["loss"] - 1))
    for n in ("a", "b", "t"):
        g, r, m = got["grad_" + n], ref["grad_" + n], ref["mag_" + n]
        err = np.abs(g - r)
        bound = RTOL * np.maximum(np.abs(r), m) + 1e-30
        assert (err <= bound).all(), (n, float(np.max(err / bound)))


def reachable(b):
    b.set_default[:] = np.where(b.rule_class[b.set_rule_off[:-1]] == 0, 1, 0)
    return b


@pytest.mark.parametrize("seed", [0, 1])
def test_soft_small_vs_oracle(ctx, orc, seed):
    X, y = synth.two_class_gaussian(3001, 8, seed)
    b = reachable(synth.random_rulesets(synth.quantile_table(X), 2, 12, (1, 8), (1, 4), seed))
    dl = np.random.default_rng(seed).uniform(-1, 2, b.P)
    got = soft_gpu(ctx, X, y, 2, b, 0.1, dl)
    ref = orc.soft(X, y, 2, b, 0.1, dloss=dl, want_mag=True)
    check_against_oracle(got, ref)


@pytest.mark.parametrize("F,P", [(160, 12), (33, 29)])
def test_soft_wide_and_odd_shapes_vs_oracle(ctx, orc, F, P):
    """F > 128 runs the per-warp kernel (features read from global memory); F <= 128 the
    staged-tile kernel, here with a set count that leaves idle warps in the last CTA group."""
    X, y = synth.two_class_gaussian(2333, F, 5)
    b = reachable(synth.random_rulesets(synth.quantile_table(X), 2, P, (1, 8), (1, 4), 5, pair_prob=0.3))
    dl = np.random.default_rng(5).uniform(-1, 2, b.P)
    got = soft_gpu(ctx, X, y, 2, b, 0.1, dl)
    ref = orc.soft(X, y, 2, b, 0.1, dloss=dl, want_mag=True)
    check_against_oracle(got, ref)


def test_soft_multiclass_probs(ctx, orc):
    rng = np.random.default_rng(4)
    X, _ = synth.gaussian_mixture(777, 6, 4, 4)
    y = rng.integers(0, 4, len(X)).astype(np.int32)
    b = synth.random_rulesets(synth.quantile_table(X), 4, 6, (3, 6), (1, 3), 4, default=3)
    for p in range(b.P):      # classes 0..2 on the first rules, 3 by default: all reachable
        r0 = b.set_rule_off[p]
        b.rule_class[r0:r0 + 3] = np.arange(3)
    got = soft_gpu(ctx, X, y, 4, b, 0.5, np.ones(b.P), probs=True)
    ref = orc.soft(X, y, 4, b, 0.5, dloss=np.ones(b.P), want_probs=True, want_mag=True)
    assert np.allclose(got["probs"].sum(axis=2), 1.0, atol=1e-5)
    assert np.allclose(got["probs"], ref["probs"], rtol=RTOL, atol=1e-30)
    assert np.array_equal(got["loss_fwd"], got["loss"])     # the forward and the fused pass agree
    check_against_oracle(got, ref)


def test_soft_ragged_and_pairs(ctx, orc):
    X, y = synth.two_class_gaussian(2049, 16, 7)
    b = reachable(synth.random_rulesets(synth.quantile_table(X), 2, 20, (1, 32), (1, 8), 7, pair_prob=0.5))
    got = soft_gpu(ctx, X, y, 2, b, 0.25, np.ones(b.P))
    ref = orc.soft(X, y, 2, b, 0.25, dloss=np.ones(b.P), want_mag=True)
    check_against_oracle(got, ref)


def _as_lists(b):
    sets = []
    for p in range(b.P):
        rules = []
        for r in range(b.set_rule_off[p], b.set_rule_off[p + 1]):
            conds = [(int(b.cond_f[c]), int(b.cond_g[c]), int(b.cond_op[c]), b.cond_a[c], b.cond_b[c], b.cond_t[c])
                     for c in range(b.rule_cond_off[r], b.rule_cond_off[r + 1])]
            rules.append((int(b.rule_class[r]), conds))
        sets.append(rules)
    return sets


@pytest.mark.parametrize("F", [8, 160])
def test_soft_rule_that_always_fires(ctx, orc, F):
    """A rule without conditions (q = 1) in the middle of a set: no later rule and not the default
    can be reached (their share and gradients are exactly 0, log of 'no earlier rule fired' is -inf
    after it), in the staged-tile and the per-warp kernel, against the oracle."""
    X, y = synth.two_class_gaussian(2500, F, 11)
    b = synth.random_rulesets(synth.quantile_table(X), 2, 14, (5, 12), (1, 4), 11, pair_prob=0.3)
    sets = _as_lists(b)
    for p, rules in enumerate(sets):
        rules[0] = (0, rules[0][1])
        rules[1] = (1, rules[1][1])                     # both labels reachable before the empty rule
        j = 2 + p % (len(rules) - 2)
        rules[j] = (rules[j][0], [])                    # fires on every sample that reaches it
    b = synth.from_lists(sets, [int(d) for d in b.set_default])
    dl = np.random.default_rng(11).uniform(-1, 2, b.P)
    got = soft_gpu(ctx, X, y, 2, b, 0.1, dl)
    ref = orc.soft(X, y, 2, b, 0.1, dloss=dl, want_mag=True)
    assert np.isfinite(ref["loss"]).all()
    check_against_oracle(got, ref)
    after = np.zeros(b.C, bool)                          # conditions of rules after the empty one
    for p in range(b.P):
        rs_ = range(b.set_rule_off[p], b.set_rule_off[p + 1])
        e = next(r for r in rs_ if b.rule_cond_off[r + 1] == b.rule_cond_off[r])
        after[b.rule_cond_off[e]:b.rule_cond_off[b.set_rule_off[p + 1]]] = True
    assert after.any()
    for n in ("a", "b", "t"):
        assert (got["grad_" + n][after] == 0).all() and (ref["grad_" + n][after] == 0).all()


@pytest.mark.parametrize("F", [8, 160])
def test_unreachable_label_gives_infinite_loss(ctx, orc, F):
    """Sets where some sample's label has no rule and is not the default: the loss is +inf, as
    in the oracle (not NaN), in both the staged-tile (F <= 128) and the per-warp kernel; the other
    sets of the batch are unaffected."""
    import torch
    from paper_2406_01821_gb300 import rs
    X, y = synth.gaussian_mixture(4000, F, 3, 9)
    b = synth.random_rulesets(synth.quantile_table(X), 2, 40, (2, 8), (1, 4), 9)   # classes 0, 1 only
    for p in range(b.P):
        r0 = b.set_rule_off[p]
        b.rule_class[r0:r0 + 2] = (0, 1)
    b.set_default[::2] = 2                                 # even sets: every label reachable
    ref = orc.soft(X, y, 3, b, 0.1)
    ds = ctx.dataset(X, y, 3)
    try:
        loss, _ = ctx.soft_fwd(ds, rs.DeviceBatch.from_host(b), 0.1)
        torch.cuda.synchronize()
        loss = loss.cpu().numpy()
    finally:
        ctx.dataset_destroy(ds)
    assert np.isposinf(ref["loss"][1::2]).all() and np.isfinite(ref["loss"][::2]).all()
    assert np.isposinf(loss[1::2]).all()
    assert np.allclose(loss[::2], ref["loss"][::2], rtol=RTOL, atol=0)


def test_soft_is_deterministic(ctx):
    X, y = synth.two_class_gaussian(5000, 8, 1)
    b = reachable(synth.random_rulesets(synth.quantile_table(X), 2, 16, (1, 8), (1, 4), 1))
    g1 = soft_gpu(ctx, X, y, 2, b, 0.1, np.ones(b.P))
    g2 = soft_gpu(ctx, X, y, 2, b, 0.1, np.ones(b.P))
    for k in g1:
        assert np.array_equal(g1[k], g2[k]), k


def test_autograd_function(ctx, orc):
    import torch
    from paper_2406_01821_gb300 import rs
    X, y = synth.two_class_gaussian(1500, 6, 2)
    b = reachable(synth.random_rulesets(synth.quantile_table(X), 2, 5, (1, 6), (1, 3), 2))
    ds = ctx.dataset(X, y, 2)
    try:
        st = rs.DeviceBatch.from_host(b)
        a = st.t["cond_a"].clone().requires_grad_(True)
        bb = st.t["cond_b"].clone().requires_grad_(True)
        t = st.t["cond_t"].clone().requires_grad_(True)
        loss = rs.rule_soft_loss(a, bb, t, ctx, ds, st, 0.1)
        w = torch.linspace(0.5, 1.5, b.P, device="cuda")
        (loss * w).sum().backward()
        ref = orc.soft(X, y, 2, b, 0.1, dloss=w.cpu().numpy().astype(np.float64), want_mag=True)
        got = {"loss": loss.detach().cpu().numpy(), "grad_a": a.grad.cpu().numpy(),
               "grad_b": bb.grad.cpu().numpy(), "grad_t": t.grad.cpu().numpy()}
        check_against_oracle(got, ref)
    finally:
        ctx.dataset_destroy(ds)


def test_soft_rejects_malformed(ctx):
    from paper_2406_01821_gb300 import rs
    import torch
    X, y = synth.two_class_gaussian(100, 3, 0)
    b = synth.random_rulesets(synth.quantile_table(X), 2, 3, 2, 2, 0)
    b.cond_f[0] = 3
    ds = ctx.dataset(X, y, 2)
    try:
        with pytest.raises(rs.RsError):
            ctx.soft_bwd(ds, rs.DeviceBatch.from_host(b), 0.1, torch.ones(3, device="cuda"))
    finally:
        ctx.dataset_destroy(ds)


def test_soft_full_size_sampled(ctx, orc):
    """The fine-tuning workload at full size (P=1024 x R=32 x C=4, N=262144, F=64, tau=0.1):
    loss and gradients of sampled sets against the float64 oracle."""
    import torch
    from paper_2406_01821_gb300 import rs
    w = synth.soft_tune(seed=0)
    b = reachable(w.batch)
    ds = ctx.dataset(w.X, w.y, w.K)
    try:
        db = rs.DeviceBatch.from_host(b)
        dl = torch.ones(b.P, device="cuda")
        ga, gb, gt, loss = ctx.soft_bwd(ds, db, w.tau, dl)
        torch.cuda.synchronize()
        got_all = {"loss": loss.cpu().numpy(), "grad_a": ga.cpu().numpy(),
                   "grad_b": gb.cpu().numpy(), "grad_t": gt.cpu().numpy()}
    finally:
        ctx.dataset_destroy(ds)
    sample = np.array([0, 517, 1023])
    sub = b.subset(sample)
    ref = orc.soft(w.X, w.y, w.K, sub, w.tau, dloss=np.ones(len(sample)), want_mag=True)
    conds = np.concatenate([np.arange(b.rule_cond_off[b.set_rule_off[p]],
                                      b.rule_cond_off[b.set_rule_off[p + 1]]) for p in sample])
    got = {"loss": got_all["loss"][sample]}
    for n in ("a", "b", "t"):
        got["grad_" + n] = got_all["grad_" + n][conds]
    check_against_oracle(got, ref)


# ------------------------------------------------- large margins (fine-tuned coefficients)

def large_margin_sets(M):
    """Sets whose samples meet rules with margins of about M tau (tau = 0.1; x0..x2 in [0.5, 1.5])
    before the rule of their label: a single huge condition, a rule of three huge conditions (where
    1 - q rounds to 0 in float32 and must come from the margins), two huge rules in a row, a rule
    that is huge only on some samples, and mixed signs."""
    A = np.float32(M / 10.0)
    mod = (3, -1, synth.GT, np.float32(0.7), 0.0, np.float32(0.1))          # a moderate condition
    T = lambda f, a, op=synth.GT: (f, -1, op, np.float32(a), 0.0, np.float32(0.0))
    sets = [
        [(0, [T(0, A)]), (1, [mod])],                                        # huge, then the label
        [(0, [T(0, A), T(1, 1.3 * A), T(2, 0.7 * A)]), (1, [mod])],          # all three huge
        [(0, [T(0, A)]), (0, [T(1, A)]), (1, [mod])],                        # two huge rules
        [(1, [T(0, A), T(3, 3.0)]), (0, [T(2, -A, synth.LT)]), (1, [mod])],  # huge '<' with -a
        [(0, [T(0, A), T(3, A)])],                                           # sign of x3 decides
    ]
    return synth.from_lists(sets, [1, 1, 0, 0, 1])


def large_margin_data(N, seed):
    rng = np.random.default_rng(seed)
    X = np.empty((N, 4), np.float32)
    X[:, :3] = rng.uniform(0.5, 1.5, (N, 3))
    X[:, 3] = rng.normal(size=N)
    y = rng.integers(0, 2, N).astype(np.int32)
    return X, y


@pytest.mark.parametrize("M", [50.0, 103.0, 200.0, 1000.0])
def test_soft_large_margins_vs_oracle(ctx, orc, M):
    """Margins of 50 to 1000 tau on every sample of some rules: loss and gradients within the
    soft tolerance of the float64 oracle (pinned at such margins by closed forms and
    arbitrary-precision references), class probabilities within 1e-5 relative."""
    X, y = large_margin_data(5003, int(M))
    b = large_margin_sets(M)
    tau = np.float32(0.1)
    dl = np.linspace(0.5, 1.5, b.P)
    got = soft_gpu(ctx, X, y, 2, b, tau, dl, probs=True)
    ref = orc.soft(X, y, 2, b, tau, dloss=dl, want_mag=True, want_probs=True)
    assert np.isfinite(got["loss"]).all() and np.isfinite(ref["loss"]).all()
    assert (ref["loss"] > 0.2 * M).any()              # the huge margins reach the loss
    check_against_oracle(got, ref)
    assert np.array_equal(got["loss_fwd"], got["loss"])
    assert np.allclose(got["probs"], ref["probs"], rtol=RTOL, atol=1e-30)


def test_soft_fig1c_rule_vs_oracle(ctx, orc):
    """The fine-tuned rule set of Fig. 1c (pair coefficient -7275.88) on data of the worked
    example's scale: margins of thousands of tau on the pair condition."""
    rng = np.random.default_rng(11)
    N = 4001
    X = np.stack([rng.uniform(6, 28, N),            # mean radius
                  rng.uniform(0.001, 0.03, N),      # fractal dimension error
                  rng.uniform(0.03, 1.06, N),       # worst compactness
                  rng.uniform(0.15, 0.66, N),       # worst symmetry
                  rng.uniform(0.75, 22.0, N),       # perimeter error
                  rng.uniform(140, 2500, N)], axis=1).astype(np.float32)
    y = rng.integers(0, 2, N).astype(np.int32)
    f = np.float32
    rules = [(0, [(0, -1, synth.GT, f(1), 0.0, f(0.06)), (1, 2, synth.GT, f(-1), f(-7275.88), 0.0),
                  (3, -1, synth.GT, f(1), 0.0, f(-3.69))]),
             (1, [(4, -1, synth.GT, f(-1), 0.0, f(-0.98)), (5, -1, synth.GT, f(-1), 0.0, f(-0.24))])]
    b = synth.from_lists([rules, rules[::-1]], [1, 0])
    for tau in (0.1, 1.0):
        got = soft_gpu(ctx, X, y, 2, b, tau, np.ones(b.P))
        ref = orc.soft(X, y, 2, b, tau, dloss=np.ones(b.P), want_mag=True)
        assert np.isfinite(got["loss"]).all()
        check_against_oracle(got, ref)


def test_log1p_unit_against_float64(ctx):
    """The soft kernels' log(1 + e) on [0, 1] (e p(e), p the degree-8 Remez fit of log1p(e) / e)
    against float64 log1p, on every float32 in [1, 2^-26] at a stride of 61 bit patterns plus the
    edges: at most 2.5 ulp of the float32 result (the documented bound is 2)."""
    from paper_2406_01821_gb300 import rs
    lo, hi = np.float32(2.0 ** -26).view(np.uint32), np.float32(1.0).view(np.uint32)
    bits = np.concatenate([np.arange(lo, hi + 1, 61, dtype=np.uint32),
                           np.array([0, 1, hi - 1, hi], np.uint32),
                           np.float32([2.0 ** -24, 2.0 ** -23, 0.5, 0.25]).view(np.uint32)])
    e = bits.view(np.float32)
    out = np.empty_like(e)
    rs.check(rs.lib().rs_selftest_log1p_unit(ctx.h, rs._ptr(e), len(e), rs._ptr(out)))
    ref = np.log1p(e.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    err = np.abs(out.astype(np.float64) - ref) / ulp
    assert err.max() <= 2.5, (float(err.max()), float(e[np.argmax(err)]))
    assert out[e == 0].tolist() == [0.0]


def test_log1m_exp_against_float64(ctx):
    """The soft forward's log(1 - e^s) (a polynomial in q = e^s for q <= e^-1/2, log t + t b(t) with
    a range-reduced hardware logarithm for t = -s < 1/2) against float64 log(-expm1(s)) for s from
    -100 to -1e-38, both sides of the split and the special values: an absolute error of at most
    4e-7 plus one ulp of the result (the log domain: lu sums these terms), and a relative error of
    at most 1e-5 where e^s is a normal float (s >= -80)."""
    from paper_2406_01821_gb300 import rs
    rng = np.random.default_rng(3)
    t = np.concatenate([10.0 ** rng.uniform(-38, 2, 200_000), rng.uniform(0.3, 0.7, 50_000),
                        rng.uniform(0, 100, 50_000)]).astype(np.float32)
    half = np.float32(0.5)
    t = np.concatenate([t, np.float32([half, np.nextafter(half, np.float32(0)), np.nextafter(half, np.float32(1)),
                                       1e-45, 1e-40, 2.0 ** -126, 87.0, 100.0])])
    s = -t
    out = np.empty_like(s)
    rs.check(rs.lib().rs_selftest_log1m_exp(ctx.h, rs._ptr(s), len(s), rs._ptr(out)))
    sd = s.astype(np.float64)
    # float64 reference in the form that is accurate on each side (1 - e^s rounds to 1 for s << 0)
    with np.errstate(divide="ignore"):
        ref = np.where(sd < -np.log(2.0), np.log1p(-np.exp(sd)), np.log(-np.expm1(np.minimum(sd, -1e-300))))
    got = out.astype(np.float64)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    err = np.abs(got - ref)
    assert (err <= 4e-7 + ulp).all(), (float((err - ulp).max()), float(s[np.argmax(err - ulp)]))
    normal = sd >= -80.0
    rel = err[normal] / np.abs(ref[normal])
    assert rel.max() <= 1e-5, (float(rel.max()), float(s[normal][np.argmax(rel)]))
    sp = np.float32([0.0, -0.0, -np.inf])
    o = np.empty_like(sp)
    rs.check(rs.lib().rs_selftest_log1m_exp(ctx.h, rs._ptr(sp), 3, rs._ptr(o)))
    assert o[0] == -np.inf and o[1] == -np.inf and o[2] == 0.0
