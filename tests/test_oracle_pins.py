"""Pins for the CPU oracle: each check compares it with something other than itself.

* Fig. 1 worked example (Sec. 3, Fig. 1a/1b/1c): decoding the tensor rows, their readable form,
  hand-placed points on both sides of every boundary, the first-fire order, and the sign-flipped
  tuned form of Fig. 1c.
* The paper's dense tensor form  sum_j w_j x_j + bias > 0  (Sec. 3), evaluated the way a matrix
  product would be (float32 products and left-to-right sums), vectorised with numpy, against the
  oracle's compare form on boundary-crowded inputs.
* A single-condition set reduces to a numpy one-liner; invariants of the counts.
* Soft path: probabilities sum to one; one rule with one or two conditions is logistic regression
  (closed form via scipy's expit); the linear-domain product form agrees with the log domain;
  tau -> 0 recovers the hard predictions; central finite differences pin the adjoint.
"""
import os

import numpy as np
import pytest
from scipy.special import expit, log_expit

from paper_2406_01821_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1.txt")
FEATS = ["mean radius", "fractal dimension error", "worst compactness", "worst symmetry",
         "perimeter error", "mean area"]
CLASSES = {"malignant": 0, "benign": 1}


# ------------------------------------------------------------------------ Fig. 1 fixtures

def read_fig1():
    sec, out = None, {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.rstrip("\n")
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                sec = line.strip("[]")
                out[sec] = []
                continue
            out[sec].append(line)
    return out


def decode_rows(lines):
    """Fig. 1a rows -> rules of conditions (f, g, op, a, b, t).

    A row with one non-zero weight w at f and bias beta reads w*x_f + beta > 0, i.e. a threshold
    condition a*x_f > t with a = w, t = -beta. A row with two non-zeros reads w_f x_f + w_g x_g > 0,
    i.e. a*x_f > b*x_g with a = w_f, b = -w_g (Sec. 3: "[0, 1.0, -0.38, 0, 0, 0] with a bias of 0").
    """
    rules = []
    for ln in lines:
        tok = ln.split()
        if tok[0] == "rule":
            rules.append((CLASSES[tok[3]], []))
            continue
        w = [float(v) for v in tok[1:7]]
        bias = float(tok[8])
        nz = [j for j, v in enumerate(w) if v != 0.0]
        if len(nz) == 1:
            f = nz[0]
            rules[-1][1].append((f, -1, synth.GT, w[f], 0.0, -bias))
        else:
            f, g = nz
            assert bias == 0.0
            rules[-1][1].append((f, g, synth.GT, w[f], -w[g], 0.0))
    return rules


def fmt(v):
    return f"{v:.2f}"


def render(rules):
    """Readable form in the layout of Fig. 1b/1c."""
    names = {v: k for k, v in CLASSES.items()}
    out = []
    for i, (cls, conds) in enumerate(rules):
        parts = []
        for f, g, op, a, b, t in conds:
            sym = ">" if op == synth.GT else "<"
            lhs = FEATS[f] if a == 1.0 else ("-" + FEATS[f] if a == -1.0 else f"{fmt(a)} x {FEATS[f]}")
            rhs = fmt(t) if g < 0 else f"{fmt(b)} x {FEATS[g]}"
            parts.append(f"({lhs} {sym} {rhs})")
        out.append(f"{i + 1}. " + " & ".join(parts) + f" -> {names[cls]}")
    return out


def parse_readable(lines):
    """Fig. 1c text -> rules (inverse of ``render`` for unit coefficients)."""
    rules = []
    for ln in lines:
        body, cls = ln.split(" -> ")
        body = body.split(". ", 1)[1]
        conds = []
        for part in body.split(" & "):
            lhs, rhs = part.strip("()").split(" > ")
            a = -1.0 if lhs.startswith("-") else 1.0
            f = FEATS.index(lhs.lstrip("-"))
            if " x " in rhs:
                b, name = rhs.split(" x ")
                conds.append((f, FEATS.index(name), synth.GT, a, float(b), 0.0))
            else:
                conds.append((f, -1, synth.GT, a, 0.0, float(rhs)))
        rules.append((CLASSES[cls], conds))
    return rules


def test_fig1a_decodes_to_fig1b():
    fig = read_fig1()
    rules = decode_rows(fig["a"])
    assert [len(c) for _, c in rules] == [3, 2]
    assert render(rules) == fig["b"]


def test_fig1c_roundtrip():
    fig = read_fig1()
    rules = parse_readable(fig["c"])
    assert render(rules) == fig["c"]


def _points_fig1b():
    """Hand-placed 6-feature points and the class Fig. 1b assigns them (7 = the default)."""
    base = [3.0, 1.0, 1.0, 0.5, 0.5, 0.5]          # satisfies rule 1 and rule 2
    f32 = np.float32
    cases = [
        ({}, 0),                                    # both rules fire -> the first wins
        ({0: 2.03}, 0),                             # just above 2.02
        ({0: f32(2.02)}, 1),                        # on the boundary: false -> rule 2
        ({0: 2.01}, 1),                             # below -> rule 2
        ({1: 0.39, 2: 1.0}, 0),                     # 0.39 > 0.38 x 1.0
        ({1: 0.37, 2: 1.0}, 1),                     # 0.37 < 0.38 x 1.0 -> rule 2
        ({1: f32(0.38), 2: 1.0}, 1),                # on the pair boundary: false -> rule 2
        ({3: 0.30}, 0),
        ({3: 0.28}, 1),
        ({3: 0.28, 4: 0.42}, 7),                    # neither rule -> default
        ({3: 0.28, 5: f32(0.29)}, 7),               # mean area on its boundary -> default
    ]
    pts, want = [], []
    for changes, cls in cases:
        x = list(base)
        for j, v in changes.items():
            x[j] = v
        pts.append(x)
        want.append(cls)
    return np.array(pts, np.float32), want


@pytest.mark.parametrize("default", [0, 1])
def test_fig1b_points(orc, default):
    rules = decode_rows(read_fig1()["a"])
    batch = synth.from_lists([rules], [default])
    X, want = _points_fig1b()
    want = [default if w == 7 else w for w in want]
    y = np.zeros(len(X), np.int32)
    _, _, preds = orc.eval_hard(X, y, 2, batch, want_preds=True)
    assert preds[0].tolist() == want


def test_fig1c_sign_flip_equivalence(orc):
    """-x > -c (Fig. 1c) is the same test as x < c; the large pair coefficient stays exact."""
    rules_c = parse_readable(read_fig1()["c"])
    flipped = []
    for cls, conds in rules_c:
        nc = []
        for f, g, op, a, b, t in conds:
            if a == -1.0:
                nc.append((f, g, synth.LT, 1.0, -b, -t))
            else:
                nc.append((f, g, op, a, b, t))
        flipped.append((cls, nc))
    rng = np.random.default_rng(5)
    X = rng.standard_normal((4000, 6)).astype(np.float32) * 3
    X[:100, 1] = np.float32(7275.88) * X[:100, 2]        # exactly on the pair boundary
    y = rng.integers(0, 2, 4000).astype(np.int32)
    b1 = synth.from_lists([rules_c], [1])
    b2 = synth.from_lists([flipped], [1])
    _, _, p1 = orc.eval_hard(X, y, 2, b1, want_preds=True)
    _, _, p2 = orc.eval_hard(X, y, 2, b2, want_preds=True)
    assert np.array_equal(p1, p2)
    # a direct reading of rule 1 of Fig. 1c
    r1 = (X[:, 0] > np.float32(0.06)) & (-X[:, 1] > np.float32(-7275.88) * X[:, 2]) \
        & (X[:, 3] > np.float32(-3.69))
    r2 = (-X[:, 4] > np.float32(-0.98)) & (-X[:, 5] > np.float32(-0.24))
    want = np.where(r1, 0, np.where(r2, 1, 1))
    assert np.array_equal(p1[0], want)


# ------------------------------------------------------------------- dense tensor form

def dense_eval(X, batch):
    """The paper's tensor evaluation (Sec. 3): one dense row per condition, margin
    z = sum_j w_j x_j + bias in float32 (products rounded, summed left to right), z > 0 true;
    rule = all its rows true; prediction = first firing rule, else default. '<' is the negated row.
    """
    N, F = X.shape
    C = batch.C
    truth = np.zeros((C, N), bool)
    for c in range(C):
        w = np.zeros(F, np.float32)
        f, g = int(batch.cond_f[c]), int(batch.cond_g[c])
        a, b, t = batch.cond_a[c], batch.cond_b[c], batch.cond_t[c]
        if g < 0:
            w[f] = a
            bias = -t
        else:
            w[f] = a
            w[g] = -b
            bias = np.float32(0)
        if batch.cond_op[c] == synth.LT:
            w, bias = -w, -bias
        z = np.zeros(N, np.float32)
        for j in range(F):
            z = (z + (w[j] * X[:, j]).astype(np.float32)).astype(np.float32)
        z = (z + np.float32(bias)).astype(np.float32)
        truth[c] = z > 0
    fires = np.ones((batch.R, N), bool)
    for r in range(batch.R):
        c0, c1 = batch.rule_cond_off[r], batch.rule_cond_off[r + 1]
        if c1 > c0:
            fires[r] = truth[c0:c1].all(axis=0)
    preds = np.zeros((batch.P, N), np.int32)
    for p in range(batch.P):
        r0, r1 = batch.set_rule_off[p], batch.set_rule_off[p + 1]
        if r1 == r0:
            preds[p] = batch.set_default[p]
            continue
        fr = fires[r0:r1]
        first = fr.argmax(axis=0)
        anyf = fr.any(axis=0)
        preds[p] = np.where(anyf, batch.rule_class[r0:r1][first], batch.set_default[p])
    return preds


@pytest.mark.parametrize("seed", range(6))
def test_dense_form_agrees_on_boundaries(orc, seed):
    rng = np.random.default_rng(seed)
    F = int(rng.integers(1, 5))
    K = int(rng.integers(2, 4))
    N = 300
    qtab = synth.quantile_table(rng.standard_normal((512, F)).astype(np.float32))
    batch = synth.random_rulesets(qtab, K, 6, (1, 4), (1, 3), seed, pair_prob=0.4 if F > 1 else 0.0)
    X = synth.boundary_samples(batch, F, N, seed)
    y = rng.integers(0, K, N).astype(np.int32)
    _, _, preds = orc.eval_hard(X, y, K, batch, want_preds=True)
    assert np.array_equal(preds, dense_eval(X, batch))


def test_boundary_samples_really_hit_boundaries():
    """The generator puts products exactly on the threshold for some samples."""
    rng = np.random.default_rng(1)
    qtab = synth.quantile_table(rng.standard_normal((512, 3)).astype(np.float32))
    batch = synth.random_rulesets(qtab, 2, 4, 3, 2, 1, pair_prob=0.0)
    X = synth.boundary_samples(batch, 3, 400, 1)
    hits = 0
    for c in range(batch.C):
        prod = (batch.cond_a[c] * X[:, batch.cond_f[c]]).astype(np.float32)
        hits += int((prod == batch.cond_t[c]).sum())
    assert hits > 0


def test_single_condition_one_liner(orc):
    rng = np.random.default_rng(3)
    X, y = synth.two_class_gaussian(1000, 5, 3)
    for op in (synth.GT, synth.LT):
        a, t, f = np.float32(0.7), np.float32(0.3), 2
        batch = synth.from_lists([[(1, [(f, -1, op, a, 0.0, t)])]], [0])
        correct, per_class, _ = orc.eval_hard(X, y, 2, batch)
        cond = (a * X[:, f] > t) if op == synth.GT else (a * X[:, f] < t)
        want = int((cond & (y == 1)).sum() + (~cond & (y == 0)).sum())
        assert correct[0] == want
        assert per_class[0, 1] == int((cond & (y == 1)).sum())


def test_nan_and_inf_compare_false(orc):
    X = np.array([[np.nan, 0.0], [np.inf, 0.0], [-np.inf, 0.0], [0.0, 0.0], [-0.0, 0.0]], np.float32)
    y = np.zeros(5, np.int32)
    rules = [(1, [(0, -1, synth.GT, 1.0, 0.0, 0.0)]), (1, [(0, -1, synth.LT, 1.0, 0.0, 0.0)])]
    _, _, preds = orc.eval_hard(X, y, 2, synth.from_lists([rules], [0]), want_preds=True)
    # NaN: both false -> default; +inf > 0; -inf < 0; +-0 is neither > 0 nor < 0
    assert preds[0].tolist() == [0, 1, 1, 0, 0]


# ----------------------------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def small():
    return synth.plain_hard(seed=0)


def test_empty_set_gives_default_count(orc, small):
    b = synth.from_lists([[], []], [0, 1])
    correct, per_class, _ = orc.eval_hard(small.X, small.y, 2, b)
    assert correct.tolist() == [int((small.y == 0).sum()), int((small.y == 1).sum())]


def test_rules_naming_default_give_default_count(orc, small):
    b = small.batch.subset(range(8))
    b.rule_class[:] = 1
    b.set_default[:] = 1
    correct, _, _ = orc.eval_hard(small.X, small.y, 2, b)
    assert (correct == int((small.y == 1).sum())).all()


def test_permutation_invariance_and_class_sum(orc, small):
    c1, pc1, p1 = orc.eval_hard(small.X, small.y, 2, small.batch, want_preds=True)
    perm = np.random.default_rng(9).permutation(small.N)
    c2, pc2, p2 = orc.eval_hard(small.X[perm], small.y[perm], 2, small.batch, want_preds=True)
    assert np.array_equal(c1, c2) and np.array_equal(pc1, pc2)
    assert np.array_equal(p1[:, perm], p2)
    assert np.array_equal(pc1.sum(axis=1), c1)


def test_empty_rule_fires(orc):
    X = np.zeros((3, 2), np.float32)
    y = np.array([0, 1, 2], np.int32)
    b = synth.from_lists([[(2, [(0, -1, synth.GT, 1.0, 0.0, 5.0)]), (1, []), (0, [])]], [0])
    _, _, preds = orc.eval_hard(X, y, 3, b, want_preds=True)
    assert preds[0].tolist() == [1, 1, 1]


def test_threads_do_not_change_results(orc):
    w = synth.plain_hard(seed=1)
    a = orc.eval_hard(w.X, w.y, 2, w.batch, nthreads=1)
    b = orc.eval_hard(w.X, w.y, 2, w.batch, nthreads=4)
    assert all(np.array_equal(u, v) for u, v in zip(a[:2], b[:2]))


# ------------------------------------------------------------------------------ soft path

def _soft_case(seed, R, C, K=2, N=200, F=4, pair_prob=0.3):
    X, y = synth.two_class_gaussian(N, F, seed)
    if K > 2:
        y = np.random.default_rng(seed).integers(0, K, N).astype(np.int32)
    b = synth.random_rulesets(synth.quantile_table(X), K, 3, R, C, seed, pair_prob=pair_prob)
    if K == 2:   # every class reachable, so that no label has probability zero (infinite loss)
        b.set_default[:] = 1 - b.rule_class[b.set_rule_off[:-1]]
    return X, y, b


def test_soft_probabilities_sum_to_one(orc):
    X, y, b = _soft_case(0, (1, 5), (1, 3), K=3)
    out = orc.soft(X, y, 3, b, 0.5, want_probs=True)
    assert np.allclose(out["probs"].sum(axis=2), 1.0, atol=1e-12, rtol=0)
    # loss is the mean negative log-probability of the label
    py = out["probs"][:, np.arange(len(y)), y]
    with np.errstate(divide="ignore"):
        assert np.allclose(out["loss"], (-np.log(py)).mean(axis=1), rtol=1e-12, atol=0)


def test_unreachable_label_has_infinite_loss(orc):
    """A label with no rule of its class and another default class has probability exactly 0 in
    the ordered mixture of Sec. 3 (every path ends in a rule or the default), so -log p is +inf;
    a set where every label is reachable stays finite."""
    X, _ = synth.two_class_gaussian(50, 2, 3)
    y = np.zeros(len(X), np.int32)
    y[7] = 2                                                   # class 2 appears in no set below
    cond = (0, -1, synth.GT, 1.0, 0.0, 0.0)
    b = synth.from_lists([[(0, [cond])], [(2, [cond])]], [1, 0])
    out = orc.soft(X, y, 3, b, 0.5, want_probs=True)
    assert np.isposinf(out["loss"][0]) and out["probs"][0, 7, 2] == 0.0
    assert np.isfinite(out["loss"][1])


@pytest.mark.parametrize("op", [synth.GT, synth.LT])
@pytest.mark.parametrize("pair", [False, True])
def test_one_rule_one_condition_is_logistic_regression(orc, op, pair):
    X, y = synth.two_class_gaussian(500, 3, 4)
    tau = np.float32(0.25)
    a, bb, t = np.float32(0.8), np.float32(-0.4), np.float32(0.35)
    cond = (0, 2 if pair else -1, op, a, bb if pair else 0.0, 0.0 if pair else t)
    batch = synth.from_lists([[(1, [cond])]], [0])
    out = orc.soft(X, y, 2, batch, tau, dloss=1.0)
    s = 1.0 if op == synth.GT else -1.0
    x0 = X[:, 0].astype(np.float64)
    rhs = (np.float64(bb) * X[:, 2].astype(np.float64)) if pair else np.float64(t)
    u = s * (np.float64(a) * x0 - rhs) / np.float64(tau)
    is1 = (y == 1)
    loss = -np.where(is1, log_expit(u), log_expit(-u)).mean()
    assert np.isclose(out["loss"][0], loss, rtol=1e-12, atol=0)
    dldu = expit(u) - is1                      # logistic regression gradient
    ga = (dldu * s * x0 / np.float64(tau)).mean()
    assert np.isclose(out["grad_a"][0], ga, rtol=1e-10, atol=1e-14)
    if pair:
        gb = (dldu * -s * X[:, 2].astype(np.float64) / np.float64(tau)).mean()
        assert np.isclose(out["grad_b"][0], gb, rtol=1e-10, atol=1e-14)
        assert out["grad_t"][0] == 0.0
    else:
        gt = (dldu * -s / np.float64(tau)).mean()
        assert np.isclose(out["grad_t"][0], gt, rtol=1e-10, atol=1e-14)
        assert out["grad_b"][0] == 0.0


def test_one_rule_two_conditions_product(orc):
    X, y = synth.two_class_gaussian(300, 3, 6)
    tau = np.float32(0.5)
    conds = [(0, -1, synth.GT, 0.9, 0.0, 0.2), (1, 2, synth.LT, -0.6, 0.3, 0.0)]
    batch = synth.from_lists([[(0, conds)]], [1])
    out = orc.soft(X, y, 2, batch, tau)
    x = X.astype(np.float64)
    u1 = (np.float64(np.float32(0.9)) * x[:, 0] - np.float64(np.float32(0.2))) / np.float64(tau)
    u2 = -(np.float64(np.float32(-0.6)) * x[:, 1] - np.float64(np.float32(0.3)) * x[:, 2]) / np.float64(tau)
    q = expit(u1) * expit(u2)                  # class 0 iff the rule fires
    loss = -np.where(y == 0, np.log(q), np.log1p(-q)).mean()
    assert np.isclose(out["loss"][0], loss, rtol=1e-11, atol=0)


def linear_domain_probs(X, batch, tau, K):
    """Soft first-fire in the linear domain: q_r = prod sigmoid(u_c), P(rule r first) =
    q_r prod_{j<r} (1 - q_j), default takes prod_j (1 - q_j)."""
    x = X.astype(np.float64)
    N = len(X)
    out = np.zeros((batch.P, N, K))
    for p in range(batch.P):
        none_yet = np.ones(N)
        for r in range(batch.set_rule_off[p], batch.set_rule_off[p + 1]):
            q = np.ones(N)
            for c in range(batch.rule_cond_off[r], batch.rule_cond_off[r + 1]):
                f, g = batch.cond_f[c], batch.cond_g[c]
                lhs = np.float64(batch.cond_a[c]) * x[:, f]
                rhs = np.float64(batch.cond_t[c]) if g < 0 else np.float64(batch.cond_b[c]) * x[:, g]
                s = 1.0 if batch.cond_op[c] == synth.GT else -1.0
                q = q * expit(s * (lhs - rhs) / np.float64(np.float32(tau)))
            out[p, :, batch.rule_class[r]] += q * none_yet
            none_yet = none_yet * (1.0 - q)
        out[p, :, batch.set_default[p]] += none_yet
    return out


def test_linear_domain_agrees(orc):
    X, y, b = _soft_case(2, (1, 6), (1, 3), K=3)
    out = orc.soft(X, y, 3, b, 1.0, want_probs=True)
    assert np.allclose(out["probs"], linear_domain_probs(X, b, 1.0, 3), rtol=1e-10, atol=1e-13)


def test_low_temperature_recovers_hard_predictions(orc):
    X, y, b = _soft_case(3, (2, 6), (1, 3), K=2, N=400)
    _, _, hard = orc.eval_hard(X, y, 2, b, want_preds=True)
    out = orc.soft(X, y, 2, b, 1e-4, want_probs=True)
    soft_pred = out["probs"].argmax(axis=2)
    # exclude samples within 1e-3 of any boundary (|u| < 10: there the relaxed decision may differ)
    x = X.astype(np.float64)
    near = np.zeros(len(X), bool)
    for c in range(b.C):
        lhs = np.float64(b.cond_a[c]) * x[:, b.cond_f[c]]
        rhs = np.float64(b.cond_t[c]) if b.cond_g[c] < 0 else np.float64(b.cond_b[c]) * x[:, b.cond_g[c]]
        near |= np.abs(lhs - rhs) < 1e-3
    assert (~near).sum() > 100
    assert np.array_equal(soft_pred[:, ~near], hard[:, ~near])


@pytest.mark.parametrize("seed", [0, 1])
def test_adjoint_matches_central_differences(orc, seed):
    X, y, b = _soft_case(10 + seed, (2, 5), (1, 3), K=2, N=150)
    tau = 0.3
    dl = np.array([1.0, -0.5, 2.0])
    out = orc.soft(X, y, 2, b, tau, dloss=dl)
    h = 1e-3

    def total(bb):
        return float((orc.soft(X, y, 2, bb, tau)["loss"] * dl).sum())

    for c in range(b.C):
        for name, arr in (("a", "cond_a"), ("t", "cond_t"), ("b", "cond_b")):
            if name == "t" and b.cond_g[c] >= 0:
                continue
            if name == "b" and b.cond_g[c] < 0:
                continue
            plus, minus = synth.Batch(**b.arrays()), synth.Batch(**b.arrays())
            for bb, sgn in ((plus, 1), (minus, -1)):
                v = getattr(b, arr).copy()
                v[c] = np.float32(v[c] + sgn * h)
                setattr(bb, arr, v)
            step = np.float64(getattr(plus, arr)[c]) - np.float64(getattr(minus, arr)[c])
            fd = (total(plus) - total(minus)) / step
            g = out["grad_" + name][c]
            assert abs(fd - g) <= 1e-3 * max(abs(g), 1e-3), (c, name, fd, g)


# ----------------------------------------------------- soft path at large margins (|u| >> 1)
#
# Fine-tuned coefficients (Fig. 1c: a pair coefficient of 7275.88) give margins of hundreds or
# thousands of temperatures. There q_r = 1 - e^{-u} (or e^{u}) to any float precision, and
# 1 - q_r, products of such factors and the gradient factors sigmoid(-u) are far below the float64
# range while the loss and the gradients stay moderate. Two references that do not share the
# oracle's log-domain form pin it there: closed forms of a single condition, and the linear-domain
# definition evaluated in arbitrary precision (mpmath), with 1 - q_r written as the positive sum
# sum_c sigmoid(-u_c) prod_{c' < c} sigmoid(u_c') (no cancellation) and gradients by central
# differences in that precision.

LARGE_U = np.array([50.0, 103.0, 200.0, 1000.0, 18000.0])


@pytest.mark.parametrize("op", [synth.GT, synth.LT])
@pytest.mark.parametrize("pair", [False, True])
def test_large_margin_single_condition_closed_form(orc, op, pair):
    tau = np.float32(0.1)
    u_target = np.concatenate([LARGE_U, -LARGE_U])
    s = 1.0 if op == synth.GT else -1.0
    a, bb, t = np.float32(1.5), np.float32(-2.0), np.float32(0.25)
    x2 = np.float32(0.5)
    rhs = np.float64(bb) * np.float64(x2) if pair else np.float64(t)
    x0 = ((s * u_target * np.float64(tau) + rhs) / np.float64(a)).astype(np.float32)
    X = np.zeros((2 * len(x0), 3), np.float32)
    X[:, 0] = np.tile(x0, 2)
    X[:, 2] = x2
    y = np.repeat(np.array([1, 0], np.int32), len(x0))           # both labels at every margin
    cond = (0, 2 if pair else -1, op, a, bb if pair else 0.0, 0.0 if pair else t)
    batch = synth.from_lists([[(1, [cond])]], [0])
    out = orc.soft(X, y, 2, batch, tau, dloss=1.0, want_mag=True)
    u = s * (np.float64(a) * X[:, 0].astype(np.float64) - rhs) / np.float64(tau)
    assert np.all(np.abs(np.abs(u) / np.tile(np.abs(u_target), 2) - 1) < 1e-3)
    is1 = y == 1
    ell = np.where(is1, np.logaddexp(0.0, -u), np.logaddexp(0.0, u))     # -log sigmoid(+-u)
    assert np.isfinite(out["loss"][0])
    assert np.isclose(out["loss"][0], ell.mean(), rtol=1e-13, atol=0)
    dldu = expit(u) - is1
    terms_a = dldu * s * X[:, 0].astype(np.float64) / np.float64(tau)
    terms_2 = dldu * -s * (X[:, 2].astype(np.float64) if pair else 1.0) / np.float64(tau)
    # the per-sample terms of both labels cancel in the mean: compare against their magnitude
    for got, terms in ((out["grad_a"][0], terms_a), (out["grad_b" if pair else "grad_t"][0], terms_2)):
        assert abs(got - terms.mean()) <= 1e-12 * np.abs(terms).mean(), (got, terms.mean())


def mp_set_loss(X, y, b, p, tau, dps=40, param=None):
    """Mean -log p_y of set p in the linear domain, in `dps` decimal digits; `param` =
    (array name, condition, mpf value) replaces one parameter (for differences)."""
    import mpmath as mp
    with mp.workdps(dps):
        tau_m = mp.mpf(float(tau))

        def val(name, c):
            if param is not None and param[0] == name and param[1] == c:
                return param[2]
            return mp.mpf(float(getattr(b, name)[c]))

        def sig(u):
            return 1 / (1 + mp.exp(-u))

        total = mp.mpf(0)
        for n in range(len(X)):
            x = [mp.mpf(float(v)) for v in X[n]]
            U, py = mp.mpf(1), mp.mpf(0)
            for r in range(b.set_rule_off[p], b.set_rule_off[p + 1]):
                pos, neg = [], []
                for c in range(b.rule_cond_off[r], b.rule_cond_off[r + 1]):
                    rhs = val("cond_t", c) if b.cond_g[c] < 0 else val("cond_b", c) * x[b.cond_g[c]]
                    s = 1 if b.cond_op[c] == synth.GT else -1
                    u = s * (val("cond_a", c) * x[b.cond_f[c]] - rhs) / tau_m
                    pos.append(sig(u))
                    neg.append(sig(-u))
                q = mp.fprod(pos)
                one_minus_q = mp.fsum(neg[c] * mp.fprod(pos[:c]) for c in range(len(pos)))
                if b.rule_class[r] == y[n]:
                    py += q * U
                U *= one_minus_q
            if b.set_default[p] == y[n]:
                py += U
            total += -mp.log(py)
        return total / len(X)


def large_margin_case(seed, N=10):
    """Small sets with coefficients of tens to thousands (margins of ~10 to ~20,000 tau at
    tau = 0.1), including a Fig. 1c-shaped pair condition (coefficient -7275.88), every label
    reachable."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(N, 3)).astype(np.float32)
    y = rng.integers(0, 2, N).astype(np.int32)
    sets = []
    for p in range(3):
        rules = []
        for r in range(int(rng.integers(1, 4))):
            conds = []
            for c in range(int(rng.integers(1, 4))):
                f = int(rng.integers(0, 3))
                op = int(rng.integers(0, 2))
                a = np.float32(rng.choice([-1, 1]) * 10 ** rng.uniform(1, 3))
                if rng.uniform() < 0.3:
                    g = (f + 1 + int(rng.integers(0, 2))) % 3
                    conds.append((f, g, op, a, np.float32(rng.choice([-1, 1]) * 10 ** rng.uniform(1, 3)), 0.0))
                else:
                    conds.append((f, -1, op, a, 0.0, np.float32(a * X[int(rng.integers(0, N)), f])))
            rules.append((int(rng.integers(0, 2)), conds))
        sets.append(rules)
    sets.append([(1, [(0, -1, synth.GT, np.float32(0.06), 0.0, np.float32(0.0)),
                      (1, 2, synth.GT, np.float32(-1.0), np.float32(-7275.88), 0.0)]),
                 (0, [(2, -1, synth.LT, np.float32(1.0), 0.0, np.float32(0.24))])])
    b = synth.from_lists(sets, [0, 1, 0, 0])
    b.set_default[:] = 1 - b.rule_class[b.set_rule_off[:-1]]
    return X, y, b


@pytest.mark.parametrize("seed", [0, 1])
def test_large_margins_match_arbitrary_precision(orc, seed):
    import mpmath as mp
    X, y, b = large_margin_case(seed)
    tau = np.float32(0.1)
    out = orc.soft(X, y, 2, b, tau, dloss=1.0, want_mag=True)
    for p in range(b.P):
        ref = float(mp_set_loss(X, y, b, p, tau))
        assert np.isfinite(out["loss"][p]) and np.isclose(out["loss"][p], ref, rtol=1e-12, atol=0), \
            (p, out["loss"][p], ref)
        h = mp.mpf(10) ** -30
        for c in range(b.rule_cond_off[b.set_rule_off[p]], b.rule_cond_off[b.set_rule_off[p + 1]]):
            for name, grad in (("cond_a", "a"), ("cond_t" if b.cond_g[c] < 0 else "cond_b",
                                                  "t" if b.cond_g[c] < 0 else "b")):
                with mp.workdps(110):
                    v = mp.mpf(float(getattr(b, name)[c]))
                    fd = (mp_set_loss(X, y, b, p, tau, 110, (name, c, v + h)) -
                          mp_set_loss(X, y, b, p, tau, 110, (name, c, v - h))) / (2 * h)
                g, m = out["grad_" + grad][c], out["mag_" + grad][c]
                # differences of losses below ~1e3 resolve gradients down to ~1e-77 at 110 digits
                assert np.isfinite(g) and abs(g - float(fd)) <= 1e-10 * max(abs(float(fd)), m) + 1e-75, \
                    (p, c, name, g, float(fd))
