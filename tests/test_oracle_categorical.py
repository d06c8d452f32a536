"""Pins of the oracle's categorical conditions (membership of an integer category code in a set;
categorical features are the future work of Sec. 5). Exact values written out by hand, numpy's
isin as a second formulation, the band form of a single code, and closed forms of the soft path
where a membership test is an exact indicator with no gradient."""
import numpy as np
import pytest
from scipy.special import expit

from paper_2406_01821_gb300 import synth

EDGE_X = np.array([0.0, -0.0, 1.0, 2.5, 63.0, 64.0, -1.0, np.nan, np.inf, -np.inf, 1e9, 31.0, 32.0,
                   33.0, np.float32(5.0000005)], np.float32)


def _member_preds(orc, x, codes):
    """Predictions of the one-rule set (x in codes -> 1), default 0, on the values x."""
    X = np.asarray(x, np.float32)[:, None]
    b = synth.from_lists([[(1, [(0, -1, synth.IN, 0.0, 0.0, 0.0, codes)])]], [0])
    _, _, preds = orc.eval_hard(X, np.zeros(len(X), np.int32), 2, b, want_preds=True)
    return preds[0].astype(bool)


@pytest.mark.parametrize("codes,want", [
    (range(64), [1, 1, 1, 0, 1, 0, 0, 0, 0, 0, 0, 1, 1, 1, 0]),
    ([0, 31, 32, 63], [1, 1, 0, 0, 1, 0, 0, 0, 0, 0, 0, 1, 1, 0, 0]),
    ([5], [0] * 15),
    ([], [0] * 15),
])
def test_membership_edge_values(orc, codes, want):
    """Integer codes 0..63 only: -0 is code 0; fractions, negatives, 64 and above, NaN and
    infinities are in no set; bit k is code k (0, 31, 32 and 63 included)."""
    assert synth.category_mask(list(codes)) < (1 << 64)
    assert _member_preds(orc, EDGE_X, list(codes)).astype(int).tolist() == want


def test_membership_bit_order(orc):
    x = np.arange(64, dtype=np.float32)
    for k in (0, 1, 7, 31, 32, 40, 62, 63):
        got = _member_preds(orc, x, [k])
        assert got.sum() == 1 and got[k], k


def reference_preds(X, batch):
    """First-fire predictions with numpy: np.isin for membership tests (on integer-valued data in
    0..63), rounded float32 products and IEEE compares for the inequalities."""
    N = len(X)
    truth = np.zeros((batch.C, N), bool)
    for c in range(batch.C):
        f, g, op = int(batch.cond_f[c]), int(batch.cond_g[c]), int(batch.cond_op[c])
        if op == synth.IN:
            ok = (X[:, f] >= 0) & (X[:, f] <= 63) & (X[:, f] == np.floor(X[:, f]))
            truth[c] = ok & np.isin(X[:, f], synth.category_codes(int(batch.cond_set[c])))
            continue
        lhs = (np.float32(batch.cond_a[c]) * X[:, f]).astype(np.float32)
        rhs = np.float32(batch.cond_t[c]) if g < 0 else (np.float32(batch.cond_b[c]) * X[:, g]).astype(np.float32)
        truth[c] = lhs > rhs if op == synth.GT else lhs < rhs
    preds = np.zeros((batch.P, N), np.int32)
    for p in range(batch.P):
        pred = np.full(N, batch.set_default[p], np.int32)
        open_ = np.ones(N, bool)
        for r in range(batch.set_rule_off[p], batch.set_rule_off[p + 1]):
            c0, c1 = batch.rule_cond_off[r], batch.rule_cond_off[r + 1]
            fire = truth[c0:c1].all(axis=0) & open_
            pred[fire] = batch.rule_class[r]
            open_ &= ~fire
        preds[p] = pred
    return preds


@pytest.mark.parametrize("seed", range(4))
def test_mixed_rulesets_match_isin_formulation(orc, seed):
    X, y = synth.categorical_mixture(2000, 10, 4, seed, n_cat=4, n_codes=16)
    b = synth.random_rulesets(synth.quantile_table(X), 4, 12, (1, 8), (1, 4), seed, cat_from=6)
    assert (b.cond_op == synth.IN).sum() > 10
    _, _, preds = orc.eval_hard(X, y, 4, b, want_preds=True)
    assert np.array_equal(preds, reference_preds(X, b))
    # a perturbed copy of the data (fractional codes, out-of-range codes) changes nothing in the
    # isin formulation's treatment of those values either
    X2 = X.copy()
    X2[::7, 6] += np.float32(0.25)
    X2[1::7, 7] = 64.0
    _, _, preds2 = orc.eval_hard(X2, y, 4, b, want_preds=True)
    assert np.array_equal(preds2, reference_preds(X2, b))


def test_single_code_equals_band(orc):
    """On integer-valued data, membership of the single code k equals k - 0.5 < x < k + 0.5."""
    rng = np.random.default_rng(3)
    X = rng.integers(0, 12, (500, 1)).astype(np.float32)
    y = rng.integers(0, 2, 500).astype(np.int32)
    for k in (0, 5, 11):
        m = synth.from_lists([[(1, [(0, -1, synth.IN, 0, 0, 0, [k])])]], [0])
        band = synth.from_lists([[(1, [(0, -1, synth.GT, 1.0, 0.0, k - 0.5),
                                       (0, -1, synth.LT, 1.0, 0.0, k + 0.5)])]], [0])
        assert np.array_equal(orc.eval_hard(X, y, 2, m, want_preds=True)[2],
                              orc.eval_hard(X, y, 2, band, want_preds=True)[2])


def test_soft_membership_is_exact_indicator(orc):
    """Rule (x0 in S) & (a*x1 > t) -> class 1, default 0: p_1 = [x0 in S] * sigmoid(u), so the
    loss and the gradients of a and t are logistic regression over the members of S (labels
    outside S are 0), and the membership test gets no gradient."""
    rng = np.random.default_rng(8)
    N = 400
    x0 = rng.integers(0, 8, N).astype(np.float32)
    x1 = rng.standard_normal(N).astype(np.float32)
    S = [1, 2, 6]
    member = np.isin(x0, S)
    y = np.where(member, (x1 > 0.2).astype(np.int32) ^ (rng.random(N) < 0.2), 0).astype(np.int32)
    X = np.stack([x0, x1], axis=1)
    a, t, tau = np.float32(0.7), np.float32(0.1), 0.5
    b = synth.from_lists([[(1, [(0, -1, synth.IN, 0, 0, 0, S), (1, -1, synth.GT, a, 0.0, t)])]], [0])
    out = orc.soft(X, y, 2, b, tau, dloss=1.0, want_probs=True)
    u = (np.float64(a) * x1.astype(np.float64) - np.float64(t)) / tau
    p1 = np.where(member, expit(u), 0.0)
    assert np.allclose(out["probs"][0, :, 1], p1, rtol=1e-12, atol=0)
    ell = -np.log(np.where(y == 1, p1, 1.0 - p1))
    assert np.isclose(out["loss"][0], ell.mean(), rtol=1e-12, atol=0)
    r = np.where(member, expit(u) - y, 0.0)                      # d ell / d u
    assert np.isclose(out["grad_a"][1], (r * x1 / tau).mean(), rtol=1e-9, atol=1e-15)
    assert np.isclose(out["grad_t"][1], (-r / tau).mean(), rtol=1e-9, atol=1e-15)
    assert out["grad_a"][0] == 0 and out["grad_b"][0] == 0 and out["grad_t"][0] == 0
