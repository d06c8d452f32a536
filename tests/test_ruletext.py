"""Readable and tensor forms of rule sets (Fig. 1 layouts): the paper's worked example and exact
round trips of random batches."""
import os

import numpy as np
import pytest

from paper_2406_01821_gb300 import ruletext, synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1.txt")
FEATS = ["mean radius", "fractal dimension error", "worst compactness", "worst symmetry",
         "perimeter error", "mean area"]
CLASSES = ["malignant", "benign"]


def sections():
    sec, out = None, {}
    for line in open(GOLDEN):
        line = line.rstrip("\n")
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            sec = line.strip("[]")
            out[sec] = []
        else:
            out[sec].append(line)
    return out


def fig1a_rows():
    rows, sizes = [], []
    for ln in sections()["a"]:
        tok = ln.split()
        if tok[0] == "rule":
            cls = CLASSES.index(tok[3])
            sizes.append(0)
            continue
        rows.append((cls, [float(v) for v in tok[1:7]], float(tok[8])))
        sizes[-1] += 1
    return rows, sizes


def test_fig1a_rows_read_as_fig1b():
    rows, sizes = fig1a_rows()
    rules = ruletext.from_tensor_rows(rows, sizes)
    assert ruletext.render_rules(rules, FEATS, CLASSES, digits=2) == sections()["b"]


def test_fig1c_text_round_trip():
    lines = sections()["c"]
    rules, default = ruletext.parse_rules(lines, FEATS, CLASSES)
    assert default is None and [len(c) for _, c in rules] == [3, 2]
    assert ruletext.render_rules(rules, FEATS, CLASSES, digits=2) == lines


def test_fig1b_rows_round_trip():
    rules, _ = ruletext.parse_rules(sections()["b"], FEATS, CLASSES)
    rows = ruletext.tensor_rows(rules, len(FEATS))
    back = ruletext.from_tensor_rows(rows, [len(c) for _, c in rules])
    assert ruletext.render_rules(back, FEATS, CLASSES, digits=2) == sections()["b"]


def special(rng, n):
    pool = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -3e-39, 3.4028235e38, 1.0, -1.0, 0.1],
                    np.float32)
    return pool[rng.integers(0, len(pool), n)]


@pytest.mark.parametrize("seed", range(3))
def test_random_batches_round_trip_bit_exactly(seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((300, 7)).astype(np.float32)
    b = synth.random_rulesets(synth.quantile_table(X), 3, 9, (1, 6), (1, 4), seed, pair_prob=0.4)
    for arr in (b.cond_a, b.cond_b, b.cond_t):
        m = rng.random(len(arr)) < 0.2
        arr[m] = special(rng, int(m.sum()))
    feats = [f"f{j}" for j in range(7)]
    classes = ["no", "yes", "maybe"]
    texts = [ruletext.render(b, p, feats, classes) for p in range(b.P)]
    back = ruletext.parse(texts, feats, classes)
    for name in ("set_rule_off", "rule_cond_off", "rule_class", "set_default", "cond_f", "cond_g",
                 "cond_op"):
        assert np.array_equal(getattr(back, name), getattr(b, name)), name
    thr = b.cond_g < 0
    for name, mask in (("cond_a", slice(None)), ("cond_b", ~thr), ("cond_t", thr)):
        x, y = getattr(back, name)[mask], getattr(b, name)[mask]
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32)), name


def test_tensor_rows_keep_the_evaluation(orc):
    """Rules -> Fig. 1a rows -> rules: '<' conditions come back as negated '>' ones; every
    prediction and count is unchanged (negation is exact in float32)."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((2000, 6)).astype(np.float32)
    y = rng.integers(0, 2, 2000).astype(np.int32)
    b = synth.random_rulesets(synth.quantile_table(X), 2, 6, (1, 5), (1, 4), 5, pair_prob=0.3)
    sets = []
    for p in range(b.P):
        rules, _ = ruletext.set_rules(b, p)
        rules = [(c, [cd for cd in conds if cd[1] != cd[0]]) for c, conds in rules]
        rules = [(c, conds) for c, conds in rules if conds]
        sets.append(rules)
    b1 = synth.from_lists(sets, list(b.set_default))
    sets2 = [ruletext.from_tensor_rows(ruletext.tensor_rows(r, 6), [len(c) for _, c in r]) for r in sets]
    b2 = synth.from_lists(sets2, list(b.set_default))
    assert (b2.cond_op == synth.GT).all()
    w1, w2 = orc.eval_hard(X, y, 2, b1, want_preds=True), orc.eval_hard(X, y, 2, b2, want_preds=True)
    for u, v in zip(w1, w2):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("seed", range(2))
def test_membership_conditions_round_trip(seed, orc):
    """'(name in {codes})' reads back to the same category set; the predictions are unchanged;
    a membership test has no Fig. 1a row."""
    X, y = synth.categorical_mixture(800, 9, 3, seed, n_cat=3, n_codes=40)
    b = synth.random_rulesets(synth.quantile_table(X), 3, 7, (1, 5), (1, 4), seed, cat_from=6, n_codes=40)
    assert (b.cond_op == synth.IN).any()
    feats = [f"f{j}" for j in range(9)]
    classes = ["a", "b", "c"]
    texts = [ruletext.render(b, p, feats, classes) for p in range(b.P)]
    assert any(" in {" in ln for t in texts for ln in t)
    back = ruletext.parse(texts, feats, classes)
    m = b.cond_op == synth.IN
    assert np.array_equal(back.cond_op, b.cond_op)
    assert np.array_equal(back.cond_set[m], b.cond_set[m])
    for u, v in zip(orc.eval_hard(X, y, 3, b, want_preds=True), orc.eval_hard(X, y, 3, back, want_preds=True)):
        assert np.array_equal(u, v)
    p = int(np.flatnonzero(m)[0])
    rule = int(np.searchsorted(b.rule_cond_off, p, side="right") - 1)
    s = int(np.searchsorted(b.set_rule_off, rule, side="right") - 1)
    with pytest.raises(ValueError):
        ruletext.tensor_rows(ruletext.set_rules(b, s)[0], 9)
