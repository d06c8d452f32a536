"""Pins for the oracle's evolution step (Sec. 3: tournament selection, offspring with randomized
coefficients). The generator is checked against numpy's Philox4x64-10 bit generator (a library
routine); the step against its invariants."""
import numpy as np
import pytest

from paper_2406_01821_gb300 import synth


def test_philox_matches_numpy(orc):
    rng = np.random.default_rng(0)
    for _ in range(20):
        ctr = rng.integers(0, 2**63, 4, dtype=np.uint64)
        key = rng.integers(0, 2**63, 2, dtype=np.uint64)
        prev = ctr.copy()
        prev[0] = prev[0] - np.uint64(1)          # numpy advances the counter before each block
        want = np.random.Philox(counter=prev, key=key).random_raw(4).astype(np.uint64)
        assert np.array_equal(orc.philox4x64_10(ctr, key), want)


@pytest.fixture(scope="module")
def setup():
    X, y = synth.two_class_gaussian(800, 7, 1)
    pop = synth.initial_population(X, y, 2, 120, 10, 4, seed=1)
    return X, y, pop


def _fitness(orc, X, y, pop):
    c, _, _ = orc.eval_hard(X, y, 2, synth.batch_from_population(pop))
    return c


def _indiv(pop, i):
    n = pop["nrule"][i]
    out = [int(n), int(pop["deflt"][i])]
    for j in range(n):
        k = pop["ncond"][i, j]
        out.append((int(pop["rcls"][i, j]), int(k),
                    tuple(pop[f][i, j, :k].tobytes() for f in ("cf", "cg", "cop", "ca", "cb", "ct"))))
    return tuple(out)


def test_elites_are_the_ranked_top(orc, setup):
    X, y, pop = setup
    fit = _fitness(orc, X, y, pop)
    E = 12
    out = orc.evolve_step(pop, fit, 3, 0, E, X, 2)
    order = np.lexsort((np.arange(len(fit)), -fit))       # fitness desc, index asc
    for c in range(E):
        assert _indiv(out, c) == _indiv(pop, order[c])


def test_children_are_valid(orc, setup):
    X, y, pop = setup
    fit = _fitness(orc, X, y, pop)
    out = orc.evolve_step(pop, fit, 4, 1, 2, X, 2)
    P, RMAX, CMAX = out["cf"].shape
    F = X.shape[1]
    assert ((out["nrule"] >= 1) & (out["nrule"] <= RMAX)).all()
    for i in range(P):
        for j in range(out["nrule"][i]):
            k = out["ncond"][i, j]
            assert 1 <= k <= CMAX
            assert 0 <= out["rcls"][i, j] < 2
            f, g = out["cf"][i, j, :k], out["cg"][i, j, :k]
            assert ((f >= 0) & (f < F)).all() and ((g >= -1) & (g < F)).all() and (g != f).all()
            assert np.isin(out["cop"][i, j, :k], (0, 1)).all()
            a = out["ca"][i, j, :k]
            assert ((a >= -1) & (a < 1)).all()
    # the slot batch of the children evaluates
    _fitness(orc, X, y, out)


def test_deterministic_and_seeded(orc, setup):
    X, y, pop = setup
    fit = _fitness(orc, X, y, pop)
    a = orc.evolve_step(pop, fit, 5, 2, 2, X, 2)
    b = orc.evolve_step(pop, fit, 5, 2, 2, X, 2)
    c = orc.evolve_step(pop, fit, 6, 2, 2, X, 2)
    d = orc.evolve_step(pop, fit, 5, 3, 2, X, 2)
    assert all(np.array_equal(a[k], b[k]) for k in a)
    assert not all(np.array_equal(a[k], c[k]) for k in a)
    assert not all(np.array_equal(a[k], d[k]) for k in a)


def test_selection_pressure(orc, setup):
    """Binary tournaments favour fitter parents: children that are plain copies of an individual
    (no crossover, no mutation) come from the upper half more often than from the lower half."""
    X, y, pop = setup
    fit = _fitness(orc, X, y, pop)
    order = np.lexsort((np.arange(len(fit)), -fit))
    rank = np.empty_like(order)
    rank[order] = np.arange(len(order))
    index = {}
    for i in range(len(fit)):
        index.setdefault(_indiv(pop, i), i)
    upper = lower = 0
    for gen in range(30):
        out = orc.evolve_step(pop, fit, 9, gen, 1, X, 2)
        for c in range(1, len(fit)):
            src = index.get(_indiv(out, c))
            if src is not None:
                if rank[src] < len(fit) // 2:
                    upper += 1
                else:
                    lower += 1
    assert upper + lower > 50
    assert upper > 2 * lower


def test_all_elites_is_a_sort(orc, setup):
    X, y, pop = setup
    fit = _fitness(orc, X, y, pop)
    out = orc.evolve_step(pop, fit, 1, 0, len(fit), X, 2)
    order = np.lexsort((np.arange(len(fit)), -fit))
    for c in range(len(fit)):
        assert _indiv(out, c) == _indiv(pop, order[c])


# ------------------------------------------------------------------ operator mix (reading 12)
#
# A population built so that every change a child carries can be read off: every individual has
# R0 = 6 rules of 2 or 3 threshold conditions (RMAX 8, CMAX 4: no add/delete is ever a no-op),
# distinct class ids out of K = 2^20 (a new class is almost surely visible), and each inherited
# condition carries a tag in its unused pair coefficient b (individual, rule, condition), which no
# operator touches. A child's rule is then traced to its origin (individual i, rule j), and its
# difference from that origin names the mutation. Equal fitness for all: tournaments take the
# lower of two uniform draws, which the statistics below do not depend on.

MIX_P, MIX_R0, MIX_RMAX, MIX_CMAX, MIX_K, MIX_F = 500, 6, 8, 4, 1 << 20, 16


def mix_population(seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(400, MIX_F)).astype(np.float32)
    P, R, C = MIX_P, MIX_RMAX, MIX_CMAX
    pop = {"nrule": np.full(P, MIX_R0, np.int32), "deflt": np.zeros(P, np.int32),
           "rcls": np.zeros((P, R), np.int32), "ncond": np.zeros((P, R), np.int32),
           "cf": np.zeros((P, R, C), np.int32), "cg": np.full((P, R, C), -1, np.int32),
           "cop": np.zeros((P, R, C), np.int8), "ca": np.zeros((P, R, C), np.float32),
           "cb": np.zeros((P, R, C), np.float32), "ct": np.zeros((P, R, C), np.float32)}
    for i in range(P):
        for j in range(MIX_R0):
            k = int(rng.integers(2, 4))
            pop["ncond"][i, j] = k
            pop["rcls"][i, j] = int(rng.integers(0, MIX_K))
            for q in range(k):
                f = int(rng.integers(0, MIX_F))
                a = np.float32(rng.uniform(-1, 1))
                pop["cf"][i, j, q] = f
                pop["cop"][i, j, q] = int(rng.integers(0, 2))
                pop["ca"][i, j, q] = a
                pop["ct"][i, j, q] = a * X[int(rng.integers(0, len(X))), f]
                pop["cb"][i, j, q] = 1 + (i * MIX_RMAX + j) * MIX_CMAX + q      # the tag
    return X, pop


def _tag(b):
    t = int(b) - 1
    return t // (MIX_RMAX * MIX_CMAX), (t // MIX_CMAX) % MIX_RMAX, t % MIX_CMAX


def _cond(pop, i, j, q):
    return tuple(pop[n][i, j, q].item() for n in ("cf", "cg", "cop", "ca", "cb", "ct"))


def classify_child(pop, out, c):
    """(origins, kind, new_conditions, redrawn_thresholds) of child c: the individuals its tagged
    rules come from, the mutation kind (0 coefficients, 1 feature, 2 comparison, 3 add condition,
    4 delete condition, 5 add rule, 6 delete rule, 7 class; None for no mutation), the conditions
    it created and the thresholds it drew again (feature, a, t)."""
    n = int(out["nrule"][c])
    origins, kinds, new_conds, redrawn = [], [], [], []
    if n == MIX_R0 + 1:
        kinds.append(5)
    elif n == MIX_R0 - 1:
        kinds.append(6)
    else:
        assert n == MIX_R0
    shift = 0
    for p in range(n):
        k = int(out["ncond"][c, p])
        tags = [out["cb"][c, p, q] for q in range(k) if out["cg"][c, p, q] < 0 and out["cb"][c, p, q] >= 1]
        if not tags:                               # a rule this child created
            assert kinds == [5]
            new_conds += [_cond(out, c, p, q) for q in range(k)]
            shift = -1
            continue
        i, j, _ = _tag(tags[0])
        assert all(_tag(t)[:2] == (i, j) for t in tags)
        if j != p + shift:                         # a rule was deleted before this position
            assert kinds == [6] and j == p + 1
            shift = 1
        origins.append(i)
        if out["rcls"][c, p] != pop["rcls"][i, j]:
            kinds.append(7)
        k0 = int(pop["ncond"][i, j])
        if k == k0 + 1:
            kinds.append(3)
            new_conds.append(_cond(out, c, p, k - 1))
            k = k0
        elif k == k0 - 1:
            kinds.append(4)
            continue
        for q in range(k):
            now, was = _cond(out, c, p, q), _cond(pop, i, j, q)
            if now == was:
                continue
            if now[3] != was[3]:
                kinds.append(0)
            elif now[0] != was[0] or now[5] != was[5]:
                kinds.append(1)
            else:
                assert now[2] == 1 - was[2] and now[:2] == was[:2] and now[3:] == was[3:]
                kinds.append(2)
            redrawn.append((now[0], now[3], now[5]))
    assert len(kinds) <= 1, kinds
    return origins, (kinds[0] if kinds else None), new_conds, redrawn


def _mix_stats(o, gens=24):
    X, pop = mix_population()
    fit = np.zeros(MIX_P, np.int32)
    stats = {"children": 0, "mixed": 0, "mutated": 0, "kinds": np.zeros(8, np.int64),
             "split": [], "new": [], "redrawn": []}
    for g in range(gens):
        out = o.evolve_step(pop, fit, 77, g, 1, X, MIX_K)
        for c in range(1, MIX_P):
            origins, kind, new, redrawn = classify_child(pop, out, c)
            stats["children"] += 1
            if len(set(origins)) > 1:
                assert len(set(origins)) == 2
                stats["mixed"] += 1
                lo = min(origins)
                if kind not in (5, 6):
                    stats["split"].append(sum(1 for x in origins if x == lo))
            if kind is not None:
                stats["mutated"] += 1
                stats["kinds"][kind] += 1
            stats["new"] += new
            stats["redrawn"] += redrawn
    return X, stats


def _within(count, n, p, sigmas=5.0):
    mean, sd = n * p, (n * p * (1 - p)) ** 0.5
    return abs(count - mean) <= sigmas * sd


def check_operator_mix(o):
    """Crossover with probability 1/2 and, per position, 1/2; one mutation with probability 9/10,
    uniform over the eight kinds; a new condition is a pair with probability 1/5. Bounds are five
    binomial standard deviations over about 12,000 children."""
    from scipy import stats as st
    X, s = _mix_stats(o)
    n = s["children"]
    # visible crossover: the two parents differ (equal-fitness tournaments: P(A = B) = sum of
    # squared probabilities that i is the lower of two draws) and not all or none of the six
    # positions were taken from B
    P = MIX_P
    pmin = np.array([(2 * (P - i) - 1) / P**2 for i in range(P)])
    p_mixed = 0.5 * (1 - (pmin**2).sum()) * (1 - 2 / 2**MIX_R0)
    assert _within(s["mixed"], n, p_mixed), (s["mixed"], n * p_mixed)
    # positions taken from the lower-indexed parent: Binomial(6, 1/2) given 1..5
    split = np.bincount(np.array(s["split"]), minlength=MIX_R0 + 1)[1:MIX_R0]
    pmf = np.array([st.binom.pmf(k, MIX_R0, 0.5) for k in range(1, MIX_R0)])
    chi = st.chisquare(split, pmf / pmf.sum() * split.sum())
    assert chi.pvalue > 1e-6, (split, chi)
    # mutation rate and kinds (kind 7 is invisible only if the same class is drawn: 2^-20)
    assert _within(s["mutated"], n, 0.9), (s["mutated"], 0.9 * n)
    for k in range(8):
        assert _within(s["kinds"][k], s["mutated"], 1 / 8), (k, s["kinds"])
    # new conditions: pairs with probability 1/5
    new = s["new"]
    pairs = sum(1 for c in new if c[1] >= 0)
    assert len(new) > 1500 and _within(pairs, len(new), 0.2), (pairs, len(new))
    for f, g, op, a, b, t in new:
        assert 0 <= f < MIX_F and op in (0, 1) and -1 <= a < 1
        if g >= 0:
            assert g != f and 0 <= g < MIX_F and -1 <= b < 1 and t == 0
        else:
            assert b == 0


def check_thresholds_from_data(o):
    """Every threshold the step draws (new conditions and redrawn ones) is fl32(a * x[n][f]) for a
    row n of the data, with f the condition's own feature."""
    X, s = _mix_stats(o, gens=6)
    drawn = [(c[0], c[3], c[5]) for c in s["new"] if c[1] < 0] + s["redrawn"]
    assert len(drawn) > 500
    for f, a, t in drawn:
        cand = np.float32(a) * X[:, f]               # float32 products, one rounding each
        assert (cand == np.float32(t)).any(), (f, a, t)


def test_operator_mix(orc):
    check_operator_mix(orc)


def test_thresholds_drawn_from_the_condition_feature(orc):
    check_thresholds_from_data(orc)
