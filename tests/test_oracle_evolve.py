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
