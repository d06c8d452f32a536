"""GPU parity of the device-resident evolution loop and of fine-tuning.

Without fine-tuning every step is exact (integer fitness, Philox draws, float32 operations that
both sides perform identically), so the GPU trajectory must equal the oracle's bit for bit."""
import numpy as np
import pytest

from paper_2406_01821_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2406_01821_gb300 import build, rs
    build.build()
    c = rs.Context(0)
    yield c
    c.close()


def oracle_run(orc, X, y, K, pop, generations, elite, seed):
    best, mean = [], []
    for g in range(generations + 1):
        fit, _, _ = orc.eval_hard(X, y, K, synth.batch_from_population(pop))
        best.append(int(fit.max()))
        mean.append(float(fit.mean()))
        if g == generations:
            return pop, fit, np.array(best), np.array(mean)
        pop = orc.evolve_step(pop, fit, seed, g, elite, X, K)


@pytest.mark.parametrize("seed,K", [(3, 2), (4, 3)])
def test_evolution_matches_oracle_bit_exact(ctx, orc, seed, K):
    X, y = synth.gaussian_mixture(3001, 9, K, seed)
    pop = synth.initial_population(X, y, K, 96, RMAX=8, CMAX=4, seed=seed)
    ds = ctx.dataset(X, y, K)
    try:
        got, fit, best, mean = ctx.evolve(ds, pop, generations=4, elite=3, seed=seed)
    finally:
        ctx.dataset_destroy(ds)
    want, wfit, wbest, wmean = oracle_run(orc, X, y, K, pop, 4, 3, seed)
    for k in want:
        assert np.array_equal(got[k], want[k]), k
    assert np.array_equal(fit, wfit)
    assert np.array_equal(best, wbest)
    assert np.allclose(mean, wmean, rtol=0, atol=1e-12)


@pytest.mark.parametrize("tile", [21, 18, 23])
def test_forced_tile_configuration_gives_the_same_evolution(ctx, orc, tile):
    """rs_set_tile_config applies to the loop's evaluations too: a forced configuration (another
    evaluator form) gives the oracle's trajectory bit for bit, as the default one does."""
    from paper_2406_01821_gb300 import rs
    X, y = synth.gaussian_mixture(2501, 7, 3, 21)
    pop = synth.initial_population(X, y, 3, 64, RMAX=6, CMAX=3, seed=21)
    c2 = rs.Context(0)
    ds = c2.dataset(X, y, 3)
    try:
        c2.set_tile_config(tile)
        got, fit, best, mean = c2.evolve(ds, pop, generations=3, elite=2, seed=21)
    finally:
        c2.dataset_destroy(ds)
        c2.close()
    want, wfit, wbest, _ = oracle_run(orc, X, y, 3, pop, 3, 2, 21)
    for k in want:
        assert np.array_equal(got[k], want[k]), k
    assert np.array_equal(fit, wfit)
    assert np.array_equal(best, wbest)


def test_lamarckian_tuning_keeps_best_monotone(ctx, orc):
    X, y = synth.two_class_gaussian(4000, 8, 5)
    pop = synth.initial_population(X, y, 2, 64, RMAX=6, CMAX=3, seed=5)
    ds = ctx.dataset(X, y, 2)
    try:
        got, fit, best, mean = ctx.evolve(ds, pop, generations=6, elite=2, seed=5, tune_every=2,
                                          tune_top=8, tune_steps=5, tau=0.1, lr=1e-2, lamarckian=True)
    finally:
        ctx.dataset_destroy(ds)
    assert (np.diff(best) >= 0).all(), best
    # the returned fitness is the exact evaluation of the returned genomes
    wfit, _, _ = orc.eval_hard(X, y, 2, synth.batch_from_population(got))
    assert np.array_equal(fit, wfit)


def test_baldwinian_tuning_runs_and_keeps_valid_genomes(ctx, orc):
    X, y = synth.two_class_gaussian(4000, 8, 6)
    pop = synth.initial_population(X, y, 2, 64, RMAX=6, CMAX=3, seed=6)
    ds = ctx.dataset(X, y, 2)
    try:
        got, fit, best, mean = ctx.evolve(ds, pop, generations=4, elite=2, seed=6, tune_every=1,
                                          tune_top=8, tune_steps=3)
    finally:
        ctx.dataset_destroy(ds)
    wfit, _, _ = orc.eval_hard(X, y, 2, synth.batch_from_population(got))
    assert np.array_equal(fit, wfit)


def test_finetune_matches_float64_adam(ctx, orc):
    """Three Adam steps of the library against float64 Adam on the oracle's gradients."""
    import torch
    from paper_2406_01821_gb300 import rs
    X, y = synth.two_class_gaussian(3000, 6, 7)
    b = synth.random_rulesets(synth.quantile_table(X), 2, 6, (1, 5), (1, 3), 7, pair_prob=0.3)
    b.set_default[:] = np.where(b.rule_class[b.set_rule_off[:-1]] == 0, 1, 0)
    tau, lr, steps = 0.25, 1e-2, 3
    ds = ctx.dataset(X, y, 2)
    try:
        a, bb, t, trace = ctx.finetune(ds, rs.DeviceBatch.from_host(b), tau, lr, steps)
        torch.cuda.synchronize()
        a, bb, t = a.cpu().numpy(), bb.cpu().numpy(), t.cpu().numpy()
    finally:
        ctx.dataset_destroy(ds)
    # float64 reference: Adam on the oracle's gradients
    pair = b.cond_g >= 0
    th = [b.cond_a.astype(np.float64), np.where(pair, b.cond_b, b.cond_t).astype(np.float64)]
    m = [np.zeros(b.C), np.zeros(b.C)]
    v = [np.zeros(b.C), np.zeros(b.C)]
    ref_trace = []
    well = np.ones(b.C, bool)
    for step in range(1, steps + 1):
        cur = synth.Batch(**b.arrays())
        cur.cond_a = th[0].astype(np.float32)
        cur.cond_b = np.where(pair, th[1], 0).astype(np.float32)
        cur.cond_t = np.where(pair, 0, th[1]).astype(np.float32)
        out = orc.soft(X, y, 2, cur, tau, dloss=np.ones(b.P), want_mag=True)
        ref_trace.append(out["loss"])
        g = [out["grad_a"], np.where(pair, out["grad_b"], out["grad_t"])]
        mag = [out["mag_a"], np.where(pair, out["mag_b"], out["mag_t"])]
        for k in range(2):
            well &= np.abs(g[k]) > 1e-3 * mag[k]          # the sign of the step is well determined
            m[k] = 0.9 * m[k] + 0.1 * g[k]
            v[k] = 0.999 * v[k] + 0.001 * g[k] ** 2
            mh, vh = m[k] / (1 - 0.9 ** step), v[k] / (1 - 0.999 ** step)
            th[k] = th[k] - lr * mh / (np.sqrt(vh) + 1e-8)
    assert np.allclose(trace, np.array(ref_trace), rtol=1e-5, atol=0)
    got2 = np.where(pair, bb, t)
    assert well.sum() > 0.5 * b.C
    assert np.allclose(a[well], th[0][well], rtol=0, atol=1e-5)
    assert np.allclose(got2[well], th[1][well], rtol=0, atol=1e-5)


def test_finetune_rejects_malformed_batch_before_any_step(ctx):
    """A batch naming a class outside 0..K-1 is refused by the one validation before the steps."""
    import torch
    from paper_2406_01821_gb300 import rs
    X, y = synth.two_class_gaussian(500, 4, 9)
    b = synth.random_rulesets(synth.quantile_table(X), 2, 5, (1, 4), (1, 3), 9, pair_prob=0.3)
    b.rule_class[2] = 2
    ds = ctx.dataset(X, y, 2)
    try:
        db = rs.DeviceBatch.from_host(b)
        with pytest.raises(rs.RsError) as e:
            ctx.finetune(ds, db, 0.2, 1e-2, 5)
        assert e.value.code == -1
        torch.cuda.synchronize()
    finally:
        ctx.dataset_destroy(ds)


@pytest.mark.parametrize("tune", [False, True])
def test_checkpoint_resume_continues_exactly(ctx, tmp_path, tune):
    """A run of 7 generations equals 3 generations, a checkpoint written and read back, and 4 more
    generations resumed from it (random counters and the tuning schedule use the absolute
    generation index)."""
    from paper_2406_01821_gb300 import rs
    X, y = synth.two_class_gaussian(3000, 8, 9)
    pop = synth.initial_population(X, y, 2, 80, RMAX=6, CMAX=3, seed=9)
    kw = dict(elite=2, seed=9)
    if tune:
        kw.update(tune_every=2, tune_top=6, tune_steps=3, tau=0.2, lr=1e-2)
    ds = ctx.dataset(X, y, 2)
    try:
        full, ffit, fbest, _ = ctx.evolve(ds, pop, generations=7, **kw)
        part, _, pbest, _ = ctx.evolve(ds, pop, generations=3, **kw)
        path = str(tmp_path / "ckpt.npz")
        rs.Context.save_population(path, part, 9, 3)
        pop2, seed2, g2 = rs.Context.load_population(path)
        assert seed2 == 9 and g2 == 3
        rest, rfit, rbest, _ = ctx.evolve(ds, pop2, generations=4, first_generation=g2, **kw)
    finally:
        ctx.dataset_destroy(ds)
    for k in full:
        assert np.array_equal(rest[k], full[k]), k
    assert np.array_equal(rfit, ffit)
    assert np.array_equal(np.concatenate([pbest[:3], rbest]), fbest)


@pytest.mark.parametrize("lamarckian", [False, True])
def test_captured_generations_equal_direct_launches(ctx, lamarckian):
    """Generations replayed from captured graphs (the generation index read on the device) give
    the same populations, fitness and statistics as generations launched one kernel at a time,
    with fine-tuning every third generation (generations 2, 5 and 8 of 10, counted from 3): each
    (parity, tuning) graph is used, and all but (odd, tuned) are replayed."""
    from paper_2406_01821_gb300 import rs
    X, y = synth.two_class_gaussian(3000, 8, 11)
    pop = synth.initial_population(X, y, 2, 48, RMAX=6, CMAX=3, seed=11)
    direct = rs.Context(0, flags=rs.CTX_NO_GRAPH)
    kw = dict(generations=9, elite=2, seed=11, tune_every=3, tune_top=8, tune_steps=4, tau=0.1, lr=1e-2,
              lamarckian=lamarckian, first_generation=3)
    try:
        results = []
        for c in (ctx, direct):
            ds = c.dataset(X, y, 2)
            try:
                results.append(c.evolve(ds, pop, **kw))
            finally:
                c.dataset_destroy(ds)
    finally:
        direct.close()
    (ga, gfit, gbest, gmean), (da, dfit, dbest, dmean) = results
    for k in ga:
        assert np.array_equal(ga[k], da[k]), k
    assert np.array_equal(gfit, dfit) and np.array_equal(gbest, dbest) and np.array_equal(gmean, dmean)


@pytest.mark.parametrize("what", ["nrule", "ncond"])
def test_population_counts_checked_before_any_kernel(ctx, what):
    """A slot count beyond RMAX / CMAX (which would send the slot readers past a set's row) is
    refused with RS_ERR_INVALID before anything runs."""
    from paper_2406_01821_gb300 import rs
    X, y = synth.two_class_gaussian(400, 4, 12)
    pop = synth.initial_population(X, y, 2, 16, RMAX=4, CMAX=3, seed=12)
    if what == "nrule":
        pop["nrule"][15] = 5
    else:
        pop["ncond"][15, 0] = 4
    ds = ctx.dataset(X, y, 2)
    try:
        with pytest.raises(rs.RsError) as e:
            ctx.evolve(ds, pop, generations=2, elite=1, seed=12)
        assert e.value.code == -1
    finally:
        ctx.dataset_destroy(ds)
