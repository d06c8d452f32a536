"""Sample-sharded evaluation (one exchange step): each rank evaluates every rule set on its own
sample range, and one all-reduce of the int32 counts (or a rank-ordered sum of the weighted soft
results) gives the whole-dataset result. Two gloo ranks on the CPU run the collective with the
oracle standing in for the GPU kernels; on one GPU, two shards evaluated by the library add up to
the whole-dataset counts and soft results."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2406_01821_gb300 import shard, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("N,world", [(0, 1), (1, 2), (10, 3), (1000, 4), (1 << 20, 8), (7, 7), (5, 8)])
def test_sample_ranges_partition(N, world):
    r = shard.sample_ranges(N, world)
    assert len(r) == world and r[0][0] == 0 and r[-1][1] == N
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    sizes = [b - a for a, b in r]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1 and sum(sizes) == N


def _case():
    X, y = synth.gaussian_mixture(3001, 12, 4, 17)
    b = synth.random_rulesets(synth.quantile_table(X), 4, 40, (1, 12), (1, 5), 17, pair_prob=0.3)
    return X, y, b


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X, y, b = _case()

    def hard(Xs, ys, K, batch):
        c, pc, _ = oracle.eval_hard(Xs, ys, K, batch)
        return c, pc

    def soft(Xs, ys, K, batch, tau, dl):
        return oracle.soft(Xs, ys, K, batch, tau, dloss=dl)

    sh = shard.SampleShard(X, y, 4, rank, world, evaluate=hard, soft_evaluate=soft)
    c, pc = sh.eval_hard(b)
    dl = np.linspace(0.5, 1.5, b.P)
    s = sh.soft(b, 0.3, dl)
    out[rank] = {"c": c.numpy().copy(), "pc": pc.numpy().copy(), "n_local": sh.n_local,
                 **{k: v.numpy().copy() for k, v in s.items()}}
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reduce_to_whole_dataset(orc, world):
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:     # no fork: the parent may hold a CUDA context
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    X, y, b = _case()
    want = orc.eval_hard(X, y, 4, b)
    dl = np.linspace(0.5, 1.5, b.P)
    ref = orc.soft(X, y, 4, b, 0.3, dloss=dl, want_mag=True)
    assert sum(res[r]["n_local"] for r in range(world)) == len(X)
    for r in range(world):
        assert np.array_equal(res[r]["c"], want[0])                 # exact on every rank
        assert np.array_equal(res[r]["pc"], want[1].reshape(b.P, 4))
        assert np.array_equal(res[r]["loss"], res[0]["loss"])       # the same sum on every rank
        fin = np.isfinite(ref["loss"])
        assert fin.sum() >= 10 and (np.isinf(res[r]["loss"]) == ~fin).all()
        assert np.allclose(res[r]["loss"][fin], ref["loss"][fin], rtol=1e-12, atol=0)
        ok = _finite_set_conditions(b, fin)        # a set with an unreachable label has no gradient
        for n in ("a", "b", "t"):
            err = np.abs(res[r]["grad_" + n] - ref["grad_" + n])[ok]
            bound = 1e-12 * np.maximum(np.abs(ref["grad_" + n]), ref["mag_" + n])[ok]
            assert (err <= bound + 1e-300).all()


def _finite_set_conditions(b, fin):
    ok = np.zeros(b.C, bool)
    for p in np.nonzero(fin)[0]:
        ok[b.rule_cond_off[b.set_rule_off[p]]:b.rule_cond_off[b.set_rule_off[p + 1]]] = True
    return ok


@pytest.mark.gpu
def test_two_shards_on_one_gpu_add_up(orc):
    """The library path of a rank: each shard registered as its own dataset (its own label
    grouping and rank tables) and evaluated by the kernels; the two shards' counts add up to the
    whole dataset's, and their weighted soft results to the whole-dataset soft pass."""
    import torch
    from paper_2406_01821_gb300 import build, rs
    build.build()
    X, y, b = _case()
    with rs.Context(0) as ctx:
        shards = [shard.SampleShard(X, y, 4, r, 2, ctx=ctx) for r in range(2)]
        db = rs.DeviceBatch.from_host(b)
        local = [s.local_hard(db) for s in shards]
        torch.cuda.synchronize()
        total = (local[0] + local[1]).cpu().numpy()
        want = orc.eval_hard(X, y, 4, b)
        assert np.array_equal(total[:b.P], want[0])
        assert np.array_equal(total[b.P:].reshape(b.P, 4), want[1].reshape(b.P, 4))
        dl = np.linspace(0.5, 1.5, b.P)
        parts = [s.local_soft(db, 0.3, dl) for s in shards]
        soft = (parts[0] + parts[1]).cpu().numpy().astype(np.float64)
        ref = orc.soft(X, y, 4, b, 0.3, dloss=dl, want_mag=True)
        fin = np.isfinite(ref["loss"])
        assert np.allclose(soft[:b.P][fin], ref["loss"][fin], rtol=1e-5, atol=0)
        ok = _finite_set_conditions(b, fin)
        for i, n in enumerate(("a", "b", "t")):
            g = soft[b.P + i * b.C:b.P + (i + 1) * b.C]
            err = np.abs(g - ref["grad_" + n])[ok]
            bound = 1e-5 * np.maximum(np.abs(ref["grad_" + n]), ref["mag_" + n])[ok]
            assert (err <= bound + 1e-30).all(), n
        for s in shards:
            s.close()
