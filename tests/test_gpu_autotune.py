"""The tile autotuner (rs_autotune) and its JSON cache, through the C ABI.

  - the tuner returns a compiled configuration whose counts equal the oracle's, and the next call
    of the same batch shape uses it (rs_tile_config_pick);
  - it writes the cache file, and a new context created with that file picks the same
    configuration for the same shape key without tuning again;
  - a corrupt, truncated or foreign cache file, or one that names a configuration the library
    does not have, is ignored: the context is created, uses the built-in heuristic and evaluates
    exactly;
  - a context created with RS_CTX_NO_AUTOTUNE never reads the file."""
import json

import numpy as np
import pytest

from paper_2406_01821_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def work():
    X, y = synth.gaussian_mixture(20011, 24, 5, 31)
    b = synth.random_rulesets(synth.quantile_table(X), 5, 300, (1, 30), (1, 6), 31)
    return X, y, b


def _counts(ctx, ds, b, K):
    import torch
    from paper_2406_01821_gb300 import rs
    c, pc, _ = ctx.eval_hard(ds, rs.DeviceBatch.from_host(b), K)
    torch.cuda.synchronize()
    return c.cpu().numpy(), pc.cpu().numpy()


def test_autotune_picks_exact_config_and_caches_it(tmp_path, work, orc):
    from paper_2406_01821_gb300 import build, rs
    build.build()
    X, y, b = work
    cache = tmp_path / "tune.json"
    want = orc.eval_hard(X, y, 5, b)
    with rs.Context(0, autotune_cache=str(cache)) as ctx:
        ds = ctx.dataset(X, y, 5)
        db = rs.DeviceBatch.from_host(b)
        heuristic = ctx.tile_pick(ds, db)
        best = ctx.autotune(ds, db)
        assert 0 <= best < rs.lib().rs_tile_config_count()
        assert ctx.tile_pick(ds, db) == best
        c, pc = _counts(ctx, ds, b, 5)
        assert np.array_equal(c, want[0]) and np.array_equal(pc, want[1].reshape(b.P, 5))
        ctx.set_tile_config(best)                    # the same configuration forced explicitly
        c2, _ = _counts(ctx, ds, b, 5)
        assert np.array_equal(c2, want[0])
        ctx.set_tile_config(-1)
        ctx.dataset_destroy(ds)
    table = json.loads(cache.read_text())
    assert best in table.values() and len(table) == 1
    # a new context reads the file at creation and picks the tuned configuration without tuning
    with rs.Context(0, autotune_cache=str(cache)) as ctx:
        ds = ctx.dataset(X, y, 5)
        db = rs.DeviceBatch.from_host(b)
        assert ctx.tile_pick(ds, db) == best
        c, _ = _counts(ctx, ds, b, 5)
        assert np.array_equal(c, want[0])
        # another shape key (another class count) is not in the table: the heuristic applies
        ds2 = ctx.dataset(X, np.minimum(y, 3).astype(np.int32), 4)
        assert ctx.tile_pick(ds2, db) == heuristic
        ctx.dataset_destroy(ds2)
        ctx.dataset_destroy(ds)
    # NO_AUTOTUNE contexts ignore the file
    with rs.Context(0, flags=rs.CTX_NO_AUTOTUNE, autotune_cache=str(cache)) as ctx:
        ds = ctx.dataset(X, y, 5)
        assert ctx.tile_pick(ds, rs.DeviceBatch.from_host(b)) == heuristic
        ctx.dataset_destroy(ds)


CORRUPT = [
    b"",
    b"{",
    b'{"F24|K5|C',
    b'{"F24|K5|C7|N14": 3',                 # no closing brace
    b'{"F24|K5|C7|N14": x}',
    b'{"F24|K5|C7|N14": -1}',
    b'{"F24|K5|C7|N14": 99999}',            # no such configuration
    b'{"F24|K5|C7|N14": 3,}',
    b'{"F24|K5|C7|N14": 3} trailing',
    b"[1, 2, 3]",
    bytes(range(256)),
]


@pytest.mark.parametrize("i", range(len(CORRUPT)))
def test_corrupt_cache_is_ignored(tmp_path, work, orc, i):
    from paper_2406_01821_gb300 import build, rs
    build.build()
    X, y, b = work
    with rs.Context(0) as plain:                       # the heuristic, for comparison
        ds = plain.dataset(X, y, 5)
        heuristic = plain.tile_pick(ds, rs.DeviceBatch.from_host(b))
        plain.dataset_destroy(ds)
    cache = tmp_path / "tune.json"
    cache.write_bytes(CORRUPT[i])
    with rs.Context(0, autotune_cache=str(cache)) as ctx:
        ds = ctx.dataset(X, y, 5)
        assert ctx.tile_pick(ds, rs.DeviceBatch.from_host(b)) == heuristic
        c, _ = _counts(ctx, ds, b, 5)
        assert np.array_equal(c, orc.eval_hard(X, y, 5, b)[0])
        ctx.dataset_destroy(ds)


def test_valid_cache_entry_for_this_shape_is_used(tmp_path, work):
    """A well-formed file written by hand: its entry for the batch's shape key is used."""
    from paper_2406_01821_gb300 import build, rs
    build.build()
    X, y, b = work
    cache = tmp_path / "tune.json"
    with rs.Context(0, autotune_cache=str(cache)) as ctx:
        ds = ctx.dataset(X, y, 5)
        best = ctx.autotune(ds, rs.DeviceBatch.from_host(b))
        ctx.dataset_destroy(ds)
    key = next(iter(json.loads(cache.read_text())))
    other = 5 if best != 5 else 3                       # another configuration that fits F = 24
    cache.write_text(json.dumps({key: other, "F7|K2|C2|N9": 1}, indent=1))
    with rs.Context(0, autotune_cache=str(cache)) as ctx:
        ds = ctx.dataset(X, y, 5)
        assert ctx.tile_pick(ds, rs.DeviceBatch.from_host(b)) == other
        ctx.dataset_destroy(ds)
