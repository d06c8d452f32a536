"""The C ABI used from C: tests/abi_consumer.c registers a dataset and evaluates a population
through rs.h alone (host arrays in, host counts out) and must give the oracle's counts exactly;
it also reports the latency of one synchronous call without the Python binding."""
import os
import sys

import numpy as np
import pytest

from paper_2406_01821_gb300 import synth

pytestmark = pytest.mark.gpu
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("case", ["plain", "ragged"])
def test_c_program_counts_equal_oracle(orc, tmp_path, case):
    import c_consumer
    from paper_2406_01821_gb300 import build
    build.build()
    if case == "plain":                              # the paper's shape: 64 sets on 569 x 30
        w = synth.plain_hard(seed=0)
        X, y, K, b = w.X, w.y, w.K, w.batch
    else:                                            # ragged sets over several tiles and a ragged tail
        X, y = synth.gaussian_mixture(3001, 24, 5, 9)
        b = synth.random_rulesets(synth.quantile_table(X), 5, 96, (1, 20), (1, 6), 9)
        K = 5
    exe = c_consumer.build(str(tmp_path))
    path = str(tmp_path / "input.bin")
    c_consumer.write_input(path, X, y, K, b)
    correct, per_class, us = c_consumer.run(exe, path, calls=200)
    want_c, want_pc, _ = orc.eval_hard(X, y, K, b)
    assert np.array_equal(correct, want_c)
    assert np.array_equal(per_class, np.asarray(want_pc).ravel())
    print(f"{case}: {us:.1f} us per synchronous rs_eval_hard call from C (host batch, host counts)")
