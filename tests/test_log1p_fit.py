"""The soft kernels' log(1 + e) polynomial (csrc/soft.cu, log1p_unit) is the one its derivation
script produces: a Remez fit of log1p(e) / e on [0, 1], rounded to float32, within 2.5 ulp of
float64 log1p when evaluated as the kernels do (no GPU: the evaluation is simulated in numpy)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def kernel_coefficients():
    src = open(os.path.join(ROOT, "paper_2406_01821_gb300", "csrc", "soft.cu")).read()
    body = src[src.index("float log1p_unit(float e)"):]
    body = body[:body.index("return e * p;")]
    nums = re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)
    first = float(nums[0])                       # the leading (degree 8) coefficient
    rest = [float(x) for x in nums[1:]]
    return [*reversed(rest), first]              # constant term first


def test_coefficients_match_the_remez_fit():
    pytest.importorskip("mpmath")
    from paper_2406_01821_gb300 import log1p_fit
    fit, err = log1p_fit.remez(8, grid_points=4000, iters=12)
    assert err < 3.1e-8
    got = kernel_coefficients()
    assert len(got) == 9
    assert np.allclose(got, np.float32(fit), rtol=1e-6, atol=0)


def test_float32_evaluation_within_bound():
    from paper_2406_01821_gb300 import log1p_fit
    assert log1p_fit.float32_error_ulp(kernel_coefficients(), samples=400_000) <= 2.5
