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


def log1m_exp_coefficients():
    """The two polynomials of log1m_exp in csrc/soft.cu, constant term first: a (the q piece,
    Horner in q) and b (the t piece, Horner in t)."""
    src = open(os.path.join(ROOT, "paper_2406_01821_gb300", "csrc", "soft.cu")).read()
    body = src[src.index("float log1m_exp(float s)"):]
    body = body[:body.index("const bool sub")]
    a_src = body[body.index("float pa ="):body.index("const float ra")]
    b_src = body[body.index("float pb ="):]
    coef = lambda txt: [float(x) for x in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", txt)][::-1]
    return coef(a_src), coef(b_src)


def test_log1m_exp_coefficients_match_the_remez_fits():
    pytest.importorskip("mpmath")
    from paper_2406_01821_gb300 import log1p_fit
    a, b = log1m_exp_coefficients()
    fa, ea = log1p_fit.remez_log1m_exp_small_q()
    fb, eb = log1p_fit.remez_log1m_exp_near_one()
    assert ea < 1.3e-8 and eb < 7e-9
    assert len(a) == 11 and len(b) == 4
    assert np.allclose(a, np.float32(fa), rtol=1e-6, atol=0)
    assert np.allclose(b, np.float32(fb), rtol=1e-6, atol=0)


def test_log1m_exp_pieces_within_bound():
    """Given exact q = e^s and log t, the float32 evaluation of each piece is within 2 ulp."""
    from paper_2406_01821_gb300 import log1p_fit
    a, b = log1m_exp_coefficients()
    ua, ub = log1p_fit.log1m_exp_pieces_error_ulp(a, b, samples=300_000)
    assert ua <= 2.0 and ub <= 1.5, (ua, ub)


def test_log1m_exp_pieces_catch_a_wrong_coefficient():
    """A planted error in one coefficient of each piece leaves its bound (the check has teeth)."""
    from paper_2406_01821_gb300 import log1p_fit
    a, b = log1m_exp_coefficients()
    a_bad = list(a)
    a_bad[5] *= 1.0001
    b_bad = list(b)
    b_bad[1] *= 1.001
    ua, _ = log1p_fit.log1m_exp_pieces_error_ulp(a_bad, b, samples=100_000)
    _, ub = log1p_fit.log1m_exp_pieces_error_ulp(a, b_bad, samples=100_000)
    assert ua > 2.0 and ub > 1.5, (ua, ub)
