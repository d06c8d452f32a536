"""Derivation of the polynomials behind the soft kernels' logarithms (csrc/soft.cu), each a
polynomial of least maximum relative error found by the Remez exchange in 50-digit arithmetic
(mpmath), rounded to float32 and checked as the kernels evaluate it (Horner's rule in fused
multiply-adds) against float64:

* `log1p_unit`: log(1 + e) on [0, 1] as e p(e), p of degree 8 fitted to log1p(e) / e.
* `log1m_exp`: log(1 - e^s) for s <= 0, the log-probability that a rule with log q = s does not
  fire, in two pieces split at s = -1/2:
  - q = e^s <= e^(-1/2): log1p(-q) = -q a(q), a of degree 10 fitted to -log1p(-q) / q on
    [0, e^(-1/2)] (relative accuracy of log1p(-q) as q goes to 0);
  - t = -s < 1/2: log(1 - e^-t) = log t + t b(t), b of degree 3 fitted to
    log((1 - e^-t) / t) / t on [0, 1/2] (a smooth function; log t carries the singularity).

Run: python -m paper_2406_01821_gb300.log1p_fit   (needs mpmath; not used at run time)
"""
from __future__ import annotations

import numpy as np

LOG1M_EXP_SPLIT = 0.5      # t = -s at which log1m_exp changes piece


def remez_rel(q, a, b, n: int, grid_points: int = 20000, iters: int = 30):
    """Coefficients (constant term first) of the degree-n polynomial p with the least maximum of
    |p(x) - q(x)| / |q(x)| over [a, b] (q without zeros there), and that maximum, by the Remez
    exchange on a uniform grid: solve for equal relative errors of alternating sign on n + 2
    reference points, then move the references to the extrema of the error's runs of one sign."""
    import mpmath as mp
    mp.mp.dps = 50
    a, b = mp.mpf(a), mp.mpf(b)
    m = n + 2
    xs = [(a + b) / 2 - (b - a) * mp.cos(mp.pi * i / (m - 1)) / 2 for i in range(m)]  # Chebyshev start
    grid = [a + (b - a) * mp.mpf(i) / grid_points for i in range(grid_points + 1)]
    qg = [q(x) for x in grid]
    ev = []
    c = []
    for _ in range(iters):
        A = mp.matrix(m, m)
        rhs = mp.matrix(m, 1)
        for i, x in enumerate(xs):
            qx = q(x)
            for j in range(n + 1):
                A[i, j] = x ** j
            A[i, n + 1] = (-1) ** i * qx
            rhs[i] = qx
        sol = mp.lu_solve(A, rhs)
        c = [sol[j] for j in range(n + 1)]

        def rel_err(k):
            x = grid[k]
            p = mp.mpf(0)
            for cj in reversed(c):
                p = p * x + cj
            return (p - qg[k]) / qg[k]

        ev = [rel_err(k) for k in range(len(grid))]
        runs, start = [], 0
        for k in range(1, len(grid)):
            if ev[k] != 0 and mp.sign(ev[k]) != mp.sign(ev[start]):
                runs.append((start, k - 1))
                start = k
        runs.append((start, len(grid) - 1))
        pts = [max(range(s0, s1 + 1), key=lambda k: abs(ev[k])) for s0, s1 in runs]
        while len(pts) > m:
            pts.pop(0 if abs(ev[pts[0]]) < abs(ev[pts[-1]]) else -1)
        if len(pts) < m:
            break
        xs = [grid[k] for k in pts]
    return [float(x) for x in c], float(max(abs(e) for e in ev))


def remez(n: int, grid_points: int = 20000, iters: int = 30):
    """log1p_unit: log1p(e) / e on [0, 1]."""
    import mpmath as mp

    def q(x):
        return mp.mpf(1) if x == 0 else mp.log1p(x) / x

    return remez_rel(q, 0, 1, n, grid_points, iters)


def remez_log1m_exp_small_q(n: int = 10, grid_points: int = 6000, iters: int = 30):
    """log1m_exp, q <= e^(-1/2): -log1p(-q) / q on [0, e^(-1/2)]."""
    import mpmath as mp

    def q(w):
        return mp.mpf(1) if w == 0 else -mp.log1p(-w) / w

    return remez_rel(q, 0, mp.exp(-mp.mpf(LOG1M_EXP_SPLIT)), n, grid_points, iters)


def remez_log1m_exp_near_one(n: int = 3, grid_points: int = 6000, iters: int = 30):
    """log1m_exp, t = -s < 1/2: log((1 - e^-t) / t) / t on [0, 1/2] (-1/2 at t = 0)."""
    import mpmath as mp

    def q(t):
        return mp.mpf(-1) / 2 if t == 0 else mp.log(-mp.expm1(-t) / t) / t

    return remez_rel(q, 0, LOG1M_EXP_SPLIT, n, grid_points, iters)


def _horner32(coeffs, x):
    """Horner's rule in float32 fused multiply-adds (each step rounded once), in float64 arrays."""
    cf = np.asarray(coeffs, np.float32).astype(np.float64)
    p = np.full_like(x, cf[-1])
    for cj in cf[-2::-1]:
        p = (p * x + cj).astype(np.float32).astype(np.float64)
    return p


def float32_error_ulp(coeffs, samples: int = 2_000_000, seed: int = 0) -> float:
    """Largest error in float32 ulps of e * Horner(coeffs, e) over [0, 1] (uniform and
    log-uniform samples, the edges included), against float64 log1p."""
    rng = np.random.default_rng(seed)
    e = np.concatenate([rng.random(samples), 10.0 ** rng.uniform(-30, 0, samples // 2),
                        [0.0, 1.0, 2.0 ** -24, 2.0 ** -126]]).astype(np.float32)
    ed = e.astype(np.float64)
    r = (ed * _horner32(coeffs, ed)).astype(np.float32).astype(np.float64)
    ref = np.log1p(ed)
    ulp = np.maximum(np.spacing(ref.astype(np.float32)).astype(np.float64), 2.0 ** -149)
    return float((np.abs(r - ref) / ulp).max())


def log1m_exp_pieces_error_ulp(small_q, near_one, samples: int = 1_000_000, seed: int = 0):
    """Largest errors in float32 ulps of the two pieces of log1m_exp as the kernels evaluate them,
    given exact values of q = e^s and of log t (the device takes these from the hardware
    exponential and logarithm, whose own errors the GPU self-test covers): -q * a(q) against
    log1p(-q) on [0, e^(-1/2)], and fma(t, b(t), log t) against log(-expm1(-t)) on (0, 1/2)."""
    rng = np.random.default_rng(seed)
    w0 = np.exp(-LOG1M_EXP_SPLIT)
    q = np.concatenate([rng.random(samples) * w0, 10.0 ** rng.uniform(-38, 0, samples // 4) * w0,
                        [0.0, np.float32(w0)]]).astype(np.float32).astype(np.float64)
    ra = (-(q * _horner32(small_q, q))).astype(np.float32).astype(np.float64)
    refa = np.log1p(-q)
    ulpa = np.maximum(np.spacing(np.abs(refa).astype(np.float32)).astype(np.float64), 2.0 ** -149)
    t = np.concatenate([rng.random(samples) * LOG1M_EXP_SPLIT,
                        10.0 ** rng.uniform(-38, np.log10(LOG1M_EXP_SPLIT), samples // 4)])
    t = t[t > 0].astype(np.float32).astype(np.float64)
    t = t[t < LOG1M_EXP_SPLIT]
    lt = np.log(t).astype(np.float32).astype(np.float64)
    rb = (t * _horner32(near_one, t) + lt).astype(np.float32).astype(np.float64)
    refb = np.log(-np.expm1(-t))
    ulpb = np.spacing(np.abs(refb).astype(np.float32)).astype(np.float64)
    return float((np.abs(ra - refa) / ulpa).max()), float((np.abs(rb - refb) / ulpb).max())


if __name__ == "__main__":
    coeffs, err = remez(8)
    c32 = [float(np.float32(c)) for c in coeffs]
    print(f"log1p_unit, degree 8: max relative error {err:.3g} before rounding")
    print("float32 coefficients, constant term first:", ", ".join("%.9e" % c for c in c32))
    print(f"float32 evaluation: at most {float32_error_ulp(c32):.2f} ulp of log1p")
    ca, ea = remez_log1m_exp_small_q()
    cb, eb = remez_log1m_exp_near_one()
    print(f"log1m_exp, q <= e^-1/2, degree {len(ca) - 1}: max relative error {ea:.3g}")
    print("float32 coefficients, constant term first:", ", ".join("%.9e" % np.float32(c) for c in ca))
    print(f"log1m_exp, t < 1/2, degree {len(cb) - 1}: max relative error {eb:.3g}")
    print("float32 coefficients, constant term first:", ", ".join("%.9e" % np.float32(c) for c in cb))
    ua, ub = log1m_exp_pieces_error_ulp(ca, cb)
    print(f"float32 evaluation: {ua:.2f} ulp (q piece), {ub:.2f} ulp (t piece, log t exact)")
