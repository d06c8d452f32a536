"""Derivation of the polynomial behind the soft kernels' log(1 + e) on [0, 1] (`log1p_unit` in
csrc/soft.cu): p of degree 8 with the least maximum relative error of e p(e) against log1p(e),
i.e. of p against log1p(e) / e, found by the Remez exchange in 50-digit arithmetic (mpmath), then
rounded to float32 and checked as the kernels evaluate it (Horner's rule in fused multiply-adds,
then one multiply by e) against float64 log1p.

Run: python -m paper_2406_01821_gb300.log1p_fit   (needs mpmath; not used at run time)
"""
from __future__ import annotations

import numpy as np


def remez(n: int, grid_points: int = 20000, iters: int = 30):
    import mpmath as mp
    mp.mp.dps = 50

    def q(x):
        return mp.mpf(1) if x == 0 else mp.log1p(x) / x

    m = n + 2
    xs = [mp.mpf(1) / 2 - mp.cos(mp.pi * i / (m - 1)) / 2 for i in range(m)]   # Chebyshev start
    grid = [mp.mpf(i) / grid_points for i in range(grid_points + 1)]
    for _ in range(iters):
        # p(x_i) - q(x_i) = (-1)^i E q(x_i): equal relative error of alternating sign
        A = mp.matrix(m, m)
        rhs = mp.matrix(m, 1)
        for i, x in enumerate(xs):
            for j in range(n + 1):
                A[i, j] = x ** j
            A[i, n + 1] = (-1) ** i * q(x)
            rhs[i] = q(x)
        sol = mp.lu_solve(A, rhs)
        c = [sol[j] for j in range(n + 1)]

        def rel_err(x):
            p = mp.mpf(0)
            for cj in reversed(c):
                p = p * x + cj
            return (p - q(x)) / q(x)

        ev = [rel_err(x) for x in grid]
        # the new reference: the largest error of each run of one sign
        runs, start = [], 0
        for k in range(1, len(grid)):
            if ev[k] != 0 and mp.sign(ev[k]) != mp.sign(ev[start]):
                runs.append((start, k - 1))
                start = k
        runs.append((start, len(grid) - 1))
        pts = [max(range(a, b + 1), key=lambda k: abs(ev[k])) for a, b in runs]
        while len(pts) > m:
            pts.pop(0 if abs(ev[pts[0]]) < abs(ev[pts[-1]]) else -1)
        if len(pts) < m:
            break
        xs = [grid[k] for k in pts]
    return [float(x) for x in c], float(max(abs(e) for e in ev))


def float32_error_ulp(coeffs, samples: int = 2_000_000, seed: int = 0) -> float:
    """Largest error in float32 ulps of e * Horner(coeffs, e) over [0, 1] (uniform and
    log-uniform samples, the edges included), against float64 log1p."""
    cf = np.asarray(coeffs, np.float32)
    rng = np.random.default_rng(seed)
    e = np.concatenate([rng.random(samples), 10.0 ** rng.uniform(-30, 0, samples // 2),
                        [0.0, 1.0, 2.0 ** -24, 2.0 ** -126]]).astype(np.float32)
    ed = e.astype(np.float64)
    p = np.full_like(ed, np.float64(cf[-1]))
    for cj in cf[-2::-1]:
        p = (p * ed + np.float64(cj)).astype(np.float32).astype(np.float64)   # a float32 FMA
    r = (ed * p).astype(np.float32).astype(np.float64)
    ref = np.log1p(ed)
    ulp = np.maximum(np.spacing(ref.astype(np.float32)).astype(np.float64), 2.0 ** -149)
    return float((np.abs(r - ref) / ulp).max())


if __name__ == "__main__":
    coeffs, err = remez(8)
    c32 = [float(np.float32(c)) for c in coeffs]
    print(f"degree 8: max relative error {err:.3g} before rounding")
    print("float32 coefficients, constant term first:", ", ".join("%.9e" % c for c in c32))
    print(f"float32 evaluation: at most {float32_error_ulp(c32):.2f} ulp of log1p")
