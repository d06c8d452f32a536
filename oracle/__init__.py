"""CPU oracle for ordered rule-set evaluation -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The library under ``paper_2406_01821_gb300`` never imports, links or calls
it, and the two share no code: the only common ground is the input layout and the seeded
generators in ``paper_2406_01821_gb300.synth`` (which hold none of the method's arithmetic).

Functions (each follows the paper, "GPU-Accelerated Rule Evaluation and Evolution"):
  eval_hard   Sec. 3 / Fig. 1a-b: inequalities with a strict sign activation, conjunction per
              rule, first firing rule of the ordered list (Sec. 1 list grammar), default class
              otherwise; fitness = correct counts (Sec. 1). float32 products, no FMA. Categorical
              membership conditions (Sec. 5 future work): x[f] an integer code 0..63 in a set.
  soft        Sec. 3: sigmoid relaxation for back-propagation of coefficients and thresholds
              (Fig. 1c). float64, log domain. Loss, class probabilities and the adjoint.
  evolve_step Sec. 3: tournament selection and offspring with randomized coefficients.

Parity status: eval_hard and soft are pinned by tests (worked example of Fig. 1, a second
dense formulation, brute force, closed forms, invariants, finite differences; membership tests
by hand-written edge values, numpy's isin and the band form of a single code). The paper's
example accuracies (21.05% -> 92.40%) are parity unpinned: the dataset and optimizer behind
them are not available.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC", "-std=c11"]


def build(force: bool = False, plant: int = 0) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so.

    ``plant`` > 0 builds a deliberately wrong variant (liboracle_plantN.so) for the test that
    checks that the pins catch it; it is never used otherwise.
    """
    srcs = [os.path.join(_HERE, f) for f in ("oracle.c", "evolve.c")]
    srcs = [s for s in srcs if os.path.exists(s)]
    so = _SO if plant == 0 else _SO.replace(".so", f"_plant{plant}.so")
    os.makedirs(os.path.dirname(so), exist_ok=True)
    if not force and os.path.exists(so):
        so_m = os.path.getmtime(so)
        if all(os.path.getmtime(s) <= so_m for s in srcs):
            return so
    tmp = so + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, f"-DORC_PLANT={int(plant)}", *srcs, "-o", tmp, "-lm"])
    os.replace(tmp, so)
    return so


class _Batch(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32),
                ("set_rule_off", ctypes.c_void_p), ("rule_cond_off", ctypes.c_void_p),
                ("rule_class", ctypes.c_void_p), ("set_default", ctypes.c_void_p),
                ("cond_f", ctypes.c_void_p), ("cond_g", ctypes.c_void_p),
                ("cond_op", ctypes.c_void_p), ("cond_a", ctypes.c_void_p),
                ("cond_b", ctypes.c_void_p), ("cond_t", ctypes.c_void_p),
                ("cond_set", ctypes.c_void_p)]


def _load(path):
    h = ctypes.CDLL(path)
    h.orc_eval_hard.restype = ctypes.c_int
    h.orc_soft.restype = ctypes.c_int
    h.orc_num_threads.restype = ctypes.c_int
    h.orc_evolve_step.restype = ctypes.c_int
    return h


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _cbatch(b):
    keep = {
        "set_rule_off": np.ascontiguousarray(b.set_rule_off, np.int32),
        "rule_cond_off": np.ascontiguousarray(b.rule_cond_off, np.int32),
        "rule_class": np.ascontiguousarray(b.rule_class, np.int32),
        "set_default": np.ascontiguousarray(b.set_default, np.int32),
        "cond_f": np.ascontiguousarray(b.cond_f, np.int32),
        "cond_g": np.ascontiguousarray(b.cond_g, np.int32),
        "cond_op": np.ascontiguousarray(b.cond_op, np.int8),
        "cond_a": np.ascontiguousarray(b.cond_a, np.float32),
        "cond_b": np.ascontiguousarray(b.cond_b, np.float32),
        "cond_t": np.ascontiguousarray(b.cond_t, np.float32),
        "cond_set": (np.ascontiguousarray(b.cond_set, np.uint64)
                     if getattr(b, "cond_set", None) is not None else None),
    }
    cb = _Batch(int(keep["set_default"].shape[0]), *[_ptr(keep[k]) for k in
                ("set_rule_off", "rule_cond_off", "rule_class", "set_default", "cond_f", "cond_g",
                 "cond_op", "cond_a", "cond_b", "cond_t", "cond_set")])
    return cb, keep


def num_threads(requested: int = 0) -> int:
    return int(lib().orc_num_threads(int(requested)))


def eval_hard(X, y, K, batch, want_preds=False, want_per_class=True, nthreads=0, _h=None):
    """Returns (correct[P], per_class[P,K] or None, preds[P,N] or None)."""
    X = np.ascontiguousarray(X, np.float32)
    y = np.ascontiguousarray(y, np.int32)
    N, F = X.shape
    cb, keep = _cbatch(batch)
    P = cb.P
    correct = np.zeros(P, np.int32)
    per_class = np.zeros((P, K), np.int32) if want_per_class else None
    preds = np.zeros((P, N), np.int32) if want_preds else None
    (_h or lib()).orc_eval_hard(_ptr(X), ctypes.c_int64(N), ctypes.c_int32(F), _ptr(y), ctypes.c_int32(K),
                        ctypes.byref(cb), _ptr(correct), _ptr(per_class), _ptr(preds),
                        ctypes.c_int(nthreads))
    return correct, per_class, preds


def soft(X, y, K, batch, tau, dloss=None, want_probs=False, want_mag=False, nthreads=0, _h=None):
    """float64 soft forward (+ adjoint when dloss is given).

    Returns a dict with 'loss' [P], optionally 'probs' [P,N,K], 'grad_a','grad_b','grad_t' [C]
    and 'mag_a','mag_b','mag_t' [C]. ``tau`` is used as the float64 value of the float32 number.
    """
    X = np.ascontiguousarray(X, np.float32)
    y = np.ascontiguousarray(y, np.int32)
    N, F = X.shape
    cb, keep = _cbatch(batch)
    P, C = cb.P, int(keep["cond_f"].shape[0])
    out = {"loss": np.zeros(P, np.float64)}
    probs = np.zeros((P, N, K), np.float64) if want_probs else None
    g = [None] * 6
    dl = None
    if dloss is not None:
        dl = np.ascontiguousarray(np.broadcast_to(np.asarray(dloss, np.float64), (P,)), np.float64)
        g[:3] = [np.zeros(C, np.float64) for _ in range(3)]
        if want_mag:
            g[3:] = [np.zeros(C, np.float64) for _ in range(3)]
    (_h or lib()).orc_soft(_ptr(X), ctypes.c_int64(N), ctypes.c_int32(F), _ptr(y), ctypes.c_int32(K),
                   ctypes.byref(cb), ctypes.c_double(float(np.float32(tau))), _ptr(out["loss"]),
                   _ptr(probs), _ptr(dl), *[_ptr(a) for a in g], ctypes.c_int(nthreads))
    if probs is not None:
        out["probs"] = probs
    if dl is not None:
        out["grad_a"], out["grad_b"], out["grad_t"] = g[:3]
        if want_mag:
            out["mag_a"], out["mag_b"], out["mag_t"] = g[3:]
    return out


def planted(plant: int):
    """A namespace with ``eval_hard`` / ``soft`` backed by a deliberately wrong build, for the
    test that checks that the pins detect each planted mistake."""
    import functools
    import types
    h = _load(build(plant=plant))
    return types.SimpleNamespace(eval_hard=functools.partial(eval_hard, _h=h),
                                 soft=functools.partial(soft, _h=h),
                                 evolve_step=functools.partial(evolve_step, _h=h), build=build)


# ------------------------------------------------------------------------------ evolution

class _Pop(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("RMAX", ctypes.c_int32), ("CMAX", ctypes.c_int32)] + \
               [(n, ctypes.c_void_p) for n in ("nrule", "deflt", "rcls", "ncond", "cf", "cg", "cop",
                                               "ca", "cb", "ct")]


POP_FIELDS = {"nrule": np.int32, "deflt": np.int32, "rcls": np.int32, "ncond": np.int32,
              "cf": np.int32, "cg": np.int32, "cop": np.int8, "ca": np.float32, "cb": np.float32,
              "ct": np.float32}


def _cpop(pop):
    arrs = {k: np.ascontiguousarray(pop[k], t) for k, t in POP_FIELDS.items()}
    P, RMAX, CMAX = arrs["cf"].shape
    return _Pop(P, RMAX, CMAX, *[_ptr(arrs[k]) for k in POP_FIELDS]), arrs


def philox4x64_10(ctr, key):
    """Philox4x64-10 block for counter[4], key[2] (uint64)."""
    out = np.zeros(4, np.uint64)
    c = np.ascontiguousarray(ctr, np.uint64)
    k = np.ascontiguousarray(key, np.uint64)
    lib().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def evolve_step(pop, fit, seed, gen, elite, X, K, _h=None):
    """One generation (tournament selection, crossover, mutation with randomized coefficients).
    ``pop`` is a dict of slot arrays (see POP_FIELDS; condition arrays are [P, RMAX, CMAX])."""
    cin, keep_in = _cpop(pop)
    out = {k: np.zeros_like(v) for k, v in keep_in.items()}
    cout, keep_out = _cpop(out)
    fit = np.ascontiguousarray(fit, np.int32)
    X = np.ascontiguousarray(X, np.float32)
    rc = (_h or lib()).orc_evolve_step(ctypes.byref(cin), _ptr(fit), ctypes.byref(cout), ctypes.c_uint64(seed),
                               ctypes.c_uint64(gen), ctypes.c_int32(elite), _ptr(X),
                               ctypes.c_int64(X.shape[0]), ctypes.c_int32(X.shape[1]),
                               ctypes.c_int32(K))
    if rc != 0:
        raise ValueError("population shape not supported by the oracle")
    return keep_out
