"""ctypes binding of librs.so (include/rs.h): argument marshalling only.

Every evaluation step runs in the library's CUDA kernels; this module turns tensors into the
pointers and sizes the C ABI takes. PyTorch is used for device memory and streams. If the
library has not been built (``paper_2406_01821_gb300.build``) the first call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "librs.so")

OK, PENDING = 0, 1
ERR = {-1: "RS_ERR_INVALID", -2: "RS_ERR_TOO_LARGE", -3: "RS_ERR_OOM", -4: "RS_ERR_TIMEOUT",
       -5: "RS_ERR_DEVICE", -6: "RS_ERR_UNSUPPORTED", -7: "RS_ERR_NOT_FOUND", -8: "RS_ERR_CANCELLED"}
MEM_HOST, MEM_DEVICE = 0, 1
OP_GT, OP_LT, OP_IN = 0, 1, 2          # cond_op values (OP_IN: category membership)
CTX_ASYNC, CTX_NO_GRAPH, CTX_NO_AUTOTUNE, CTX_PROFILE, CTX_COUNT_WORK = 1, 2, 4, 8, 16


class RsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR.get(code, code)}: {msg}")
        self.code = code


class rs_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("mem_budget_bytes", ctypes.c_uint64), ("autotune_cache", ctypes.c_char_p)]


class rs_batch(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("R", ctypes.c_int32), ("C", ctypes.c_int32),
                ("mem", ctypes.c_int32),
                ("set_rule_off", ctypes.c_void_p), ("rule_cond_off", ctypes.c_void_p),
                ("rule_class", ctypes.c_void_p), ("set_default", ctypes.c_void_p),
                ("cond_f", ctypes.c_void_p), ("cond_g", ctypes.c_void_p),
                ("cond_op", ctypes.c_void_p), ("cond_a", ctypes.c_void_p),
                ("cond_b", ctypes.c_void_p), ("cond_t", ctypes.c_void_p),
                ("cond_set", ctypes.c_void_p)]


class rs_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("hard_launches", ctypes.c_int64),
                ("hard_ms", ctypes.c_double), ("soft_launches", ctypes.c_int64),
                ("soft_ms", ctypes.c_double), ("hard_records_walked", ctypes.c_int64),
                ("hard_rows_walked", ctypes.c_int64), ("hard_rule_ends_walked", ctypes.c_int64),
                ("hard_set_tiles", ctypes.c_int64)]


class rs_pipe_rates(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("ffma", "fmul", "lop3", "popc", "ex2", "fset")]


class rs_population(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("nrule", "deflt", "rcls", "ncond", "cf", "cg", "cop",
                                               "ca", "cb", "ct", "fitness")]


class rs_ticket_info(ctypes.Structure):
    _fields_ = [("submit_ns", ctypes.c_int64), ("admit_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64)]


class rs_serving_stats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("active", ctypes.c_int64),
                ("device_bytes_in_use", ctypes.c_uint64), ("units_published", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_int64)]


class rs_dataset_stats(ctypes.Structure):
    _fields_ = [("datasets", ctypes.c_int64), ("resident", ctypes.c_int64),
                ("resident_bytes", ctypes.c_uint64), ("evictions", ctypes.c_int64),
                ("rebuilds", ctypes.c_int64)]


class rs_evolve_config(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("RMAX", ctypes.c_int32), ("CMAX", ctypes.c_int32),
                ("generations", ctypes.c_int32), ("elite", ctypes.c_int32),
                ("tune_every", ctypes.c_int32), ("tune_top", ctypes.c_int32),
                ("tune_steps", ctypes.c_int32), ("tau", ctypes.c_float), ("lr", ctypes.c_float),
                ("lamarckian", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("first_generation", ctypes.c_int32)]


_lib = None

_SIGS = {
    "rs_create": (ctypes.c_int32, [ctypes.POINTER(rs_config), ctypes.POINTER(ctypes.c_void_p)]),
    "rs_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "rs_last_error": (ctypes.c_char_p, []),
    "rs_version": (ctypes.c_char_p, []),
    "rs_check": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p]),
    "rs_dataset_create": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_uint64)]),
    "rs_dataset_destroy": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64]),
    "rs_set_dataset_budget": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64]),
    "rs_dataset_stats_read": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(rs_dataset_stats)]),
    "rs_dataset_info": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "rs_eval_hard": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(rs_batch),
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "rs_eval_hard_static": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(rs_batch),
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "rs_eval_soft_fwd": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(rs_batch),
                                          ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "rs_eval_soft_bwd": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(rs_batch),
                                          ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "rs_profile_read": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(rs_profile), ctypes.c_int32]),
    "rs_submit": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(rs_batch),
                                   ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]),
    "rs_poll": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.POINTER(rs_ticket_info)]),
    "rs_cancel": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64]),
    "rs_serving_stats_read": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(rs_serving_stats)]),
    "rs_evolve": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(rs_evolve_config),
                                   ctypes.POINTER(rs_population), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "rs_finetune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(rs_batch),
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "rs_tile_config_count": (ctypes.c_int32, []),
    "rs_tile_config_info": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "rs_tile_config_form": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "rs_set_tile_config": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "rs_submit_soft": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(rs_batch), ctypes.c_float,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "rs_poll_soft": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.POINTER(rs_ticket_info)]),
    "rs_tile_config_pick": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(rs_batch),
                                             ctypes.POINTER(ctypes.c_int32)]),
    "rs_autotune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(rs_batch),
                                     ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "rs_selftest_threshold_rewrite": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p,
                                                       ctypes.c_void_p, ctypes.c_void_p,
                                                       ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64)]),
    "rs_measure_pipe_rates": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(rs_pipe_rates)]),
    "rs_selftest_log1p_unit": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "rs_selftest_log1m_exp": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "rs_inject_alloc_failures": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32]),
    "rs_selftest_bounded_wait": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
}


def lib():
    """Load librs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise RuntimeError(f"librs.so not built ({_SO}); run paper_2406_01821_gb300/build.py")
        h = ctypes.CDLL(_SO)
        for name, (res, args) in _SIGS.items():
            fn = getattr(h, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def exported_symbols():
    return list(_SIGS)


def check(code):
    if code < 0:
        raise RsError(code, lib().rs_last_error().decode())
    return code


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return ctypes.c_void_p(0)
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------------------- batches

_FIELDS = ("set_rule_off", "rule_cond_off", "rule_class", "set_default", "cond_f", "cond_g",
           "cond_op", "cond_a", "cond_b", "cond_t")
_DTYPES = {"cond_op": np.int8, "cond_a": np.float32, "cond_b": np.float32, "cond_t": np.float32}
_ALL_FIELDS = _FIELDS + ("cond_set",)


class DeviceBatch:
    """A rule-set batch held in device memory (torch tensors), ready for the C ABI."""

    def __init__(self, tensors: dict):
        self.t = tensors
        self.P = int(tensors["set_default"].numel())
        self.R = int(tensors["rule_class"].numel())
        self.C = int(tensors["cond_f"].numel())
        self._c = None

    @classmethod
    def from_host(cls, batch, device="cuda"):
        import torch
        t = {}
        for f in _FIELDS:
            a = np.ascontiguousarray(getattr(batch, f), _DTYPES.get(f, np.int32))
            t[f] = torch.from_numpy(a).to(device)
        cs = getattr(batch, "cond_set", None)
        if cs is not None:        # 64-bit category sets, carried as int64 bit patterns
            t["cond_set"] = torch.from_numpy(np.ascontiguousarray(cs, np.uint64).view(np.int64)).to(device)
        return cls(t)

    def with_params(self, a=None, b=None, t=None) -> "DeviceBatch":
        d = dict(self.t)
        if a is not None:
            d["cond_a"] = a
        if b is not None:
            d["cond_b"] = b
        if t is not None:
            d["cond_t"] = t
        return DeviceBatch(d)

    def c(self) -> rs_batch:
        # Building the ctypes structure is most of the host time of a small call, so it is kept
        # and rebuilt only when an array's address has changed.
        addrs = tuple(0 if x is None else x.data_ptr() for x in map(self.t.get, _ALL_FIELDS))
        key = (self.P, self.R, self.C, addrs)
        if self._c is None or self._c[0] != key:
            self._c = (key, rs_batch(self.P, self.R, self.C, MEM_DEVICE, *addrs))
        return self._c[1]


class HostBatch:
    """A rule-set batch in host memory (numpy); the library copies it to the device per call."""

    def __init__(self, batch):
        self.a = {f: np.ascontiguousarray(getattr(batch, f), _DTYPES.get(f, np.int32)) for f in _FIELDS}
        cs = getattr(batch, "cond_set", None)
        self.a["cond_set"] = None if cs is None else np.ascontiguousarray(cs, np.uint64)
        self.P = int(self.a["set_default"].shape[0])
        self.R = int(self.a["rule_class"].shape[0])
        self.C = int(self.a["cond_f"].shape[0])

    def c(self) -> rs_batch:
        return rs_batch(self.P, self.R, self.C, MEM_HOST, *[_ptr(self.a[f]) for f in _FIELDS],
                        _ptr(self.a["cond_set"]))


# ------------------------------------------------------------------------------- context

class Context:
    def __init__(self, device: int = 0, flags: int = 0, mem_budget_bytes: int = 0,
                 autotune_cache: str | None = None):
        cfg = rs_config(device, flags, mem_budget_bytes,
                        autotune_cache.encode() if autotune_cache else None)
        h = ctypes.c_void_p()
        check(lib().rs_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            check(lib().rs_destroy(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # datasets
    def dataset(self, X, y, K: int, stream=None) -> int:
        """Register X (N x F float32) and y (int32[N]); numpy -> host path, torch cuda -> device."""
        import torch
        if isinstance(X, np.ndarray):
            Xc = np.ascontiguousarray(X, np.float32)
            yc = np.ascontiguousarray(y, np.int32)
            mem = MEM_HOST
        else:
            Xc = X.contiguous().to(torch.float32)
            yc = y.contiguous().to(torch.int32)
            mem = MEM_DEVICE if Xc.is_cuda else MEM_HOST
        N, F = Xc.shape
        out = ctypes.c_uint64()
        check(lib().rs_dataset_create(self.h, _ptr(Xc), _ptr(yc), N, F, K, mem,
                                      _stream_ptr(stream), ctypes.byref(out)))
        return out.value

    def dataset_destroy(self, ds: int):
        check(lib().rs_dataset_destroy(self.h, ds))

    def set_dataset_budget(self, nbytes: int):
        """Device-memory budget of this context's datasets (0: no limit); least recently used
        datasets not in use are evicted beyond it and rebuilt when next named."""
        check(lib().rs_set_dataset_budget(self.h, int(nbytes)))

    def dataset_stats(self) -> dict:
        st = rs_dataset_stats()
        check(lib().rs_dataset_stats_read(self.h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in rs_dataset_stats._fields_}

    def dataset_info(self, ds: int):
        N, F, K = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        check(lib().rs_dataset_info(self.h, ds, ctypes.byref(N), ctypes.byref(F), ctypes.byref(K), None))
        cc = np.zeros(K.value, np.int64)
        check(lib().rs_dataset_info(self.h, ds, None, None, None, _ptr(cc)))
        return N.value, F.value, K.value, cc

    # hard
    def eval_hard(self, ds: int, batch, K: int, N: int | None = None, per_class=True, preds=False,
                  out=None, stream=None):
        """Returns (correct, per_class or None, preds or None) as torch tensors (device batch)
        or numpy arrays (host batch)."""
        cb = batch.c()
        P = cb.P
        if cb.mem == MEM_DEVICE:
            import torch
            dev = batch.t["set_default"].device
            if out is not None:
                correct, pc, pr = out
            else:
                correct = torch.empty(P, dtype=torch.int32, device=dev)
                pc = torch.empty((P, K), dtype=torch.int32, device=dev) if per_class else None
                pr = torch.empty((P, N), dtype=torch.int32, device=dev) if preds else None
        else:
            correct = np.zeros(P, np.int32)
            pc = np.zeros((P, K), np.int32) if per_class else None
            pr = np.zeros((P, N), np.int32) if preds else None
        check(lib().rs_eval_hard(self.h, ds, ctypes.byref(cb), _ptr(correct), _ptr(pc), _ptr(pr),
                                 _stream_ptr(stream)))
        return correct, pc, pr

    # soft
    def soft_fwd(self, ds: int, batch, tau: float, N: int | None = None, K: int | None = None,
                 probs=False, stream=None):
        import torch
        cb = batch.c()
        dev = batch.t["set_default"].device
        loss = torch.empty(cb.P, dtype=torch.float32, device=dev)
        pr = torch.empty((cb.P, N, K), dtype=torch.float32, device=dev) if probs else None
        check(lib().rs_eval_soft_fwd(self.h, ds, ctypes.byref(cb), float(tau), _ptr(loss), _ptr(pr),
                                     _stream_ptr(stream)))
        return loss, pr

    def soft_bwd(self, ds: int, batch, tau: float, dloss, want_loss=True, stream=None):
        import torch
        cb = batch.c()
        dev = batch.t["set_default"].device
        ga = torch.empty(cb.C, dtype=torch.float32, device=dev)
        gb = torch.empty(cb.C, dtype=torch.float32, device=dev)
        gt = torch.empty(cb.C, dtype=torch.float32, device=dev)
        loss = torch.empty(cb.P, dtype=torch.float32, device=dev) if want_loss else None
        dl = dloss.contiguous().to(torch.float32)
        check(lib().rs_eval_soft_bwd(self.h, ds, ctypes.byref(cb), float(tau), _ptr(dl), _ptr(ga),
                                     _ptr(gb), _ptr(gt), _ptr(loss), _stream_ptr(stream)))
        return ga, gb, gt, loss

    # tuning
    def set_tile_config(self, cfg_id: int):
        check(lib().rs_set_tile_config(self.h, cfg_id))

    def tile_pick(self, ds: int, batch) -> int:
        """The tile configuration the next hard evaluation of `batch` on `ds` would use."""
        cid = ctypes.c_int32(-1)
        cb = batch.c()
        check(lib().rs_tile_config_pick(self.h, ds, ctypes.byref(cb), ctypes.byref(cid)))
        return cid.value

    def autotune(self, ds: int, batch, stream=None) -> int:
        best = ctypes.c_int32(-1)
        cb = batch.c()
        check(lib().rs_autotune(self.h, ds, ctypes.byref(cb), _stream_ptr(stream), ctypes.byref(best)))
        return best.value

    def pipe_rates(self) -> dict:
        """Measured lane operations per second of the GPU's arithmetic pipes (rs_measure_pipe_rates)."""
        r = rs_pipe_rates()
        check(lib().rs_measure_pipe_rates(self.h, ctypes.byref(r)))
        return {f: getattr(r, f) for f, _ in rs_pipe_rates._fields_}

    def profile(self, reset=False) -> dict:
        p = rs_profile()
        check(lib().rs_profile_read(self.h, ctypes.byref(p), int(reset)))
        return {f: getattr(p, f) for f, _ in rs_profile._fields_}

    # serving
    def submit(self, ds: int, batch) -> int:
        """Queue a hard-evaluation request (HostBatch or DeviceBatch); returns its ticket."""
        t = ctypes.c_uint64()
        cb = batch.c()
        check(lib().rs_submit(self.h, ds, ctypes.byref(cb), 0, ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, P: int, K: int, timeout_us: int = 0):
        """Returns None while pending, else (correct[P], per_class[P,K], info dict)."""
        c = np.zeros(P, np.int32)
        pc = np.zeros((P, K), np.int32)
        info = rs_ticket_info()
        rc = lib().rs_poll(self.h, ticket, int(timeout_us), _ptr(c), _ptr(pc), ctypes.byref(info))
        if rc == PENDING:
            return None
        check(rc)
        return c, pc, {"submit_ns": info.submit_ns, "admit_ns": info.admit_ns, "done_ns": info.done_ns}

    def submit_soft(self, ds: int, batch, tau: float) -> int:
        """Queue a soft-loss request (forward at temperature tau); returns its ticket."""
        t = ctypes.c_uint64()
        cb = batch.c()
        check(lib().rs_submit_soft(self.h, ds, ctypes.byref(cb), float(tau), ctypes.byref(t)))
        return t.value

    def poll_soft(self, ticket: int, P: int, timeout_us: int = 0):
        """Returns None while pending, else (loss[P] float32, info dict)."""
        loss = np.zeros(P, np.float32)
        info = rs_ticket_info()
        rc = lib().rs_poll_soft(self.h, ticket, int(timeout_us), _ptr(loss), ctypes.byref(info))
        if rc == PENDING:
            return None
        check(rc)
        return loss, {"submit_ns": info.submit_ns, "admit_ns": info.admit_ns, "done_ns": info.done_ns}

    def cancel(self, ticket: int) -> int:
        return lib().rs_cancel(self.h, ticket)

    def serving_stats(self) -> dict:
        st = rs_serving_stats()
        check(lib().rs_serving_stats_read(self.h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in rs_serving_stats._fields_}

    def evolve(self, ds: int, pop: dict, generations: int, elite: int, seed: int, tune_every=0,
               tune_top=0, tune_steps=0, tau=0.1, lr=1e-2, lamarckian=False, first_generation=0,
               stream=None):
        """Device-resident evolution. ``pop`` = dict of fixed-slot numpy arrays (nrule [P],
        deflt [P], rcls/ncond [P,RMAX], cf/cg/cop/ca/cb/ct [P,RMAX,CMAX]); returns
        (final population dict, fitness [P], best [G+1], mean [G+1])."""
        kinds = {"nrule": np.int32, "deflt": np.int32, "rcls": np.int32, "ncond": np.int32,
                 "cf": np.int32, "cg": np.int32, "cop": np.int8, "ca": np.float32, "cb": np.float32,
                 "ct": np.float32}
        arr = {k: np.ascontiguousarray(pop[k], t).copy() for k, t in kinds.items()}
        P, RMAX, CMAX = arr["cf"].shape
        fitness = np.zeros(P, np.int32)
        best = np.zeros(generations + 1, np.int32)
        mean = np.zeros(generations + 1, np.float64)
        cp = rs_population(*[_ptr(arr[k]) for k in kinds], _ptr(fitness))
        cfg = rs_evolve_config(P, RMAX, CMAX, generations, elite, tune_every, tune_top, tune_steps,
                               tau, lr, int(lamarckian), seed, int(first_generation))
        check(lib().rs_evolve(self.h, ds, ctypes.byref(cfg), ctypes.byref(cp), _ptr(best), _ptr(mean),
                              _stream_ptr(stream)))
        return arr, fitness, best, mean

    @staticmethod
    def save_population(path: str, pop: dict, seed: int, next_generation: int):
        """Checkpoint of an evolution run: the fixed-slot population, the seed and the index of
        the next generation (a plain numpy .npz file)."""
        np.savez(path, seed=np.uint64(seed), next_generation=np.int64(next_generation),
                 **{k: np.asarray(v) for k, v in pop.items()})

    @staticmethod
    def load_population(path: str):
        """(population dict, seed, next generation) of a checkpoint; resume with
        evolve(..., seed=seed, first_generation=next_generation)."""
        with np.load(path) as z:
            pop = {k: z[k].copy() for k in z.files if k not in ("seed", "next_generation")}
            return pop, int(z["seed"]), int(z["next_generation"])

    def finetune(self, ds: int, batch: DeviceBatch, tau: float, lr: float, steps: int, stream=None):
        """Adam fine-tuning of a device batch; returns (a, b, t, loss_trace [steps, P])."""
        a = batch.t["cond_a"].clone()
        b = batch.t["cond_b"].clone()
        t = batch.t["cond_t"].clone()
        trace = np.zeros((steps, batch.P), np.float32)
        cb = batch.c()
        check(lib().rs_finetune(self.h, ds, ctypes.byref(cb), _ptr(a), _ptr(b), _ptr(t), float(tau),
                                float(lr), int(steps), _ptr(trace), _stream_ptr(stream)))
        return a, b, t, trace

    def check_async(self, stream=None):
        check(lib().rs_check(self.h, _stream_ptr(stream)))

    def selftest_threshold_rewrite(self, a, t, op) -> int:
        a = np.ascontiguousarray(a, np.float32)
        t = np.ascontiguousarray(t, np.float32)
        op = np.ascontiguousarray(op, np.int8)
        mm = ctypes.c_uint64()
        check(lib().rs_selftest_threshold_rewrite(self.h, _ptr(a), _ptr(t), _ptr(op), len(a),
                                                  ctypes.byref(mm)))
        return mm.value


def tile_configs():
    out = []
    for i in range(lib().rs_tile_config_count()):
        s, w, v, f = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(lib().rs_tile_config_info(i, ctypes.byref(s), ctypes.byref(w), ctypes.byref(v)))
        check(lib().rs_tile_config_form(i, ctypes.byref(f)))
        out.append({"id": i, "samples_per_tile": s.value, "warps": w.value, "samples_per_lane": v.value,
                    "form": f.value})
    return out


# ------------------------------------------------------------------------------- autograd

def _make_soft_fn():
    import torch

    class RuleSoftFn(torch.autograd.Function):
        """loss[P] = soft first-fire cross-entropy of every set; gradients w.r.t. the condition
        coefficients a, b and thresholds t come from the library's adjoint kernel."""

        @staticmethod
        def forward(ctx, a, b, t, rsctx, ds, structure, tau):
            batch = structure.with_params(a.detach().contiguous(), b.detach().contiguous(),
                                          t.detach().contiguous())
            loss, _ = rsctx.soft_fwd(ds, batch, tau)
            ctx.save_for_backward(a, b, t)
            ctx.rs = (rsctx, ds, structure, tau)
            return loss

        @staticmethod
        def backward(ctx, dloss):
            a, b, t = ctx.saved_tensors
            rsctx, ds, structure, tau = ctx.rs
            batch = structure.with_params(a.detach().contiguous(), b.detach().contiguous(),
                                          t.detach().contiguous())
            ga, gb, gt, _ = rsctx.soft_bwd(ds, batch, tau, dloss, want_loss=False)
            return ga, gb, gt, None, None, None, None

    return RuleSoftFn


_soft_fn = None


def rule_soft_loss(a, b, t, rsctx: Context, ds: int, structure: DeviceBatch, tau: float):
    """Differentiable per-set loss (torch.autograd.Function over rs_eval_soft_fwd/bwd)."""
    global _soft_fn
    if _soft_fn is None:
        _soft_fn = _make_soft_fn()
    return _soft_fn.apply(a, b, t, rsctx, ds, structure, tau)
