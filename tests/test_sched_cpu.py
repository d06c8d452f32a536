"""The serving scheduler on the CPU, through a fake device (no GPU).

The state machine that the server's scheduler thread runs (``csrc/serve_sched.h``: FIFO admission
under a device-memory budget and the persistent kernel's slot table, relaunch of the kernel after
it idles out, completion, release) is compiled with g++ against ``tests/sched_fake.cpp``, a device
whose allocations fail on script, whose kernel claims work units between scheduler passes and
whose result copies can report a device error. The same header is what ``serve.cu`` includes.
"""
import ctypes
import os
import random
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2406_01821_gb300", "csrc")

QUEUED, RUNNING, COPYING, DONE = 0, 2, 3, 4
CANCELLED, COPY_ERROR = -8, -5


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("sched") / "libsched_fake.so")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-shared", "-fPIC",
                           "-I", CSRC, os.path.join(HERE, "sched_fake.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
    sig = {
        "fs_create": (vp, [u64, i32]), "fs_destroy": (None, [vp]),
        "fs_submit": (u64, [vp, u64, i32, i32]), "fs_cancel": (i32, [vp, u64]),
        "fs_script_alloc": (None, [vp, i32]), "fs_fail_copy": (None, [vp, u64]),
        "fs_step": (i32, [vp]), "fs_device_tick": (None, [vp, i32]),
        "fs_state": (i32, [vp, u64]), "fs_status": (i32, [vp, u64]), "fs_slot": (i32, [vp, u64]),
        "fs_used": (u64, [vp]), "fs_free_slots": (i32, [vp]), "fs_launches": (ctypes.c_int64, [vp]),
        "fs_fatal": (i32, [vp]), "fs_kernel_live": (i32, [vp]), "fs_idle": (i32, [vp]),
        "fs_admitted": (i32, [vp, ctypes.POINTER(u64), i32]),
        "fs_released": (i32, [vp, ctypes.POINTER(u64), i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    return L


class Sim:
    def __init__(self, L, budget, slots):
        self.L, self.h, self.slots = L, L.fs_create(budget, slots), slots

    def __del__(self):
        self.L.fs_destroy(self.h)

    def submit(self, nbytes, units, hard=True):
        return self.L.fs_submit(self.h, nbytes, units, 1 if hard else 0)

    def step(self):
        return bool(self.L.fs_step(self.h))

    def tick(self, units=1):
        self.L.fs_device_tick(self.h, units)

    def state(self, t):
        return self.L.fs_state(self.h, t)

    def _list(self, fn):
        buf = (ctypes.c_uint64 * 4096)()
        n = fn(self.h, buf, 4096)
        return list(buf[:n])

    def admitted(self):
        return self._list(self.L.fs_admitted)

    def released(self):
        return self._list(self.L.fs_released)

    @property
    def used(self):
        return self.L.fs_used(self.h)

    @property
    def free_slots(self):
        return self.L.fs_free_slots(self.h)

    def drain(self, limit=10000):
        """Steps and device ticks until the scheduler is idle."""
        for _ in range(limit):
            if self.L.fs_idle(self.h):
                return
            self.step()
            self.tick(4)
        raise AssertionError("scheduler did not drain")


def test_budget_blocks_head_of_line(lib):
    """A request that does not fit the budget stops admission: the small one behind it waits."""
    s = Sim(lib, budget=100, slots=8)
    a, b, c = s.submit(60, 3), s.submit(60, 3), s.submit(10, 1)
    assert s.step()
    assert s.admitted() == [a] and s.used == 60
    assert s.state(b) == QUEUED and s.state(c) == QUEUED
    while s.state(a) != DONE:             # until a's memory returns, b does not fit, c waits
        assert s.admitted() == [a]
        s.tick(1)
        s.step()
    assert s.used == 0
    s.step()                              # the next pass admits b and c together
    assert s.admitted() == [a, b, c] and s.used == 70
    s.drain()
    assert s.released() == [a, b, c]
    assert s.used == 0 and s.free_slots == 8
    assert all(s.state(t) == DONE and lib.fs_status(s.h, t) == 0 for t in (a, b, c))


def test_request_larger_than_budget_never_admitted_alone(lib):
    """Exactly the budget fits; nothing above it is admitted while others hold memory."""
    s = Sim(lib, budget=100, slots=4)
    a = s.submit(100, 1)
    b = s.submit(1, 1)
    s.step()
    assert s.admitted() == [a] and s.state(b) == QUEUED
    s.drain()
    assert s.admitted() == [a, b]


def test_slots_exhausted(lib):
    """Hard requests take a slot of the kernel's table; with none free, admission waits."""
    s = Sim(lib, budget=1 << 30, slots=2)
    h1, h2, h3 = s.submit(1, 5), s.submit(1, 5), s.submit(1, 5)
    s.step()
    assert s.admitted() == [h1, h2] and s.free_slots == 0
    assert {lib.fs_slot(s.h, h1), lib.fs_slot(s.h, h2)} == {0, 1}
    assert s.state(h3) == QUEUED and lib.fs_slot(s.h, h3) == -1
    s.drain()
    assert s.admitted() == [h1, h2, h3] and s.free_slots == 2


def test_soft_takes_no_slot_but_keeps_order(lib):
    """A soft request needs no slot, yet it does not overtake a hard request waiting for one."""
    s = Sim(lib, budget=1 << 30, slots=1)
    h1, h2 = s.submit(1, 4), s.submit(1, 4)
    f = s.submit(1, 0, hard=False)
    s.step()
    assert s.admitted() == [h1] and s.state(f) == QUEUED
    s.drain()
    assert s.admitted() == [h1, h2, f] and lib.fs_slot(s.h, f) == -1

    s2 = Sim(lib, budget=1 << 30, slots=1)
    g1 = s2.submit(1, 4)
    g2 = s2.submit(1, 0, hard=False)      # the slot is held, the soft request still runs
    s2.step()
    assert s2.admitted() == [g1, g2] and s2.free_slots == 0


def test_cancel_queued_and_admitted(lib):
    s = Sim(lib, budget=50, slots=4)
    a, b, c = s.submit(50, 2), s.submit(10, 1), s.submit(10, 1)
    s.step()
    assert lib.fs_cancel(s.h, a) == 0                 # already admitted: runs to completion
    assert lib.fs_cancel(s.h, b) == 1                 # queued: dropped
    assert s.state(b) == DONE and lib.fs_status(s.h, b) == CANCELLED
    assert lib.fs_cancel(s.h, b) == 0                 # a second cancel changes nothing
    s.drain()
    assert s.admitted() == [a, c] and b not in s.released()
    assert lib.fs_status(s.h, a) == 0 and s.used == 0


def test_allocation_failure_retried_in_order(lib):
    """A failed device allocation takes nothing and is retried first on the next pass."""
    s = Sim(lib, budget=1 << 20, slots=4)
    lib.fs_script_alloc(s.h, 0)
    lib.fs_script_alloc(s.h, 0)
    a, b = s.submit(100, 1), s.submit(100, 1)
    assert not s.step()
    assert s.admitted() == [] and s.used == 0 and s.free_slots == 4
    assert s.state(a) == QUEUED and lib.fs_slot(s.h, a) == -1
    s.step()
    assert s.admitted() == [] and s.state(b) == QUEUED
    s.step()
    assert s.admitted() == [a, b] and s.used == 200 and s.free_slots == 2
    s.drain()
    assert s.used == 0 and s.free_slots == 4


def test_kernel_relaunched_after_idle_exit(lib):
    s = Sim(lib, budget=1 << 20, slots=4)
    a = s.submit(1, 2)
    s.step()
    assert lib.fs_launches(s.h) == 1 and lib.fs_kernel_live(s.h)
    s.drain()
    for _ in range(3):                    # the kernel idles out
        s.tick(1)
    assert not lib.fs_kernel_live(s.h)
    b = s.submit(1, 2)
    s.step()
    assert lib.fs_launches(s.h) == 2
    s.drain()
    assert s.state(a) == DONE and s.state(b) == DONE


def test_no_work_no_launch(lib):
    """A request with no work units (an empty batch) completes without a kernel launch."""
    s = Sim(lib, budget=1 << 20, slots=4)
    a = s.submit(16, 0)
    s.drain()
    assert s.state(a) == DONE and lib.fs_launches(s.h) == 0 and lib.fs_status(s.h, a) == 0


def test_copy_error_is_fatal(lib):
    s = Sim(lib, budget=1 << 20, slots=4)
    a, b = s.submit(10, 1), s.submit(10, 1)
    lib.fs_fail_copy(s.h, a)
    s.drain()
    assert lib.fs_fatal(s.h) == COPY_ERROR
    assert s.state(a) == DONE and lib.fs_status(s.h, a) == COPY_ERROR
    assert lib.fs_status(s.h, b) == 0
    assert a not in s.released()          # the device's state is unknown: nothing is freed


@pytest.mark.parametrize("seed", range(12))
def test_random_schedules_keep_invariants(lib, seed):
    """Random arrivals, cancels, allocation failures and device progress against a model of the
    rules: budget and slots never exceeded, memory accounting exact, admission in arrival order
    with no request admitted while an earlier live one waits, every request finishing."""
    rng = random.Random(seed)
    budget, slots = rng.choice([64, 256, 1024]), rng.choice([1, 2, 3, 8])
    s = Sim(lib, budget=budget, slots=slots)
    reqs = {}                             # ticket -> (bytes, hard)
    order, cancelled = [], set()
    for _ in range(400):
        op = rng.random()
        if op < 0.3:
            nb = rng.randint(0, budget)
            hard = rng.random() < 0.7
            t = s.submit(nb, rng.randint(0, 6), hard)
            reqs[t] = (nb, hard)
            order.append(t)
        elif op < 0.4 and order:
            t = rng.choice(order)
            was_queued = s.state(t) == QUEUED
            ok = lib.fs_cancel(s.h, t)
            assert ok == was_queued
            if ok:
                cancelled.add(t)
        elif op < 0.45:
            lib.fs_script_alloc(s.h, 0)
        elif op < 0.7:
            s.tick(rng.randint(0, 5))
        else:
            s.step()
        adm = s.admitted()
        live = [t for t in adm if s.state(t) in (RUNNING, COPYING)]
        assert s.used == sum(reqs[t][0] for t in live) <= budget
        held = [t for t in live if reqs[t][1]]
        assert s.free_slots + len(held) == slots
        assert len({lib.fs_slot(s.h, t) for t in held}) == len(held)
        assert adm == [t for t in order if t in set(adm)]
        if adm:                           # every request before the last admitted one is settled
            last = order.index(adm[-1])
            assert all(t in adm or t in cancelled for t in order[:last])
    s.drain()
    for t in order:
        assert s.state(t) == DONE
        assert lib.fs_status(s.h, t) == (CANCELLED if t in cancelled else 0)
    assert s.used == 0 and s.free_slots == slots
    assert s.admitted() == [t for t in order if t not in cancelled]
    assert sorted(s.released()) == sorted(s.admitted())
