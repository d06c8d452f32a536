"""The dataset-eviction policy (csrc/dataset_lru.h: least recently used first, never a dataset in
use, without a host copy or being made resident) on the CPU, compiled with g++ from the header the
library uses."""
import ctypes
import os
import random
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2406_01821_gb300", "csrc")


@pytest.fixture(scope="module")
def victims(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("lru") / "liblru.so")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-shared", "-fPIC", "-I", CSRC,
                           os.path.join(HERE, "lru_cases.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    L.lru_victims.restype = ctypes.c_int
    L.lru_victims.argtypes = [u64p, u64p, u64p, u8p, u8p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                              ctypes.c_uint64, ctypes.c_uint64, u64p]

    def call(entries, used, need, budget, keep=0):
        n = len(entries)
        arr = lambda t, xs: (t * max(n, 1))(*xs)
        ids = arr(ctypes.c_uint64, [e[0] for e in entries])
        by = arr(ctypes.c_uint64, [e[1] for e in entries])
        lu = arr(ctypes.c_uint64, [e[2] for e in entries])
        res = arr(ctypes.c_uint8, [int(e[3]) for e in entries])
        ev = arr(ctypes.c_uint8, [int(e[4]) for e in entries])
        out = (ctypes.c_uint64 * max(n, 1))()
        k = L.lru_victims(ids, by, lu, res, ev, n, used, need, budget, keep, out)
        return list(out[:k])
    return call


def test_no_budget_or_fits(victims):
    e = [(1, 100, 5, True, True), (2, 100, 1, True, True)]
    assert victims(e, 200, 50, 0) == []          # no limit
    assert victims(e, 200, 50, 250) == []        # fits


def test_least_recently_used_first(victims):
    e = [(1, 100, 5, True, True), (2, 100, 1, True, True), (3, 100, 3, True, True)]
    assert victims(e, 300, 100, 300) == [2]
    assert victims(e, 300, 150, 300) == [2, 3]


def test_skips_in_use_not_resident_and_kept(victims):
    e = [(1, 100, 1, True, False),               # in use (or no host copy)
         (2, 100, 2, False, True),               # already evicted
         (3, 100, 3, True, True),
         (4, 100, 4, True, True)]
    assert victims(e, 300, 100, 300, keep=3) == [4]
    assert victims(e, 300, 300, 300) == [3, 4]   # as many as help: the budget is then exceeded


def test_random_against_a_model(victims):
    rng = random.Random(5)
    for _ in range(300):
        n = rng.randint(0, 12)
        entries = [(i + 1, rng.randint(1, 50), rng.randint(0, 100), rng.random() < 0.8, rng.random() < 0.7)
                   for i in range(n)]
        used = sum(e[1] for e in entries if e[3])
        need = rng.randint(0, 60)
        budget = rng.randint(1, 400)
        keep = rng.randint(0, n)
        got = victims(entries, used, need, budget, keep)
        # model: walk candidates in (last_use, id) order until it fits
        want, u = [], used
        if used + need > budget:
            for e in sorted(entries, key=lambda e: (e[2], e[0])):
                if u + need <= budget:
                    break
                if e[3] and e[4] and e[0] != keep:
                    want.append(e[0])
                    u -= e[1]
        assert got == want
        chosen = {e[0]: e for e in entries if e[0] in got}
        assert all(e[3] and e[4] and e[0] != keep for e in chosen.values())
