"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every function
declared in include/rs.h, and fails cleanly where a device would be required."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_01821_gb300 import build, rs
    build.build()
    return rs.lib()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(rs_[a-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("rs_create", "rs_destroy", "rs_eval_hard", "rs_eval_soft_fwd", "rs_eval_soft_bwd",
                 "rs_dataset_create", "rs_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2406_01821_gb300 import rs
    missing = [n for n in declared_functions() if n not in rs.exported_symbols()]
    assert not missing, missing


def test_tile_configs_describe_themselves(lib):
    from paper_2406_01821_gb300 import rs
    cfgs = rs.tile_configs()
    assert len(cfgs) >= 4
    for c in cfgs:
        assert c["samples_per_tile"] == 32 * c["samples_per_lane"]
        assert c["warps"] in (4, 8, 16, 32)
    assert lib.rs_tile_config_info(len(cfgs), None, None, None) == -1


def test_version_and_null_handling(lib):
    assert lib.rs_version().startswith(b"rulesgpu")
    assert lib.rs_create(None, None) == -1           # out pointer is NULL -> RS_ERR_INVALID
    assert lib.rs_destroy(None) == -1


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.rs_create(None, ctypes.byref(h))
    assert rc == -6                                  # RS_ERR_UNSUPPORTED
    assert h.value is None
    assert b"device" in lib.rs_last_error()


def test_device_batch_struct_follows_its_arrays():
    """DeviceBatch keeps its ctypes structure between calls and rebuilds it when an array is
    replaced or a size changes (CPU tensors stand in for device ones: only addresses are read)."""
    import numpy as np
    import torch
    from paper_2406_01821_gb300 import rs, synth
    b = synth.random_rulesets(synth.quantile_table(np.random.default_rng(0).normal(size=(50, 4))),
                              2, 5, 3, 2, 0)
    t = {f: torch.from_numpy(np.ascontiguousarray(getattr(b, f), rs._DTYPES.get(f, np.int32)))
         for f in rs._FIELDS}
    db = rs.DeviceBatch(t)
    c1 = db.c()
    assert db.c() is c1
    assert (c1.P, c1.R, c1.C, c1.mem) == (b.P, b.R, b.C, rs.MEM_DEVICE)
    assert c1.cond_t == t["cond_t"].data_ptr() and not c1.cond_set
    t["cond_t"] = t["cond_t"].clone()
    c2 = db.c()
    assert c2 is not c1 and c2.cond_t == t["cond_t"].data_ptr()
    t["cond_set"] = torch.zeros(b.C, dtype=torch.int64)
    assert db.c().cond_set == t["cond_set"].data_ptr()
    db.P -= 1
    assert db.c().P == b.P - 1


def test_c_consumer_compiles_and_links(lib, tmp_path):
    """A strict C99 program that includes rs.h and calls the library through it compiles without
    warnings and links against librs.so: the header is valid C and agrees with the exports."""
    import c_consumer
    try:
        exe = c_consumer.build(str(tmp_path))
    except FileNotFoundError:
        pytest.skip("no C compiler")
    assert os.path.exists(exe)
