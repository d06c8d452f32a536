"""Build and feed tests/abi_consumer.c, a C program that uses the library only through its C ABI
(include/rs.h and librs.so), for the host and GPU tests of the boundary."""
import os
import shutil
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2406_01821_gb300")


def build(out_dir: str) -> str:
    """Compile the consumer as strict C99 against the header and link it against librs.so."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise FileNotFoundError("no C compiler")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = os.path.join(out_dir, "abi_consumer")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-O2",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_consumer.c"),
           "-o", exe, "-L", PKG, "-l:librs.so", f"-Wl,-rpath,{PKG}",
           f"-Wl,-rpath-link,{os.path.join(cuda, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stdout + r.stderr)
    return exe


def write_input(path: str, X, y, K: int, batch) -> None:
    """The consumer's input file (layout in abi_consumer.c)."""
    X = np.ascontiguousarray(X, np.float32)
    N, F = X.shape
    with open(path, "wb") as f:
        f.write(np.int64(N).tobytes())
        f.write(np.array([F, K, batch.P, batch.R, batch.C], np.int32).tobytes())
        f.write(X.tobytes())
        f.write(np.ascontiguousarray(y, np.int32).tobytes())
        for name, dt in (("set_rule_off", np.int32), ("rule_cond_off", np.int32), ("rule_class", np.int32),
                         ("set_default", np.int32), ("cond_f", np.int32), ("cond_g", np.int32),
                         ("cond_op", np.int8), ("cond_a", np.float32), ("cond_b", np.float32),
                         ("cond_t", np.float32)):
            f.write(np.ascontiguousarray(getattr(batch, name), dt).tobytes())


def run(exe: str, path: str, calls: int = 200):
    """(correct[P], per_class[P*K] flat, microseconds per call) printed by the consumer."""
    r = subprocess.run([exe, path, str(calls)], capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(r.stdout + r.stderr)
    lines = {ln.split()[0]: ln.split()[1:] for ln in r.stdout.splitlines() if ln.strip()}
    return (np.array(lines["correct"], np.int64), np.array(lines["per_class"], np.int64),
            float(lines["us_per_call"][0]))
