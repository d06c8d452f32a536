"""GB300-native (sm_103a) evaluation of populations of ordered rule sets.

The compute lives in ``librs.so`` (CUDA kernels behind a C ABI, declared in ``include/rs.h``);
``paper_2406_01821_gb300.rs`` is the thin ctypes binding with the same names. Importing this
package does not load the library; the first call into ``rs`` does, and fails loudly if the
library is missing.
"""
from . import synth  # noqa: F401

__all__ = ["synth"]
