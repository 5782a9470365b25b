"""GB300-native failureless Aho-Corasick (PFAC) matching.

The CUDA library (``_build/libpfac.so``, built by ``build.build()``) does all
matching; ``api`` is a thin ctypes binding of its C ABI (``include/ac.h``).
``workloads`` makes seeded synthetic inputs.
"""
from .api import (  # noqa: F401
    AC_KERNEL_SIMPLE,
    AC_KERNEL_TILED,
    AcError,
    Automaton,
    ac_compile,
    ac_count,
    ac_destroy,
    ac_device_status,
    ac_export_tables,
    ac_info,
    ac_match,
    ac_match_compact,
    ac_match_host,
    ac_set_kernel,
    ac_status_string,
)
