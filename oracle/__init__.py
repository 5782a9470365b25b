"""CPU oracle for failureless Aho-Corasick matching -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The library itself never does, and
this package imports nothing from the library: the two share no code.

``ac_oracle.c`` is the classic serial machine of the paper's section II
(goto, failure and output functions, one pass over the text).  This module
compiles it with gcc and wraps it with ctypes.  The functions here follow:

* ``pfac_ids``  -- per-start longest keyword id, the result the failureless
  machine reports (section II: no sub-pattern outputs); -1 where no keyword
  starts.  Computed by converting the full machine's (end, id) occurrences.
* ``full_occurrences`` -- every (end, id) occurrence, sub-patterns included
  (the original machine's output function, section II).
* ``compact`` / ``count`` -- the derived forms: ascending (position, id) pairs
  of the matched starts, and their number.
* ``walk_steps`` -- the number of goto evaluations a failureless walk makes
  from every start (a work statistic for the lookup-rate ceiling, not a
  result).

Every function is pinned in ``tests/test_oracle_pins.py`` against worked
examples, closed forms, brute force and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "ac_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

_lock = threading.Lock()
_libs: dict[str, ctypes.CDLL] = {}


def compile_source(src: str, out: str) -> str:
    """Compile an oracle C source into a shared object with gcc."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``ac_oracle.c`` into ``oracle/_build/liboracle.so``."""
    with _lock:
        if force or not os.path.exists(LIB_PATH) or (
            os.path.getmtime(LIB_PATH) < os.path.getmtime(SOURCE)
        ):
            compile_source(SOURCE, LIB_PATH)
    return LIB_PATH


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    p = ctypes.c_void_p
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.oracle_ac_build.argtypes = [u8p, u64p, ctypes.c_uint32]
    lib.oracle_ac_build.restype = p
    lib.oracle_ac_free.argtypes = [p]
    lib.oracle_ac_free.restype = None
    lib.oracle_ac_states.argtypes = [p]
    lib.oracle_ac_states.restype = ctypes.c_uint32
    lib.oracle_ac_depth_counts.argtypes = [p, u64p, ctypes.c_uint32]
    lib.oracle_ac_depth_counts.restype = ctypes.c_uint32
    lib.oracle_ac_full.argtypes = [p, u8p, ctypes.c_uint64, u64p, i32p, ctypes.c_uint64]
    lib.oracle_ac_full.restype = ctypes.c_uint64
    lib.oracle_ac_pfac_ids.argtypes = [p, u8p, ctypes.c_uint64, i32p]
    lib.oracle_ac_pfac_ids.restype = None
    lib.oracle_ac_walk_steps.argtypes = [p, u8p, ctypes.c_uint64, u64p]
    lib.oracle_ac_walk_steps.restype = ctypes.c_uint64
    return lib


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (building if needed) the oracle library, or another compiled variant."""
    if path is None:
        path = build()
    with _lock:
        if path not in _libs:
            _libs[path] = _bind(ctypes.CDLL(path))
        return _libs[path]


def _as_u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(a), dtype=np.uint8)
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint8:
        raise TypeError("text must be uint8")
    return a


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Machine:
    """The serial Aho-Corasick machine for one keyword set."""

    def __init__(self, patterns, lib: ctypes.CDLL | None = None):
        self._lib = lib if lib is not None else load()
        pats = [bytes(p) for p in patterns]
        if not pats:
            raise ValueError("empty keyword set")
        if any(len(p) == 0 for p in pats):
            raise ValueError("empty keyword")
        self.patterns = pats
        self.lengths = np.array([len(p) for p in pats], dtype=np.int64)
        blob = np.frombuffer(b"".join(pats), dtype=np.uint8).copy()
        off = np.zeros(len(pats) + 1, dtype=np.uint64)
        off[1:] = np.cumsum(self.lengths)
        if blob.size == 0:
            blob = np.zeros(1, dtype=np.uint8)
        self._h = self._lib.oracle_ac_build(_ptr(blob, ctypes.c_uint8), _ptr(off, ctypes.c_uint64), len(pats))
        if not self._h:
            raise MemoryError("oracle build failed")

    def close(self):
        if self._h:
            self._lib.oracle_ac_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n_states(self) -> int:
        return int(self._lib.oracle_ac_states(self._h))

    def depth_counts(self) -> np.ndarray:
        cap = int(self.lengths.max()) + 1
        counts = np.zeros(cap, dtype=np.uint64)
        self._lib.oracle_ac_depth_counts(self._h, _ptr(counts, ctypes.c_uint64), cap)
        return counts

    def pfac_ids(self, text) -> np.ndarray:
        t = _as_u8(text)
        out = np.empty(t.size, dtype=np.int32)
        if t.size:
            self._lib.oracle_ac_pfac_ids(self._h, _ptr(t, ctypes.c_uint8), t.size, _ptr(out, ctypes.c_int32))
        return out

    def full_occurrences(self, text):
        """All (end, id) occurrences in scan order (sub-patterns included)."""
        t = _as_u8(text)
        if t.size == 0:
            return np.zeros(0, np.uint64), np.zeros(0, np.int32)
        dummy_e = np.zeros(1, np.uint64)
        dummy_i = np.zeros(1, np.int32)
        total = self._lib.oracle_ac_full(
            self._h, _ptr(t, ctypes.c_uint8), t.size, _ptr(dummy_e, ctypes.c_uint64), _ptr(dummy_i, ctypes.c_int32), 0
        )
        ends = np.zeros(max(total, 1), np.uint64)
        ids = np.zeros(max(total, 1), np.int32)
        self._lib.oracle_ac_full(
            self._h, _ptr(t, ctypes.c_uint8), t.size, _ptr(ends, ctypes.c_uint64), _ptr(ids, ctypes.c_int32), total
        )
        return ends[:total], ids[:total]

    def walk_steps(self, text):
        """(total goto evaluations of failureless walks from every start, longest walk)."""
        t = _as_u8(text)
        if t.size == 0:
            return 0, 0
        mx = np.zeros(1, np.uint64)
        tot = self._lib.oracle_ac_walk_steps(self._h, _ptr(t, ctypes.c_uint8), t.size, _ptr(mx, ctypes.c_uint64))
        return int(tot), int(mx[0])


def pfac_ids(patterns, text, lib: ctypes.CDLL | None = None) -> np.ndarray:
    """Per-start longest keyword id (-1 = none) for ``text``."""
    with Machine(patterns, lib) as m:
        return m.pfac_ids(text)


def full_occurrences(patterns, text, lib: ctypes.CDLL | None = None):
    with Machine(patterns, lib) as m:
        return m.full_occurrences(text)


def compact(ids: np.ndarray):
    """Ascending (position, id) pairs of matched starts (derived from pfac_ids)."""
    pos = np.nonzero(ids >= 0)[0].astype(np.uint32)
    return pos, ids[pos].astype(np.uint32)


def count(ids: np.ndarray) -> int:
    """Number of matched start positions."""
    return int(np.count_nonzero(ids >= 0))
