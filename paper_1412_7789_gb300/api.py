"""Thin Python binding of the C ABI in ``include/ac.h`` (ctypes).

Argument marshalling only: every matching step runs in the CUDA library.  The
library must have been built (``paper_1412_7789_gb300.build.build()``); when
it is missing every call raises -- there is no fallback.

PyTorch supplies device memory and streams: texts are ``torch.uint8`` CUDA
tensors, outputs ``torch.int32`` / ``torch.uint32``-compatible tensors, and the
stream defaults to the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

# ---- status codes (mirror of ac_status) ---------------------------------------
AC_OK = 0
AC_ERR_INVALID_ARG = 1
AC_ERR_EMPTY_PATTERN = 2
AC_ERR_TOO_MANY_STATES = 3
AC_ERR_OOM = 4
AC_ERR_CUDA = 5
AC_ERR_OVERFLOW = 6
AC_ERR_BUDGET = 7
AC_ERR_TIMEOUT = 8
AC_ERR_NOT_FOUND = 9
AC_ERR_CANCELLED = 10
AC_REQ_HOST_TEXT = 1

AC_KERNEL_TILED = 0
AC_KERNEL_SIMPLE = 1
AC_KERNEL_WALK_SLOTS = 2
AC_KERNEL_THREAD_JUMP = 3
AC_KERNEL_THREAD_JUMP_L1 = 4
KERNELS = {"tiled": AC_KERNEL_TILED, "simple": AC_KERNEL_SIMPLE, "walk_slots": AC_KERNEL_WALK_SLOTS,
           "thread_jump": AC_KERNEL_THREAD_JUMP, "thread_jump_l1": AC_KERNEL_THREAD_JUMP_L1}


class AcError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, ac_status_string(status), status))


class ac_options(ctypes.Structure):
    _fields_ = [
        ("index_width", ctypes.c_int32),
        ("class_compress", ctypes.c_int32),
        ("host_only", ctypes.c_int32),
        ("jump_bytes", ctypes.c_uint32),
        ("stride_bytes", ctypes.c_uint64),
        ("dev_alloc", ctypes.c_void_p),
        ("dev_free", ctypes.c_void_p),
        ("alloc_ctx", ctypes.c_void_p),
        ("no_chains", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class ac_info_t(ctypes.Structure):
    _fields_ = [
        ("n_keywords", ctypes.c_uint32),
        ("n_states", ctypes.c_uint32),
        ("n_classes", ctypes.c_uint32),
        ("row_width", ctypes.c_uint32),
        ("index_width", ctypes.c_uint32),
        ("code_bits", ctypes.c_uint32),
        ("jump_depth", ctypes.c_uint32),
        ("stride_depth", ctypes.c_uint32),
        ("min_len", ctypes.c_uint32),
        ("max_len", ctypes.c_uint32),
        ("table_bytes", ctypes.c_uint64),
        ("depth_base_jump", ctypes.c_uint32),
        ("count_jump", ctypes.c_uint32),
        ("class_hash_shift", ctypes.c_int32),
        ("match_windows_ppm", ctypes.c_uint32),
        ("class_direct_shift", ctypes.c_int32),
    ]


class ac_tuning(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint32) for name in ("block", "stages", "halo", "per_thread", "filter_bytes",
                                                     "survivor_list")]


_lock = threading.Lock()
_LIB: ctypes.CDLL | None = None

_H = ctypes.c_void_p
_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_SIGS = {
    "ac_default_options": (None, [ctypes.POINTER(ac_options)]),
    "ac_compile": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32,
                                  ctypes.POINTER(ac_options), ctypes.POINTER(_H)]),
    "ac_destroy": (ctypes.c_int, [_H]),
    "ac_info": (ctypes.c_int, [_H, ctypes.POINTER(ac_info_t)]),
    "ac_export_tables": (ctypes.c_int, [_H, _P, _P, _P]),
    "ac_match": (ctypes.c_int, [_H, _P, _U64, _P, _P]),
    "ac_match_compact": (ctypes.c_int, [_H, _P, _U64, _P, _P, _U64, _P, _P]),
    "ac_match_full": (ctypes.c_int, [_H, _P, _U64, _P, _P, _U64, _P, _P]),
    "ac_export_full": (ctypes.c_int, [_H, _P, _P, ctypes.POINTER(ctypes.c_uint32)]),
    "ac_export_stride": (ctypes.c_int, [_H, _P, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)]),
    "ac_export_jump": (ctypes.c_int, [_H, _P, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                      ctypes.POINTER(ctypes.c_uint64)]),
    "ac_export_hash": (ctypes.c_int, [_H, _P, _P] + [ctypes.POINTER(ctypes.c_uint32)] * 4),
    "ac_export_filter": (ctypes.c_int, [_H, _P, _P, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "ac_count": (ctypes.c_int, [_H, _P, _U64, _P, _P]),
    "ac_match_host": (ctypes.c_int, [_H, _P, _U64, _P, _P]),
    "ac_match_compact_static": (ctypes.c_int, [_H, _P, _U64, _P, _P, _U64, _P, _P]),
    "ac_set_kernel": (ctypes.c_int, [_H, ctypes.c_int]),
    "ac_set_wait_limit": (ctypes.c_int, [_H, ctypes.c_uint64, ctypes.c_int32]),
    "ac_get_tuning": (ctypes.c_int, [_H, ctypes.POINTER(ac_tuning)]),
    "ac_set_tuning": (ctypes.c_int, [_H, ctypes.POINTER(ac_tuning)]),
    "ac_export_chains": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_uint32), _P, _P, ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "ac_match_batch": (ctypes.c_int, [_P, ctypes.c_uint32, _P, _P, ctypes.c_uint32, _P, _P]),
    "ac_batch_create": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)]),
    "ac_batch_run": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint32, _P, _P]),
    "ac_batch_capture": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint32, _P]),
    "ac_batch_replay": (ctypes.c_int, [_P, _P]),
    "ac_batch_destroy": (ctypes.c_int, [_P]),
    "ac_batch_reserve_lists": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "ac_autotune": (ctypes.c_int, [_H, _P, _U64, ctypes.c_uint32, _P, ctypes.POINTER(ctypes.c_uint32),
                                   ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]),
    "ac_server_create": (ctypes.c_int, [_P, ctypes.c_uint32, _P, ctypes.POINTER(ctypes.c_void_p)]),
    "ac_server_submit": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "ac_server_replay": (ctypes.c_int, [_P, _P, ctypes.c_uint32, _P, _P]),
    "ac_server_poll": (ctypes.c_int, [_P, _P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32]),
    "ac_server_drain": (ctypes.c_int, [_P]),
    "ac_server_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "ac_server_destroy": (ctypes.c_int, [_P]),
    "ac_scratch_pool_usage": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                             ctypes.c_int32]),
    "ac_device_status": (ctypes.c_int, []),
    "ac_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def library_path() -> str:
    return _build.LIB_PATH


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _LIB
    with _lock:
        if _LIB is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    "libpfac.so is not built (expected at %s); run paper_1412_7789_gb300.build.build()" % path)
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _LIB = L
        return _LIB


def _check(status: int, what: str):
    if status != AC_OK:
        raise AcError(status, what)


def ac_status_string(status: int) -> str:
    try:
        return lib().ac_status_string(status).decode()
    except Exception:
        return "status %d" % status


def _stream_ptr(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _dev_ptr(t, dtype_bytes: int | None = None) -> int:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype_bytes is not None and t.element_size() != dtype_bytes:
        raise ValueError("wrong element size")
    return int(t.data_ptr())


# ---- C-named functions ----------------------------------------------------------
def ac_compile(patterns, index_width: int = 0, class_compress: bool = True, host_only: bool = False,
               jump_bytes: int = 0, stride_bytes: int = 0, chains: bool = True) -> int:
    """Compile keywords (sequence of bytes-like) -> raw handle (int)."""
    pats = [bytes(p) for p in patterns]
    k = len(pats)
    bufs = [ctypes.create_string_buffer(p, max(1, len(p))) for p in pats]
    arr = (ctypes.c_void_p * max(1, k))(*[ctypes.cast(b, ctypes.c_void_p) for b in bufs])
    lens = (ctypes.c_uint32 * max(1, k))(*[len(p) for p in pats])
    opt = ac_options()
    lib().ac_default_options(ctypes.byref(opt))
    opt.index_width = index_width
    opt.class_compress = 1 if class_compress else 0
    opt.host_only = 1 if host_only else 0
    opt.jump_bytes = jump_bytes
    opt.stride_bytes = stride_bytes
    opt.no_chains = 0 if chains else 1
    h = _H()
    _check(lib().ac_compile(arr, lens, k, ctypes.byref(opt), ctypes.byref(h)), "ac_compile")
    return int(h.value)


def ac_destroy(h: int):
    _check(lib().ac_destroy(h), "ac_destroy")


def ac_info(h: int) -> dict:
    info = ac_info_t()
    _check(lib().ac_info(h, ctypes.byref(info)), "ac_info")
    return {name: getattr(info, name) for name, _ in ac_info_t._fields_}


def ac_export_tables(h: int):
    """(cls int16[256], goto table int16/int32 [n_states, row_width], depth counts uint32[max_len+1])."""
    info = ac_info(h)
    cls = np.zeros(256, dtype=np.int16)
    dt = np.int16 if info["index_width"] == 16 else np.int32
    G = np.zeros((info["n_states"], info["row_width"]), dtype=dt)
    depth = np.zeros(info["max_len"] + 1, dtype=np.uint32)
    _check(lib().ac_export_tables(h, cls.ctypes.data, G.ctypes.data, depth.ctypes.data), "ac_export_tables")
    return cls, G, depth


def ac_export_chains(h: int):
    """(s_chain, records uint32[n, 4], bytes uint8[m]) -- see ac.h."""
    sc = ctypes.c_uint32()
    nr = ctypes.c_uint64()
    nb = ctypes.c_uint64()
    _check(lib().ac_export_chains(h, ctypes.byref(sc), None, None, ctypes.byref(nr), ctypes.byref(nb)),
           "ac_export_chains")
    rec = np.zeros((nr.value, 4), dtype=np.uint32)
    byt = np.zeros(nb.value, dtype=np.uint8)
    _check(lib().ac_export_chains(h, ctypes.byref(sc), rec.ctypes.data, byt.ctypes.data, ctypes.byref(nr),
                                  ctypes.byref(nb)), "ac_export_chains")
    return int(sc.value), rec, byt


def ac_export_full(h: int, n_keywords: int):
    """(records uint32[n_keywords, 4], dups uint32[n_keywords], max_chain) -- see ac.h."""
    rec = np.zeros((n_keywords, 4), dtype=np.uint32)
    dups = np.zeros(n_keywords, dtype=np.uint32)
    mc = ctypes.c_uint32()
    _check(lib().ac_export_full(h, rec.ctypes.data, dups.ctypes.data, ctypes.byref(mc)), "ac_export_full")
    return rec, dups, int(mc.value)


def ac_export_filter(h: int):
    """(B, k, F uint32[...], JK int32[...]) of a 2-/4-bit-code automaton, or (0, 0, empty, empty)."""
    B, k = ctypes.c_uint32(), ctypes.c_uint32()
    nf, nj = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().ac_export_filter(h, None, None, ctypes.byref(B), ctypes.byref(k), ctypes.byref(nf), ctypes.byref(nj)),
           "ac_export_filter")
    F = np.zeros(nf.value, dtype=np.uint32)
    JK = np.zeros(nj.value, dtype=np.int32)
    _check(lib().ac_export_filter(h, F.ctypes.data, JK.ctypes.data, ctypes.byref(B), ctypes.byref(k), ctypes.byref(nf),
                                  ctypes.byref(nj)), "ac_export_filter")
    return int(B.value), int(k.value), F, JK


def ac_export_stride(h: int):
    """(k2, base_k, count_k, J2 int32[...]) -- see ac.h."""
    k2, bk, ck = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    ne = ctypes.c_uint64()
    _check(lib().ac_export_stride(h, None, ctypes.byref(k2), ctypes.byref(bk), ctypes.byref(ck), ctypes.byref(ne)),
           "ac_export_stride")
    J2 = np.zeros(ne.value, dtype=np.int32)
    _check(lib().ac_export_stride(h, J2.ctypes.data, ctypes.byref(k2), ctypes.byref(bk), ctypes.byref(ck),
                                  ctypes.byref(ne)), "ac_export_stride")
    return int(k2.value), int(bk.value), int(ck.value), J2


def ac_export_hash(h: int):
    """(kh, fbits, hk_bits, probes, F uint32[...], HK uint32[n_buckets, 4]) of an 8-bit-code automaton -- see ac.h."""
    v = [ctypes.c_uint32() for _ in range(4)]
    _check(lib().ac_export_hash(h, None, None, *[ctypes.byref(x) for x in v]), "ac_export_hash")
    kh, fbits, hk_bits, probes = (int(x.value) for x in v)
    F = np.zeros((1 << fbits) // 32 if kh else 0, dtype=np.uint32)
    HK = np.zeros(((1 << hk_bits) if kh else 0, 4), dtype=np.uint32)
    _check(lib().ac_export_hash(h, F.ctypes.data, HK.ctypes.data, *[ctypes.byref(x) for x in v]), "ac_export_hash")
    return kh, fbits, hk_bits, probes, F, HK


def ac_export_jump(h: int):
    """(k, base_k, J int16[...]) of an 8-bit-code automaton -- see ac.h."""
    k, bk = ctypes.c_uint32(), ctypes.c_uint32()
    ne = ctypes.c_uint64()
    _check(lib().ac_export_jump(h, None, ctypes.byref(k), ctypes.byref(bk), ctypes.byref(ne)), "ac_export_jump")
    J = np.zeros(ne.value, dtype=np.int16)
    _check(lib().ac_export_jump(h, J.ctypes.data, ctypes.byref(k), ctypes.byref(bk), ctypes.byref(ne)),
           "ac_export_jump")
    return int(k.value), int(bk.value), J


def ac_match(h: int, text, n: int, out, stream=None):
    _check(lib().ac_match(h, _dev_ptr(text), n, _dev_ptr(out, 4), _stream_ptr(stream)), "ac_match")


def ac_match_compact(h: int, text, n: int, pos, ids, cap: int, count, stream=None):
    _check(lib().ac_match_compact(h, _dev_ptr(text), n, _dev_ptr(pos, 4) if cap else 0,
                                  _dev_ptr(ids, 4) if cap else 0, cap, _dev_ptr(count, 8),
                                  _stream_ptr(stream)), "ac_match_compact")


def ac_match_full(h: int, text, n: int, end, ids, cap: int, count, stream=None):
    _check(lib().ac_match_full(h, _dev_ptr(text), n, _dev_ptr(end, 4) if cap else 0,
                               _dev_ptr(ids, 4) if cap else 0, cap, _dev_ptr(count, 8),
                               _stream_ptr(stream)), "ac_match_full")


# Largest text ac_match_compact_static accepts (AC_STATIC_MAX_TEXT in ac.h).
AC_STATIC_MAX_TEXT = 16 << 20


def ac_match_compact_static(h: int, text, n: int, pos, ids, cap: int, count, stream=None):
    """ac_match_compact without device allocation (shared static scratch; see ac.h)."""
    _check(lib().ac_match_compact_static(h, _dev_ptr(text), n, _dev_ptr(pos, 4) if cap else 0,
                                         _dev_ptr(ids, 4) if cap else 0, cap, _dev_ptr(count, 8),
                                         _stream_ptr(stream)), "ac_match_compact_static")


def ac_count(h: int, text, n: int, count, stream=None):
    _check(lib().ac_count(h, _dev_ptr(text), n, _dev_ptr(count, 8), _stream_ptr(stream)), "ac_count")


def ac_match_host(h: int, text_ptr: int, n: int, out_ptr: int, stream=None):
    """Host-buffer dense matching: text_ptr / out_ptr are host addresses."""
    _check(lib().ac_match_host(h, text_ptr, n, out_ptr, _stream_ptr(stream)), "ac_match_host")


def ac_set_kernel(h: int, kernel: int):
    _check(lib().ac_set_kernel(h, kernel), "ac_set_kernel")


def ac_set_wait_limit(h: int, limit_ns: int = 0, stall_help: bool = False):
    _check(lib().ac_set_wait_limit(h, limit_ns, 1 if stall_help else 0), "ac_set_wait_limit")


def ac_device_status() -> int:
    return int(lib().ac_device_status())


def ac_scratch_pool_usage(reset_high: bool = False) -> tuple[int, int]:
    """(bytes of the library's scratch pool in use now, high-water mark since the last reset)."""
    now, high = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().ac_scratch_pool_usage(ctypes.byref(now), ctypes.byref(high), 1 if reset_high else 0),
           "ac_scratch_pool_usage")
    return int(now.value), int(high.value)


# ---- batches ---------------------------------------------------------------------
# numpy mirror of ac_batch_item (32 bytes)
BATCH_ITEM = np.dtype([("text_off", "<u8"), ("len", "<u8"), ("out_off", "<u8"), ("automaton", "<u4"),
                       ("reserved", "<u4")])
assert BATCH_ITEM.itemsize == 32


def batch_items(text_off, lens, out_off, automaton) -> np.ndarray:
    """A host array of ac_batch_item (copy it to the device for the calls)."""
    k = len(lens)
    it = np.zeros(k, dtype=BATCH_ITEM)
    it["text_off"] = np.asarray(text_off, dtype=np.uint64)
    it["len"] = np.asarray(lens, dtype=np.uint64)
    it["out_off"] = np.asarray(out_off, dtype=np.uint64)
    it["automaton"] = np.asarray(automaton, dtype=np.uint32)
    return it


def items_to_device(items: np.ndarray, device="cuda"):
    """The item array as a uint8 CUDA tensor (the bytes the kernels read)."""
    import torch

    return torch.from_numpy(items.view(np.uint8).copy()).to(device)


def _handles(hs):
    arr = (ctypes.c_void_p * max(1, len(hs)))(*[int(h) for h in hs])
    return arr


def ac_match_batch(hs, texts, items, nitems: int, out, stream=None):
    """hs: handles; texts: uint8 CUDA tensor; items: device bytes of nitems ac_batch_item; out: int32 tensor."""
    arr = _handles(hs)
    _check(lib().ac_match_batch(ctypes.cast(arr, ctypes.c_void_p), len(hs), _dev_ptr(texts), _dev_ptr(items), nitems,
                                _dev_ptr(out, 4), _stream_ptr(stream)), "ac_match_batch")


def ac_get_tuning(h: int) -> dict:
    """The filter kernel's launch shape for h (ac_tuning fields but reserved)."""
    t = ac_tuning()
    _check(lib().ac_get_tuning(h, ctypes.byref(t)), "ac_get_tuning")
    return {name: int(getattr(t, name)) for name, _ in ac_tuning._fields_}


def ac_set_tuning(h: int, **fields) -> None:
    """Change fields of h's tuning (the others keep their values; filter_bytes
    defaults to 0, keep the root tables)."""
    cur = ac_get_tuning(h)
    cur["filter_bytes"] = 0
    unknown = set(fields) - set(cur)
    if unknown:
        raise TypeError("unknown tuning fields: %s" % sorted(unknown))
    cur.update(fields)
    t = ac_tuning(**cur)
    _check(lib().ac_set_tuning(h, ctypes.byref(t)), "ac_set_tuning")


def ac_autotune(h: int, sample, n: int | None = None, reps: int = 0, stream=None) -> tuple[int, int, str]:
    """Pick the fastest kernel and launch shape for h on a device sample;
    returns (block, stages, kernel name)."""
    b = ctypes.c_uint32()
    s = ctypes.c_uint32()
    k = ctypes.c_uint32()
    n = sample.numel() if n is None else n
    _check(lib().ac_autotune(h, _dev_ptr(sample), n, reps, _stream_ptr(stream), ctypes.byref(b), ctypes.byref(s),
                             ctypes.byref(k)), "ac_autotune")
    names = {v: name for name, v in KERNELS.items()}
    return int(b.value), int(s.value), names.get(int(k.value), "tiled")


class BatchPlan:
    """ac_batch_create / run / capture / replay / destroy."""

    def __init__(self, handles, max_items: int):
        self.handles = [int(h) for h in handles]
        arr = _handles(self.handles)
        p = ctypes.c_void_p()
        _check(lib().ac_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(self.handles), max_items,
                                     ctypes.byref(p)), "ac_batch_create")
        self.plan = int(p.value)
        self.max_items = max_items

    def reserve_lists(self, text_bytes: int):
        """Survivor lists for the phased form of the plan's 8-bit-code automata
        (ac_batch_reserve_lists); drops a captured graph."""
        _check(lib().ac_batch_reserve_lists(self.plan, int(text_bytes)), "ac_batch_reserve_lists")

    def run(self, texts, items, nitems: int, out, stream=None):
        _check(lib().ac_batch_run(self.plan, _dev_ptr(texts), _dev_ptr(items), nitems, _dev_ptr(out, 4),
                                  _stream_ptr(stream)), "ac_batch_run")

    def capture(self, texts, items, nitems: int, out):
        _check(lib().ac_batch_capture(self.plan, _dev_ptr(texts), _dev_ptr(items), nitems, _dev_ptr(out, 4)),
               "ac_batch_capture")

    def replay(self, stream=None):
        _check(lib().ac_batch_replay(self.plan, _stream_ptr(stream)), "ac_batch_replay")

    def close(self):
        if getattr(self, "plan", None):
            lib().ac_batch_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- object wrapper ----------------------------------------------------------------
class Automaton:
    """A compiled keyword set resident on the current CUDA device."""

    def __init__(self, patterns, **kw):
        self.patterns = [bytes(p) for p in patterns]
        self.handle = ac_compile(self.patterns, **kw)

    def close(self):
        if getattr(self, "handle", None):
            ac_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def info(self) -> dict:
        return ac_info(self.handle)

    def export_tables(self):
        return ac_export_tables(self.handle)

    def set_kernel(self, kernel: str | int):
        if isinstance(kernel, str):
            kernel = KERNELS[kernel]
        ac_set_kernel(self.handle, kernel)

    def match(self, text, out=None, stream=None):
        import torch

        n = text.numel()
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=text.device)
        ac_match(self.handle, text, n, out, stream)
        return out

    def count(self, text, out=None, stream=None):
        import torch

        if out is None:
            out = torch.zeros(1, dtype=torch.int64, device=text.device)
        ac_count(self.handle, text, text.numel(), out, stream)
        return out

    def match_compact(self, text, cap: int | None = None, stream=None):
        """(pos, ids, count): pos/ids hold min(count, cap) entries."""
        import torch

        n = text.numel()
        if cap is None:
            cap = max(1, n // 64)
        pos = torch.empty(max(cap, 1), dtype=torch.int32, device=text.device)
        ids = torch.empty(max(cap, 1), dtype=torch.int32, device=text.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=text.device)
        ac_match_compact(self.handle, text, n, pos, ids, cap, cnt, stream)
        return pos, ids, cnt

    def match_full(self, text, cap: int | None = None, stream=None):
        """(end, ids, count): every keyword occurrence (sub-patterns included),
        ordered by start, end, id; end/ids hold min(count, cap) entries."""
        import torch

        n = text.numel()
        if cap is None:
            cap = max(1, n // 64)
        end = torch.empty(max(cap, 1), dtype=torch.int32, device=text.device)
        ids = torch.empty(max(cap, 1), dtype=torch.int32, device=text.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=text.device)
        ac_match_full(self.handle, text, n, end, ids, cap, cnt, stream)
        return end, ids, cnt

    def export_full(self):
        return ac_export_full(self.handle, self.info()["n_keywords"])

    def autotune(self, sample, reps: int = 0, stream=None) -> tuple[int, int, str]:
        return ac_autotune(self.handle, sample, reps=reps, stream=stream)

    def tuning(self) -> dict:
        return ac_get_tuning(self.handle)

    def set_tuning(self, **fields):
        ac_set_tuning(self.handle, **fields)

    def match_host(self, text, out=None, stream=None):
        """text: CPU uint8 tensor (pinned for overlap); returns a CPU int32 tensor."""
        import torch

        n = text.numel()
        if out is None:
            out = torch.empty(n, dtype=torch.int32, pin_memory=text.is_pinned())
        ac_match_host(self.handle, int(text.data_ptr()), n, int(out.data_ptr()), stream)
        return out


# ---- serving ----------------------------------------------------------------------
class ac_server_options(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_wave", ctypes.c_uint32),
                ("waves_in_flight", ctypes.c_uint32), ("fifo", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("dev_alloc", ctypes.c_void_p), ("dev_free", ctypes.c_void_p), ("alloc_ctx", ctypes.c_void_p)]


# C types of the server's optional scratch allocator (ac_server_options)
DEV_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
DEV_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

# numpy mirrors of ac_server_request (56 bytes) and ac_server_completion (40 bytes)
SERVER_REQUEST = np.dtype([("automaton", "<u4"), ("flags", "<u4"), ("d_text", "<u8"), ("n", "<u8"),
                           ("d_pos", "<u8"), ("d_ids", "<u8"), ("cap", "<u8"), ("d_count", "<u8")])
SERVER_COMPLETION = np.dtype([("ticket", "<u8"), ("status", "<i4"), ("wave_size", "<u4"),
                              ("t_submit_us", "<f8"), ("t_launch_us", "<f8"), ("t_done_us", "<f8")])
assert SERVER_REQUEST.itemsize == 56 and SERVER_COMPLETION.itemsize == 40


class Server:
    """ac_server_*: continuous batching of compacted-match requests."""

    def __init__(self, handles, hbm_budget: int = 0, max_wave: int = 0, waves_in_flight: int = 0,
                 fifo: bool = False, dev_alloc=None, dev_free=None):
        """dev_alloc(bytes) -> device address (0 = failure) and dev_free(address):
        optional Python allocator of the waves' device scratch (called from
        the server's worker thread)."""
        self.handles = [int(h) for h in handles]
        arr = _handles(self.handles)
        opt = ac_server_options(hbm_budget, max_wave, waves_in_flight, 1 if fifo else 0, 0)
        self._hooks = None
        if dev_alloc is not None:
            self._hooks = (DEV_ALLOC(lambda n, ctx: dev_alloc(int(n)) or None),
                           DEV_FREE(lambda p, ctx: dev_free(int(p or 0))))
            opt.dev_alloc = ctypes.cast(self._hooks[0], ctypes.c_void_p)
            opt.dev_free = ctypes.cast(self._hooks[1], ctypes.c_void_p)
        p = ctypes.c_void_p()
        _check(lib().ac_server_create(ctypes.cast(arr, ctypes.c_void_p), len(self.handles), ctypes.byref(opt),
                                      ctypes.byref(p)), "ac_server_create")
        self.srv = int(p.value)

    @staticmethod
    def request(automaton: int, text, n: int, pos, ids, cap: int, count) -> np.ndarray:
        """A request record; a CPU (pinned) text tensor makes it a host-text request."""
        r = np.zeros(1, dtype=SERVER_REQUEST)
        r["automaton"] = automaton
        r["flags"] = 0 if (n == 0 or text.is_cuda) else AC_REQ_HOST_TEXT
        r["d_text"] = int(text.data_ptr()) if n else 0
        r["n"] = n
        r["d_pos"] = int(pos.data_ptr()) if cap else 0
        r["d_ids"] = int(ids.data_ptr()) if cap else 0
        r["cap"] = cap
        r["d_count"] = int(count.data_ptr())
        return r

    def submit(self, req) -> int:
        """Submit one request (a SERVER_REQUEST record or a length-1 array)."""
        req = np.ascontiguousarray(np.array(req, dtype=SERVER_REQUEST).reshape(-1)[:1])
        t = ctypes.c_uint64()
        _check(lib().ac_server_submit(self.srv, req.ctypes.data, ctypes.byref(t)), "ac_server_submit")
        return int(t.value)

    def replay(self, reqs: np.ndarray, arrival_us: np.ndarray) -> np.ndarray:
        """Submit reqs[i] at arrival_us[i] after the call starts; returns the tickets."""
        reqs = np.ascontiguousarray(reqs, dtype=SERVER_REQUEST)
        arr = np.ascontiguousarray(arrival_us, dtype=np.float64)
        tickets = np.zeros(len(reqs), dtype=np.uint64)
        _check(lib().ac_server_replay(self.srv, reqs.ctypes.data, len(reqs), arr.ctypes.data, tickets.ctypes.data),
               "ac_server_replay")
        return tickets

    def poll(self, max_n: int = 4096, wait_us: int = 0) -> np.ndarray:
        out = np.zeros(max_n, dtype=SERVER_COMPLETION)
        k = ctypes.c_uint32()
        _check(lib().ac_server_poll(self.srv, out.ctypes.data, max_n, ctypes.byref(k), wait_us), "ac_server_poll")
        return out[:k.value]

    def drain(self):
        _check(lib().ac_server_drain(self.srv), "ac_server_drain")

    def cancel(self, ticket: int):
        """Cancel a request not yet in a wave (raises AcError(AC_ERR_NOT_FOUND) otherwise)."""
        _check(lib().ac_server_cancel(self.srv, ticket), "ac_server_cancel")

    def close(self):
        if getattr(self, "srv", None):
            lib().ac_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
