"""Python binding of the PI batch library (include/pi.h), for tests and benchmarks.

Argument marshalling only: every step of the batch path runs in the CUDA library
(paper_1601_00159_gb300/_build/libpi.so). PyTorch supplies device memory and streams.
uint64 keys and values travel as torch.int64 tensors holding the same bits.
There is no fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpi.so")

PI_OP_SEARCH, PI_OP_INSERT, PI_OP_DELETE = 0, 1, 2
PI_R_ABSENT, PI_R_PRESENT, PI_R_INVALID = 0, 1, 2
PI_OK, PI_ERR_INVALID_ARG, PI_ERR_OOM, PI_ERR_CUDA, PI_ERR_TIMEOUT, PI_ERR_NOT_BUILT = 0, -1, -2, -3, -4, -5
PI_MAX_BATCH = 1 << 28
PI_MAX_KEYS = (1 << 30) - 2

EXPORTED = ["pi_create", "pi_create_ex", "pi_execute_batch", "pi_execute_batch_host", "pi_destroy",
            "pi_last_error", "pi_status", "pi_info", "pi_size", "pi_test_fail_allocations",
            "pi_selftest_wait", "pi_num_levels", "pi_export", "pi_export_level", "pi_export_storage", "pi_profile",
            "pi_profile_read", "pi_profile_kernels", "pi_execute_batch_noalloc", "pi_flush",
            "pi_range_search", "pi_multi_create", "pi_multi_execute", "pi_multi_destroy", "pi_multi_kernels_per_call",
            "pi_server_create", "pi_server_submit", "pi_server_wait", "pi_server_stats", "pi_server_replay",
            "pi_server_destroy"]
PI_MULTI_MAX_CLASSES = 4
PI_MULTI_MAX_BATCH = 1 << 20
PI_NOALLOC_MAX_BATCH = 1 << 16
PI_TEST_WALK_LEVELS = 1
PI_TEST_SORT_FULL = 2
PI_TEST_OWNER_CHECK = 0x100


def PI_TEST_SORT_PREFIX(k: int) -> int:
    """test_flags value: sort batches with k = 1..4 radix passes plus the prefix fix-up."""
    return k << 4
STAGES = ["sort", "descend", "apply", "merge", "layout", "rebuild", "rebuild_write", "locate"]


class PiError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what} failed with code {code}")
        self.code = code


class PiConfig(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("rebuild_policy", ctypes.c_uint32),
                ("rebuild_threshold_pct", ctypes.c_uint32), ("smem_top_entries", ctypes.c_uint32),
                ("storage_capacity", ctypes.c_uint64), ("index_capacity", ctypes.c_uint64),
                ("test_flags", ctypes.c_uint32), ("lowest_level", ctypes.c_uint32),
                ("sort_passes", ctypes.c_uint32), ("small_batches", ctypes.c_uint32)]


class PiMultiClass(ctypes.Structure):
    _fields_ = [("max_log2_size", ctypes.c_uint32), ("warps", ctypes.c_uint32),
                ("radix_bits", ctypes.c_uint32), ("cluster", ctypes.c_uint32)]


class PiMultiConfig(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("num_classes", ctypes.c_uint32),
                ("cls", PiMultiClass * 4)]


class PiMultiBatch(ctypes.Structure):
    _fields_ = [("index", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("ops", ctypes.c_void_p),
                ("keys", ctypes.c_void_p), ("values", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("results", ctypes.c_void_p)]


class PiServerConfig(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("max_batch", ctypes.c_uint32), ("slots", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("ring_queries", ctypes.c_uint64)]


class PiServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("queries", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("max_in_flight", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("p50_s", ctypes.c_double),
                ("p99_s", ctypes.c_double), ("max_s", ctypes.c_double), ("mean_batch", ctypes.c_double)]


class PiInfo(ctypes.Structure):
    _fields_ = [("size", ctypes.c_uint64), ("live", ctypes.c_uint64), ("tombstones", ctypes.c_uint64),
                ("top_level", ctypes.c_uint32), ("bottom_built", ctypes.c_uint32),
                ("smem_low_level", ctypes.c_uint32), ("promote_shift", ctypes.c_uint32),
                ("level_size", ctypes.c_uint64 * 34), ("storage_capacity", ctypes.c_uint64),
                ("index_capacity", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("rebuilds", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("incremental_rebuilds", ctypes.c_uint64), ("owner_checked_writes", ctypes.c_uint64),
                ("routed_batches", ctypes.c_uint64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "level_size"}
        d["level_size"] = list(self.level_size)
        return d


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpi.so and declare its signatures. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"PI CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, u64, i32, dbl = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    lib.pi_create.restype = vp
    lib.pi_create.argtypes = [vp, vp, u64, dbl, u64]
    lib.pi_create_ex.restype = vp
    lib.pi_create_ex.argtypes = [vp, vp, u64, dbl, u64, ctypes.POINTER(PiConfig)]
    lib.pi_execute_batch.restype = i32
    lib.pi_execute_batch.argtypes = [vp, vp, vp, vp, u64, vp, vp]
    lib.pi_execute_batch_noalloc.restype = i32
    lib.pi_execute_batch_noalloc.argtypes = [vp, vp, vp, vp, u64, vp, vp]
    lib.pi_execute_batch_host.restype = i32
    lib.pi_execute_batch_host.argtypes = [vp, vp, vp, vp, u64, vp, vp]
    lib.pi_destroy.restype = None
    lib.pi_destroy.argtypes = [vp]
    lib.pi_last_error.restype = i32
    lib.pi_last_error.argtypes = []
    lib.pi_status.restype = i32
    lib.pi_status.argtypes = [vp, vp]
    lib.pi_info.restype = i32
    lib.pi_info.argtypes = [vp, ctypes.POINTER(PiInfo), vp]
    lib.pi_test_fail_allocations.restype = None
    lib.pi_test_fail_allocations.argtypes = [ctypes.c_uint32]
    lib.pi_selftest_wait.restype = i32
    lib.pi_selftest_wait.argtypes = [ctypes.POINTER(ctypes.c_uint32), vp]
    lib.pi_size.restype = i32
    lib.pi_size.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), vp]
    lib.pi_num_levels.restype = i32
    lib.pi_num_levels.argtypes = [vp, vp]
    lib.pi_export.restype = i32
    lib.pi_export.argtypes = [vp, vp, vp, u64, ctypes.POINTER(u64), vp]
    lib.pi_export_level.restype = i32
    lib.pi_export_level.argtypes = [vp, i32, vp, vp, u64, ctypes.POINTER(u64), vp]
    lib.pi_export_storage.restype = i32
    lib.pi_export_storage.argtypes = [vp, vp, vp, u64, ctypes.POINTER(u64), vp]
    lib.pi_flush.restype = i32
    lib.pi_flush.argtypes = [vp, vp]
    lib.pi_profile.restype = i32
    lib.pi_profile.argtypes = [vp, i32]
    lib.pi_profile_read.restype = i32
    lib.pi_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u64), vp]
    lib.pi_profile_kernels.restype = i32
    lib.pi_profile_kernels.argtypes = [vp, ctypes.c_char_p, u64, vp]
    lib.pi_range_search.restype = i32
    lib.pi_range_search.argtypes = [vp, vp, vp, u64, vp, vp, vp, u64, vp]
    lib.pi_multi_create.restype = vp
    lib.pi_multi_create.argtypes = [ctypes.POINTER(vp), ctypes.c_uint32, ctypes.POINTER(PiMultiConfig)]
    lib.pi_multi_execute.restype = i32
    lib.pi_multi_execute.argtypes = [vp, ctypes.POINTER(PiMultiBatch), ctypes.c_uint32, vp]
    lib.pi_multi_kernels_per_call.restype = u64
    lib.pi_multi_kernels_per_call.argtypes = [vp]
    lib.pi_server_create.restype = vp
    lib.pi_server_create.argtypes = [vp, ctypes.POINTER(PiServerConfig)]
    lib.pi_server_submit.restype = i32
    lib.pi_server_submit.argtypes = [vp, vp, vp, vp, ctypes.c_uint32, ctypes.POINTER(u64)]
    lib.pi_server_wait.restype = i32
    lib.pi_server_wait.argtypes = [vp, u64, vp, ctypes.POINTER(ctypes.c_double)]
    lib.pi_server_stats.restype = i32
    lib.pi_server_stats.argtypes = [vp, ctypes.POINTER(PiServerStats), i32]
    lib.pi_server_replay.restype = i32
    lib.pi_server_replay.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_uint32, vp, vp]
    lib.pi_server_destroy.restype = None
    lib.pi_server_destroy.argtypes = [vp]
    lib.pi_multi_destroy.restype = None
    lib.pi_multi_destroy.argtypes = [vp]
    _lib = lib
    return lib


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_dev(t, dtype, name):
    import torch
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")


def _chk(rc: int, what: str):
    if rc != PI_OK:
        raise PiError(rc, what)


def test_fail_allocations(count: int) -> None:
    """The next `count` device allocations of the library on this thread fail as out of
    memory (pi_test_fail_allocations)."""
    load_library().pi_test_fail_allocations(count)


def selftest_wait(stream=None):
    """(return code, error word) of pi_selftest_wait: a bounded wait on a flag that nothing
    sets must give up with PI_ERR_TIMEOUT."""
    w = ctypes.c_uint32(0)
    rc = load_library().pi_selftest_wait(ctypes.byref(w), _stream_handle(stream))
    return rc, w.value


def _kernel_identifier(mangled: str) -> str:
    """The kernel's own identifier (k_...) in an Itanium-mangled name: a decimal length
    followed by that many characters; the digits before it may run into other digits."""
    import re
    for m in re.finditer(r"(\d+)(k_[a-z0-9_]+)", mangled):
        digits, rest = m.group(1), mangled[m.start(2):]
        for j in range(len(digits)):
            n = int(digits[j:])
            if 0 < n <= len(rest) and re.fullmatch(r"k_[a-z0-9_]+", rest[:n]) and \
                    (n == len(rest) or not re.match(r"[a-z0-9_]", rest[n])):
                if rest[n:n + 1] == "I":  # a template instance: keep its arguments apart
                    return rest[:n] + "<" + rest[n + 1:].split("EE")[0] + ">"
                return rest[:n]
    return mangled


class Index:
    """One PI index resident on the current CUDA device (pi_create ... pi_destroy)."""

    def __init__(self, keys, vals, promote_p: float, seed: int, config: dict | None = None):
        import torch
        lib = load_library()
        _check_dev(keys, torch.int64, "keys")
        _check_dev(vals, torch.int64, "vals")
        if keys.numel() != vals.numel():
            raise ValueError("keys and vals differ in length")
        torch.cuda.current_stream().synchronize()
        if config:
            cfg = PiConfig(ctypes.sizeof(PiConfig), 0, 0, 0, 0, 0, 0, 0, 0, 0)
            for k, v in config.items():
                setattr(cfg, k, v)
            h = lib.pi_create_ex(keys.data_ptr(), vals.data_ptr(), keys.numel(), float(promote_p),
                                 seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(cfg))
        else:
            h = lib.pi_create(keys.data_ptr(), vals.data_ptr(), keys.numel(), float(promote_p),
                              seed & 0xFFFFFFFFFFFFFFFF)
        if not h:
            raise PiError(lib.pi_last_error(), "pi_create")
        self._h = ctypes.c_void_p(h)
        self.lib = lib

    def execute(self, ops, keys, vals, results=None, stream=None):
        """pi_execute_batch on device tensors; returns results as int64 [n, 2]:
        column 0 = value bits, column 1 = status (low 32 bits)."""
        import torch
        n = ops.numel()
        _check_dev(ops, torch.uint8, "ops")
        _check_dev(keys, torch.int64, "keys")
        _check_dev(vals, torch.int64, "vals")
        if keys.numel() != n or vals.numel() != n:
            raise ValueError("ops, keys and vals differ in length")
        if results is None:
            results = torch.empty((n, 2), dtype=torch.int64, device=ops.device)
        rc = self.lib.pi_execute_batch(self._h, ops.data_ptr(), keys.data_ptr(), vals.data_ptr(), n,
                                       results.data_ptr(), _stream_handle(stream))
        _chk(rc, "pi_execute_batch")
        return results

    def execute_noalloc(self, ops, keys, vals, results, stream=None):
        """pi_execute_batch_noalloc: device tensors; `results` (int64 [n, 2]) must exist."""
        import torch
        _check_dev(ops, torch.uint8, "ops")
        _check_dev(keys, torch.int64, "keys")
        _check_dev(vals, torch.int64, "vals")
        _check_dev(results, torch.int64, "results")
        rc = self.lib.pi_execute_batch_noalloc(self._h, ops.data_ptr(), keys.data_ptr(), vals.data_ptr(),
                                               ops.numel(), results.data_ptr(), _stream_handle(stream))
        _chk(rc, "pi_execute_batch_noalloc")
        return results

    def execute_host(self, ops, keys, vals, results, stream=None):
        """pi_execute_batch_host on host (ideally pinned) CPU tensors."""
        n = ops.numel()
        rc = self.lib.pi_execute_batch_host(self._h, ops.data_ptr(), keys.data_ptr(), vals.data_ptr(), n,
                                            results.data_ptr(), _stream_handle(stream))
        _chk(rc, "pi_execute_batch_host")
        return results

    def status(self, stream=None) -> int:
        return self.lib.pi_status(self._h, _stream_handle(stream))

    def info(self, stream=None) -> dict:
        out = PiInfo()
        _chk(self.lib.pi_info(self._h, ctypes.byref(out), _stream_handle(stream)), "pi_info")
        return out.as_dict()

    def size(self, stream=None) -> int:
        """Live keys (pi_size)."""
        n = ctypes.c_uint64(0)
        _chk(self.lib.pi_size(self._h, ctypes.byref(n), _stream_handle(stream)), "pi_size")
        return n.value

    def num_levels(self, stream=None) -> int:
        """H, the number of levels (pi_num_levels)."""
        h = self.lib.pi_num_levels(self._h, _stream_handle(stream))
        _chk(min(h, 0), "pi_num_levels")
        return h

    def export(self, stream=None):
        """Live (keys, vals) in key order as int64 CUDA tensors."""
        import torch
        n = ctypes.c_uint64(0)
        _chk(self.lib.pi_export(self._h, None, None, 0, ctypes.byref(n), _stream_handle(stream)), "pi_export")
        k = torch.empty(max(n.value, 1), dtype=torch.int64, device="cuda")
        v = torch.empty(max(n.value, 1), dtype=torch.int64, device="cuda")
        _chk(self.lib.pi_export(self._h, k.data_ptr(), v.data_ptr(), n.value, ctypes.byref(n),
                                _stream_handle(stream)), "pi_export")
        return k[: n.value], v[: n.value]

    def export_level(self, level: int, stream=None):
        """(keys int64, down int32) of built level `level` >= 2, or None if not built."""
        import torch
        n = ctypes.c_uint64(0)
        rc = self.lib.pi_export_level(self._h, level, None, None, 0, ctypes.byref(n), _stream_handle(stream))
        if rc == PI_ERR_NOT_BUILT:
            return None
        _chk(rc, "pi_export_level")
        k = torch.empty(max(n.value, 1), dtype=torch.int64, device="cuda")
        d = torch.empty(max(n.value, 1), dtype=torch.int32, device="cuda")
        _chk(self.lib.pi_export_level(self._h, level, k.data_ptr(), d.data_ptr(), n.value, ctypes.byref(n),
                                      _stream_handle(stream)), "pi_export_level")
        return k[: n.value], d[: n.value]

    def export_storage(self, stream=None):
        """(keys int64, meta uint8) of the storage layer as stored, delete-flagged nodes
        included (pi_export_storage)."""
        import torch
        n = ctypes.c_uint64(0)
        _chk(self.lib.pi_export_storage(self._h, None, None, 0, ctypes.byref(n), _stream_handle(stream)),
             "pi_export_storage")
        k = torch.empty(max(n.value, 1), dtype=torch.int64, device="cuda")
        m = torch.empty(max(n.value, 1), dtype=torch.uint8, device="cuda")
        _chk(self.lib.pi_export_storage(self._h, k.data_ptr(), m.data_ptr(), n.value, ctypes.byref(n),
                                        _stream_handle(stream)), "pi_export_storage")
        return k[: n.value], m[: n.value]

    def range_search(self, lo, hi, cap=None, stream=None):
        """pi_range_search on int64 CUDA tensors of bounds: (offsets int64 [n + 1], keys,
        vals), query i's pairs at [offsets[i], offsets[i + 1]). Calls again with more room
        when the first capacity is too small (reading offsets[n] synchronises)."""
        import torch
        _check_dev(lo, torch.int64, "lo")
        _check_dev(hi, torch.int64, "hi")
        n = lo.numel()
        if hi.numel() != n:
            raise ValueError("lo and hi differ in length")
        offs = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        cap = int(cap) if cap is not None else max(1024, 16 * n)
        for _ in range(2):
            k = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
            v = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
            _chk(self.lib.pi_range_search(self._h, lo.data_ptr(), hi.data_ptr(), n, offs.data_ptr(), k.data_ptr(),
                                          v.data_ptr(), cap, _stream_handle(stream)), "pi_range_search")
            total = int(offs[n].item())
            if total <= cap:
                return offs, k[:total], v[:total]
            cap = total
        raise RuntimeError("range results did not fit after resizing")

    def flush(self, stream=None):
        """pi_flush: make the stream wait for the index's background work."""
        _chk(self.lib.pi_flush(self._h, _stream_handle(stream)), "pi_flush")

    def profile(self, enable):
        """pi_profile: False/0 off, True/1 stage times, 2 stage and per-kernel times."""
        _chk(self.lib.pi_profile(self._h, int(enable)), "pi_profile")

    def profile_read(self, stream=None):
        """(dict stage -> summed ms, batches covered)."""
        ms = (ctypes.c_double * len(STAGES))()
        nb = ctypes.c_uint64(0)
        _chk(self.lib.pi_profile_read(self._h, ms, ctypes.byref(nb), _stream_handle(stream)), "pi_profile_read")
        return dict(zip(STAGES, list(ms))), nb.value

    def profile_kernels(self, stream=None):
        """{kernel name: (launches, summed ms)} recorded since pi_profile(idx, 2)."""
        import re
        need = self.lib.pi_profile_kernels(self._h, None, 0, _stream_handle(stream))
        _chk(min(need, 0), "pi_profile_kernels")
        buf = ctypes.create_string_buffer(need)
        self.lib.pi_profile_kernels(self._h, buf, need, _stream_handle(stream))
        out = {}
        for line in buf.value.decode().splitlines():
            name, cnt, ms = line.split("\t")
            out[_kernel_identifier(name)] = (int(cnt), float(ms))
        return out

    def close(self):
        if getattr(self, "_h", None):
            self.lib.pi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Prepared:
    """A checked descriptor array for MultiSet.execute (from MultiSet.prepare)."""

    def __init__(self, arr, count, refs):
        self.arr, self.count, self._refs = arr, count, refs


class MultiSet:
    """A set of indices run one batch each per call (pi_multi_create / pi_multi_execute).
    classes: list of (max_log2_size, warps, radix_bits[, cluster]), or None for the
    built-in table; cluster > 1 gives each batch of the class that many CTAs."""

    def __init__(self, indices, classes=None):
        lib = load_library()
        self.indices = list(indices)
        arr = (ctypes.c_void_p * len(self.indices))(*[ix._h.value for ix in self.indices])
        cfgp = None
        if classes is not None:
            cfg = PiMultiConfig()
            cfg.struct_size = ctypes.sizeof(PiMultiConfig)
            cfg.num_classes = len(classes)
            for i, c in enumerate(classes):
                lg, w, b = c[:3]
                cfg.cls[i] = PiMultiClass(lg, w, b, c[3] if len(c) > 3 else 0)
            cfgp = ctypes.byref(cfg)
        h = lib.pi_multi_create(arr, len(self.indices), cfgp)
        if not h:
            raise PiError(lib.pi_last_error(), "pi_multi_create")
        self._h = ctypes.c_void_p(h)
        self.lib = lib

    def prepare(self, batches):
        """The descriptor array of a list of batches (see execute), checked once, for calls
        that reuse it: pi_multi_execute reads the descriptors only during the call. The
        result keeps the tensors referenced."""
        import torch
        arr = (PiMultiBatch * len(batches))()
        for i, (ix, ops, keys, vals, res) in enumerate(batches):
            n = ops.numel()
            _check_dev(ops, torch.uint8, "ops")
            _check_dev(keys, torch.int64, "keys")
            _check_dev(vals, torch.int64, "vals")
            _check_dev(res, torch.int64, "results")
            if keys.numel() != n or vals.numel() != n or res.numel() != 2 * n:
                raise ValueError("batch arrays differ in length")
            arr[i] = PiMultiBatch(ix, 0, ops.data_ptr(), keys.data_ptr(), vals.data_ptr(), n, res.data_ptr())
        return _Prepared(arr, len(batches), list(batches))

    def execute(self, batches, stream=None):
        """batches: list of (index position, ops u8, keys i64, vals i64, results i64[n, 2]) with
        CUDA tensors, or the result of prepare(); results are written in place (value bits,
        status)."""
        p = batches if isinstance(batches, _Prepared) else self.prepare(batches)
        _chk(self.lib.pi_multi_execute(self._h, p.arr, p.count, _stream_handle(stream)), "pi_multi_execute")

    def kernels_per_call(self) -> int:
        return int(self.lib.pi_multi_kernels_per_call(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self.lib.pi_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server over one index (pi_server_*). Host numpy arrays in and
    out; results come back as int64 [n, 2] (value bits, status)."""

    def __init__(self, index, max_batch: int = 0, slots: int = 0, ring_queries: int = 0):
        lib = load_library()
        cfg = PiServerConfig(ctypes.sizeof(PiServerConfig), max_batch, slots, 0, ring_queries)
        h = lib.pi_server_create(index._h, ctypes.byref(cfg))
        if not h:
            raise PiError(lib.pi_last_error(), "pi_server_create")
        self._h = ctypes.c_void_p(h)
        self.lib = lib
        self.index = index

    @staticmethod
    def _host(a, dtype):
        import numpy as np
        a = np.ascontiguousarray(a)
        if a.dtype != dtype:
            a = a.astype(dtype) if dtype != np.uint64 else a.view(np.uint64)
        return a

    def submit(self, ops, keys, vals) -> int:
        import numpy as np
        ops = self._host(ops, np.uint8)
        keys = self._host(keys, np.uint64)
        vals = self._host(vals, np.uint64)
        t = ctypes.c_uint64(0)
        _chk(self.lib.pi_server_submit(self._h, ops.ctypes.data, keys.ctypes.data, vals.ctypes.data, len(ops),
                                       ctypes.byref(t)), "pi_server_submit")
        return t.value

    def wait(self, ticket: int, n: int):
        """(results int64 [n, 2], latency seconds) of the oldest uncollected request."""
        import numpy as np
        out = np.empty((n, 2), dtype=np.int64)
        lat = ctypes.c_double(0)
        _chk(self.lib.pi_server_wait(self._h, ticket, out.ctypes.data, ctypes.byref(lat)), "pi_server_wait")
        return out, lat.value

    def stats(self, reset: bool = False) -> dict:
        st = PiServerStats()
        _chk(self.lib.pi_server_stats(self._h, ctypes.byref(st), 1 if reset else 0), "pi_server_stats")
        return {f: getattr(st, f) for f, _ in st._fields_ if f != "reserved"}

    def replay(self, ops, keys, vals, sizes, arrivals, want_results: bool = True):
        """pi_server_replay: (results int64 [sum(sizes), 2] or None, latencies seconds)."""
        import numpy as np
        ops = self._host(ops, np.uint8)
        keys = self._host(keys, np.uint64)
        vals = self._host(vals, np.uint64)
        sizes = np.ascontiguousarray(sizes, dtype=np.uint32)
        arrivals = np.ascontiguousarray(arrivals, dtype=np.float64)
        total = int(sizes.sum())
        if total > len(ops):
            raise ValueError("sizes exceed the query arrays")
        res = np.empty((total, 2), dtype=np.int64) if want_results else None
        lat = np.empty(len(sizes), dtype=np.float64)
        _chk(self.lib.pi_server_replay(self._h, ops.ctypes.data, keys.ctypes.data, vals.ctypes.data,
                                       sizes.ctypes.data, arrivals.ctypes.data, len(sizes),
                                       res.ctypes.data if res is not None else None, lat.ctypes.data),
             "pi_server_replay")
        return res, lat

    def close(self):
        if getattr(self, "_h", None):
            self.lib.pi_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
