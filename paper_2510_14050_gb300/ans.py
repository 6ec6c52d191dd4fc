"""ctypes binding of ``include/ans.h`` (libans.so).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI.  PyTorch supplies device memory (tensors) and
streams.  If libans.so cannot be loaded the import of this module fails; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Sequence

import numpy as np

from . import buildlib

OK = 0
ERR_INVALID_ARG = -1
ERR_BUDGET = -2
ERR_OOM = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5
ERR_INTERNAL = -6

BATCH_MATRICES = 0x1
BATCH_SUM = 0x2
BATCH_SYNC = 0x4

QUANTITY_NAMES = (
    "valid_packets",
    "unique_links",
    "max_link_packets",
    "unique_sources",
    "max_source_packets",
    "max_source_fanout",
    "unique_destinations",
    "max_destination_packets",
    "max_destination_fanin",
)

# Every symbol the header declares.
EXPORTS = (
    "ans_ctx_create", "ans_ctx_destroy", "ans_build_window", "ans_sum_windows", "ans_network_quantities",
    "ans_batch_submit", "ans_wait", "ans_matrix_view", "ans_matrix_quantities", "ans_matrix_free",
    "ans_status_string", "ans_last_error", "ans_profile_enable", "ans_profile_read",
    "ans_window_quantities_noalloc", "ans_get_tuning", "ans_set_tuning", "ans_autotune", "ans_matrix_retain",
    "ans_ctx_memory", "ans_batch_bytes", "ans_matrix_import", "ans_batch_submit_windows", "ans_combine",
    "ans_set_wait_limit", "ans_probe_wait_expiry", "ans_batch_submit_host", "ans_set_batch_capacity",
    "ans_matrix_split_rows", "ans_probe_guards",
)

# The allocator hook types of ans_ctx_create.
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Quantities(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in QUANTITY_NAMES]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n in QUANTITY_NAMES}


class Tuning(C.Structure):
    _fields_ = [(n, C.c_uint32) for n in ("key_threads", "key_rank", "key_blocks", "kv_threads", "kv_rank",
                                            "kv_blocks", "col_threads", "col_rank", "col_blocks",
                                            "win_path", "win_threads", "win_rank", "sum_path",
                                            "agg_path", "graph", "col_hash", "merge_tile")]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class AnsError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str):
        super().__init__(f"{what}: {detail or status_string(code)} (status {code})")
        self.code = code


_lib = None
_vp = C.c_void_p
_u64 = C.c_uint64


def load(path: str | os.PathLike | None = None):
    """Load libans.so (building it in-tree first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = buildlib.LIBANS if buildlib.LIBANS.exists() else buildlib.build_ans()
    lib = C.CDLL(str(path))
    P = C.POINTER
    sig = {
        "ans_ctx_create": ([P(_vp), C.c_int, C.c_size_t, _vp, _vp, _vp], C.c_int),
        "ans_ctx_destroy": ([_vp], C.c_int),
        "ans_build_window": ([_vp, _vp, _vp, _u64, P(_vp), _vp], C.c_int),
        "ans_sum_windows": ([_vp, P(_vp), C.c_size_t, P(_vp), _vp], C.c_int),
        "ans_network_quantities": ([_vp, _vp, _vp, _vp], C.c_int),
        "ans_batch_submit": ([_vp, _vp, _vp, _vp, C.c_size_t, C.c_uint32, _vp, P(_vp), P(_vp), P(_u64), _vp],
                             C.c_int),
        "ans_batch_submit_host": ([_vp, _vp, _vp, P(_u64), C.c_size_t, C.c_uint32, _vp, P(_vp), P(_vp), P(_u64),
                                   _vp], C.c_int),
        "ans_set_batch_capacity": ([_vp, _u64], C.c_int),
        "ans_matrix_split_rows": ([_vp, _vp, C.c_uint32, P(_vp), _vp], C.c_int),
        "ans_wait": ([_vp, _u64, _u64], C.c_int),
        "ans_matrix_view": ([_vp, P(_u64), P(_u64), P(_vp), P(_vp), P(_vp), P(_vp)], C.c_int),
        "ans_matrix_quantities": ([_vp, P(Quantities)], C.c_int),
        "ans_matrix_free": ([_vp], C.c_int),
        "ans_matrix_retain": ([_vp, P(_vp)], C.c_int),
        "ans_status_string": ([C.c_int], C.c_char_p),
        "ans_last_error": ([_vp], C.c_char_p),
        "ans_profile_enable": ([_vp, C.c_int], C.c_int),
        "ans_profile_read": ([_vp, C.c_char_p, C.c_size_t, P(C.c_size_t)], C.c_int),
        "ans_window_quantities_noalloc": ([_vp, _vp, _u64, _vp, _vp, _vp], C.c_int),
        "ans_get_tuning": ([_vp, P(Tuning)], C.c_int),
        "ans_set_tuning": ([_vp, P(Tuning)], C.c_int),
        "ans_autotune": ([_vp, _vp, _vp, P(_u64), C.c_size_t, C.c_uint32, P(Tuning), _vp], C.c_int),
        "ans_ctx_memory": ([_vp, P(C.c_size_t), P(C.c_size_t)], C.c_int),
        "ans_batch_bytes": ([_vp, P(_u64), C.c_size_t, C.c_uint32, P(C.c_size_t)], C.c_int),
        "ans_matrix_import": ([_vp, _u64, _u64, _vp, _vp, _vp, _vp, P(_vp), _vp], C.c_int),
        "ans_combine": ([_vp, P(_vp), P(C.c_int), C.c_size_t, P(_vp), _vp], C.c_int),
        "ans_batch_submit_windows": ([_vp, P(_vp), P(_vp), P(_u64), C.c_size_t, C.c_uint32, _vp, P(_vp), P(_vp),
                                      P(_u64), _vp], C.c_int),
        "ans_set_wait_limit": ([_vp, C.c_uint32], C.c_int),
        "ans_probe_wait_expiry": ([_vp, P(_vp), P(_u64), _vp], C.c_int),
        "ans_probe_guards": ([_vp, P(_u64), _vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().ans_status_string(code).decode()


def _check(rc: int, what: str, ctx=None):
    if rc != OK:
        detail = load().ans_last_error(ctx).decode()
        raise AnsError(rc, what, detail)


def _stream(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(x) -> int:
    if isinstance(x, int):
        return x
    if x.device.type != "cuda":
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return x.data_ptr()


def _pairs_ptr(x) -> int:
    """Address of a packet array the kernels may read: a CUDA tensor, or a
    page-locked host tensor (read in place over the host link)."""
    if isinstance(x, int):
        return x
    if x.device.type == "cpu" and x.is_pinned():
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    return _dev_ptr(x)


class _DevView:
    """Wrap a raw device pointer for torch.as_tensor (CUDA array interface)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


def _download(ptr: int, n: int, np_dtype) -> np.ndarray:
    import torch
    np_dtype = np.dtype(np_dtype)
    if n == 0:
        return np.zeros(0, np_dtype)
    ts = "<i4" if np_dtype.itemsize == 4 else "<i8"
    t = torch.as_tensor(_DevView(ptr, n, ts), device="cuda")
    return t.cpu().numpy().view(np_dtype)


def _device_tensor(ptr: int, n: int, itemsize: int):
    import torch
    ts = "<i4" if itemsize == 4 else "<i8"
    if n == 0:
        return torch.zeros(0, dtype=torch.int32 if itemsize == 4 else torch.int64, device="cuda")
    return torch.as_tensor(_DevView(ptr, n, ts), device="cuda")


class Matrix:
    """A DCSR traffic matrix in device memory (owned; freed by ``free()``)."""

    def __init__(self, handle: int):
        self._h = _vp(handle)

    @property
    def handle(self):
        return self._h

    def view(self):
        n_r, n_u = _u64(), _u64()
        p = [_vp() for _ in range(4)]
        _check(load().ans_matrix_view(self._h, C.byref(n_r), C.byref(n_u), *[C.byref(x) for x in p]), "view")
        return int(n_r.value), int(n_u.value), [x.value or 0 for x in p]

    @property
    def nrows(self) -> int:
        return self.view()[0]

    @property
    def nnz(self) -> int:
        return self.view()[1]

    def to_numpy(self):
        """(row_ids uint32, row_ptr uint64, col_ids uint32, vals uint64) on the host."""
        nr, nu, (pr, pp, pc, pv) = self.view()
        return (_download(pr, nr, np.uint32), _download(pp, nr + 1, np.uint64),
                _download(pc, nu, np.uint32), _download(pv, nu, np.uint64))

    def device_arrays(self):
        """Zero-copy torch views (int32/int64 reinterpretations) of the four arrays."""
        nr, nu, (pr, pp, pc, pv) = self.view()
        return (_device_tensor(pr, nr, 4), _device_tensor(pp, nr + 1, 8),
                _device_tensor(pc, nu, 4), _device_tensor(pv, nu, 8))

    def quantities(self) -> dict:
        q = Quantities()
        _check(load().ans_matrix_quantities(self._h, C.byref(q)), "matrix_quantities")
        return q.as_dict()

    def retain(self) -> "Matrix":
        """A second handle to the same device matrix (no copy)."""
        out = _vp()
        _check(load().ans_matrix_retain(self._h, C.byref(out)), "matrix_retain")
        return Matrix(out.value)

    def free(self):
        if self._h is not None and self._h.value:
            _check(load().ans_matrix_free(self._h), "matrix_free")
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class TorchAllocator:
    """Device-memory hooks for ans_ctx_create backed by torch's caching
    allocator (stream-ordered: each block is tied to the stream the library
    names).  ``fail_after`` (tests) makes allocation number ``fail_after``
    and later return NULL until it is reset to None."""

    def __init__(self, device: int = 0):
        self.device = device
        self.calls = 0
        self.fail_after = None
        self.live = {}

        def _alloc(nbytes, stream, user):
            import torch
            self.calls += 1
            if self.fail_after is not None and self.calls >= self.fail_after:
                return None
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
            except Exception:
                return None
            self.live[ptr] = int(nbytes)
            return ptr

        def _free(ptr, stream, user):
            import torch
            if ptr:
                self.live.pop(ptr, None)
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)


class Context:
    """One ans_ctx: a device, an allocator, a memory budget and scratch.

    ``allocator``: optional object with ``alloc_fn`` / ``free_fn`` ctypes hooks
    (e.g. TorchAllocator); it must outlive every matrix of the context."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, allocator=None):
        self._lib = load()
        h = _vp()
        self._allocator = allocator  # the hooks must stay alive with the context
        fa = C.cast(allocator.alloc_fn, _vp) if allocator is not None else None
        ff = C.cast(allocator.free_fn, _vp) if allocator is not None else None
        _check(self._lib.ans_ctx_create(C.byref(h), int(device), int(budget_bytes), fa, ff, None), "ctx_create")
        self._h = h
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            _check(self._lib.ans_ctx_destroy(self._h), "ctx_destroy")
        self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points ------------------------------------------------------
    def build_window(self, src, dst, n: int | None = None, stream=None) -> Matrix:
        if n is None:
            n = src.numel()
        out = _vp()
        _check(self._lib.ans_build_window(self._h, _vp(_dev_ptr(src)), _vp(_dev_ptr(dst)), int(n),
                                          C.byref(out), _vp(_stream(stream))), "build_window", self._h)
        return Matrix(out.value)

    def import_matrix(self, row_ids, row_ptr, col_ids, vals, stream=None) -> Matrix:
        """A matrix of this context from DCSR arrays (CUDA tensors, or host
        numpy arrays / CPU tensors: uint32 row ids and column ids, uint64 row
        pointers and values; int32/int64 tensors are taken bit for bit).
        The arrays are copied; non-canonical input raises ERR_INVALID_ARG."""
        keep = []

        def ptr(x, dt):
            if hasattr(x, "data_ptr"):  # torch tensor, device or host
                if not x.is_contiguous():
                    raise ValueError("expected a contiguous tensor")
                keep.append(x)
                return x.data_ptr() if x.numel() else None
            a = np.ascontiguousarray(np.asarray(x, dtype=dt))
            keep.append(a)
            return a.ctypes.data if a.size else None

        nrows = len(row_ids)
        nnz = len(col_ids)
        if len(row_ptr) != nrows + 1 or len(vals) != nnz:
            raise ValueError("row_ptr needs nrows + 1 entries and vals nnz")
        out = _vp()
        _check(self._lib.ans_matrix_import(self._h, nrows, nnz, _vp(ptr(row_ids, np.uint32)),
                                           _vp(ptr(row_ptr, np.uint64)), _vp(ptr(col_ids, np.uint32)),
                                           _vp(ptr(vals, np.uint64)), C.byref(out), _vp(_stream(stream))),
               "matrix_import", self._h)
        return Matrix(out.value)

    def combine(self, mats: Sequence[Matrix], signs: Sequence[int], stream=None) -> Matrix:
        """sum_i signs[i] * mats[i] (signs +1 / -1); cancelled links are dropped."""
        arr = (_vp * max(len(mats), 1))(*[m.handle for m in mats])
        sg = (C.c_int * max(len(signs), 1))(*[int(x) for x in signs])
        if len(signs) != len(mats):
            raise ValueError("one sign per matrix")
        out = _vp()
        _check(self._lib.ans_combine(self._h, arr, sg, len(mats), C.byref(out), _vp(_stream(stream))),
               "combine", self._h)
        return Matrix(out.value)

    def sum_windows(self, mats: Sequence[Matrix], stream=None) -> Matrix:
        arr = (_vp * max(len(mats), 1))(*[m.handle for m in mats])
        out = _vp()
        _check(self._lib.ans_sum_windows(self._h, arr, len(mats), C.byref(out), _vp(_stream(stream))),
               "sum_windows", self._h)
        return Matrix(out.value)

    def split_rows(self, m: Matrix, nparts: int, stream=None) -> list:
        """m's rows split by owner rank (a hash of the source address mod
        nparts), one new matrix per owner."""
        arr = (_vp * nparts)()
        _check(self._lib.ans_matrix_split_rows(self._h, m.handle, int(nparts), arr, _vp(_stream(stream))),
               "matrix_split_rows", self._h)
        return [Matrix(arr[i]) for i in range(nparts)]

    def network_quantities(self, m: Matrix, out=None, stream=None) -> dict | None:
        """Recompute the nine quantities of ``m`` on the device.  With ``out``
        (a device or pinned uint64 tensor of 9 elements) the call is
        asynchronous and returns None; otherwise a dict is returned."""
        if out is not None:
            _check(self._lib.ans_network_quantities(self._h, m.handle, _vp(out.data_ptr()), _vp(_stream(stream))),
                   "network_quantities", self._h)
            return None
        q = Quantities()
        _check(self._lib.ans_network_quantities(self._h, m.handle, _vp(C.addressof(q)), _vp(_stream(stream))),
               "network_quantities", self._h)
        return q.as_dict()

    def batch_submit(self, src, dst, offsets, flags: int = 0, out=None, stream=None, want_ticket: bool = True):
        """Analyse windows [offsets[w], offsets[w+1]) of (src, dst).

        ``src``, ``dst``: int32 tensors on the device, or in page-locked host
        memory (the kernels then read the pairs in place over the host link,
        with no staging copy).  ``offsets``: nwin + 1 uint64 offsets -- a CUDA tensor (int64/uint64,
        read on the device: ans_batch_submit) or a host array-like
        (ans_batch_submit_host).  ``out``: optional tensor of nwin x 9 int64
        (device or pinned host) receiving the quantities.  Returns
        (per_window matrices or None, sum or None, ticket)."""
        on_device = hasattr(offsets, "device") and getattr(offsets.device, "type", "") == "cuda"
        if on_device:
            if offsets.element_size() != 8 or not offsets.is_contiguous():
                raise ValueError("device offsets must be a contiguous 64-bit tensor")
            nwin = offsets.numel() - 1
        else:
            offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
            nwin = len(offs) - 1
        per = (_vp * max(nwin, 1))() if flags & BATCH_MATRICES else None
        sm = _vp() if flags & BATCH_SUM else None
        tk = _u64() if want_ticket else None
        outp = _vp(out.data_ptr()) if out is not None else None
        tail = (nwin, int(flags), outp, per, C.byref(sm) if sm is not None else None,
                C.byref(tk) if tk is not None else None, _vp(_stream(stream)))
        if on_device:
            _check(self._lib.ans_batch_submit(self._h, _vp(_pairs_ptr(src)), _vp(_pairs_ptr(dst)),
                                              _vp(offsets.data_ptr()), *tail), "batch_submit", self._h)
        else:
            _check(self._lib.ans_batch_submit_host(self._h, _vp(_pairs_ptr(src)), _vp(_pairs_ptr(dst)),
                                                   offs.ctypes.data_as(C.POINTER(_u64)), *tail),
                   "batch_submit_host", self._h)
        mats = [Matrix(per[i]) for i in range(nwin)] if per is not None else None
        summ = Matrix(sm.value) if sm is not None else None
        return mats, summ, (int(tk.value) if tk is not None else None)

    def batch_submit_windows(self, windows, flags: int = 0, out=None, stream=None, want_ticket: bool = True):
        """As batch_submit, with every window in its own arrays: ``windows`` is
        a sequence of (src, dst) pairs -- int32 tensors of equal length on the
        device or in pinned host memory (read in place), or (src_ptr, dst_ptr,
        n) triples of raw addresses."""
        nwin = len(windows)
        srcs = (_vp * max(nwin, 1))()
        dsts = (_vp * max(nwin, 1))()
        lens = np.zeros(max(nwin, 1), dtype=np.uint64)
        for i, w in enumerate(windows):
            if len(w) == 3:
                srcs[i], dsts[i], lens[i] = w[0], w[1], int(w[2])
            else:
                a, b = w
                if a.numel() != b.numel():
                    raise ValueError("src and dst of a window differ in length")
                if not (a.is_contiguous() and b.is_contiguous()):
                    raise ValueError("expected contiguous tensors")
                srcs[i], dsts[i], lens[i] = a.data_ptr(), b.data_ptr(), a.numel()
        per = (_vp * max(nwin, 1))() if flags & BATCH_MATRICES else None
        sm = _vp() if flags & BATCH_SUM else None
        tk = _u64() if want_ticket else None
        outp = _vp(out.data_ptr()) if out is not None else None
        _check(self._lib.ans_batch_submit_windows(
            self._h, srcs, dsts, lens.ctypes.data_as(C.POINTER(_u64)), nwin, int(flags), outp, per,
            C.byref(sm) if sm is not None else None, C.byref(tk) if tk is not None else None,
            _vp(_stream(stream))), "batch_submit_windows", self._h)
        mats = [Matrix(per[i]) for i in range(nwin)] if per is not None else None
        summ = Matrix(sm.value) if sm is not None else None
        return mats, summ, (int(tk.value) if tk is not None else None)

    def profile(self, enable: bool = True):
        _check(self._lib.ans_profile_enable(self._h, 1 if enable else 0), "profile_enable", self._h)

    def profile_read(self) -> dict:
        """{kernel name: (launches, total ms)} since profiling was enabled."""
        need = C.c_size_t()
        _check(self._lib.ans_profile_read(self._h, None, 0, C.byref(need)), "profile_read", self._h)
        buf = C.create_string_buffer(need.value + 64)
        _check(self._lib.ans_profile_read(self._h, buf, len(buf), None), "profile_read", self._h)
        out = {}
        for line in buf.value.decode().splitlines():
            name, n, ms = line.split()
            out[name] = (int(n), float(ms))
        return out

    def memory(self) -> tuple[int, int]:
        """(device bytes held now, budget) of this context."""
        live, budget = C.c_size_t(), C.c_size_t()
        _check(self._lib.ans_ctx_memory(self._h, C.byref(live), C.byref(budget)), "ctx_memory", self._h)
        return int(live.value), int(budget.value)

    def batch_bytes(self, offsets, flags: int = 0) -> int:
        """Additional device bytes batch_submit(offsets, flags) would allocate now."""
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
        out = C.c_size_t()
        _check(self._lib.ans_batch_bytes(self._h, offs.ctypes.data_as(C.POINTER(_u64)), len(offs) - 1, int(flags),
                                         C.byref(out)), "batch_bytes", self._h)
        return int(out.value)

    def get_tuning(self) -> dict:
        t = Tuning()
        _check(self._lib.ans_get_tuning(self._h, C.byref(t)), "get_tuning", self._h)
        return t.as_dict()

    def set_tuning(self, **kw):
        t = Tuning(**{**self.get_tuning(), **kw})
        _check(self._lib.ans_set_tuning(self._h, C.byref(t)), "set_tuning", self._h)

    def autotune(self, src, dst, offsets, stream=None, flags: int = BATCH_MATRICES | BATCH_SUM) -> dict:
        """Time the candidate radix-pass configurations and paths on this
        batch, as submitted with ``flags``; returns the chosen configuration."""
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
        t = Tuning()
        _check(self._lib.ans_autotune(self._h, _vp(_dev_ptr(src)), _vp(_dev_ptr(dst)),
                                      offs.ctypes.data_as(C.POINTER(_u64)), len(offs) - 1, int(flags), C.byref(t),
                                      _vp(_stream(stream))), "autotune", self._h)
        return t.as_dict()

    def set_batch_capacity(self, max_packets: int = 0):
        """Packets a batch with device-resident offsets may hold (0: each such
        batch reads its first and last offset back to size itself)."""
        _check(self._lib.ans_set_batch_capacity(self._h, int(max_packets)), "set_batch_capacity", self._h)

    def set_wait_limit(self, polls: int = 0):
        """Poll limit of the bounded device waits (0: the default, ~1 s)."""
        _check(self._lib.ans_set_wait_limit(self._h, int(polls)), "set_wait_limit", self._h)

    def probe_wait_expiry(self, want_matrix: bool = True, stream=None):
        """Run one device wait that can only end at the poll limit; returns
        (empty matrix or None, ticket).  ans_wait on the ticket and the
        matrix's view then report ERR_INTERNAL."""
        m = _vp()
        tk = _u64()
        _check(self._lib.ans_probe_wait_expiry(self._h, C.byref(m) if want_matrix else None, C.byref(tk),
                                               _vp(_stream(stream))), "probe_wait_expiry", self._h)
        return (Matrix(m.value) if want_matrix else None), int(tk.value)

    def probe_guards(self, stream=None) -> int:
        """Fill one scratch guard, overwrite it and check it; returns the
        ticket, on which ans_wait then reports ERR_INTERNAL."""
        tk = _u64()
        _check(self._lib.ans_probe_guards(self._h, C.byref(tk), _vp(_stream(stream))), "probe_guards", self._h)
        return int(tk.value)

    def wait_status(self, ticket: int, timeout_s: float = 60.0) -> int:
        """ans_wait's status code (no exception)."""
        return int(self._lib.ans_wait(self._h, int(ticket), int(timeout_s * 1e9)))

    def wait(self, ticket: int, timeout_s: float = 60.0):
        _check(self._lib.ans_wait(self._h, int(ticket), int(timeout_s * 1e9)), "wait", self._h)


def quantities_from_tensor(t) -> list[dict]:
    """nwin x 9 int64 tensor/array -> list of quantity dicts."""
    a = t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
    a = a.view(np.uint64).reshape(-1, 9)
    return [{n: int(v) for n, v in zip(QUANTITY_NAMES, row)} for row in a]
