"""The C-ABI library builds for sm_103a, loads and exports every entry point
that include/ans.h declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2510_14050_gb300 import ans, buildlib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ans.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ans_[a-z_]+)\s*\(", text)) - {"ans_alloc_fn", "ans_free_fn"})


def test_header_lists_the_boundary():
    names = declared_functions()
    for required in ("ans_build_window", "ans_sum_windows", "ans_network_quantities", "ans_batch_submit"):
        assert required in names
    assert set(names) == set(ans.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(str(buildlib.build_ans()))
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_clean_failure_without_gpu():
    lib = ans.load()
    assert ans.status_string(ans.ERR_BUDGET) == "memory budget exceeded"
    assert ans.status_string(0) == "ok"
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except Exception:
        pass
    h = ctypes.c_void_p()
    rc = lib.ans_ctx_create(ctypes.byref(h), 0, 0, None, None, None)
    assert rc in (ans.ERR_CUDA, ans.ERR_INVALID_ARG)
    assert not h.value


def test_allocator_hooks_must_come_in_pairs():
    lib = ans.load()
    h = ctypes.c_void_p()
    fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)(lambda *a: None)
    rc = lib.ans_ctx_create(ctypes.byref(h), 0, 0, ctypes.cast(fn, ctypes.c_void_p), None, None)
    assert rc == ans.ERR_INVALID_ARG
