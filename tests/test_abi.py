"""The C-ABI library loads and exports every entry point include/moma.h
declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "moma.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(moma_[a-z_]+)\s*\(", text))


def test_header_declarations_match_binding_list(moma_lib):
    assert _declared() == set(moma_lib.EXPORTS)


def test_library_exports_every_declared_symbol(moma_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", moma_lib.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (moma_\w+)", out))
    missing = _declared() - exported
    assert not missing, missing
    L = ctypes.CDLL(moma_lib.LIB_PATH)
    for name in _declared():
        assert getattr(L, name) is not None


def test_build_targets_sm103a_only():
    from paper_2608_17844_b300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_null_handle_and_bad_args_fail_cleanly(moma_lib):
    L = moma_lib.lib()
    assert L.moma_set_blocks(None, None, 0) == 1  # MOMA_ERR_ARG
    assert L.moma_solve(None, 1, None, None, None, None, None) == 1
    assert L.moma_launch_count(None) == 0
    L.moma_destroy(None)
    assert "NULL" in moma_lib.moma_last_error()


def test_create_without_gpu_reports_status(moma_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(moma_lib.MomaError) as e:
        moma_lib.moma_create_array(4, 4, 8)
    assert e.value.status in (4, 3)  # MOMA_ERR_CUDA / MOMA_ERR_OOM, never a crash


def test_create_rejects_bad_sizes(moma_lib):
    for args in [(0, 4, 8), (4, -1, 8), (4, 4, 0)]:
        with pytest.raises(moma_lib.MomaError) as e:
            moma_lib.moma_create_array(*args)
        assert e.value.status == 1


def test_binding_fails_loudly_without_library(moma_lib, monkeypatch):
    from paper_2608_17844_b300 import moma as m
    monkeypatch.setattr(m, "_lib", None)
    monkeypatch.setattr(m, "LIB_PATH", "/nonexistent/libmoma.so")
    with pytest.raises(RuntimeError, match="missing"):
        m.lib()
