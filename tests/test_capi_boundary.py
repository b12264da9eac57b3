"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/sdm.h (no GPU needed: nothing here launches work)."""
import ctypes as C
import os
import re

import pytest

from paper_2101_06318_b300 import build, sdm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "sdm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(sdm_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    L = C.CDLL(path)
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name
    # the binding knows the same set
    assert sorted(sdm.EXPORTS) == declared


def test_host_only_calls():
    L = sdm.lib()
    assert b"sm_103a" in L.sdm_version()
    for code in range(8):
        assert L.sdm_status_str(code).startswith(b"SDM_")
    # workspace bound grows with the state size
    assert L.sdm_workspace_bytes(1 << 20, 1, 1) > L.sdm_workspace_bytes(1 << 10, 1, 1) > 0
    # argument checks happen before any CUDA call
    h = C.c_void_p()
    assert L.sdm_alloc(None, 10, 1, 1, None, None, 0) == 1
    assert L.sdm_alloc(C.byref(h), 0, 1, 1, None, None, 0) == 1
    assert L.sdm_alloc(C.byref(h), 10, 0, 1, None, None, 0) == 1
    assert L.sdm_alloc(C.byref(h), 1 << 32, 1, 1, None, None, 0) == 1
    assert L.sdm_coalescence_step(None, None, 1, None) == 1
    assert L.sdm_sync(None) == 1
    assert L.sdm_debug_wait_timeout(None, 100, 1) == 1
    assert L.sdm_debug_bucket_capacity(None, 64) == 1
    assert L.sdm_debug_stage_shortfall(None, 16, 20) == 1
    L.sdm_free(None)


def test_binding_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        sdm.State(16, 1)
