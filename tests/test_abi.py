"""The C ABI library loads and exports every function include/kpx.h declares,
and rejects invalid problems before touching the GPU (no compute calls: every
case here fails host-side validation, which runs before any CUDA call)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2602_02846_gb300 as kpx
from paper_2602_02846_gb300 import build as kbuild
from paper_2602_02846_gb300 import scenes

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kpx.h")


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return kpx.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kpx_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(kpx.EXPORTED) == set(names)


def test_status_strings(lib):
    assert lib.kpx_status_str(0) == b"ok"
    assert lib.kpx_status_str(4) == b"tree full"
    assert lib.kpx_status_str(99) == b"unknown status"


def test_workspace_size_validation(lib):
    p = scenes.di_scene(0)
    assert kpx.kpx_workspace_size(p) > 0
    assert kpx.kpx_workspace_size(p.replace(tree_cap=0)) == 0
    assert kpx.kpx_workspace_size(p.replace(k_min=0)) == 0
    assert kpx.kpx_workspace_size(p.replace(i_max=255)) == 0
    assert kpx.kpx_workspace_size(p.replace(h=-0.01)) == 0
    # sizes grow with the tree capacity
    assert kpx.kpx_workspace_size(p.replace(tree_cap=1 << 16)) > kpx.kpx_workspace_size(p)


def _create(lib, prob, ws_ptr, ws_bytes):
    d, w, o, g, c, cfg, obs, start = kpx.problem_structs(prob)
    h = C.c_void_p()
    st = lib.kpx_create(C.byref(d), C.byref(w), C.byref(o), start.ctypes.data_as(C.POINTER(C.c_float)),
                        C.byref(g), C.byref(c), C.byref(cfg), C.c_void_p(ws_ptr), C.c_size_t(ws_bytes),
                        None, C.byref(h))
    return st, h, lib.kpx_last_error(None).decode()


def _no_gpu():
    try:
        import torch
        return not torch.cuda.is_available()
    except Exception:
        return True


def test_create_rejects_invalid_inputs_before_cuda(lib):
    if not _no_gpu():
        pytest.skip("host-validation cases run on machines without a GPU only")
    p = scenes.di_scene(0)
    size = kpx.kpx_workspace_size(p)
    fake = 1 << 20  # aligned, never dereferenced: every case fails validation first
    st, h, msg = _create(lib, p, 0, size)
    assert st == kpx.KPX_E_INVALID and "null" in msg
    st, h, msg = _create(lib, p, fake + 8, size)
    assert st == kpx.KPX_E_INVALID and "aligned" in msg
    st, h, msg = _create(lib, p, fake, size - 1)
    assert st == kpx.KPX_E_NOMEM
    bad = p.replace(start=np.array([0.05, 0.05, np.nan, 0, 0, 0], np.float32))
    st, h, msg = _create(lib, bad, fake, size)
    assert st == kpx.KPX_E_INVALID and "finite" in msg
    box = p.obstacles[0]
    inside = np.array([(box[0] + box[3]) / 2, (box[1] + box[4]) / 2, (box[2] + box[5]) / 2, 0, 0, 0], np.float32)
    st, h, msg = _create(lib, p.replace(start=inside), fake, size)
    assert st == kpx.KPX_E_INVALID and "X_valid" in msg
    st, h, msg = _create(lib, p.replace(start=np.array([0.05, 0.05, 0.05, 1.5, 0, 0], np.float32)), fake, size)
    assert st == kpx.KPX_E_INVALID
    st, h, msg = _create(lib, p.replace(cost_kind=scenes.COST_EFFORT_DURATION), fake, size)
    assert st == kpx.KPX_E_INVALID and "quadcopter" in msg
    st, h, msg = _create(lib, p.replace(goal_r=-1.0), fake, size)
    assert st == kpx.KPX_E_INVALID
    flipped = p.obstacles.copy()
    flipped[0, [0, 3]] = flipped[0, [3, 0]]
    st, h, msg = _create(lib, p.replace(obstacles=flipped), fake, size)
    assert st == kpx.KPX_E_INVALID and "lo > hi" in msg


def test_null_handles(lib):
    assert lib.kpx_iterate(None, 1, None) == kpx.KPX_E_INVALID
    assert lib.kpx_destroy(None) == kpx.KPX_OK
    assert lib.kpx_reset(None) == kpx.KPX_E_INVALID
    n = C.c_int32(0)
    assert lib.kpx_best_trajectory(None, 0, None, None, None, C.byref(n), None) == kpx.KPX_E_INVALID
