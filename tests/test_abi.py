"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry
point include/memgs.h declares; ctypes layouts match the header (no GPU calls)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "memgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mgs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_13536_gb300 import _abi, build
    build.build()
    return _abi.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    from paper_2509_13536_gb300 import _abi
    assert sorted(_abi.EXPORTS) == _declared()


def test_struct_sizes_match_header(lib):
    from paper_2509_13536_gb300 import _abi
    assert C.sizeof(_abi.mgs_gaussians) == 72
    assert C.sizeof(_abi.mgs_camera) == 80
    assert C.sizeof(_abi.mgs_image) == 24
    assert C.sizeof(_abi.mgs_grads) == 64
    assert C.sizeof(_abi.mgs_merge_params) == 48


def test_host_only_queries(lib):
    from paper_2509_13536_gb300 import _abi, scenegen as sg
    from paper_2509_13536_gb300.api import _cam_array
    assert lib.mgs_version().decode().startswith("memgs")
    cams = sg.room_poses(2, 0, 320, 240)
    arr = _cam_array(cams)
    a = lib.mgs_render_workspace_size(1000, arr, 2, 0)
    b = lib.mgs_render_workspace_size(1000, arr, 2, 100000)
    assert 0 < a < b
    assert lib.mgs_render_workspace_size(-1, arr, 2, 0) == 0
    assert lib.mgs_render_workspace_size(10, arr, 0, 0) == 0
    assert lib.mgs_voxel_merge_workspace_size(1000) > lib.mgs_voxel_merge_workspace_size(10) > 0
    assert lib.mgs_sort_workspace_size(5000) > 0


def test_invalid_arguments_are_rejected_before_any_launch(lib):
    from paper_2509_13536_gb300 import _abi
    g = _abi.mgs_gaussians(10, 7, 0, 0, 0, None, None, None, None, None, None)  # bad degree
    cam = (_abi.mgs_camera * 1)()
    st = lib.mgs_render(C.byref(g), cam, 1, None, None, 0, None, None)
    assert st == _abi.MGS_ERR_INVALID
    assert b"sh_degree" in lib.mgs_last_error()
    st = lib.mgs_sort_pairs(None, None, None, 10, 5, 3, None, 0, None)
    assert st == _abi.MGS_ERR_INVALID
    p = _abi.mgs_merge_params(7.815, 1e-3, 0, 0, None, None, None, 1, 0)
    g2 = _abi.mgs_gaussians(10, 0, 0, 0, 0, 1, 1, 1, 1, 1, None)  # no birth
    st = lib.mgs_voxel_merge(C.byref(g2), 0.02, C.byref(p), None, None, None, None, None, 0, None)
    assert st == _abi.MGS_ERR_INVALID
    bad = _abi.mgs_merge_params(7.815, 1e-3, 0, 0, None, None, None, 1, 3)  # unknown solver
    g3 = _abi.mgs_gaussians(10, 0, 0, 0, 0, 16, 16, 16, 16, 16, 16)
    n_out = C.c_int64(0)
    st = lib.mgs_voxel_merge(C.byref(g3), 0.02, C.byref(bad), C.byref(g3), None, None, C.byref(n_out), None, 0, None)
    assert st == _abi.MGS_ERR_INVALID and b"solver" in lib.mgs_last_error()


def test_product_path_does_not_import_the_oracle():
    import subprocess
    import sys
    code = ("import sys; import paper_2509_13536_gb300.api as a; import paper_2509_13536_gb300.build; "
            "assert not any(m.startswith('oracle') for m in sys.modules), sorted(sys.modules)")
    subprocess.check_call([sys.executable, "-c", code], cwd=ROOT)
