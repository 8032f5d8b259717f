"""mgs_sort_pairs_noalloc, the sort entry point for callers that cannot allocate device
memory (its scratch is a static array inside the library), must give exactly what
mgs_sort_pairs gives with a caller workspace.  Called through the C ABI, twice in a
row, so the second call runs on scratch that still holds the first call's data.  This
file is collected last so that a run stopping at the first failure has run the rest."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _sort_with_workspace(lib, keys, with_vals, bits):
    n = keys.numel()
    ws = torch.empty(lib.mgs_sort_workspace_size(n), dtype=torch.uint8, device="cuda")
    k = keys.clone()
    v = torch.arange(n, dtype=torch.int32, device="cuda") * 7 + 3 if with_vals else None
    out = None if with_vals else torch.empty(n, dtype=torch.int32, device="cuda")
    st = lib.mgs_sort_pairs(_p(k), _p(v), _p(out), n, bits[0], bits[1], _p(ws), ws.numel(),
                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.mgs_last_error()
    return k, (v if with_vals else out)


def _sort_noalloc(lib, keys, with_vals, bits):
    n = keys.numel()
    k = keys.clone()
    v = torch.arange(n, dtype=torch.int32, device="cuda") * 7 + 3 if with_vals else None
    out = None if with_vals else torch.empty(n, dtype=torch.int32, device="cuda")
    st = lib.mgs_sort_pairs_noalloc(_p(k), _p(v), _p(out), n, bits[0], bits[1],
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.mgs_last_error()
    return k, (v if with_vals else out)


def test_noalloc_sort_matches_workspace_sort_twice_in_a_row():
    from paper_2509_13536_gb300 import _abi, build
    build.build()
    lib = _abi.load()
    rng = np.random.default_rng(2024)
    cases = [(1_000_003, False, (0, 32)), (_abi.MGS_SORT_NOALLOC_MAX, True, (3, 20)), (4097, False, (0, 15))]
    for n, with_vals, bits in cases:
        raw = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
        raw[: n // 4] = raw[0]  # runs of equal keys: the sort must be stable
        keys = torch.from_numpy(raw.view(np.int32)).cuda()
        k_ref, v_ref = _sort_with_workspace(lib, keys, with_vals, bits)
        k_new, v_new = _sort_noalloc(lib, keys, with_vals, bits)
        torch.cuda.synchronize()
        assert torch.equal(k_new, k_ref)
        assert torch.equal(v_new, v_ref)


def test_noalloc_sort_rejects_sizes_beyond_its_maximum():
    from paper_2509_13536_gb300 import _abi
    lib = _abi.load()
    n = _abi.MGS_SORT_NOALLOC_MAX + 1
    keys = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = lib.mgs_sort_pairs_noalloc(_p(keys), None, _p(out), n, 0, 32,
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _abi.MGS_ERR_UNSUPPORTED
    assert b"MGS_SORT_NOALLOC_MAX" in lib.mgs_last_error()


def test_noalloc_sort_of_an_offset_view():
    """Keys that start 4 bytes into an allocation (keys[1:], not 16-byte aligned) sort
    exactly as an aligned copy of them does."""
    from paper_2509_13536_gb300 import _abi
    lib = _abi.load()
    rng = np.random.default_rng(7)
    n = 200_003
    raw = rng.integers(0, 2 ** 32, n + 1, dtype=np.uint64).astype(np.uint32)
    base = torch.from_numpy(raw.view(np.int32)).cuda()
    view = base[1:]
    assert view.data_ptr() % 16 != 0
    k_ref, v_ref = _sort_with_workspace(lib, view.clone(), False, (0, 32))
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = lib.mgs_sort_pairs_noalloc(_p(view), None, _p(out), n, 0, 32,
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.mgs_last_error()
    torch.cuda.synchronize()
    assert torch.equal(view, k_ref) and torch.equal(out, v_ref)
