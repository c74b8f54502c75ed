"""asci_sort_accumulate_noalloc against asci_sort_accumulate, through the C ABI.

The no-allocation entry point is for callers that cannot allocate device
memory during a call (memory reserved by another allocator or capped, or a
policy that forbids allocation behind the caller's back); its scratch is one
fixed device array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_PAIRS = 65536  # ASCI_NOALLOC_MAX_PAIRS in include/asci.h


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_05688_gb300 as asci
    L = asci.load()
    vp, sz = ct.c_void_p, ct.c_size_t
    for name in ("asci_sort_accumulate", "asci_sort_accumulate_noalloc"):
        f = getattr(L, name)
        f.restype = ct.c_int
        f.argtypes = [vp, vp, sz, vp, vp, ct.POINTER(sz), vp]
    return L


def _call(L, name, keys, vals):
    import torch
    n = keys.shape[0]
    ok = torch.empty((max(n, 1), 2), dtype=torch.int64, device="cuda")
    os_ = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    m = ct.c_size_t(0)
    stream = torch.cuda.current_stream().cuda_stream
    code = getattr(L, name)(keys.data_ptr(), vals.data_ptr(), n, ok.data_ptr(), os_.data_ptr(),
                            ct.byref(m), stream)
    return code, ok[:m.value].cpu().numpy(), os_[:m.value].cpu().numpy()


def _case(seed, n):
    import torch
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 1 << 11, n).astype(np.int64)
    b = rng.integers(0, 1 << 7, n).astype(np.int64) << 12
    v = rng.normal(size=n) * 10.0 ** rng.uniform(-12, 1, n)
    keys = torch.tensor(np.stack([a, b], 1), device="cuda")
    return keys, torch.tensor(v, device="cuda")


def test_noalloc_matches_sort_accumulate_twice(lib):
    # two calls in a row: the shared scratch keeps the previous call's contents
    for seed, n in ((11, 50_000), (12, MAX_PAIRS)):
        keys, vals = _case(seed, n)
        c1, k1, s1 = _call(lib, "asci_sort_accumulate", keys, vals)
        c2, k2, s2 = _call(lib, "asci_sort_accumulate_noalloc", keys, vals)
        assert c1 == 0 and c2 == 0
        assert np.array_equal(k1, k2)
        assert np.allclose(s1, s2, rtol=0, atol=1e-12)


def test_noalloc_rejects_sizes_beyond_its_maximum(lib):
    keys, vals = _case(13, MAX_PAIRS + 1)
    code, _, _ = _call(lib, "asci_sort_accumulate_noalloc", keys, vals)
    assert code == -1
    lib.asci_last_error.restype = ct.c_char_p
    assert b"ASCI_NOALLOC_MAX_PAIRS" in lib.asci_last_error()
