"""asci_sort_accumulate_noalloc against asci_sort_accumulate, through the C ABI.

The no-allocation entry point is for callers that cannot allocate device
memory during a call (memory reserved by another allocator or capped, or a
policy that forbids allocation behind the caller's back); its scratch is one
fixed device array inside the library.  Both entry points run the same stable
sort and the same sequential segment sums, so their results are compared bit
for bit.  This file is collected last so that a run stopping at the first
failure has already run every other test; each test also passes alone in a
fresh process (the first call on the device loads the array).
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
    L.asci_last_error.restype = ct.c_char_p
    return L


def _call(L, name, keys, vals):
    """One call with device inputs and outputs; returns (code, keys, sums)."""
    import torch
    n = keys.shape[0]
    ok = torch.empty((max(n, 1), 2), dtype=torch.int64, device="cuda")
    os_ = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    m = ct.c_size_t(0)
    stream = torch.cuda.current_stream().cuda_stream
    code = getattr(L, name)(keys.data_ptr(), vals.data_ptr(), n, ok.data_ptr(), os_.data_ptr(),
                            ct.byref(m), stream)
    return code, ok[:m.value].cpu().numpy(), os_[:m.value].cpu().numpy()


def _call_host(L, name, keys, vals):
    """One call with host (numpy) inputs and outputs."""
    n = keys.shape[0]
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    ok = np.zeros((max(n, 1), 2), dtype=np.uint64)
    os_ = np.zeros(max(n, 1))
    m = ct.c_size_t(0)
    code = getattr(L, name)(keys.ctypes.data, vals.ctypes.data, n, ok.ctypes.data,
                            os_.ctypes.data, ct.byref(m), None)
    return code, ok[:m.value], os_[:m.value]


def _arrays(seed, n):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 1 << 11, n).astype(np.uint64)
    b = rng.integers(0, 1 << 7, n).astype(np.uint64) << np.uint64(12)
    v = rng.normal(size=n) * 10.0 ** rng.uniform(-12, 1, n)
    return np.stack([a, b], 1), v


def _case(seed, n):
    import torch
    k, v = _arrays(seed, n)
    return torch.tensor(k.view(np.int64), device="cuda"), torch.tensor(v, device="cuda")


def test_noalloc_matches_sort_accumulate_twice(lib):
    # two calls in a row: the shared scratch keeps the previous call's contents
    for seed, n in ((11, 50_000), (12, MAX_PAIRS)):
        keys, vals = _case(seed, n)
        c1, k1, s1 = _call(lib, "asci_sort_accumulate", keys, vals)
        c2, k2, s2 = _call(lib, "asci_sort_accumulate_noalloc", keys, vals)
        assert c1 == 0 and c2 == 0
        assert len(k1) < n
        assert np.array_equal(k1, k2)
        assert np.array_equal(s1, s2)


def test_noalloc_host_buffers_at_the_maximum(lib):
    keys, vals = _arrays(14, MAX_PAIRS)
    c1, k1, s1 = _call_host(lib, "asci_sort_accumulate", keys, vals)
    c2, k2, s2 = _call_host(lib, "asci_sort_accumulate_noalloc", keys, vals)
    assert c1 == 0 and c2 == 0
    assert np.array_equal(k1, k2) and np.array_equal(s1, s2)
    # against numpy: unique keys ascending (beta word high), sums in input order
    key = (keys[:, 1] << np.uint64(32)) | keys[:, 0]
    uk, inv = np.unique(key, return_inverse=True)
    assert np.array_equal((k2[:, 1] << np.uint64(32)) | k2[:, 0], uk)
    ref = np.zeros(len(uk))
    np.add.at(ref, inv, vals)
    assert np.allclose(s2, ref, rtol=1e-12, atol=1e-300)


def test_noalloc_degenerate_inputs(lib):
    import torch
    # n = 0 (valid buffers): nothing to do, nothing written
    keys, vals = _case(15, 1)
    ok = torch.full((1, 2), -1, dtype=torch.int64, device="cuda")
    m = ct.c_size_t(7)
    code = lib.asci_sort_accumulate_noalloc(keys.data_ptr(), vals.data_ptr(), 0, ok.data_ptr(),
                                            ok.data_ptr(), ct.byref(m), None)
    assert code == 0 and m.value == 0 and int(ok[0, 0]) == -1
    # every key equal: one output, the sum of all values
    n = 4097
    keys = torch.tensor(np.tile(np.array([[5, 9 << 20]], dtype=np.int64), (n, 1)), device="cuda")
    vals = torch.tensor(np.random.default_rng(16).normal(size=n), device="cuda")
    c1, k1, s1 = _call(lib, "asci_sort_accumulate", keys, vals)
    c2, k2, s2 = _call(lib, "asci_sort_accumulate_noalloc", keys, vals)
    assert c1 == 0 and c2 == 0 and len(k2) == 1
    assert np.array_equal(k1, k2) and np.array_equal(s1, s2)
    assert abs(s2[0] - float(np.sum(vals.cpu().numpy()))) <= 1e-12 * n


def test_noalloc_allocates_no_device_memory(lib):
    import torch
    keys, vals = _case(17, MAX_PAIRS)
    ok = torch.empty((MAX_PAIRS, 2), dtype=torch.int64, device="cuda")
    os_ = torch.empty(MAX_PAIRS, dtype=torch.float64, device="cuda")
    m = ct.c_size_t(0)
    stream = torch.cuda.current_stream().cuda_stream
    args = (keys.data_ptr(), vals.data_ptr(), MAX_PAIRS, ok.data_ptr(), os_.data_ptr(),
            ct.byref(m), stream)
    assert lib.asci_sort_accumulate_noalloc(*args) == 0  # warm-up: loads the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lib.asci_sort_accumulate_noalloc(*args) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_invalid_input(lib):
    keys, vals = _case(13, MAX_PAIRS + 1)
    code, _, _ = _call(lib, "asci_sort_accumulate_noalloc", keys, vals)
    assert code == -1
    assert b"ASCI_NOALLOC_MAX_PAIRS" in lib.asci_last_error()
    # a key word with a bit at or above 32 does not fit the packed key
    keys, vals = _arrays(18, 1000)
    keys[123, 0] |= np.uint64(1 << 40)
    for name in ("asci_sort_accumulate", "asci_sort_accumulate_noalloc"):
        code, _, _ = _call_host(lib, name, keys, vals)
        assert code == -1, name
        assert b"bits at or above 32" in lib.asci_last_error()
    # a valid call still works after the rejections
    keys, vals = _case(19, 1000)
    code, k, _ = _call(lib, "asci_sort_accumulate_noalloc", keys, vals)
    assert code == 0 and len(k) > 0
