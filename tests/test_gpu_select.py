"""GPU parity of the distributed selection's local steps (asci_select_histogram,
asci_select_below) against a host computation of the rank words, and the
whole distributed selection on one rank (a world-size-1 gloo group) against
asci_select_topn."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def asci():
    import paper_2303_05688_gb300 as m
    m.load()
    return m


def _case(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.permutation(1 << 20)[:n].astype(np.uint64)
    b = rng.integers(0, 1 << 12, n).astype(np.uint64)
    s = rng.normal(size=n) * 10.0 ** rng.integers(-8, 2, n)
    s[rng.random(n) < 0.2] = 0.125  # ties decided by the key
    return a, b, s


def _words(a, b, s):
    bits = np.abs(s).view(np.uint64)
    return (~bits).astype(np.uint64), (b << np.uint64(32)) | a


@pytest.mark.parametrize("n", [1, 1000, 123457])
def test_select_histogram_and_below(torch_cuda, asci, n):
    torch = torch_cuda
    a, b, s = _case(n, n)
    d = torch.tensor(np.stack([a, b], 1).view(np.int64), device="cuda")
    v = torch.tensor(s, device="cuda")
    hi, lo = _words(a, b, s)
    # the top byte, then a byte under a prefix
    h = asci.select_histogram(d, v, 15, [0, 0], [0, 0])
    assert np.array_equal(h, np.bincount((hi >> np.uint64(56)).astype(np.int64), minlength=256))
    top = int(hi[0] >> np.uint64(56))
    m = (hi >> np.uint64(56)) == np.uint64(top)
    h2 = asci.select_histogram(d, v, 2, [top << 56, 0], [0xff << 56, 0])
    want = np.bincount(((lo[m] >> np.uint64(16)) & np.uint64(0xff)).astype(np.int64), minlength=256)
    assert np.array_equal(h2, want)
    # entries at or below the rank word of a middle entry
    t = np.lexsort((lo, hi))[n // 2]
    k, sc = asci.select_below(d, v, [int(hi[t]), int(lo[t])])
    keep = (hi < hi[t]) | ((hi == hi[t]) & (lo <= lo[t]))
    got = sorted(((k.cpu().numpy().view(np.uint64)[:, 1] << np.uint64(32)) |
                  k.cpu().numpy().view(np.uint64)[:, 0]).tolist())
    assert got == sorted(lo[keep].tolist()) and len(sc) == keep.sum()


def test_distributed_topn_one_rank_equals_select_topn(torch_cuda, asci):
    torch = torch_cuda
    import torch.distributed as dist
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        a, b, s = _case(50000, 7)
        d = torch.tensor(np.stack([a, b], 1).view(np.int64), device="cuda")
        v = torch.tensor(s, device="cuda")
        for N in (1, 777, 50000, 60000):
            # gloo reduces CPU tensors: hand the local steps' results over on the host
            gk, gs = asci.distributed_topn(
                d.cpu(), v.cpu(), N,
                hist_fn=lambda dg, p, m: asci.select_histogram(d, v, dg, p, m),
                below_fn=lambda t: tuple(x.cpu() for x in asci.select_below(d, v, t)))
            rk, rs = asci.select_topn(d, v, N)
            g = sorted(zip(gk.numpy().view(np.uint64)[:, 0].tolist(),
                           gk.numpy().view(np.uint64)[:, 1].tolist(), gs.numpy().tolist()))
            r = sorted(zip(rk.cpu().numpy().view(np.uint64)[:, 0].tolist(),
                           rk.cpu().numpy().view(np.uint64)[:, 1].tolist(), rs.cpu().numpy().tolist()))
            assert g == r
    finally:
        dist.destroy_process_group()
