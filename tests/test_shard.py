"""Constraint sharding (Sec. 2.2, Alg. 3) and the exchange of the sharded
search, on the CPU: the greedy placement exported by the library, and the
candidate exchange over torch.distributed with the gloo backend (world size 2).
"""
import os
import socket

import shutil

import numpy as np
import pytest


@pytest.fixture(scope="module")
def asci():
    """The library, built here if needed (the functions used run on the host)."""
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2303_05688_gb300 as m
    from paper_2303_05688_gb300 import build
    build.build()
    m.load()
    return m


def _greedy(weights, shards, init=None):
    """Alg. 3 written out: heaviest first (ties: lower index), each class to the
    least-loaded shard (ties: lower shard)."""
    loads = list(init) if init is not None else [0] * shards
    out = [None] * len(weights)
    for c in sorted(range(len(weights)), key=lambda i: (-weights[i], i)):
        s = min(range(shards), key=lambda k: (loads[k], k))
        out[c] = s
        loads[s] += weights[c]
    return out


def test_shard_assign_is_the_greedy_placement(asci):
    rng = np.random.default_rng(5)
    for _ in range(50):
        n = int(rng.integers(0, 60))
        W = int(rng.integers(1, 9))
        w = rng.integers(0, 1000, n).tolist()
        init = rng.integers(0, 500, W).tolist() if rng.random() < 0.5 else None
        got = asci.shard_assign(w, W, init)
        assert got.tolist() == _greedy(w, W, init)


def test_shard_assign_balance_bound(asci):
    # Graham's bound for the greedy placement: makespan <= (4/3 - 1/(3W)) OPT,
    # and OPT >= max(total / W, largest weight)
    rng = np.random.default_rng(6)
    for W in (2, 3, 8):
        w = rng.integers(1, 10**6, 500)
        sh = asci.shard_assign(w, W)
        loads = np.bincount(sh, weights=w, minlength=W)
        lower = max(w.sum() / W, w.max())
        assert loads.max() <= (4 / 3 - 1 / (3 * W)) * lower * (1 + 1e-12)


def test_shard_assign_rejects_bad_arguments(asci):
    with pytest.raises(asci.AsciError):
        asci.shard_assign([1, 2], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import paper_2303_05688_gb300 as asci
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # shards hold disjoint targets; rank r has 3 + 2 r candidates
        m = 3 + 2 * rank
        keys = torch.tensor([[100 * rank + i, rank] for i in range(m)], dtype=torch.int64)
        scores = torch.tensor([(-1) ** i * (m - i) / (rank + 1.0) for i in range(m)],
                              dtype=torch.float64)
        gk, gs = asci.gather_candidates(keys, scores)
        q.put((rank, gk.numpy().tolist(), gs.numpy().tolist()))
    finally:
        dist.destroy_process_group()


def test_candidate_exchange_gloo_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, k, s = q.get(timeout=120)
        res[r] = (k, s)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank holds the union, in rank order
    want_k, want_s = [], []
    for rank in range(2):
        m = 3 + 2 * rank
        want_k += [[100 * rank + i, rank] for i in range(m)]
        want_s += [(-1) ** i * (m - i) / (rank + 1.0) for i in range(m)]
    for r in range(2):
        assert res[r][0] == want_k and res[r][1] == want_s


def test_union_of_local_topn_is_global_topn():
    # the exchange's premise: shards partition the targets, so the top N of the
    # union of each shard's top N is the top N of all (|S| descending, key
    # ascending), checked by brute force on random partitions
    rng = np.random.default_rng(8)

    def top(keys, s, N):
        o = np.lexsort((keys, -np.abs(s)))
        return keys[o[:N]]

    for _ in range(40):
        n, W, N = int(rng.integers(1, 300)), int(rng.integers(1, 5)), int(rng.integers(1, 50))
        keys = rng.permutation(10**6)[:n]
        s = rng.normal(size=n) * np.where(rng.random(n) < 0.2, 1.0, 1e-3)
        s[rng.random(n) < 0.1] = 0.5  # ties in |S|
        part = rng.integers(0, W, n)
        score_of = dict(zip(keys.tolist(), s.tolist()))
        local = [top(keys[part == r], s[part == r], N) for r in range(W)]
        uk = np.concatenate(local)
        us = np.array([score_of[k] for k in uk.tolist()])
        assert np.array_equal(top(uk, us, N), top(keys, s, N))


# --------------------------------------------------------------------------
# distributed top-N: byte-wise radix select with an all-reduce per byte
# --------------------------------------------------------------------------

def _rank_words(keys, s):
    """(hi, lo) rank words of the library's selection: ~bits(|s|), packed key
    (beta word high, alpha word low), as Python integers."""
    out = []
    for (a, b), v in zip(keys.tolist(), s.tolist()):
        bits = int(np.array([abs(v)], dtype=np.float64).view(np.uint64)[0])
        out.append((~bits & ((1 << 64) - 1), ((b & 0xffffffff) << 32) | (a & 0xffffffff)))
    return out


def _np_hist(keys, s, digit, pre, msk):
    h = np.zeros(256, dtype=np.uint64)
    for hi, lo in _rank_words(keys, s):
        if (hi & msk[0]) == pre[0] and (lo & msk[1]) == pre[1]:
            d = (hi >> (8 * (digit - 8))) & 0xff if digit >= 8 else (lo >> (8 * digit)) & 0xff
            h[d] += 1
    return h


def _np_below(keys, s, thr):
    keep = [i for i, (hi, lo) in enumerate(_rank_words(keys, s))
            if hi < thr[0] or (hi == thr[0] and lo <= thr[1])]
    import torch
    return keys[keep] if keep else keys[:0], s[keep] if keep else s[:0]


def _select_worker(rank, world, port, q, seed, N, empty_rank0=False):
    import torch
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import paper_2303_05688_gb300 as asci
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        keys, s = _select_case(seed, world)
        owner = np.arange(len(keys)) % world
        if empty_rank0:  # rank 0 holds no candidates at all
            owner[owner == 0] = 1 % world
        part = owner == rank
        k = torch.tensor(keys[part], dtype=torch.int64)
        v = torch.tensor(s[part], dtype=torch.float64)
        gk, gs = asci.distributed_topn(
            k, v, N, hist_fn=lambda d, p, m: _np_hist(k, v, d, p, m),
            below_fn=lambda t: _np_below(k, v, t))
        q.put((rank, gk.numpy().tolist(), gs.numpy().tolist()))
    finally:
        dist.destroy_process_group()


def _select_case(seed, world):
    rng = np.random.default_rng(seed)
    n = 60 + 7 * world
    alpha = rng.permutation(1000)[:n]
    beta = rng.integers(0, 4, n)
    keys = np.stack([alpha, beta], 1).astype(np.int64)
    s = rng.normal(size=n)
    s[rng.random(n) < 0.3] = 0.25   # ties in |S| decided by the key
    s[rng.random(n) < 0.1] = -0.25
    return keys, s


@pytest.mark.parametrize("world,N,empty", [(2, 17, False), (3, 40, False), (2, 500, False),
                                           (4, 1, False), (3, 25, True)])
def test_distributed_topn_gloo(world, N, empty):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    seed = 100 + world
    procs = [ctx.Process(target=_select_worker, args=(r, world, port, q, seed, N, empty))
             for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, k, s = q.get(timeout=120)
        res[r] = (k, s)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    keys, s = _select_case(seed, world)
    # brute force: |S| descending, then the packed key (beta high) ascending
    packed = (keys[:, 1] << 32) | keys[:, 0]
    o = np.lexsort((packed, -np.abs(s)))[:N]
    want = sorted(zip(packed[o].tolist(), s[o].tolist()))
    for r in range(world):
        gk = np.array(res[r][0], dtype=np.int64).reshape(-1, 2)
        got = sorted(zip(((gk[:, 1] << 32) | gk[:, 0]).tolist(), res[r][1]))
        assert got == want


def test_select_state_machine_on_the_host(asci):
    """asci_select_begin / asci_select_step (host only): fed the exact
    histograms of one list, the threshold keeps exactly the top N by rank word
    (|S| descending, key ascending); total <= N selects everything; a
    histogram short of the remaining count is rejected."""
    import ctypes as ct
    lib = asci.load()
    rng = np.random.default_rng(9)
    n = 300
    keys = np.stack([rng.permutation(5000)[:n], rng.integers(0, 3, n)], 1).astype(np.int64)
    s = rng.normal(size=n)
    s[rng.random(n) < 0.4] = 0.5          # many ties in |S|
    words = _rank_words(keys, s)
    order = sorted(range(n), key=lambda i: words[i])
    for N in (1, 2, 57, 119, 120, 299):
        st = asci._SelectState()
        assert lib.asci_select_begin(n, N, ct.byref(st)) == 0 and not st.done
        steps = 0
        while not st.done:
            h = np.ascontiguousarray(_np_hist(keys, s, st.digit, list(st.prefix), list(st.mask)))
            assert lib.asci_select_step(ct.byref(st), h.ctypes.data) == 0
            steps += 1
            assert steps <= 16
        thr = (st.threshold[0], st.threshold[1])
        kept = sorted(i for i in range(n) if words[i] <= thr)
        assert kept == sorted(order[:N]), N
    st = asci._SelectState()
    assert lib.asci_select_begin(10, 10, ct.byref(st)) == 0 and st.done
    assert st.threshold[0] == (1 << 64) - 1 and st.threshold[1] == (1 << 64) - 1
    st = asci._SelectState()
    lib.asci_select_begin(100, 50, ct.byref(st))
    short = np.zeros(256, dtype=np.uint64)
    short[3] = 10
    assert lib.asci_select_step(ct.byref(st), short.ctypes.data) == -1
