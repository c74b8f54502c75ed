"""The continuous-batching server's admission and concurrency (CPU, with a
stand-in search) and its results against standalone searches (GPU)."""
import threading
import time

import numpy as np
import pytest

import workloads as W


def _fake_search_factory(log, lock, dt=0.02):
    def fake(dets, coeffs, E0, h1, eri, ecore, C, N, **kw):
        with lock:
            log.append(("start", C, time.perf_counter()))
        time.sleep(dt)
        with lock:
            log.append(("end", C, time.perf_counter()))
        return dets[:1], coeffs[:1], {"C": C, "batch": kw.get("max_batch_pairs")}
    return fake


def _server_cpu(**kw):
    torch = pytest.importorskip("torch")
    from paper_2303_05688_gb300.serve import Server
    return torch, Server(**kw)


def test_admission_respects_budget_and_slots():
    from paper_2303_05688_gb300.serve import footprint
    log, lock = [], threading.Lock()
    fp = footprint(8, 10, 5, 100, 1 << 20)
    torch, srv = _server_cpu(slots=4, budget=int(2.5 * fp),
                             search_fn=_fake_search_factory(log, lock))
    with srv:
        srv.register("s", np.zeros((10, 2), np.int64), np.ones(10), -1.0, np.zeros((8, 8)),
                     np.zeros(8 ** 4), 0.0)
        futs = [srv.submit("s", 5, 100, batch_pairs=1 << 20) for _ in range(10)]
        res = [f.result(timeout=30) for f in futs]
    assert len(res) == 10
    assert srv.peak_running == 2          # the budget admits two at a time, not four
    assert srv.peak_bytes <= srv.budget
    # never more than two searches overlap in the log
    live, worst = 0, 0
    for ev in sorted(log, key=lambda e: e[2]):
        live += 1 if ev[0] == "start" else -1
        worst = max(worst, live)
    assert worst <= 2


def test_requests_start_in_arrival_order():
    log, lock = [], threading.Lock()
    torch, srv = _server_cpu(slots=1, budget=1 << 40, search_fn=_fake_search_factory(log, lock, 0.005))
    with srv:
        srv.register("s", np.zeros((10, 2), np.int64), np.ones(10), -1.0, np.zeros((8, 8)),
                     np.zeros(8 ** 4), 0.0)
        futs = [srv.submit("s", c, 100) for c in range(1, 9)]
        for f in futs:
            f.result(timeout=30)
    starts = [c for kind, c, _ in sorted(log, key=lambda e: e[2]) if kind == "start"]
    assert starts == list(range(1, 9))


def test_oversized_request_rejected():
    torch, srv = _server_cpu(slots=2, budget=1 << 20, search_fn=lambda *a, **k: None)
    with srv:
        srv.register("s", np.zeros((10, 2), np.int64), np.ones(10), -1.0, np.zeros((8, 8)),
                     np.zeros(8 ** 4), 0.0)
        with pytest.raises(ValueError):
            srv.submit("s", 5, 100)


def test_failed_search_reaches_its_future_and_frees_its_slot():
    """A search that raises reports through its own future; its memory and slot
    are released, so the requests behind it still run."""
    calls = []

    def flaky(dets, coeffs, E0, h1, eri, ecore, C, N, **kw):
        calls.append(C)
        if C == 3:
            raise RuntimeError("planted failure")
        return dets[:1], coeffs[:1], {"C": C}

    torch, srv = _server_cpu(slots=1, budget=1 << 40, search_fn=flaky)
    with srv:
        srv.register("s", np.zeros((10, 2), np.int64), np.ones(10), -1.0, np.zeros((8, 8)),
                     np.zeros(8 ** 4), 0.0)
        futs = [srv.submit("s", c, 100) for c in range(1, 6)]
        with pytest.raises(RuntimeError, match="planted failure"):
            futs[2].result(timeout=30)
        for i in (0, 1, 3, 4):
            assert futs[i].result(timeout=30)[2]["C"] == i + 1
    assert calls == [1, 2, 3, 4, 5]
    assert srv._in_use == 0 and srv._running == 0


def test_queued_request_can_be_cancelled():
    """A request still queued is withdrawn by its future's cancel(): it never
    runs, takes no slot, and the requests behind it run; a running request
    cannot be cancelled.  A withdrawn request at the head of the queue that
    did not fit the budget no longer holds up the smaller one behind it."""
    from paper_2303_05688_gb300.serve import footprint
    gate = threading.Event()
    calls = []

    def gated(dets, coeffs, E0, h1, eri, ecore, C, N, **kw):
        calls.append(C)
        if C == 1:
            gate.wait(30)
        return dets[:1], coeffs[:1], {"C": C}

    torch, srv = _server_cpu(slots=1, budget=1 << 40, search_fn=gated)
    with srv:
        srv.register("s", np.zeros((10, 2), np.int64), np.ones(10), -1.0, np.zeros((8, 8)),
                     np.zeros(8 ** 4), 0.0)
        futs = [srv.submit("s", c, 100) for c in (1, 2, 3)]
        t0 = time.perf_counter()
        while not futs[0].running() and time.perf_counter() - t0 < 10:
            time.sleep(0.005)
        assert futs[0].running() and not futs[0].cancel()
        assert futs[1].cancel() and futs[1].cancelled()
        gate.set()
        assert futs[0].result(timeout=30)[2]["C"] == 1
        assert futs[2].result(timeout=30)[2]["C"] == 3
    assert calls == [1, 3] and srv.cancelled == 1
    assert srv._in_use == 0 and srv._running == 0
    # budget: a running request holds most of it, a big request waits at the
    # head of the queue, a small one behind it; cancelling the big one lets
    # the small one start while the first still runs
    fp_small = footprint(8, 10, 1, 100, 1 << 20)
    fp_big = footprint(8, 10, 1, 100, 1 << 26)
    gate2, started = threading.Event(), []

    def gated2(dets, coeffs, E0, h1, eri, ecore, C, N, **kw):
        started.append(C)
        if C == 1:
            gate2.wait(30)
        return dets[:1], coeffs[:1], {"C": C}

    torch, srv = _server_cpu(slots=2, budget=fp_small + fp_big - 1, search_fn=gated2)
    with srv:
        srv.register("s", np.zeros((10, 2), np.int64), np.ones(10), -1.0, np.zeros((8, 8)),
                     np.zeros(8 ** 4), 0.0)
        f1 = srv.submit("s", 1, 100, batch_pairs=1 << 20)
        t0 = time.perf_counter()
        while not f1.running() and time.perf_counter() - t0 < 10:
            time.sleep(0.005)
        fbig = srv.submit("s", 2, 100, batch_pairs=1 << 26)
        fsmall = srv.submit("s", 3, 100, batch_pairs=1 << 20)
        time.sleep(0.05)
        assert started == [1]  # the big one does not fit beside the first; the small one waits
        assert fbig.cancel()
        assert fsmall.result(timeout=10)[2]["C"] == 3  # while the first still runs
        assert not f1.done()
        gate2.set()
        f1.result(timeout=30)
    assert started == [1, 3] and srv.cancelled == 1


def test_submit_after_close_is_refused():
    torch, srv = _server_cpu(slots=1, budget=1 << 40, search_fn=lambda *a, **k: None)
    srv.register("s", np.zeros((10, 2), np.int64), np.ones(10), -1.0, np.zeros((8, 8)),
                 np.zeros(8 ** 4), 0.0)
    srv.close()
    with pytest.raises(RuntimeError, match="closed"):
        srv.submit("s", 1, 10)


@pytest.mark.gpu
def test_served_results_equal_standalone(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_05688_gb300 as asci
    from paper_2303_05688_gb300.serve import Server
    from tests._parity import key_order, to_u64_pairs
    asci.load()
    systems = W.batched_systems(6, seed=91, scale=0.05)
    with Server(slots=4) as srv:
        for sy in systems:
            ints = oracle_mod.Ints(sy["h1"], sy["eri"], sy["ecore"])
            E0 = oracle_mod.diag(ints, (int(sy["alpha"][0]), int(sy["beta"][0]))) - 1.0
            sy["E0"] = E0
            srv.register(sy["name"], np.stack([sy["alpha"], sy["beta"]], 1).astype(np.int64),
                         sy["c"], E0, sy["h1"], sy["eri"], sy["ecore"])
        reqs = [(sy, sy["C"], sy["N"]) for sy in systems] * 3
        futs = [srv.submit(sy["name"], C, N) for sy, C, N in reqs]
        got = [f.result(timeout=300) for f in futs]
    for (sy, C, N), (k, s_, st, lat) in zip(reqs, got):
        d = torch.tensor(np.stack([sy["alpha"], sy["beta"]], 1).astype(np.int64), device="cuda")
        k1, s1, _ = asci.search(d, torch.tensor(sy["c"], device="cuda"), sy["E0"],
                                torch.tensor(sy["h1"], device="cuda"),
                                torch.tensor(sy["eri"], device="cuda"), sy["ecore"], C, N)
        a, b = to_u64_pairs(k)
        a1, b1 = to_u64_pairs(k1)
        o, o1 = key_order(a, b), key_order(a1, b1)
        assert np.array_equal(a[o], a1[o1]) and np.array_equal(b[o], b1[o1])
        assert np.array_equal(s_.cpu().numpy()[o], s1.cpu().numpy()[o1])
        assert lat > 0
