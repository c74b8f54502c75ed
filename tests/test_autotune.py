"""The batched-search autotuner's grid search (host logic, CPU): with a
stand-in for the batched search whose speed depends on the stream count and
the batch cap, tune_batched picks the fastest pair, caches it per batch
signature, honours a fixed cap, and tune_streams returns its stream count."""
import time

import numpy as np
import pytest


@pytest.fixture()
def asci(monkeypatch):
    import paper_2303_05688_gb300 as m
    monkeypatch.setattr(m, "_TUNED", {})
    calls = []

    def fake_many(systems, streams=None, max_batch_pairs=0, ctas_per_sm=0, **kw):
        calls.append((len(systems), streams, max_batch_pairs, ctas_per_sm))
        # fastest at 8 streams, the 2^22 cap and 2 CTAs per SM
        cost = (abs(np.log2(streams) - 3) + (0 if max_batch_pairs == 1 << 22 else 1)
                + (0 if ctas_per_sm == 2 else 1))
        time.sleep(0.002 * (1 + 4 * cost))
        return []

    monkeypatch.setattr(m, "search_many", fake_many)
    m._calls = calls
    return m


def _systems(k, norb=10):
    return [dict(h1=np.zeros((norb, norb))) for _ in range(k)]


def test_tune_batched_picks_the_fastest_grid_point(asci):
    t = asci.tune_batched(_systems(80))
    assert t == {"streams": 8, "max_batch_pairs": 1 << 22, "ctas_per_sm": 2}
    # every (CTAs, cap, streams) point of the grid was timed on the 64-system sample
    timed = {(s, b, c) for n, s, b, c in asci._calls if n == 64}
    assert timed == {(s, b, c) for s in (1, 2, 4, 8, 16, 32) for b in (0, 1 << 22, 1 << 20)
                     for c in (0, 2, 1)}
    # cached per signature: no new timing
    n = len(asci._calls)
    assert asci.tune_batched(_systems(90)) == t and len(asci._calls) == n
    # another orbital count is another signature
    asci.tune_batched(_systems(90, norb=12))
    assert len(asci._calls) > n


def test_fixed_cap_and_stream_tuner(asci):
    t = asci.tune_batched(_systems(70), max_batch_pairs=1 << 20)
    assert t["max_batch_pairs"] == 1 << 20 and t["streams"] == 8 and t["ctas_per_sm"] == 2
    assert {b for _, _, b, _ in asci._calls} == {1 << 20}
    n = len(asci._calls)
    t = asci.tune_batched(_systems(70), max_batch_pairs=1 << 22, ctas_per_sm=1)
    assert t["ctas_per_sm"] == 1 and {c for *_, c in asci._calls[n:]} == {1}
    assert asci.tune_streams(_systems(70), max_batch_pairs=1 << 22) == 8
    assert asci.tune_batched([]) == {"streams": 1, "max_batch_pairs": 0, "ctas_per_sm": 0}
