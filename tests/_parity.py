"""Shared helpers of the parity tests: tolerances and set comparisons.

Score tolerance (FP64 path): |dS| <= 1e-11 |S| when the sum is benign;
otherwise the error budget of the numerator's cancellation and of the
denominator E0 - H_ii is added:
    1e-11 * sum_j |H_ij c_j| / |E0 - H_ii|  +  1e-13 * (|H_ii| + |E0| + 1) * |S| / |E0 - H_ii|.
"""
from __future__ import annotations

import numpy as np


def score_tol(S, abssum, haa, E0, rel=1e-11):
    den = np.abs(E0 - haa)
    return rel * np.abs(S) + rel * abssum / den + 1e-13 * (np.abs(haa) + abs(E0) + 1.0) * np.abs(S) / den


def key_order(a, b):
    return np.lexsort((np.asarray(a), np.asarray(b)))


def to_u64_pairs(t):
    """(m, 2) torch int64 / numpy -> (alpha uint64[m], beta uint64[m])."""
    x = t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
    x = x.view(np.uint64) if x.dtype == np.int64 else x.astype(np.uint64)
    return x[:, 0].copy(), x[:, 1].copy()


def compare_candidates(got_a, got_b, got_s, ref, E0):
    """Bit-exact key sets and scores within tolerance; returns the max err/tol."""
    assert len(got_a) == len(ref.a), (len(got_a), len(ref.a))
    o1 = key_order(got_a, got_b)
    o2 = key_order(ref.a, ref.b)
    assert np.array_equal(got_a[o1], ref.a[o2]), "alpha words differ"
    assert np.array_equal(got_b[o1], ref.b[o2]), "beta words differ"
    tol = score_tol(ref.score[o2], ref.abssum[o2], ref.haa[o2], E0)
    err = np.abs(got_s[o1] - ref.score[o2])
    ratio = np.divide(err, tol, out=np.zeros_like(err), where=tol > 0)
    worst = float(np.max(ratio)) if len(err) else 0.0
    assert np.all(err <= tol), f"score error {worst:.3g} x tolerance"
    return worst


def compare_selection(got_a, got_b, ref, sel_idx, E0):
    """Selected set matches except keys whose oracle |S| is within the tie band of the cutoff."""
    if len(sel_idx) == 0:
        assert len(got_a) == 0
        return
    s = np.abs(ref.score)
    cut = s[sel_idx[-1]]
    tol = score_tol(ref.score, ref.abssum, ref.haa, E0)
    band = np.maximum(1e-12, tol)
    ref_keys = set(zip(ref.a[sel_idx].tolist(), ref.b[sel_idx].tolist()))
    got_keys = set(zip(np.asarray(got_a).tolist(), np.asarray(got_b).tolist()))
    assert len(got_keys) == len(ref_keys)
    pos = {k: i for i, k in enumerate(zip(ref.a.tolist(), ref.b.tolist()))}
    for k in ref_keys ^ got_keys:
        i = pos[k]
        assert abs(s[i] - cut) <= band[i] + 1e-12 * cut, f"selection differs away from the cutoff: {k}"
