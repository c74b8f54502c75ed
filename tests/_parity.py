"""Shared helpers of the parity tests: tolerances, set comparisons, reports.

Score tolerance of the FP64 path (the acceptance rule for scores of
Sec. 2.2's ranking, S = num / (E0 - H_ii), Eq. 1):

* benign:    |dS| <= rel |S|                        (rel = 1e-11)
* fallback:  |dS| <= rel * sum_j |H_ij c_j| / |E0 - H_ii|  +  |S| * d_den / |E0 - H_ii|

The fallback covers cancellation in the numerator (its rounding scales with
the sum of the magnitudes of its contributions, not with |num|) and the error
of the denominator.  d_den is derived from how the two sides form E0 - H_ii:

* the GPU sums H_ii exactly in fixed point after rounding each integral term
  (h_pp, J - K of a same-spin pair, J of an opposite-spin pair), ecore and E0
  once to the grid 2^-g (g = stats.diag_grid_bits): at most (T + 2) 2^-(g+1)
  with T the number of integral terms of a determinant;
* both sides round in FP64 elsewhere (the GPU forms J - K before rounding it
  to the grid; the oracle sums with Neumaier compensation, then subtracts from
  E0): at most 8 * 2^-53 * (sum |H_ii terms| + |E0|).

A key passes when either bound holds; keys that need the fallback are
counted.  Every comparison files a report (worst err / tol, fallback count)
that the test session prints at its end.
"""
from __future__ import annotations

import numpy as np

REPORTS: list = []

_U53 = 2.0 ** -53


def diag_terms(na: int, nb: int) -> int:
    """Integral terms of one diagonal element: the one-body terms of every
    electron, the same-spin pairs and the opposite-spin pairs."""
    return na + nb + na * (na - 1) // 2 + nb * (nb - 1) // 2 + na * nb


def grid_err(grid_bits: int, na: int, nb: int) -> float:
    """Bound on the fixed-point rounding carried by the GPU's E0 - H_ii."""
    if grid_bits <= 0:
        return 0.0
    return (diag_terms(na, nb) + 2) * 2.0 ** -(grid_bits + 1)


def counts_of(a, b):
    """Electron counts of the first determinant of a key list."""
    return bin(int(np.asarray(a).flat[0])).count("1"), bin(int(np.asarray(b).flat[0])).count("1")


def score_tol(S, abssum, haa, E0, haa_abs, grid, rel=1e-11, parts=False):
    """Per-key tolerance max(benign, fallback) (module docstring).  With
    parts=True also returns the benign bound alone."""
    S = np.asarray(S, dtype=np.float64)
    den = np.abs(E0 - np.asarray(haa, dtype=np.float64))
    d_den = grid + 8.0 * _U53 * (np.asarray(haa_abs, dtype=np.float64) + abs(E0))
    benign = rel * np.abs(S)
    fallback = rel * np.asarray(abssum) / den + np.abs(S) * d_den / den
    tol = np.maximum(benign, fallback)
    return (tol, benign) if parts else tol


def key_order(a, b):
    return np.lexsort((np.asarray(a), np.asarray(b)))


def to_u64_pairs(t):
    """(m, 2) torch int64 / numpy -> (alpha uint64[m], beta uint64[m])."""
    x = t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
    x = x.view(np.uint64) if x.dtype == np.int64 else x.astype(np.uint64)
    return x[:, 0].copy(), x[:, 1].copy()


def report(label: str, err, tol, benign):
    """File one comparison: worst err / tol and the keys beyond the benign bound."""
    err, tol, benign = (np.asarray(x, dtype=np.float64) for x in (err, tol, benign))
    ratio = np.divide(err, tol, out=np.zeros_like(err), where=tol > 0)
    worst = float(np.max(ratio)) if len(err) else 0.0
    nfb = int(np.sum(err > benign))
    REPORTS.append((label, len(err), worst, nfb))
    return worst, nfb


def compare_candidates(got_a, got_b, got_s, ref, E0, grid_bits, rel=1e-11, label="candidates"):
    """Bit-exact key sets and scores within tolerance; returns (worst err/tol,
    keys that needed the fallback bound)."""
    assert len(got_a) == len(ref.a), (len(got_a), len(ref.a))
    o1 = key_order(got_a, got_b)
    o2 = key_order(ref.a, ref.b)
    assert np.array_equal(got_a[o1], ref.a[o2]), "alpha words differ"
    assert np.array_equal(got_b[o1], ref.b[o2]), "beta words differ"
    if len(ref.a) == 0:
        return 0.0, 0
    na, nb = counts_of(ref.a, ref.b)
    tol, benign = score_tol(ref.score[o2], ref.abssum[o2], ref.haa[o2], E0, ref.haa_abs[o2],
                            grid_err(grid_bits, na, nb), rel=rel, parts=True)
    err = np.abs(got_s[o1] - ref.score[o2])
    worst, nfb = report(label, err, tol, benign)
    assert np.all(err <= tol), f"score error {worst:.3g} x tolerance"
    return worst, nfb


def compare_selection(got_a, got_b, ref, sel_idx, E0, grid_bits):
    """Selected set matches except keys whose oracle |S| is within the tie band
    of the cutoff (the wider of 1e-12 and the score tolerance)."""
    if len(sel_idx) == 0:
        assert len(got_a) == 0
        return
    s = np.abs(ref.score)
    cut = s[sel_idx[-1]]
    na, nb = counts_of(ref.a, ref.b)
    tol = score_tol(ref.score, ref.abssum, ref.haa, E0, ref.haa_abs, grid_err(grid_bits, na, nb))
    band = np.maximum(1e-12, tol)
    ref_keys = set(zip(ref.a[sel_idx].tolist(), ref.b[sel_idx].tolist()))
    got_keys = set(zip(np.asarray(got_a).tolist(), np.asarray(got_b).tolist()))
    assert len(got_keys) == len(ref_keys)
    pos = {k: i for i, k in enumerate(zip(ref.a.tolist(), ref.b.tolist()))}
    for k in ref_keys ^ got_keys:
        i = pos[k]
        assert abs(s[i] - cut) <= band[i] + 1e-12 * cut, f"selection differs away from the cutoff: {k}"
