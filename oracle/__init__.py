"""Plain FP64 CPU oracle for the ASCI determinant search (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  It shares no code with the GPU path; the C source
``asci_oracle.c`` is compiled with gcc into ``liboracle.so`` beside it.

Functions follow arXiv:2303.05688: Eq. 1 (the ASCI score), Algorithm 2 (the
search: core selection, single/double enumeration, sort-and-accumulate), the
duplicate-aware top-N selection of Sec. 2.2, and Algorithm 1 (the ASCI loop:
search, select, diagonalise in the selected space, repeat) with the
diagonalisation written as its definition, the lowest eigenpair of the dense
Hamiltonian restricted to the space (Sec. 2.3 computes it by Davidson,
Algorithm 5), and the ASCI-PT2 energy that ends Algorithm 1.  ``fock`` holds an independent
brute-force second-quantised Hamiltonian that pins the oracle's Slater-Condon
evaluator.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asci_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    u64p = ct.POINTER(ct.c_uint64)
    f64p = ct.POINTER(ct.c_double)
    szp = ct.POINTER(ct.c_size_t)
    lib.oracle_search.restype = ct.c_void_p
    lib.oracle_search.argtypes = [ct.c_int, f64p, f64p, ct.c_double, u64p, u64p, f64p,
                                  ct.c_size_t, ct.c_double, ct.c_size_t, ct.c_double,
                                  ct.c_uint64, ct.c_uint64]
    lib.oracle_search_parallel.restype = ct.c_void_p
    lib.oracle_search_parallel.argtypes = [ct.c_int, f64p, f64p, ct.c_double, u64p, u64p, f64p,
                                           ct.c_size_t, ct.c_double, ct.c_size_t, ct.c_double,
                                           ct.c_int]
    lib.oracle_free.argtypes = [ct.c_void_p]
    lib.oracle_result_count.restype = ct.c_size_t
    lib.oracle_result_count.argtypes = [ct.c_void_p]
    lib.oracle_result_stats.argtypes = [ct.c_void_p, szp]
    lib.oracle_result_copy.argtypes = [ct.c_void_p, u64p, u64p, f64p, f64p, f64p, f64p, f64p]
    lib.oracle_topn.restype = ct.c_size_t
    lib.oracle_topn.argtypes = [u64p, u64p, f64p, ct.c_size_t, ct.c_size_t, szp]
    lib.oracle_core_select.restype = ct.c_size_t
    lib.oracle_core_select.argtypes = [u64p, u64p, f64p, ct.c_size_t, ct.c_size_t, szp]
    lib.oracle_hij.restype = ct.c_double
    lib.oracle_hij.argtypes = [ct.c_int, f64p, f64p, ct.c_double, ct.c_uint64, ct.c_uint64,
                               ct.c_uint64, ct.c_uint64]
    lib.oracle_diag.restype = ct.c_double
    lib.oracle_diag.argtypes = [ct.c_int, f64p, f64p, ct.c_double, ct.c_uint64, ct.c_uint64]
    lib.oracle_diag_abs.restype = ct.c_double
    lib.oracle_diag_abs.argtypes = [ct.c_int, f64p, f64p, ct.c_double, ct.c_uint64, ct.c_uint64]
    lib.oracle_dense_h.argtypes = [ct.c_int, f64p, f64p, ct.c_double, u64p, u64p,
                                   ct.c_size_t, f64p]
    lib.oracle_h_rows.argtypes = [ct.c_int, f64p, f64p, ct.c_double, u64p, u64p,
                                  ct.c_size_t, szp, ct.c_size_t, f64p]
    lib.oracle_pairs.restype = ct.c_size_t
    lib.oracle_pairs.argtypes = [ct.c_int, f64p, f64p, ct.c_double, u64p, u64p, f64p,
                                 ct.c_size_t, ct.c_size_t, u64p, u64p, f64p]
    lib.oracle_numerator.restype = ct.c_double
    lib.oracle_numerator.argtypes = [ct.c_int, f64p, f64p, ct.c_double, ct.c_uint64,
                                     ct.c_uint64, u64p, u64p, f64p, ct.c_size_t, f64p]
    lib.oracle_bucket_of.restype = ct.c_uint64
    lib.oracle_bucket_of.argtypes = [ct.c_uint64, ct.c_uint64, ct.c_uint64]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ct.CDLL(_LIB))
    return _lib


class substitute:
    """Context manager for the mutation tests: every oracle function of this
    module runs on the library at `path` (a copy of asci_oracle.c with a
    planted mistake, compiled by the test) until the block ends."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        _lib = _bind(ct.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _u64(x):
    return np.ascontiguousarray(x, dtype=np.uint64)


def _p(a, t):
    return a.ctypes.data_as(ct.POINTER(t))


class Ints:
    """Integrals in the oracle's layout: h1[n, n], eri[n, n, n, n] = (pq|rs)."""

    def __init__(self, h1, eri, ecore=0.0):
        self.h1 = _f64(h1)
        self.eri = _f64(eri)
        self.n = int(self.h1.shape[0])
        self.ecore = float(ecore)

    def args(self):
        return (self.n, _p(self.h1, ct.c_double), _p(self.eri, ct.c_double), self.ecore)


def hij(ints: Ints, bra, ket) -> float:
    """<bra|H|ket> by the Slater-Condon rules (determinants as (alpha, beta))."""
    return _load().oracle_hij(*ints.args(), int(bra[0]), int(bra[1]), int(ket[0]), int(ket[1]))


def diag(ints: Ints, det) -> float:
    """<D|H|D>."""
    return _load().oracle_diag(*ints.args(), int(det[0]), int(det[1]))


def diag_abs(ints: Ints, det) -> float:
    """Sum of the magnitudes of the terms of <D|H|D> (ecore, h_pp, the
    same-spin (J - K) / 2 of ordered pairs, the opposite-spin J)."""
    return _load().oracle_diag_abs(*ints.args(), int(det[0]), int(det[1]))


def dense_h(ints: Ints, A, B) -> np.ndarray:
    """H[i, j] = <D_i|H|D_j> for the determinant list (A, B)."""
    A, B = _u64(A), _u64(B)
    out = np.empty((len(A), len(A)))
    _load().oracle_dense_h(*ints.args(), _p(A, ct.c_uint64), _p(B, ct.c_uint64), len(A),
                           _p(out, ct.c_double))
    return out


def core_select(A, B, c, C) -> np.ndarray:
    """Indices of the C largest |c| (ties: key ascending), in that order."""
    A, B, c = _u64(A), _u64(B), _f64(c)
    out = np.empty(max(len(A), 1), dtype=np.uintp)
    m = _load().oracle_core_select(_p(A, ct.c_uint64), _p(B, ct.c_uint64), _p(c, ct.c_double),
                                   len(A), int(C), _p(out, ct.c_size_t))
    return out[:m].astype(np.int64)


def pairs(ints: Ints, CA, CB, CC):
    """Pre-sort (target, H_ij c_j) pairs of Alg. 2 for the given core dets."""
    CA, CB, CC = _u64(CA), _u64(CB), _f64(CC)
    lib = _load()
    args = ints.args() + (_p(CA, ct.c_uint64), _p(CB, ct.c_uint64), _p(CC, ct.c_double), len(CA))
    n = lib.oracle_pairs(*args, 0, None, None, None)
    a = np.empty(n, dtype=np.uint64)
    b = np.empty(n, dtype=np.uint64)
    v = np.empty(n)
    lib.oracle_pairs(*args, n, _p(a, ct.c_uint64), _p(b, ct.c_uint64), _p(v, ct.c_double))
    return a, b, v


def numerator(ints: Ints, target, CA, CB, CC):
    """(sum_j <target|H|D_j> c_j, sum_j |...|) over a core list, by brute force."""
    CA, CB, CC = _u64(CA), _u64(CB), _f64(CC)
    s = ct.c_double(0.0)
    v = _load().oracle_numerator(*ints.args(), int(target[0]), int(target[1]),
                                 _p(CA, ct.c_uint64), _p(CB, ct.c_uint64), _p(CC, ct.c_double),
                                 len(CA), ct.byref(s))
    return v, s.value


def bucket_of(a: int, b: int, nbuckets: int) -> int:
    return int(_load().oracle_bucket_of(int(a), int(b), int(nbuckets)))


class SearchResult:
    """Every unique candidate outside psi (Alg. 2 before the final selection)."""

    def __init__(self, a, b, num, abssum, haa, haa_abs, score, stats):
        self.a, self.b = a, b
        self.num, self.abssum, self.haa, self.score = num, abssum, haa, score
        self.haa_abs = haa_abs
        (self.generated, self.surviving, self.unique, self.excluded, self.ncore) = stats

    @property
    def keys(self) -> np.ndarray:
        return np.stack([self.a, self.b], axis=1)

    def topn(self, N: int) -> np.ndarray:
        """Indices of the selected candidates (|S| desc, key asc)."""
        return topn(self.a, self.b, self.score, N)


def search(ints: Ints, A, B, c, E0: float, C: int, eps: float = 0.0,
           nbuckets: int = 1, bucket: int = 0, threads: int = 1) -> SearchResult:
    """Algorithm 2 + Eq. 1: all unique candidates with numerator, H_ii and score.
    threads > 1 runs the all-core form (same result bit for bit; no buckets)."""
    A, B, c = _u64(A), _u64(B), _f64(c)
    lib = _load()
    if threads > 1:
        if nbuckets > 1:
            raise ValueError("the all-core form takes no bucket filter")
        h = lib.oracle_search_parallel(*ints.args(), _p(A, ct.c_uint64), _p(B, ct.c_uint64),
                                       _p(c, ct.c_double), len(A), float(E0), int(C),
                                       float(eps), int(threads))
    else:
        h = lib.oracle_search(*ints.args(), _p(A, ct.c_uint64), _p(B, ct.c_uint64),
                              _p(c, ct.c_double), len(A), float(E0), int(C), float(eps),
                              int(nbuckets), int(bucket))
    if not h:
        raise MemoryError("oracle_search failed")
    try:
        k = lib.oracle_result_count(h)
        st = np.zeros(5, dtype=np.uintp)
        lib.oracle_result_stats(h, _p(st, ct.c_size_t))
        a = np.empty(k, dtype=np.uint64)
        b = np.empty(k, dtype=np.uint64)
        num, abss, haa, habs, sc = (np.empty(k) for _ in range(5))
        lib.oracle_result_copy(h, _p(a, ct.c_uint64), _p(b, ct.c_uint64), _p(num, ct.c_double),
                               _p(abss, ct.c_double), _p(haa, ct.c_double),
                               _p(habs, ct.c_double), _p(sc, ct.c_double))
    finally:
        lib.oracle_free(h)
    return SearchResult(a, b, num, abss, haa, habs, sc, tuple(int(x) for x in st))


def topn(a, b, score, N: int) -> np.ndarray:
    """Top-N indices by |score| descending, ties by key ascending."""
    a, b, score = _u64(a), _u64(b), _f64(score)
    out = np.empty(max(len(a), 1), dtype=np.uintp)
    m = _load().oracle_topn(_p(a, ct.c_uint64), _p(b, ct.c_uint64), _p(score, ct.c_double),
                            len(a), int(N), _p(out, ct.c_size_t))
    return out[:m].astype(np.int64)


def variational_energy(ints: Ints, A, B, c) -> float:
    """<psi|H|psi> / <psi|psi> on the given determinants (dense, small lists)."""
    H = dense_h(ints, A, B)
    c = _f64(c)
    return float(c @ H @ c / (c @ c))


def ground_state(ints: Ints, A, B):
    """Lowest eigenpair of H restricted to the determinant list (dense)."""
    H = dense_h(ints, A, B)
    w, V = np.linalg.eigh(H)
    v = V[:, 0].copy()
    if v[np.argmax(np.abs(v))] < 0:
        v = -v
    return float(w[0]), v


def h_rows(ints: Ints, A, B, rows) -> np.ndarray:
    """Dense rows H[r, :] = <D_rows[r]|H|D_j> over the determinant list (A, B)."""
    A, B = _u64(A), _u64(B)
    rows = np.ascontiguousarray(rows, dtype=np.uintp)
    out = np.empty((len(rows), len(A)))
    _load().oracle_h_rows(*ints.args(), _p(A, ct.c_uint64), _p(B, ct.c_uint64), len(A),
                          _p(rows, ct.c_size_t), len(rows), _p(out, ct.c_double))
    return out


def key_order(A, B) -> np.ndarray:
    """Indices that sort determinants by key (beta word high, alpha word low)."""
    return np.lexsort((_u64(A), _u64(B)))


def asci_merge(ints: Ints, A, B, c, E0: float, ncdets: int, ntdets: int, eps: float = 0.0):
    """Steps 2-3 of Algorithm 1 before the diagonalisation: the search
    (Algorithm 2, ncdets core), then the ntdets determinants of largest
    magnitude among the current ones (valued by c_i) and the candidates
    (valued by their score S_i, Eq. 1), ties by key ascending.  Returns
    (A', B', values, kept_min, dropped_max, changed): the kept determinants in
    key order with their values, the smallest kept and the largest dropped
    magnitude (0 when nothing is dropped), and whether the set differs from
    (A, B)."""
    A, B, c = _u64(A), _u64(B), _f64(c)
    res = search(ints, A, B, c, E0, ncdets, eps)
    ua = np.concatenate([A, res.a])
    ub = np.concatenate([B, res.b])
    val = np.concatenate([c, res.score])
    idx = topn(ua, ub, val, ntdets)
    mag = np.abs(val)
    keep = np.zeros(len(val), dtype=bool)
    keep[idx] = True
    kept_min = float(mag[keep].min()) if keep.any() else 0.0
    dropped_max = float(mag[~keep].max()) if (~keep).any() else 0.0
    na, nb, v = ua[idx], ub[idx], val[idx]
    o = key_order(na, nb)
    changed = len(idx) != len(A) or bool(np.any(idx >= len(A)))
    return na[o], nb[o], v[o], kept_min, dropped_max, changed


def asci_step(ints: Ints, A, B, c, E0: float, ncdets: int, ntdets: int, eps: float = 0.0):
    """One pass of Algorithm 1 from the wavefunction (A, B, c) with energy E0:
    asci_merge, then the ground state of the new space, the lowest eigenpair
    of H restricted to it.  Returns (A', B', c', E', changed) with the
    determinants in key order and c' normalised, largest |c'| positive."""
    na, nb, _, _, _, changed = asci_merge(ints, A, B, c, E0, ncdets, ntdets, eps)
    E, v = ground_state(ints, na, nb)
    return na, nb, v, E, changed


def asci_loop(ints: Ints, A, B, c, ncdets: int, ntdets: int, max_iter: int, etol: float = 0.0,
              eps: float = 0.0):
    """Algorithm 1: from the start (A, B, c) (energy <psi|H|psi>/<psi|psi>),
    repeat the step until the energy changes by at most etol, the determinant
    set stops changing, or max_iter steps have run.  Returns (A, B, c, E,
    history) with history a list of (size, energy) per step."""
    E = variational_energy(ints, A, B, c)
    hist = []
    for _ in range(max_iter):
        A2, B2, c2, E2, changed = asci_step(ints, A, B, c, E, ncdets, ntdets, eps)
        hist.append((len(A2), E2))
        done = abs(E2 - E) <= etol or not changed
        A, B, c, E = A2, B2, c2, E2
        if done:
            break
    return A, B, c, E, hist


def pt2(ints: Ints, A, B, c, E0: float, C: int, eps: float = 0.0) -> float:
    """ASCI-PT2 (the last step of Algorithm 1): the sum over every unique
    candidate i outside psi of num_i^2 / (E0 - H_ii), num_i = sum over the C
    core determinants of H_ij c_j (the search's numerator, Eq. 1), summed
    exactly rounded (math.fsum)."""
    import math
    res = search(ints, A, B, c, E0, C, eps)
    return math.fsum((res.num * res.num / (E0 - res.haa)).tolist())
