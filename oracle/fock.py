"""Brute-force second-quantised Hamiltonian on tiny Fock spaces (test pin).

Independent of the oracle's Slater-Condon evaluator: it builds
    H = ecore + sum_{pq,s} h_pq a+_ps a_qs
          + 1/2 sum_{pqrs,s,t} (pq|rs) a+_ps a+_rt a_st a_qs
by applying creation and annihilation operators to occupation vectors and
counting anticommutation signs explicitly.

Spin orbitals are ordered alpha 0..n-1 then beta 0..n-1 (index n + p), and
a determinant is |D> = a+_{k1} a+_{k2} ... |0> with k1 < k2 < ... in that order,
so an operator on spin orbital k picks up (-1)^(number of occupied spin
orbitals with index < k).  This is the ordering
prod_{alpha asc} a+ prod_{beta asc} a+ |0> that the oracle reads the paper with.
"""
from __future__ import annotations

import numpy as np

_POP8 = np.array([bin(i).count("1") for i in range(256)], dtype=np.int64)


def _popcount(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.int64)
    c = np.zeros_like(x)
    while np.any(x):
        c += _POP8[x & 255]
        x = x >> 8
    return c


def _annihilate(occ, valid, sign, k):
    has = ((occ >> k) & 1).astype(bool)
    valid = valid & has
    below = occ & ((1 << k) - 1)
    sign = sign * np.where(_popcount(below) % 2 == 1, -1, 1)
    return occ & ~(1 << k), valid, sign


def _create(occ, valid, sign, k):
    has = ((occ >> k) & 1).astype(bool)
    valid = valid & ~has
    below = occ & ((1 << k) - 1)
    sign = sign * np.where(_popcount(below) % 2 == 1, -1, 1)
    return occ | (1 << k), valid, sign


def spin_orbital_occupations(norb: int, A, B) -> np.ndarray:
    """Occupation integers over 2*norb spin orbitals (alpha low, beta high)."""
    A = np.asarray(A, dtype=np.int64)
    B = np.asarray(B, dtype=np.int64)
    return A | (B << norb)


def hamiltonian(norb: int, h1, eri, ecore, A, B, tol: float = 0.0) -> np.ndarray:
    """Dense H[i, j] = <D_i|H|D_j> over the determinant list (A, B).

    The list must be closed under the Hamiltonian's action for the matrix to be
    the full operator (a complete particle/spin sector is); elements leading
    outside the list are dropped.
    """
    h1 = np.asarray(h1, dtype=np.float64)
    eri = np.asarray(eri, dtype=np.float64)
    occ0 = spin_orbital_occupations(norb, A, B)
    nd = len(occ0)
    order = np.argsort(occ0)
    sorted_occ = occ0[order]
    H = np.zeros((nd, nd))
    H[np.arange(nd), np.arange(nd)] += ecore
    cols = np.arange(nd)

    def scatter(occ, valid, sign, coef):
        if not np.any(valid):
            return
        o = occ[valid]
        pos = np.searchsorted(sorted_occ, o)
        pos = np.minimum(pos, nd - 1)
        ok = sorted_occ[pos] == o
        rows = order[pos[ok]]
        np.add.at(H, (rows, cols[valid][ok]), coef * sign[valid][ok])

    ones = np.ones(nd, dtype=bool)
    unit = np.ones(nd, dtype=np.int64)
    # one-body part
    for s in range(2):
        for p in range(norb):
            for q in range(norb):
                v = h1[p, q]
                if v == 0.0 or abs(v) <= tol:
                    continue
                occ, val, sg = _annihilate(occ0, ones, unit, s * norb + q)
                occ, val, sg = _create(occ, val, sg, s * norb + p)
                scatter(occ, val, sg, v)
    # two-body part: 1/2 (pq|rs) a+_ps a+_rt a_st a_qs, rightmost operator first
    for s in range(2):
        for t in range(2):
            for p in range(norb):
                for q in range(norb):
                    for r in range(norb):
                        for u in range(norb):
                            v = eri[p, q, r, u]
                            if v == 0.0 or abs(v) <= tol:
                                continue
                            occ, val, sg = _annihilate(occ0, ones, unit, s * norb + q)
                            occ, val, sg = _annihilate(occ, val, sg, t * norb + u)
                            occ, val, sg = _create(occ, val, sg, t * norb + r)
                            occ, val, sg = _create(occ, val, sg, s * norb + p)
                            scatter(occ, val, sg, 0.5 * v)
    return H


def sector(norb: int, na: int, nb: int):
    """All determinants of one particle/spin sector, key ascending."""
    sa = [w for w in range(1 << norb) if bin(w).count("1") == na]
    sb = [w for w in range(1 << norb) if bin(w).count("1") == nb]
    A = np.array([x for y in sb for x in sa], dtype=np.uint64)
    B = np.array([y for y in sb for x in sa], dtype=np.uint64)
    return A, B
