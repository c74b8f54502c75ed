"""Seeded synthetic inputs for the ASCI determinant search.

This module is shared by the CPU oracle's tests and by the GPU path's tests and
benchmark.  It holds none of the method's arithmetic: no Hamiltonian matrix
element, diagonal energy, score or selection is computed here.  It only draws
integrals and determinant lists from seeded generators (numpy PCG64).

Determinants are pairs of occupation bitstrings (alpha word, beta word); bit p of
a word is spatial orbital p.  Every generator is deterministic for a given seed.

Recipes (the paper's Cr2 integrals, from its Sec. 3, are not available, so these
stand in with the same shapes):

* Random molecular-like integrals (``random_molecular``): orbital energies
  h_pp drawn from U(-2, 2) and sorted ascending; off-diagonal h_pq ~ N(0, 0.05^2),
  symmetric; two-electron (pq|rs) = 0.5 exp(-0.3(|p-q| + |r-s|)) (1 + N(0, 0.1^2)),
  one noise draw per canonical index (p>=q, r>=s, pq>=rs) copied to all eight
  permutations; core energy 0.
* 1D Hubbard ring (``hubbard_ring``): h_{p,p+1 mod n} = -t, (pp|pp) = U.
* Wavefunction (``random_walk_dets``): starts from the aufbau determinant and
  grows by a rank-biased random walk over single and double excitations until it
  holds the requested number of distinct determinants; ``rank_decay_coeffs``
  gives c_r = s_r / (r + 1) with seeded signs (s_0 = +1), normalised.
"""
from __future__ import annotations

import dataclasses
import json
import os
from math import comb

import numpy as np

__all__ = [
    "aufbau",
    "hubbard_ring",
    "random_molecular",
    "random_walk_dets",
    "rank_decay_coeffs",
    "all_dets",
    "n_excitations",
    "Workload",
    "WORKLOADS",
    "stored_e0",
]


def aufbau(nocc: int) -> int:
    """Bitstring with the lowest ``nocc`` orbitals occupied."""
    return (1 << nocc) - 1


def n_excitations(norb: int, na: int, nb: int) -> int:
    """Number of single plus double excitations of one determinant.

    Counts alpha and beta singles, same-spin doubles and opposite-spin doubles;
    it is a counting identity used to size buffers and to state workloads.
    """
    va, vb = norb - na, norb - nb
    return (na * va + nb * vb + comb(na, 2) * comb(va, 2) + comb(nb, 2) * comb(vb, 2)
            + na * va * nb * vb)


def hubbard_ring(norb: int, t: float, U: float):
    """1D periodic Hubbard ring in the site basis.

    Returns (h1[norb, norb], eri[norb, norb, norb, norb], ecore) with chemists'
    two-electron layout eri[p, q, r, s] = (pq|rs).
    """
    h1 = np.zeros((norb, norb))
    for p in range(norb):
        q = (p + 1) % norb
        if q != p:
            h1[p, q] = -t
            h1[q, p] = -t
    eri = np.zeros((norb,) * 4)
    for p in range(norb):
        eri[p, p, p, p] = U
    return h1, eri, 0.0


def random_molecular(norb: int, seed: int):
    """Random molecular-like integrals with 8-fold permutational symmetry.

    Returns (h1[norb, norb], eri[norb]*4, ecore) (chemists' notation).
    """
    rng = np.random.default_rng(seed)
    n = norb
    h1 = np.zeros((n, n))
    h1[np.arange(n), np.arange(n)] = np.sort(rng.uniform(-2.0, 2.0, n))
    iu = np.triu_indices(n, 1)
    off = rng.normal(0.0, 0.05, len(iu[0]))
    h1[iu] = off
    h1[(iu[1], iu[0])] = off

    # canonical compound indices pq (p >= q), ordered by pq = p(p+1)/2 + q
    P, Q = np.tril_indices(n)
    npair = len(P)
    I, J = np.tril_indices(npair)          # compound pq >= rs
    noise = rng.normal(0.0, 0.1, len(I))
    p, q, r, s = P[I], Q[I], P[J], Q[J]
    val = 0.5 * np.exp(-0.3 * (np.abs(p - q) + np.abs(r - s))) * (1.0 + noise)
    eri = np.zeros((n,) * 4)
    for (a, b, c, d) in ((p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                         (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)):
        eri[a, b, c, d] = val
    return h1, eri, 0.0


def _words_to_occ(words: np.ndarray, norb: int) -> np.ndarray:
    return ((words[:, None] >> np.arange(norb, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(bool)


def _pick(mask: np.ndarray, k: int, rng) -> np.ndarray:
    """k distinct random True columns per row (rows must hold >= k True)."""
    keys = rng.random(mask.shape)
    keys[~mask] = 2.0
    return np.argsort(keys, axis=1, kind="stable")[:, :k]


def _flip(words: np.ndarray, cols: np.ndarray, sel: np.ndarray) -> None:
    for c in range(cols.shape[1]):
        words[sel] ^= (np.uint64(1) << cols[sel, c].astype(np.uint64))


def random_walk_dets(norb: int, na: int, nb: int, ndets: int, seed: int):
    """Distinct determinants grown by a rank-biased random walk from aufbau.

    Each round draws proposals: a parent of rank floor(len * u^3) (u ~ U(0,1)),
    then an excitation kind (alpha single 1/8, beta single 1/8, alpha-alpha
    double 3/16, beta-beta double 3/16, alpha-beta double 3/8) whose holes and
    particles are uniform among the parent's occupied / empty orbitals.  New
    determinants are appended in proposal order.  Returns (alpha, beta) as
    uint64 arrays in rank order; rank 0 is the aufbau determinant.
    """
    if norb > 32:
        raise ValueError("random_walk_dets packs keys in 64 bits: norb <= 32")
    rng = np.random.default_rng(seed)
    A = np.zeros(ndets, dtype=np.uint64)
    B = np.zeros(ndets, dtype=np.uint64)
    A[0], B[0] = aufbau(na), aufbau(nb)
    cur = 1
    seen = np.array([(int(B[0]) << 32) | int(A[0])], dtype=np.uint64)
    full = np.uint64((1 << norb) - 1)
    while cur < ndets:
        m = int(min(max(cur, 64), 65536))
        u = rng.random(m)
        par = np.minimum((cur * u ** 3).astype(np.int64), cur - 1)
        kind_u = rng.random(m)
        a = A[par].copy()
        b = B[par].copy()
        occ_a = _words_to_occ(a, norb)
        occ_b = _words_to_occ(b, norb)
        h_a = _pick(occ_a, 2, rng)
        p_a = _pick(~occ_a, 2, rng)
        h_b = _pick(occ_b, 2, rng)
        p_b = _pick(~occ_b, 2, rng)
        na_, va_ = na, norb - na
        nb_, vb_ = nb, norb - nb
        s_a = kind_u < 0.125
        s_b = (kind_u >= 0.125) & (kind_u < 0.25)
        d_aa = (kind_u >= 0.25) & (kind_u < 0.4375)
        d_bb = (kind_u >= 0.4375) & (kind_u < 0.625)
        d_ab = kind_u >= 0.625
        ok = np.ones(m, dtype=bool)
        ok &= ~(s_a & ((na_ < 1) | (va_ < 1)))
        ok &= ~(s_b & ((nb_ < 1) | (vb_ < 1)))
        ok &= ~(d_aa & ((na_ < 2) | (va_ < 2)))
        ok &= ~(d_bb & ((nb_ < 2) | (vb_ < 2)))
        ok &= ~(d_ab & ((na_ < 1) | (va_ < 1) | (nb_ < 1) | (vb_ < 1)))
        _flip(a, np.stack([h_a[:, 0], p_a[:, 0]], 1), s_a | d_ab | d_aa)
        _flip(a, np.stack([h_a[:, 1], p_a[:, 1]], 1), d_aa)
        _flip(b, np.stack([h_b[:, 0], p_b[:, 0]], 1), s_b | d_ab | d_bb)
        _flip(b, np.stack([h_b[:, 1], p_b[:, 1]], 1), d_bb)
        a &= full
        b &= full
        key = (b << np.uint64(32)) | a
        key = key[ok]
        # first occurrence of each new key, in proposal order
        _, first = np.unique(key, return_index=True)
        first.sort()
        key = key[first]
        pos = np.searchsorted(seen, key)
        pos = np.minimum(pos, len(seen) - 1)
        new = seen[pos] != key
        key = key[new][: ndets - cur]
        k = len(key)
        A[cur:cur + k] = key & np.uint64(0xFFFFFFFF)
        B[cur:cur + k] = key >> np.uint64(32)
        cur += k
        seen = np.sort(np.concatenate([seen, key]))
    return A, B


def rank_decay_coeffs(ndets: int, seed: int) -> np.ndarray:
    """c_r = s_r / (r + 1) with seeded signs s_r = +-1 (s_0 = +1), normalised."""
    rng = np.random.default_rng(seed + 7919)
    s = rng.integers(0, 2, ndets).astype(np.float64) * 2.0 - 1.0
    s[0] = 1.0
    c = s / (np.arange(ndets, dtype=np.float64) + 1.0)
    return c / np.linalg.norm(c)


def all_dets(norb: int, na: int, nb: int):
    """Every determinant with na alpha and nb beta electrons in norb orbitals.

    Ordered by the 128-bit key ascending (beta word high, alpha word low).
    """
    def strings(k):
        out = []
        for w in range(1 << norb):
            if bin(w).count("1") == k:
                out.append(w)
        return out
    sa, sb = strings(na), strings(nb)
    A = np.array([x for y in sb for x in sa], dtype=np.uint64)
    B = np.array([y for y in sb for x in sa], dtype=np.uint64)
    return A, B


@dataclasses.dataclass(frozen=True)
class Workload:
    """One single-system search workload.  ``e0_key`` names its stored E0."""
    name: str
    norb: int
    na: int
    nb: int
    kind: str            # "hubbard" | "random"
    seed: int
    ndets: int           # |psi|
    C: int               # core determinants
    N: int               # determinants to select
    t: float = 1.0
    U: float = 4.0

    def integrals(self):
        if self.kind == "hubbard":
            return hubbard_ring(self.norb, self.t, self.U)
        return random_molecular(self.norb, self.seed)

    def psi(self):
        """(alpha, beta, c) of the random-walk wavefunction (random kind only)."""
        if self.kind != "random":
            raise ValueError("the Hubbard start wavefunction is built by the CI solver")
        A, B = random_walk_dets(self.norb, self.na, self.nb, self.ndets, self.seed)
        return A, B, rank_decay_coeffs(self.ndets, self.seed)

    @property
    def pairs(self) -> int:
        return min(self.C, self.ndets) * n_excitations(self.norb, self.na, self.nb)


WORKLOADS = {
    # (8e,8o) periodic Hubbard ring, t=1, U=4: 100-det start, C=100, N=1000
    "hubbard_8e8o": Workload("hubbard_8e8o", 8, 4, 4, "hubbard", 0, 100, 100, 1000),
    # random molecular-like (16e,16o): |psi| = N = 1e5, C = 1e4
    "random_16e16o": Workload("random_16e16o", 16, 8, 8, "random", 2, 100_000, 10_000, 100_000),
    # Cr2-shaped (24e,30o): |psi| = N = 1e6, C = 1e5
    "random_24e30o": Workload("random_24e30o", 30, 12, 12, "random", 3, 1_000_000, 100_000, 1_000_000),
    # small parity cases spanning several tiles with ragged tails
    "random_12e12o": Workload("random_12e12o", 12, 6, 6, "random", 12, 2_000, 200, 5_000),
    "random_10e14o": Workload("random_10e14o", 14, 5, 5, "random", 14, 600, 150, 3_000),
    "random_14e20o": Workload("random_14e20o", 20, 7, 7, "random", 20, 20_000, 400, 20_000),
}


def stored_e0(name: str) -> float:
    """E0 for a random workload, as written by ``workloads/make_e0.py``."""
    path = os.path.join(os.path.dirname(__file__), "e0.json")
    with open(path) as f:
        return float(json.load(f)[name]["E0"])


def batched_systems(count: int = 512, seed: int = 4000, scale: float = 1.0):
    """Many small uneven systems for the batched search (512 by default).

    System k: norb in {8, 10, ..., 20} (uniform), half filling, Ms = 0; even k a
    periodic Hubbard ring with t = 1 and U/t ~ U(1, 8), odd k random
    molecular-like integrals (seed 1000 + k); C ~ logU(1e3, 1e4) and
    N ~ logU(1e4, 1e5), both times ``scale``; psi holds min(2 C, a quarter of the
    determinant space) dets of the random walk (seed 1000 + k) with 1/rank
    coefficients, and C is capped by |psi|.  E0 is left to the caller (it is an
    input of the search; any value below the spectrum's top serves).
    Returns a list of dicts with keys name, h1, eri, ecore, alpha, beta, c, C, N,
    norb, na, nb.
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        norb = int(rng.choice([8, 10, 12, 14, 16, 18, 20]))
        na = nb = norb // 2
        C = int(round(scale * 10 ** rng.uniform(3, 4)))
        N = int(round(scale * 10 ** rng.uniform(4, 5)))
        if k % 2 == 0:
            h1, eri, ec = hubbard_ring(norb, 1.0, float(rng.uniform(1, 8)))
            kind = "hubbard"
        else:
            h1, eri, ec = random_molecular(norb, 1000 + k)
            kind = "random"
        space = comb(norb, na) * comb(norb, nb)
        nd = int(max(2, min(2 * C, space // 4)))
        A, B = random_walk_dets(norb, na, nb, nd, 1000 + k)
        c = rank_decay_coeffs(nd, 1000 + k)
        out.append(dict(name=f"{kind}_{2 * na}e{norb}o_{k}", h1=h1, eri=eri, ecore=ec, alpha=A,
                        beta=B, c=c, C=min(C, nd), N=N, norb=norb, na=na, nb=nb))
    return out
