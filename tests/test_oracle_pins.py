"""Pins of the CPU oracle against things other than itself (CPU only).

* The brute-force second-quantised Hamiltonian (oracle/fock.py) is pinned by
  closed forms: the Hubbard ring at U = 0 and t = 0, and the Hubbard dimer.
* The oracle's Slater-Condon evaluator is pinned element by element against
  that brute-force Hamiltonian on complete tiny sectors with random integrals.
* The oracle's search (Alg. 2 with Eq. 1) is pinned by brute force: numerators
  equal the dense product H[:, core] @ c_core, the candidate set equals the
  structural set of dets within two excitations of the core and outside psi,
  counts follow the closed form, and the single-determinant case reduces to
  Epstein-Nesbet coefficients.
* The ASCI loop (Alg. 1) with N = infinity converges to full CI on the Hubbard
  ring; each step's selection equals a brute-force sort of |c| and |S| with key
  ties, its eigenpair satisfies H v = E v on the space, and its energies stay
  above full CI (Rayleigh-Ritz).
* Mutation tests plant plausible mistakes in a copy of the oracle and check
  that a pin catches each one.
"""
import json
import math
import os
import subprocess
import ctypes as ct

import numpy as np
import pytest

import workloads as W
from oracle import fock

GOLD = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _gold():
    with open(GOLD) as f:
        return json.load(f)


def _lowest(H):
    """Lowest eigenvalue of a dense symmetric matrix (LAPACK, robust to degeneracy)."""
    import scipy.linalg as sl
    return float(sl.eigh(H, subset_by_index=[0, 0], eigvals_only=True)[0])


# --------------------------------------------------------------------------
# brute force pinned by closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", _gold()["hubbard"]["cases"], ids=lambda c: f"n{c['norb']}_t{c['t']}_U{c['U']}")
def test_bruteforce_hubbard_closed_forms(case):
    n, na, nb = case["norb"], case["na"], case["nb"]
    h1, eri, ec = W.hubbard_ring(n, case["t"], case["U"])
    A, B = fock.sector(n, na, nb)
    H = fock.hamiltonian(n, h1, eri, ec, A, B)
    assert np.allclose(H, H.T, atol=1e-14)
    assert abs(_lowest(H) - case["E"]) < 1e-9


def test_bruteforce_particle_and_spin_conservation():
    # H never couples sectors: the brute-force action on one sector lands in it
    n = 4
    h1, eri, ec = W.random_molecular(n, 5)
    A, B = fock.sector(n, 2, 1)
    A2, B2 = fock.sector(n, 1, 2)
    H = fock.hamiltonian(n, h1, eri, ec, np.concatenate([A, A2]), np.concatenate([B, B2]))
    m = len(A)
    assert np.all(H[:m, m:] == 0.0) and np.all(H[m:, :m] == 0.0)


# --------------------------------------------------------------------------
# Slater-Condon (oracle) pinned by brute force
# --------------------------------------------------------------------------

SECTORS = [(4, 1, 1, 0.0), (6, 2, 2, 0.37), (6, 3, 3, 0.0), (5, 3, 1, -1.25), (5, 2, 0, 0.0)]


@pytest.mark.parametrize("n,na,nb,ecore", SECTORS)
def test_slater_condon_matches_bruteforce(oracle_mod, n, na, nb, ecore):
    h1, eri, _ = W.random_molecular(n, 100 + n + na)
    A, B = fock.sector(n, na, nb)
    Hb = fock.hamiltonian(n, h1, eri, ecore, A, B)
    Ho = oracle_mod.dense_h(oracle_mod.Ints(h1, eri, ecore), A, B)
    assert np.max(np.abs(Ho - Hb)) < 1e-13


def test_slater_condon_hubbard_matches_bruteforce(oracle_mod):
    n = 6
    h1, eri, ec = W.hubbard_ring(n, 1.0, 3.0)
    A, B = fock.sector(n, 3, 3)
    Hb = fock.hamiltonian(n, h1, eri, ec, A, B)
    Ho = oracle_mod.dense_h(oracle_mod.Ints(h1, eri, ec), A, B)
    assert np.max(np.abs(Ho - Hb)) < 1e-13


def test_hermiticity(oracle_mod):
    n = 8
    h1, eri, _ = W.random_molecular(n, 9)
    ints = oracle_mod.Ints(h1, eri)
    A, B = fock.sector(n, 3, 3)
    rng = np.random.default_rng(0)
    idx = rng.choice(len(A), 150, replace=False)
    H = oracle_mod.dense_h(ints, A[idx], B[idx])
    assert np.max(np.abs(H - H.T)) < 1e-14


# --------------------------------------------------------------------------
# the search pinned by brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,na,nb,npsi,C", [(6, 2, 2, 20, 12), (6, 3, 3, 40, 40), (5, 3, 1, 8, 5),
                                             (7, 3, 2, 30, 17)])
def test_search_numerators_equal_dense_product(oracle_mod, n, na, nb, npsi, C):
    h1, eri, _ = W.random_molecular(n, 7 * n + na)
    ecore = 0.5
    ints = oracle_mod.Ints(h1, eri, ecore)
    A, B = fock.sector(n, na, nb)
    Hb = fock.hamiltonian(n, h1, eri, ecore, A, B)
    rng = np.random.default_rng(n + npsi)
    psi = rng.choice(len(A), npsi, replace=False)
    c = rng.normal(size=npsi)
    E0 = float(np.min(np.diag(Hb))) - 0.3
    res = oracle_mod.search(ints, A[psi], B[psi], c, E0, C)
    core = psi[np.argsort(-np.abs(c), kind="stable")][:C]   # |c| distinct a.s.
    core_c = c[np.argsort(-np.abs(c), kind="stable")][:C]
    # structural candidate set: within two excitations of a core det, not in psi
    exc = lambda i, j: (bin(int(A[i]) ^ int(A[j])).count("1") + bin(int(B[i]) ^ int(B[j])).count("1")) // 2
    expect = sorted(i for i in range(len(A)) if i not in set(psi.tolist())
                    and any(1 <= exc(i, j) <= 2 for j in core))
    key_of = {(int(A[i]), int(B[i])): i for i in range(len(A))}
    got = sorted(key_of[(int(a), int(b))] for a, b in zip(res.a, res.b))
    assert got == expect
    num_dense = Hb[:, core] @ core_c
    for k, (a, b) in enumerate(zip(res.a, res.b)):
        i = key_of[(int(a), int(b))]
        assert abs(res.num[k] - num_dense[i]) <= 1e-13 * max(1.0, res.abssum[k])
        assert abs(res.haa[k] - Hb[i, i]) <= 1e-13 * max(1.0, abs(Hb[i, i]))
        assert abs(res.score[k] - num_dense[i] / (E0 - Hb[i, i])) <= 1e-12 * abs(res.score[k]) + 1e-15
    assert res.generated == len(core) * W.n_excitations(n, na, nb)


def test_search_single_det_is_epstein_nesbet(oracle_mod):
    n, na, nb = 6, 3, 3
    h1, eri, _ = W.random_molecular(n, 77)
    ints = oracle_mod.Ints(h1, eri)
    A, B = fock.sector(n, na, nb)
    Hb = fock.hamiltonian(n, h1, eri, 0.0, A, B)
    hf = (W.aufbau(na), W.aufbau(nb))
    key_of = {(int(A[i]), int(B[i])): i for i in range(len(A))}
    i0 = key_of[hf]
    E0 = Hb[i0, i0]
    res = oracle_mod.search(ints, [hf[0]], [hf[1]], [1.0], E0, 1)
    assert res.generated == W.n_excitations(n, na, nb) == len(res.a)
    for k, (a, b) in enumerate(zip(res.a, res.b)):
        i = key_of[(int(a), int(b))]
        en = Hb[i, i0] / (E0 - Hb[i, i])
        assert abs(res.score[k] - en) <= 1e-12 * abs(en) + 1e-15


@pytest.mark.parametrize("case", _gold()["excitation_counts"]["cases"], ids=lambda c: f"n{c['norb']}")
def test_excitation_counts_closed_form(oracle_mod, case):
    n, na, nb = case["norb"], case["na"], case["nb"]
    assert W.n_excitations(n, na, nb) == case["n_exc"]
    h1 = np.zeros((n, n))
    eri = np.zeros((n,) * 4)
    ints = oracle_mod.Ints(h1, eri)
    # a non-aufbau parent so holes and particles interleave
    rng = np.random.default_rng(n)
    pa = sum(1 << int(x) for x in rng.choice(n, na, replace=False))
    pb = sum(1 << int(x) for x in rng.choice(n, nb, replace=False))
    a, b, v = oracle_mod.pairs(ints, [pa], [pb], [1.0])
    assert len(a) == case["n_exc"]
    keys = set(zip(a.tolist(), b.tolist()))
    assert len(keys) == case["n_exc"]               # every excitation is a distinct det
    for x, y in zip(a.tolist(), b.tolist()):
        assert bin(x).count("1") == na and bin(y).count("1") == nb
        lvl = (bin(x ^ pa).count("1") + bin(y ^ pb).count("1")) // 2
        assert 1 <= lvl <= 2


# --------------------------------------------------------------------------
# invariants of the search
# --------------------------------------------------------------------------

def _small_random_case():
    w = W.WORKLOADS["random_10e14o"]
    h1, eri, ec = w.integrals()
    A, B, c = w.psi()
    return w, h1, eri, ec, A, B, c


def test_invariants_permutation_sign_and_buckets(oracle_mod):
    w, h1, eri, ec, A, B, c = _small_random_case()
    ints = oracle_mod.Ints(h1, eri, ec)
    E0 = -20.0
    C = 60
    r0 = oracle_mod.search(ints, A, B, c, E0, C)
    perm = np.random.default_rng(1).permutation(len(A))
    r1 = oracle_mod.search(ints, A[perm], B[perm], c[perm], E0, C)
    assert np.array_equal(r0.a, r1.a) and np.array_equal(r0.b, r1.b)
    assert np.array_equal(r0.score, r1.score)
    r2 = oracle_mod.search(ints, A, B, -c, E0, C)
    assert np.array_equal(r0.a, r2.a) and np.array_equal(r0.score, -r2.score)
    parts = [oracle_mod.search(ints, A, B, c, E0, C, nbuckets=3, bucket=k) for k in range(3)]
    ka = np.concatenate([p.a for p in parts])
    kb = np.concatenate([p.b for p in parts])
    sc = np.concatenate([p.score for p in parts])
    o = np.lexsort((ka, kb))
    assert np.array_equal(ka[o], r0.a) and np.array_equal(kb[o], r0.b)
    assert np.array_equal(sc[o], r0.score)
    assert sum(p.generated for p in parts) == 3 * r0.generated


def test_invariant_alpha_beta_swap(oracle_mod):
    w, h1, eri, ec, A, B, c = _small_random_case()
    ints = oracle_mod.Ints(h1, eri, ec)
    E0, C = -20.0, 60
    r0 = oracle_mod.search(ints, A, B, c, E0, C)
    r1 = oracle_mod.search(ints, B, A, c, E0, C)
    o0 = np.lexsort((r0.a, r0.b))
    o1 = np.lexsort((r1.b, r1.a))  # swapped keys
    assert np.array_equal(r0.a[o0], r1.b[o1]) and np.array_equal(r0.b[o0], r1.a[o1])
    # the reordering phase (-1)^(na nb) is global, so |S| is unchanged
    s0, s1 = np.abs(r0.score[o0]), np.abs(r1.score[o1])
    assert np.all(np.abs(s0 - s1) <= 1e-12 * s0 + 1e-300)


def test_topn_is_duplicate_aware_selection(oracle_mod):
    # |{a > a_k}| < k <= |{a >= a_k}| (Sec. 2.2), ties broken by key ascending
    rng = np.random.default_rng(3)
    n = 500
    a = rng.integers(0, 1 << 20, n).astype(np.uint64)
    b = rng.integers(0, 1 << 20, n).astype(np.uint64)
    s = rng.choice([-3.0, -1.0, 0.5, 1.0, 2.0, 3.0], n)
    for N in (1, 7, 100, 250, 499, 500, 800):
        idx = oracle_mod.topn(a, b, s, N)
        assert len(idx) == min(N, n)
        k = len(idx)
        ak = np.abs(s[idx[-1]])
        assert np.sum(np.abs(s) > ak) < k <= np.sum(np.abs(s) >= ak)
        sel = set(idx.tolist())
        ties = [i for i in range(n) if np.abs(s[i]) == ak]
        tie_sel = sorted((int(b[i]), int(a[i])) for i in ties if i in sel)
        tie_all = sorted((int(b[i]), int(a[i])) for i in ties)
        assert tie_sel == tie_all[:len(tie_sel)]


# --------------------------------------------------------------------------
# full CI through the ASCI loop (Alg. 1 with N = infinity)
# --------------------------------------------------------------------------

def test_asci_loop_reaches_full_ci_on_hubbard_ring(oracle_mod):
    n, na, nb = 8, 4, 4
    h1, eri, ec = W.hubbard_ring(n, 1.0, 4.0)
    ints = oracle_mod.Ints(h1, eri, ec)
    A, B = fock.sector(n, na, nb)
    E_fci = _lowest(fock.hamiltonian(n, h1, eri, ec, A, B))
    from tests.golden.make_golden import hubbard_start
    pa, pb, c, E0 = hubbard_start(oracle_mod)
    big = 10 ** 6
    pa, pb, c, E, hist = oracle_mod.asci_loop(ints, pa, pb, c, big, big, max_iter=10)
    assert len(pa) == len(A) == 4900
    assert abs(E - E_fci) < 1e-9
    # the last step found nothing new: the sector is closed under H
    assert hist[-1][0] == 4900 and len(hist) < 10


def test_asci_step_selects_by_magnitude_with_key_ties(oracle_mod):
    """The next space is the ntdets largest of |c_i| (current dets) and |S_i|
    (candidates), ties by key ascending: brute force with Python sorting."""
    n, na, nb = 6, 3, 3
    h1, eri, ec = W.random_molecular(n, 11)
    ints = oracle_mod.Ints(h1, eri, ec)
    A, B = W.random_walk_dets(n, na, nb, 12, seed=5)
    c = W.rank_decay_coeffs(12, seed=5)
    E0 = oracle_mod.variational_energy(ints, A, B, c)
    res = oracle_mod.search(ints, A, B, c, E0, 6)
    pool = [(abs(float(v)), int(b), int(a)) for a, b, v in zip(A, B, c)]
    pool += [(abs(float(v)), int(b), int(a)) for a, b, v in zip(res.a, res.b, res.score)]
    pool.sort(key=lambda t: (-t[0], t[1], t[2]))
    for ntd in (1, 5, 12, 30, 10 ** 6):
        ma, mb, mv, kept_min, dropped_max, _ = oracle_mod.asci_merge(ints, A, B, c, E0, 6, ntd)
        assert kept_min >= dropped_max and len(ma) == min(ntd, len(pool))
        assert np.isclose(kept_min, np.min(np.abs(mv)))
        na_, nb_, v, E, changed = oracle_mod.asci_step(ints, A, B, c, E0, 6, ntd)
        assert np.array_equal(na_, ma) and np.array_equal(nb_, mb)
        want = sorted((b, a) for _, b, a in pool[:ntd])
        assert [(int(b), int(a)) for a, b in zip(na_, nb_)] == want
        # c' is the ground vector of the dense H on that space
        H = fock.hamiltonian(n, h1, eri, ec, na_, nb_)
        assert abs(E - _lowest(H)) < 1e-10
        assert np.allclose(H @ v, E * v, atol=1e-9) and abs(np.linalg.norm(v) - 1) < 1e-12
        assert v[np.argmax(np.abs(v))] > 0
        assert changed == (set(want) != set(zip(B.tolist(), A.tolist())))


def test_asci_loop_energies_are_variational(oracle_mod):
    """Every step's energy lies above full CI of the sector (Rayleigh-Ritz) and
    the loop's output is that step's ground state."""
    n, na, nb = 8, 4, 4
    h1, eri, ec = W.random_molecular(n, 3)
    ints = oracle_mod.Ints(h1, eri, ec)
    A, B = fock.sector(n, na, nb)
    E_fci = _lowest(fock.hamiltonian(n, h1, eri, ec, A, B))
    a0 = np.array([W.aufbau(na)], dtype=np.uint64)
    b0 = np.array([W.aufbau(nb)], dtype=np.uint64)
    pa, pb, c, E, hist = oracle_mod.asci_loop(ints, a0, b0, np.ones(1), 50, 400, max_iter=6)
    assert len(hist) >= 3
    for size, e in hist:
        assert e >= E_fci - 1e-10 and size <= 400
    assert hist[-1][1] == E and E - E_fci < 0.05 * abs(E_fci)


def test_h_rows_equal_bruteforce_rows(oracle_mod):
    n, na, nb = 5, 2, 3
    h1, eri, ec = W.random_molecular(n, 7)
    ints = oracle_mod.Ints(h1, eri, ec)
    A, B = fock.sector(n, na, nb)
    H = fock.hamiltonian(n, h1, eri, ec, A, B)
    rows = [0, 3, len(A) - 1, 17]
    assert np.allclose(oracle_mod.h_rows(ints, A, B, rows), H[rows], atol=1e-13, rtol=0)


# --------------------------------------------------------------------------
# ASCI-PT2 (last step of Alg. 1) against the dense brute-force Hamiltonian
# --------------------------------------------------------------------------

@pytest.mark.parametrize("npsi,C", [(1, 1), (30, 30), (30, 12)])
def test_pt2_equals_dense_second_order_sum(oracle_mod, npsi, C):
    """E_PT2 = sum_{i not in psi} ((H c_core)_i)^2 / (E0 - H_ii) over the whole
    sector, with H from the second-quantised brute force."""
    n, na, nb = 6, 3, 3
    h1, eri, ec = W.random_molecular(n, 21)
    ec = 0.4
    ints = oracle_mod.Ints(h1, eri, ec)
    SA, SB = fock.sector(n, na, nb)
    H = fock.hamiltonian(n, h1, eri, ec, SA, SB)
    rng = np.random.default_rng(npsi + C)
    idx = rng.choice(len(SA), npsi, replace=False)
    A, B = SA[idx], SB[idx]
    c = rng.normal(size=npsi)
    E0 = float(np.min(np.diag(H))) - 0.5  # below every H_ii: no vanishing denominator
    core = oracle_mod.core_select(A, B, c, C)
    y = H[:, idx[core]] @ c[core]
    out = np.ones(len(SA), dtype=bool)
    out[idx] = False
    ref = float(np.sum(y[out] ** 2 / (E0 - np.diag(H)[out])))
    got = oracle_mod.pt2(ints, A, B, c, E0, C)
    assert abs(got - ref) <= 1e-12 * abs(ref)
    assert got < 0


def test_pt2_pin_catches_planted_mistakes(oracle_mod):
    """Plausible mistakes in the PT2 sum (a sign, the denominator's order, the
    numerator's absolute sum, targets inside psi kept) each break the dense
    brute-force pin."""
    import math
    n, na, nb = 6, 3, 3
    h1, eri, ec = W.random_molecular(n, 21)
    ints = oracle_mod.Ints(h1, eri, ec)
    SA, SB = fock.sector(n, na, nb)
    H = fock.hamiltonian(n, h1, eri, ec, SA, SB)
    rng = np.random.default_rng(3)
    idx = rng.choice(len(SA), 30, replace=False)
    A, B, c = SA[idx], SB[idx], rng.normal(size=30)
    E0 = float(np.min(np.diag(H))) - 0.5
    y = H[:, idx] @ c
    out = np.ones(len(SA), dtype=bool)
    out[idx] = False
    ref = float(np.sum(y[out] ** 2 / (E0 - np.diag(H)[out])))
    res = oracle_mod.search(ints, A, B, c, E0, 30)
    mutants = {
        "sign": -math.fsum((res.num ** 2 / (E0 - res.haa)).tolist()),
        "denominator_order": math.fsum((res.num ** 2 / (res.haa - E0 + 1e-3)).tolist()),
        "absolute_numerator": math.fsum((res.abssum ** 2 / (E0 - res.haa)).tolist()),
        "psi_not_excluded": math.fsum((res.num ** 2 / (E0 - res.haa)).tolist())
        + float(np.sum(y[~out] ** 2 / (E0 - np.diag(H)[~out]))),
    }
    assert abs(oracle_mod.pt2(ints, A, B, c, E0, 30) - ref) <= 1e-12 * abs(ref)
    for name, v in mutants.items():
        assert abs(v - ref) > 1e-6 * abs(ref), name


# --------------------------------------------------------------------------
# Alg. 2's partial-score screen, the brute-force numerator and the core order
# --------------------------------------------------------------------------

def _excitation_level(A, B, i_idx, j_idx):
    """Excitation level between determinants i and j of (A, B), as a matrix."""
    a, b = A.astype(np.int64), B.astype(np.int64)
    xa = a[i_idx][:, None] ^ a[j_idx][None, :]
    xb = b[i_idx][:, None] ^ b[j_idx][None, :]
    pop = np.vectorize(lambda x: bin(int(x)).count("1"))
    return (pop(xa) + pop(xb)) // 2


def _screen_bruteforce(H, A, B, psi, c, E0, C, eps):
    """Alg. 2 over the dense brute-force H: the generated pairs are (i, j) with j
    a core determinant (the C largest |c|, distinct here) and i one or two
    excitations away (H_ij = 0 included); a pair survives when
    |H_ij c_j / (E0 - H_ii)| > eps (eps = 0: every pair).  Returns the surviving
    pair count and {i: (numerator, sum |H_ij c_j|)} over targets outside psi."""
    order = np.argsort(-np.abs(c), kind="stable")[:C]
    core, cc = psi[order], c[order]
    lvl = _excitation_level(A, B, np.arange(len(A)), core)
    inpsi = np.zeros(len(A), dtype=bool)
    inpsi[psi] = True
    surv, out = 0, {}
    for jj, j in enumerate(core):
        for i in np.nonzero((lvl[:, jj] == 1) | (lvl[:, jj] == 2))[0]:
            v = H[i, j] * cc[jj]
            if eps > 0.0 and not abs(v / (E0 - H[i, i])) > eps:
                continue
            surv += 1
            if not inpsi[i]:
                n0, a0 = out.get(i, (0.0, 0.0))
                out[i] = (n0 + v, a0 + abs(v))
    return surv, out


def _partial_scores(H, A, B, psi, c, E0, C):
    order = np.argsort(-np.abs(c), kind="stable")[:C]
    core, cc = psi[order], c[order]
    lvl = _excitation_level(A, B, np.arange(len(A)), core)
    ps = []
    for jj, j in enumerate(core):
        for i in np.nonzero((lvl[:, jj] == 1) | (lvl[:, jj] == 2))[0]:
            ps.append(abs(H[i, j] * cc[jj] / (E0 - H[i, i])))
    return np.array(ps)


def _check_screen(om, ints, H, A, B, psi, c, E0, C, eps):
    surv, want = _screen_bruteforce(H, A, B, psi, c, E0, C, eps)
    res = om.search(ints, A[psi], B[psi], c, E0, C, eps=eps)
    assert res.surviving == surv, (eps, res.surviving, surv)
    key_of = {(int(A[i]), int(B[i])): i for i in range(len(A))}
    got = {key_of[(int(a), int(b))]: k for k, (a, b) in enumerate(zip(res.a, res.b))}
    assert set(got) == set(want), eps
    for i, k in got.items():
        num, mag = want[i]
        assert abs(res.num[k] - num) <= 1e-13 * max(1.0, mag)
    return surv


def pin_eps_screen(om):
    """The oracle's eps screen equals the brute-force screen on a complete
    sector with random integrals, for eps at quantiles of the partial scores and
    within 1e-13 relative of one pair's partial score on either side; and, on
    the Hubbard ring where every quantity is exact, a pair whose partial score
    equals eps is dropped (the screen is strict)."""
    n, na, nb = 6, 3, 3
    h1, eri, _ = W.random_molecular(n, 41)
    ec = 0.25
    ints = om.Ints(h1, eri, ec)
    A, B = fock.sector(n, na, nb)
    H = fock.hamiltonian(n, h1, eri, ec, A, B)
    rng = np.random.default_rng(17)
    psi = rng.choice(len(A), 30, replace=False)
    c = rng.normal(size=30)
    C = 14
    E0 = float(np.min(np.diag(H))) - 0.4
    ps = np.sort(_partial_scores(H, A, B, psi, c, E0, C))
    ps = ps[ps > 0]
    counts = []
    for q in (0.1, 0.5, 0.9):
        counts.append(_check_screen(om, ints, H, A, B, psi, c, E0, C, float(np.quantile(ps, q))))
    assert counts[0] > counts[1] > counts[2] > 0
    # a partial score isolated from its neighbours by more than 1e-12 relative
    gaps = np.minimum(np.diff(ps)[:-1], np.diff(ps)[1:]) / ps[1:-1]
    k = 1 + int(np.argmax(gaps > 1e-9))
    p = float(ps[k])
    above = _check_screen(om, ints, H, A, B, psi, c, E0, C, p * (1.0 - 1e-13))
    below = _check_screen(om, ints, H, A, B, psi, c, E0, C, p * (1.0 + 1e-13))
    assert above == below + 1
    # exact arithmetic: Hubbard ring, c powers of two, E0 exact
    h1, eri, ec = W.hubbard_ring(n, 1.0, 4.0)
    ints = om.Ints(h1, eri, ec)
    H = fock.hamiltonian(n, h1, eri, ec, A, B)
    assert np.array_equal(H, om.dense_h(ints, A, B))
    psi = rng.choice(len(A), 12, replace=False)
    c = np.array([(-1.0) ** k * 2.0 ** -k for k in range(12)])
    E0 = -3.5
    ps = _partial_scores(H, A, B, psi, c, E0, 12)
    p = float(np.unique(ps[ps > 0])[len(np.unique(ps[ps > 0])) // 2])
    tied = int(np.sum(ps == p))
    at = _check_screen(om, ints, H, A, B, psi, c, E0, 12, p)
    just_below = _check_screen(om, ints, H, A, B, psi, c, E0, 12, float(np.nextafter(p, 0.0)))
    assert tied > 0 and just_below == at + tied


def pin_numerator(om):
    """oracle.numerator(target, core) = sum over core j != target of
    H_target,j c_j, for every determinant of two complete sectors (inside and
    outside the core), with the brute-force H; also its sum of magnitudes."""
    for n, na, nb, ncore in ((6, 3, 3, 25), (7, 3, 2, 40)):
        h1, eri, _ = W.random_molecular(n, 5 * n + nb)
        ec = -0.6
        ints = om.Ints(h1, eri, ec)
        A, B = fock.sector(n, na, nb)
        H = fock.hamiltonian(n, h1, eri, ec, A, B)
        rng = np.random.default_rng(n)
        core = rng.choice(len(A), ncore, replace=False)
        cc = rng.normal(size=ncore)
        Hoff = H - np.diag(np.diag(H))
        want = Hoff[:, core] @ cc
        want_abs = np.abs(Hoff[:, core]) @ np.abs(cc)
        for i in range(len(A)):
            got, mag = om.numerator(ints, (A[i], B[i]), A[core], B[core], cc)
            assert abs(got - want[i]) <= 1e-13 * max(1.0, want_abs[i]), i
            assert abs(mag - want_abs[i]) <= 1e-13 * max(1.0, want_abs[i]), i


def pin_core_ties(om):
    """core_select under tied |c| equals a plain sort by (|c| descending, beta
    word, alpha word), for C across the ties."""
    A, B = fock.sector(6, 3, 2)
    rng = np.random.default_rng(23)
    idx = rng.choice(len(A), 70, replace=False)
    A, B = A[idx], B[idx]
    c = rng.choice([-0.5, 0.5, -0.25, 0.25, 0.125], 70)
    want = sorted(range(70), key=lambda i: (-abs(c[i]), int(B[i]), int(A[i])))
    for C in (1, 3, 10, 25, 40, 69, 70, 100):
        assert list(om.core_select(A, B, c, C)) == want[:C], C


def test_eps_screen_equals_bruteforce(oracle_mod):
    pin_eps_screen(oracle_mod)


def test_numerator_equals_dense_product(oracle_mod):
    pin_numerator(oracle_mod)


def test_core_select_ties_by_key(oracle_mod):
    pin_core_ties(oracle_mod)


@pytest.mark.parametrize("eps", [0.0, 2e-6])
def test_all_core_oracle_equals_single_core(oracle_mod, eps):
    """The all-core form of the search returns the single-core result bit for
    bit (keys, numerators, sums of magnitudes, diagonals, scores, counters)."""
    w, h1, eri, ec, A, B, c = _small_random_case()
    ints = oracle_mod.Ints(h1, eri, ec)
    E0 = -20.0
    r1 = oracle_mod.search(ints, A, B, c, E0, 60, eps=eps)
    for threads in (2, 5):
        r2 = oracle_mod.search(ints, A, B, c, E0, 60, eps=eps, threads=threads)
        for f in ("a", "b", "num", "abssum", "haa", "haa_abs", "score"):
            assert np.array_equal(getattr(r1, f), getattr(r2, f)), f
        assert (r1.generated, r1.surviving, r1.unique, r1.excluded, r1.ncore) == \
            (r2.generated, r2.surviving, r2.unique, r2.excluded, r2.ncore)
    if eps > 0:
        assert r1.surviving < r1.generated


def test_diag_abs_is_sum_of_term_magnitudes(oracle_mod):
    """diag_abs: |ecore| + sum |h_pp| + sum over same-spin pairs p<q |J - K| +
    sum over opposite-spin pairs |J|, written out with numpy."""
    n = 7
    h1, eri, _ = W.random_molecular(n, 8)
    ints = oracle_mod.Ints(h1, eri, -1.5)
    for a, b in ((0b0010111, 0b1000011), (0b1110000, 0b0000111)):
        oa = [p for p in range(n) if a >> p & 1]
        ob = [p for p in range(n) if b >> p & 1]
        J = lambda p, q: eri[p, p, q, q]
        K = lambda p, q: eri[p, q, q, p]
        want = 1.5 + sum(abs(h1[p, p]) for p in oa + ob)
        for o in (oa, ob):
            want += sum(abs(J(p, q) - K(p, q)) for p in o for q in o if p < q)
        want += sum(abs(J(p, q)) for p in oa for q in ob)
        assert abs(oracle_mod.diag_abs(ints, (a, b)) - want) <= 1e-13 * want


# --------------------------------------------------------------------------
# planted mistakes: each must be caught by a pin
# --------------------------------------------------------------------------

MUTATIONS = {
    "drop_single_exchange": ("ERI(I, i, a, k, k) - ERI(I, i, k, k, a)", "ERI(I, i, a, k, k)"),
    "flip_double_sign": ("return sg * (ERI(I, i, a, j, b) - ERI(I, i, b, j, a));",
                         "return -sg * (ERI(I, i, a, j, b) - ERI(I, i, b, j, a));"),
    "transpose_double_operand": ("ERI(I, i, a, j, b) - ERI(I, i, b, j, a)",
                                 "ERI(I, i, j, a, b) - ERI(I, i, b, j, a)"),
    "drop_cross_coulomb": ("if (occupied(a, p) && occupied(b, q)) diag_term(&acc, &mag, ERI(I, p, p, q, q));",
                           ""),
    "wrong_phase_range": ("for (k = lo + 1; k < hi; k++)", "for (k = lo; k < hi; k++)"),
    "opposite_spin_sign": ("int s = single_sign(ket_a, ha[0], pa[0]) * single_sign(ket_b, hb[0], pb[0]);",
                           "int s = single_sign(ket_a, ha[0], pa[0]);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistakes(tmp_path, name):
    src = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "asci_oracle.c")).read()
    old, new = MUTATIONS[name]
    assert old in src, f"mutation site for {name} not found"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"])
    lib = ct.CDLL(str(so))
    f64p = ct.POINTER(ct.c_double)
    u64p = ct.POINTER(ct.c_uint64)
    lib.oracle_dense_h.argtypes = [ct.c_int, f64p, f64p, ct.c_double, u64p, u64p, ct.c_size_t, f64p]
    caught = False
    for (n, na, nb, ecore) in SECTORS:
        h1, eri, _ = W.random_molecular(n, 100 + n + na)
        A, B = fock.sector(n, na, nb)
        Hb = fock.hamiltonian(n, h1, eri, ecore, A, B)
        h1c, eric = np.ascontiguousarray(h1), np.ascontiguousarray(eri)
        A, B = np.ascontiguousarray(A), np.ascontiguousarray(B)
        out = np.empty((len(A), len(A)))
        lib.oracle_dense_h(n, h1c.ctypes.data_as(f64p), eric.ctypes.data_as(f64p), ecore,
                           A.ctypes.data_as(u64p), B.ctypes.data_as(u64p), len(A), out.ctypes.data_as(f64p))
        if np.max(np.abs(out - Hb)) >= 1e-13:
            caught = True
            break
    assert caught, f"planted mistake {name} went unnoticed"


# mistakes in the search's screen, the brute-force numerator and the core order,
# each with the pin that must catch it
SEARCH_MUTATIONS = {
    "screen_on_value_alone": ("if (!(fabs(v / (g->E0 - hii)) > g->eps)) return;",
                              "if (!(fabs(v) > g->eps)) return;", "pin_eps_screen"),
    "screen_not_strict": ("if (!(fabs(v / (g->E0 - hii)) > g->eps)) return;",
                          "if (!(fabs(v / (g->E0 - hii)) >= g->eps)) return;", "pin_eps_screen"),
    "screen_denominator_sign": ("if (!(fabs(v / (g->E0 - hii)) > g->eps)) return;",
                                "if (!(fabs(v / (g->E0 + hii)) > g->eps)) return;",
                                "pin_eps_screen"),
    "numerator_skips_doubles": ("if (count_bits(xa) + count_bits(xb) > 4 || (xa == 0 && xb == 0)) continue;",
                                "if (count_bits(xa) + count_bits(xb) >= 4 || (xa == 0 && xb == 0)) continue;",
                                "pin_numerator"),
    "numerator_keeps_diagonal": ("if (count_bits(xa) + count_bits(xb) > 4 || (xa == 0 && xb == 0)) continue;",
                                 "if (count_bits(xa) + count_bits(xb) > 4) continue;", "pin_numerator"),
    "core_ties_reversed": ("if (p->absc != q->absc) return p->absc > q->absc ? -1 : 1;\n"
                           "  return key_cmp(p->a, p->b, q->a, q->b);",
                           "if (p->absc != q->absc) return p->absc > q->absc ? -1 : 1;\n"
                           "  return key_cmp(q->a, q->b, p->a, p->b);", "pin_core_ties"),
    "core_ties_alpha_high": ("if (p->absc != q->absc) return p->absc > q->absc ? -1 : 1;\n"
                             "  return key_cmp(p->a, p->b, q->a, q->b);",
                             "if (p->absc != q->absc) return p->absc > q->absc ? -1 : 1;\n"
                             "  return key_cmp(p->b, p->a, q->b, q->a);", "pin_core_ties"),
}


@pytest.mark.parametrize("name", sorted(SEARCH_MUTATIONS))
def test_search_pins_catch_planted_mistakes(tmp_path, oracle_mod, name):
    src = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "asci_oracle.c")).read()
    old, new, pin = SEARCH_MUTATIONS[name]
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"])
    with oracle_mod.substitute(str(so)):
        with pytest.raises(AssertionError):
            globals()[pin](oracle_mod)
