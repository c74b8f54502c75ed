"""GPU parity of the variational step (Sec. 2.3) and the ASCI loop (Alg. 1)
through the C ABI, against the CPU oracle.

* asci_hamiltonian: the CSR matrix, densified, equals the oracle's dense H
  element by element (sizes spanning several 256-row CTAs and column slices
  with ragged tails, the full (8e,8o) Hubbard sector, one determinant, a list
  with no connections, 32 orbitals), rows hold ascending columns and the
  diagonal, off-diagonal entries are nonzero; at 5e4 determinants, sampled
  rows against the oracle's dense rows.
* asci_spmv: y = H x against the dense product.
* asci_davidson: the lowest eigenpair of the dense matrix (LAPACK), with and
  without a guess, with restarts (small subspace), and at n <= subspace.
* asci_loop: step by step against the oracle's step from the same input
  (selected set equal except magnitudes tied at the cutoff within 1e-9,
  energies within 1e-9, vectors within 1e-6), a whole loop, and full CI of
  the Hubbard ring when nothing is truncated.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fock
from tests._parity import key_order, to_u64_pairs

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


def _dev(torch, A, B):
    return torch.tensor(np.stack([np.asarray(A, dtype=np.uint64), np.asarray(B, dtype=np.uint64)],
                                 1).view(np.int64), device="cuda")


def _dense(H, n):
    rp, col, val = (t.cpu().numpy() for t in H)
    D = np.zeros((n, n))
    for i in range(n):
        cols = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0), f"row {i}: columns not ascending"
        assert i in cols, f"row {i}: diagonal missing"
        D[i, cols] = val[rp[i]:rp[i + 1]]
        off = val[rp[i]:rp[i + 1]][cols != i]
        assert np.all(off != 0.0), f"row {i}: stored zero"
    return D


def _ints_sys(kind, norb, seed):
    if kind == "hubbard":
        return W.hubbard_ring(norb, 1.0, 4.0)
    return W.random_molecular(norb, seed)


# ------------------------------------------------------------- the build ---

CASES = [
    # (kind, norb, na, nb, ndets, seed)
    ("random", 8, 4, 4, 700, 1),       # 3 row CTAs, ragged tail
    ("random", 10, 5, 4, 2500, 2),     # several column slices
    ("random", 12, 6, 6, 1, 3),        # one determinant
    ("random", 32, 3, 2, 300, 4),      # 32 orbitals: bits up to 31
    ("hubbard", 8, 4, 4, None, 0),     # the full sector (4900)
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}{c[1]}o_{c[4]}")
def test_hamiltonian_equals_oracle_dense(torch_cuda, asci, oracle_mod, case):
    torch = torch_cuda
    kind, norb, na, nb, nd, seed = case
    h1, eri, ec = _ints_sys(kind, norb, seed)
    ec = 0.75 if kind == "random" else ec
    if nd is None:
        A, B = fock.sector(norb, na, nb)
    else:
        A, B = W.random_walk_dets(norb, na, nb, nd, seed=seed)
    n = len(A)
    H = asci.hamiltonian(_dev(torch, A, B), h1, eri, ec)
    D = _dense(H, n)
    ref = oracle_mod.dense_h(oracle_mod.Ints(h1, eri, ec), A, B)
    assert np.allclose(D, ref, rtol=1e-12, atol=1e-12)
    # every connection the oracle finds nonzero is stored
    big = np.abs(ref) > 1e-12
    assert np.all(D[big] != 0.0)
    assert np.array_equal(D, D.T) or np.allclose(D, D.T, rtol=0, atol=1e-13)


def test_hamiltonian_without_connections(torch_cuda, asci, oracle_mod):
    """Determinants pairwise more than two excitations apart: diagonal only."""
    torch = torch_cuda
    h1, eri, ec = W.random_molecular(12, 9)
    A = np.array([0b000000000111, 0b000000111000, 0b000111000000, 0b111000000000], dtype=np.uint64)
    B = A.copy()
    rp, col, val = asci.hamiltonian(_dev(torch, A, B), h1, eri, ec)
    assert rp.cpu().tolist() == [0, 1, 2, 3, 4]
    assert col.cpu().tolist() == [0, 1, 2, 3]
    ints = oracle_mod.Ints(h1, eri, ec)
    ref = [oracle_mod.diag(ints, (a, b)) for a, b in zip(A, B)]
    assert np.allclose(val.cpu().numpy(), ref, rtol=1e-13, atol=1e-12)


def test_hamiltonian_sampled_rows_at_5e4(torch_cuda, asci, oracle_mod):
    torch = torch_cuda
    norb, na, nb = 16, 8, 8
    h1, eri, ec = W.random_molecular(norb, 2)
    A, B = W.random_walk_dets(norb, na, nb, 50000, seed=2)
    n = len(A)
    rp, col, val = (t.cpu().numpy() for t in asci.hamiltonian(_dev(torch, A, B), h1, eri, ec))
    rng = np.random.default_rng(0)
    rows = np.concatenate([[0, n - 1], rng.choice(n, 14, replace=False)])
    ref = oracle_mod.h_rows(oracle_mod.Ints(h1, eri, ec), A, B, rows)
    for r, i in enumerate(rows):
        got = np.zeros(n)
        got[col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
        assert np.allclose(got, ref[r], rtol=1e-12, atol=1e-12), i
        assert np.all(got[np.abs(ref[r]) > 1e-12] != 0.0)


def test_hamiltonian_size_query_and_errors(torch_cuda, asci):
    import ctypes as ct
    torch = torch_cuda
    lib = asci.load()
    h1, eri, ec = W.random_molecular(8, 1)
    A, B = W.random_walk_dets(8, 4, 4, 100, seed=1)
    d = _dev(torch, A, B)
    keep = []
    ints, _ = asci._ints(h1, eri, ec, keep)
    rp = torch.empty(101, dtype=torch.int64, device="cuda")
    nnz = ct.c_size_t(0)
    assert lib.asci_hamiltonian(d.data_ptr(), 100, ct.byref(ints), rp.data_ptr(), None, None, 0,
                                ct.byref(nnz), None) == 0
    assert nnz.value == int(rp[-1].item()) > 100
    # duplicates and mixed electron counts are rejected
    dup = torch.cat([d, d[:1]])
    rp2 = torch.empty(102, dtype=torch.int64, device="cuda")
    assert lib.asci_hamiltonian(dup.data_ptr(), 101, ct.byref(ints), rp2.data_ptr(), None, None,
                                0, ct.byref(nnz), None) == -1
    bad = d.clone()
    bad[0, 0] = 0b1
    assert lib.asci_hamiltonian(bad.data_ptr(), 100, ct.byref(ints), rp.data_ptr(), None, None,
                                0, ct.byref(nnz), None) == -1


# ------------------------------------------------------ products, Davidson ---

def test_spmv_equals_dense_product(torch_cuda, asci, oracle_mod):
    torch = torch_cuda
    h1, eri, ec = W.random_molecular(10, 5)
    A, B = W.random_walk_dets(10, 5, 5, 3000, seed=5)
    H = asci.hamiltonian(_dev(torch, A, B), h1, eri, ec)
    D = oracle_mod.dense_h(oracle_mod.Ints(h1, eri, ec), A, B)
    x = np.random.default_rng(1).normal(size=len(A))
    y = asci.spmv(H, torch.tensor(x, device="cuda")).cpu().numpy()
    ref = D @ x
    assert np.allclose(y, ref, rtol=1e-11, atol=1e-11 * np.abs(D).sum(1).max())
    # fixed summation order: the same bits on a second call
    y2 = asci.spmv(H, torch.tensor(x, device="cuda")).cpu().numpy()
    assert np.array_equal(y, y2)


@pytest.mark.parametrize("sub,guess,nd", [(24, False, 2000), (4, True, 2000), (24, True, 3),
                                          (24, False, 1), (8, False, 600)])
def test_davidson_equals_lowest_eigenpair(torch_cuda, asci, oracle_mod, sub, guess, nd):
    torch = torch_cuda
    import scipy.linalg as sl
    h1, eri, ec = W.random_molecular(10, 7)
    A, B = W.random_walk_dets(10, 5, 5, nd, seed=7)
    H = asci.hamiltonian(_dev(torch, A, B), h1, eri, ec)
    D = oracle_mod.dense_h(oracle_mod.Ints(h1, eri, ec), A, B)
    w, V = sl.eigh(D)
    v0 = V[:, 0] * np.sign(V[np.argmax(np.abs(V[:, 0])), 0])
    g = None
    if guess:
        g = torch.tensor(np.abs(V[:, 0]) + 0.3, device="cuda")  # a rough guess
    E, v, iters, res = asci.davidson(H, g, max_subspace=sub, tol=1e-10, max_iter=2000)
    v = v.cpu().numpy()
    assert abs(E - w[0]) < 1e-9 * max(1.0, abs(w[0]))
    assert res <= 1e-10 and abs(np.linalg.norm(v) - 1.0) < 1e-12
    if len(w) > 1:
        assert w[1] - w[0] > 1e-4  # nondegenerate: the vector is unique up to sign
    assert np.max(np.abs(v - v0)) < 1e-7
    assert v[np.argmax(np.abs(v))] > 0
    assert iters >= 1


# ------------------------------------------------------------- the loop ---

def _hubbard_start():
    """The (8e,8o) Hubbard start: the 100 lowest-H_ii determinants with their
    CI ground vector (its energy lies below every other determinant's H_ii)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "hubbard_8e8o_psi.json")) as f:
        d = json.load(f)
    return (np.array(d["alpha"], dtype=np.uint64), np.array(d["beta"], dtype=np.uint64),
            np.array(d["c"]))


def _start(norb, na, nb):
    a0 = np.array([W.aufbau(na)], dtype=np.uint64)
    b0 = np.array([W.aufbau(nb)], dtype=np.uint64)
    return a0, b0, np.ones(1)


def _check_step(oracle_mod, ints, A, B, c, E0, ncd, ntd, gA, gB, gc, gE):
    """The GPU step from (A, B, c, E0) against the oracle's step from the same
    input.  Returns False when the selected sets differ (allowed only for
    magnitudes tied at the cutoff); the energies and vectors are compared
    when the sets agree."""
    import scipy.linalg as sl
    res = oracle_mod.search(ints, A, B, c, E0, ncd)
    mag = {(int(b), int(a)): abs(float(v)) for a, b, v in
           zip(np.concatenate([A, res.a]), np.concatenate([B, res.b]), np.concatenate([c, res.score]))}
    na, nb, vals, kept_min, dropped_max, _ = oracle_mod.asci_merge(ints, A, B, c, E0, ncd, ntd)
    want = set(zip(nb.tolist(), na.tolist()))
    got = set(zip(gB.tolist(), gA.tolist()))
    assert len(got) == len(want)
    o = key_order(gA, gB)
    assert np.array_equal(gA[o], gA) and np.array_equal(gB[o], gB), "output not in key order"
    if want != got:
        band = 1e-9 * kept_min + 1e-15
        for k in want ^ got:
            assert k in mag, "selected a determinant that is neither in psi nor a candidate"
            assert abs(mag[k] - kept_min) <= band, "sets differ away from the cutoff"
        return False
    D = oracle_mod.dense_h(ints, na, nb)
    w, V = sl.eigh(D)
    assert abs(gE - w[0]) < 1e-9 * max(1.0, abs(w[0]))
    assert abs(np.linalg.norm(gc) - 1.0) < 1e-12 and gc[np.argmax(np.abs(gc))] > 0
    if len(w) == 1 or w[1] - w[0] > 1e-6:  # nondegenerate: the vector is unique
        v0 = V[:, 0] * np.sign(V[np.argmax(np.abs(V[:, 0])), 0])
        assert np.max(np.abs(gc - v0)) < 1e-6
    return True


@pytest.mark.parametrize("kind,norb,na,nb,ncd,ntd", [("random", 8, 4, 4, 20, 300),
                                                      ("random", 10, 5, 5, 50, 800),
                                                      ("hubbard", 8, 4, 4, 30, 400)])
def test_asci_loop_stepwise_equals_oracle(torch_cuda, asci, oracle_mod, kind, norb, na, nb, ncd,
                                          ntd):
    torch = torch_cuda
    h1, eri, ec = _ints_sys(kind, norb, 3)
    ints = oracle_mod.Ints(h1, eri, ec)
    A, B, c = _hubbard_start() if kind == "hubbard" else _start(norb, na, nb)
    E = oracle_mod.variational_energy(ints, A, B, c)
    matched = 0
    for step in range(4):
        d, gc, gE, st = asci.asci_loop(_dev(torch, A, B), torch.tensor(c, device="cuda"), h1, eri,
                                       ec, ncdets=ncd, ntdets=ntd, max_steps=1, tol=1e-10)
        gA, gB = to_u64_pairs(d)
        gc = gc.cpu().numpy()
        assert abs(st.start_energy - E) < 1e-9 * max(1.0, abs(E))
        assert st.ndets == [len(gA)] and len(st.energy) == 1 and st.energy[0] == gE
        matched += _check_step(oracle_mod, ints, A, B, c, E, ncd, ntd, gA, gB, gc, gE)
        A, B, c, E = gA, gB, gc, oracle_mod.variational_energy(ints, gA, gB, gc)
    assert matched >= 3


def test_asci_loop_rejects_undefined_scores(torch_cuda, asci):
    """From the Hubbard ring's aufbau determinant, doubles that keep the double
    occupancy have H_ii = E_0 (and a zero numerator): the score 0/0 is
    undefined and the loop says so."""
    torch = torch_cuda
    h1, eri, ec = W.hubbard_ring(8, 1.0, 4.0)
    A, B, c = _start(8, 4, 4)
    with pytest.raises(asci.AsciError, match="not finite"):
        asci.asci_loop(_dev(torch, A, B), torch.tensor(c, device="cuda"), h1, eri, ec, ncdets=5,
                       ntdets=50, max_steps=2)


def test_asci_loop_whole_run_equals_oracle(torch_cuda, asci, oracle_mod):
    torch = torch_cuda
    h1, eri, ec = W.random_molecular(8, 3)
    ints = oracle_mod.Ints(h1, eri, ec)
    A, B, c = _start(8, 4, 4)
    pa, pb, pc, pE, hist = oracle_mod.asci_loop(ints, A, B, c, 40, 500, max_iter=6, etol=1e-7)
    d, gc, gE, st = asci.asci_loop(_dev(torch, A, B), torch.tensor(c, device="cuda"), h1, eri, ec,
                                   ncdets=40, ntdets=500, max_steps=6, etol=1e-7, tol=1e-10)
    gA, gB = to_u64_pairs(d)
    assert [int(x) for x in st.ndets] == [h[0] for h in hist]
    assert np.allclose(st.energy, [h[1] for h in hist], rtol=0, atol=1e-9)
    # energies agree at every step.  With n_alpha = n_beta the ground state is
    # spin-symmetric, so a determinant and its alpha-beta swap carry equal |c|
    # and |S|; where the cutoff falls between such a pair, the key tie-break
    # meets values that the two runs round differently, and the runs may keep
    # different partners.  Compared modulo that swap, the final spaces agree.
    from collections import Counter

    def canon(a, b):
        return Counter(min((int(x), int(y)), (int(y), int(x))) for x, y in zip(a, b))
    cg, cp = canon(gA, gB), canon(pa, pb)
    assert sum((cg & cp).values()) >= 0.99 * len(pa)
    assert abs(gE - pE) < 1e-9
    assert all(t >= 0 for t in st.t_search_ms + st.t_hamiltonian_ms + st.t_davidson_ms)
    assert st.new_dets[0] == st.ndets[0] - 1


def test_asci_loop_reaches_full_ci(torch_cuda, asci, oracle_mod):
    """Nothing truncated: the loop closes the (8e,8o) Hubbard sector and its
    energy is full CI."""
    torch = torch_cuda
    import scipy.linalg as sl
    h1, eri, ec = W.hubbard_ring(8, 1.0, 4.0)
    S_A, S_B = fock.sector(8, 4, 4)
    E_fci = float(sl.eigh(fock.hamiltonian(8, h1, eri, ec, S_A, S_B), subset_by_index=[0, 0],
                          eigvals_only=True)[0])
    A, B, c = _hubbard_start()
    d, gc, gE, st = asci.asci_loop(_dev(torch, A, B), torch.tensor(c, device="cuda"), h1, eri, ec,
                                   ncdets=10 ** 6, ntdets=10 ** 4, max_steps=12, etol=0.0,
                                   tol=1e-10)
    assert len(d) == 4900 and st.ndets[-1] == 4900
    assert abs(gE - E_fci) < 1e-9
    assert st.new_dets[-1] == 0  # the last step found the sector closed


def test_asci_loop_rejects_bad_options(torch_cuda, asci):
    torch = torch_cuda
    h1, eri, ec = W.random_molecular(8, 1)
    A, B, c = _start(8, 4, 4)
    with pytest.raises(asci.AsciError):
        asci.asci_loop(_dev(torch, A, B), torch.tensor(c, device="cuda"), h1, eri, ec, ncdets=0,
                       ntdets=10)
    with pytest.raises(asci.AsciError):
        asci.asci_loop(_dev(torch, A, B), torch.tensor(c, device="cuda"), h1, eri, ec, ncdets=5,
                       ntdets=10, max_subspace=1)


# ------------------------------------------------------- host-memory paths ---

def test_host_pointer_paths(torch_cuda, asci, oracle_mod):
    """asci_hamiltonian, asci_spmv, asci_davidson and asci_loop with every
    array in host memory (the library stages them) give what the device paths
    give."""
    import ctypes as ct
    torch = torch_cuda
    lib = asci.load()
    h1, eri, ec = W.random_molecular(8, 5)
    A, B = W.random_walk_dets(8, 4, 4, 500, seed=5)
    n = len(A)
    dets = np.ascontiguousarray(np.stack([A, B], 1).astype(np.uint64))
    keep = []
    ints, _ = asci._ints(h1, eri, ec, keep)
    rp = np.empty(n + 1, dtype=np.int64)
    nnz = ct.c_size_t(0)
    assert lib.asci_hamiltonian(dets.ctypes.data, n, ct.byref(ints), rp.ctypes.data, None, None,
                                0, ct.byref(nnz), None) == 0
    col = np.empty(nnz.value, dtype=np.int32)
    val = np.empty(nnz.value, dtype=np.float64)
    assert lib.asci_hamiltonian(dets.ctypes.data, n, ct.byref(ints), rp.ctypes.data,
                                col.ctypes.data, val.ctypes.data, nnz.value, ct.byref(nnz),
                                None) == 0
    Hd = asci.hamiltonian(_dev(torch, A, B), h1, eri, ec)
    assert np.array_equal(rp, Hd[0].cpu().numpy()) and np.array_equal(col, Hd[1].cpu().numpy())
    assert np.array_equal(val, Hd[2].cpu().numpy())
    x = np.random.default_rng(2).normal(size=n)
    y = np.empty(n)
    assert lib.asci_spmv(rp.ctypes.data, col.ctypes.data, val.ctypes.data, n, x.ctypes.data,
                         y.ctypes.data, None) == 0
    assert np.array_equal(y, asci.spmv(Hd, torch.tensor(x, device="cuda")).cpu().numpy())
    o = asci._DavOpts(16, 500, 1e-10)
    e, it, res = ct.c_double(0), ct.c_int32(0), ct.c_double(0)
    vec = np.empty(n)
    assert lib.asci_davidson(rp.ctypes.data, col.ctypes.data, val.ctypes.data, n, None,
                             ct.byref(o), ct.byref(e), vec.ctypes.data, ct.byref(it),
                             ct.byref(res), None) == 0
    Ed, vd, _, _ = asci.davidson(Hd, None, max_subspace=16, max_iter=500, tol=1e-10)
    assert e.value == Ed and np.array_equal(vec, vd.cpu().numpy())
    # the loop with numpy inputs returns numpy outputs equal to the device run
    a0 = np.array([W.aufbau(4)], dtype=np.uint64)
    hd, hc, hE, _ = asci.asci_loop(np.stack([a0, a0], 1), np.ones(1), h1, eri, ec, ncdets=5,
                                   ntdets=300, max_steps=2, tol=1e-10)
    dd, dc, dE, _ = asci.asci_loop(_dev(torch, a0, a0), torch.ones(1, dtype=torch.float64,
                                                                    device="cuda"),
                                   h1, eri, ec, ncdets=5, ntdets=300, max_steps=2, tol=1e-10)
    assert isinstance(hd, np.ndarray) and hE == dE
    assert np.array_equal(hd.view(np.int64), dd.cpu().numpy()) and np.array_equal(hc, dc.cpu().numpy())


def test_asci_loop_truncates_a_large_start(torch_cuda, asci, oracle_mod):
    """A start larger than N_tdets: the first step keeps the N_tdets largest of
    |c| and |S| (some of the start's determinants are dropped), as the oracle's
    step does."""
    torch = torch_cuda
    h1, eri, ec = W.random_molecular(10, 4)
    ints = oracle_mod.Ints(h1, eri, ec)
    A, B = W.random_walk_dets(10, 5, 5, 400, seed=4)
    c = W.rank_decay_coeffs(400, seed=4)
    E = oracle_mod.variational_energy(ints, A, B, c)
    d, gc, gE, st = asci.asci_loop(_dev(torch, A, B), torch.tensor(c, device="cuda"), h1, eri, ec,
                                   ncdets=60, ntdets=150, max_steps=1, tol=1e-10)
    gA, gB = to_u64_pairs(d)
    assert len(gA) == 150 and st.ndets == [150]
    assert len(set(zip(gA.tolist(), gB.tolist())) & set(zip(A.tolist(), B.tolist()))) < 150 or \
        st.new_dets[0] == 0
    _check_step(oracle_mod, ints, A, B, c, E, 60, 150, gA, gB, gc.cpu().numpy(), gE)
