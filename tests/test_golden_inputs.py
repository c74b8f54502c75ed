"""Stored inputs stay consistent with the oracle scripts that wrote them (CPU)."""
import json
import os

import numpy as np

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def test_hubbard_start_wavefunction_matches_oracle(oracle_mod):
    from tests.golden.make_golden import hubbard_start
    with open(os.path.join(HERE, "golden", "hubbard_8e8o_psi.json")) as f:
        d = json.load(f)
    pa, pb, c, E0 = hubbard_start(oracle_mod)
    assert [int(x) for x in pa] == d["alpha"] and [int(x) for x in pb] == d["beta"]
    assert abs(E0 - d["E0"]) < 1e-12
    # eigenvector sign fixed by the largest |c| being positive
    assert np.max(np.abs(np.abs(c) - np.abs(np.array(d["c"])))) < 1e-10
    # the recipe: 70 dets with H_ii = 0 then 30 from the H_ii = U shell
    ints = oracle_mod.Ints(*W.hubbard_ring(8, 1.0, 4.0))
    hii = sorted(oracle_mod.diag(ints, (a, b)) for a, b in zip(pa, pb))
    assert hii.count(0.0) == 70 and all(abs(h - 4.0) < 1e-12 for h in hii[70:])


def test_stored_e0_matches_oracle(oracle_mod):
    name = "random_10e14o"
    w = W.WORKLOADS[name]
    A, B, c = w.psi()
    k = min(2000, len(A))
    E0 = oracle_mod.variational_energy(oracle_mod.Ints(*w.integrals()), A[:k], B[:k], c[:k])
    assert abs(E0 - W.stored_e0(name)) < 1e-9 * abs(E0)


def test_workload_generators_are_seeded_and_valid():
    w = W.WORKLOADS["random_12e12o"]
    A1, B1, c1 = w.psi()
    A2, B2, c2 = w.psi()
    assert np.array_equal(A1, A2) and np.array_equal(B1, B2) and np.array_equal(c1, c2)
    keys = (B1 << np.uint64(32)) | A1
    assert len(np.unique(keys)) == len(keys)
    pa = np.array([bin(int(x)).count("1") for x in A1])
    pb = np.array([bin(int(x)).count("1") for x in B1])
    assert np.all(pa == w.na) and np.all(pb == w.nb)
    assert abs(np.linalg.norm(c1) - 1.0) < 1e-12 and c1[0] > 0
    h1, eri, _ = w.integrals()
    assert np.allclose(h1, h1.T)
    for perm in ((1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)):
        assert np.array_equal(eri, eri.transpose(perm))
