"""GPU parity of ASCI-PT2 (the last step of Alg. 1) through the C ABI against
the oracle: the value within 1e-10 relative, bit-identical under any constraint
batching (the sum is exact fixed point), the precision variants within 1e-6,
and vanishing denominators reported as errors."""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


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


def _system(name):
    if name == "hubbard":
        with open(os.path.join(HERE, "golden", "hubbard_8e8o_psi.json")) as f:
            d = json.load(f)
        h1, eri, ec = W.hubbard_ring(8, 1.0, 4.0)
        return (h1, eri, ec, np.array(d["alpha"], dtype=np.uint64),
                np.array(d["beta"], dtype=np.uint64), np.array(d["c"]), d["E0"])
    w = W.WORKLOADS[name]
    h1, eri, ec = w.integrals()
    A, B, c = w.psi()
    return h1, eri, ec, A, B, c, W.stored_e0(name)


def _dev(torch, A, B):
    return torch.tensor(np.stack([A, B], 1).view(np.int64), device="cuda")


@pytest.mark.parametrize("name,C", [("hubbard", 100), ("hubbard", 30), ("random_12e12o", 2000),
                                    ("random_12e12o", 200), ("random_10e14o", 600)])
def test_pt2_equals_oracle(torch_cuda, asci, oracle_mod, name, C):
    torch = torch_cuda
    h1, eri, ec, A, B, c, E0 = _system(name)
    ref = oracle_mod.pt2(oracle_mod.Ints(h1, eri, ec), A, B, c, E0, C)
    e, st = asci.pt2(_dev(torch, A, B), torch.tensor(c, device="cuda"), E0, h1, eri, ec, C)
    assert abs(e - ref) <= 1e-10 * abs(ref), (e, ref)
    res = oracle_mod.search(oracle_mod.Ints(h1, eri, ec), A, B, c, E0, C)
    assert st.unique - st.excluded == len(res.a) and st.selected == 0


def test_pt2_is_independent_of_batching(torch_cuda, asci):
    torch = torch_cuda
    h1, eri, ec, A, B, c, E0 = _system("random_14e20o")
    d, cf = _dev(torch, A, B), torch.tensor(c, device="cuda")
    ref, st0 = asci.pt2(d, cf, E0, h1, eri, ec, 400)
    for bmax, lvl in [(1 << 14, 0), (1 << 16, 3), (1 << 20, 5)]:
        e, st = asci.pt2(d, cf, E0, h1, eri, ec, 400, max_batch_pairs=bmax,
                         max_constraint_level=lvl)
        assert st.batches > st0.batches
        assert e == ref  # exact fixed-point sum: the same bits


@pytest.mark.parametrize("prec", [1, 2])
def test_pt2_precision_variants(torch_cuda, asci, oracle_mod, prec):
    torch = torch_cuda
    h1, eri, ec, A, B, c, E0 = _system("random_12e12o")
    ref = oracle_mod.pt2(oracle_mod.Ints(h1, eri, ec), A, B, c, E0, 2000)
    e, _ = asci.pt2(_dev(torch, A, B), torch.tensor(c, device="cuda"), E0, h1, eri, ec, 2000,
                    precision=prec)
    assert abs(e - ref) <= 1e-6 * abs(ref)


def test_pt2_rejects_vanishing_denominators(torch_cuda, asci):
    """From the Hubbard ring's aufbau determinant with E0 = its H_ii,
    same-occupancy doubles have E0 - H_ii = 0."""
    torch = torch_cuda
    h1, eri, ec = W.hubbard_ring(8, 1.0, 4.0)
    A = np.array([W.aufbau(4)], dtype=np.uint64)
    E0 = float(np.trace(h1[:4, :4]) * 2 + 4 * 4.0)
    with pytest.raises(asci.AsciError, match="PT2 term"):
        asci.pt2(_dev(torch, A, A.copy()), torch.tensor([1.0], device="cuda"), E0, h1, eri, ec, 1)


def test_pt2_with_screening(torch_cuda, asci, oracle_mod):
    """eps_search > 0 screens pairs as Alg. 2 does (|H_ij c_j / (E0 - H_ii)| >
    eps) before the PT2 sum."""
    torch = torch_cuda
    h1, eri, ec, A, B, c, E0 = _system("random_12e12o")
    for eps in (1e-6, 1e-4):
        ref = oracle_mod.pt2(oracle_mod.Ints(h1, eri, ec), A, B, c, E0, 2000, eps)
        e, st = asci.pt2(_dev(torch, A, B), torch.tensor(c, device="cuda"), E0, h1, eri, ec, 2000,
                         eps=eps)
        assert abs(e - ref) <= 1e-9 * abs(ref), (eps, e, ref)
        assert st.surviving < st.generated
