"""The error path of a scratch allocation failure (GPU; the failure is made on
the host by the library's fault injector, not by exhausting the device): the
call returns ASCI_ENOMEM after releasing its scratch, and the next call gives
the same result as before, bit for bit."""
import numpy as np
import pytest

import workloads as W
from tests._parity import key_order, to_u64_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def asci():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2303_05688_gb300 as m
    m.load()
    return m


def _case(torch):
    w = W.WORKLOADS["random_12e12o"]
    h1, eri, ec = w.integrals()
    A, B, c = w.psi()
    d = torch.tensor(np.stack([A, B], 1).astype(np.int64), device="cuda")
    return (d, torch.tensor(c, device="cuda"), W.stored_e0(w.name),
            torch.tensor(h1, device="cuda"), torch.tensor(eri, device="cuda"), ec)


def _same(r1, r2):
    a1, b1 = to_u64_pairs(r1[0])
    a2, b2 = to_u64_pairs(r2[0])
    o1, o2 = key_order(a1, b1), key_order(a2, b2)
    return (np.array_equal(a1[o1], a2[o2]) and np.array_equal(b1[o1], b2[o2])
            and np.array_equal(r1[1].cpu().numpy()[o1], r2[1].cpu().numpy()[o2]))


@pytest.mark.parametrize("entry", ["search", "pt2"])
def test_injected_allocation_failure_returns_enomem_then_recovers(asci, entry):
    import torch
    lib = asci.load()
    d, c, E0, h1, eri, ec = _case(torch)
    run = ((lambda: asci.search(d, c, E0, h1, eri, ec, 200, 5000)) if entry == "search"
           else (lambda: asci.pt2(d, c, E0, h1, eri, ec, 200)))
    ref = run()
    failed = 0
    for after in (0, 1, 4, 11, 30, 70):
        lib.asci_debug_fail_allocation(after)
        try:
            run()
        except asci.AsciError as e:
            assert e.code == -2 and "injected allocation failure" in str(e), str(e)
            failed += 1
        finally:
            lib.asci_debug_fail_allocation(-1)
        torch.cuda.synchronize()
        got = run()  # the library works normally after the failure
        if entry == "search":
            assert _same(ref, got)
        else:
            assert got[0] == ref[0]
    assert failed >= 4
