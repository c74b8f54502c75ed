"""Writes the stored inputs and expected values under tests/golden/.

Calls only the CPU oracle (and the seeded generators in ``workloads``).
Run from the repository root:  python -m tests.golden.make_golden
"""
from __future__ import annotations

import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def hubbard_start(oracle, norb=8, na=4, nb=4, t=1.0, U=4.0, ndets=100):
    """Start wavefunction of the (8e,8o) Hubbard workload.

    The ``ndets`` determinants of lowest H_ii in the full sector, ties broken by
    the 128-bit key ascending (beta word high), with c the ground vector of the
    CI in that space (largest |c| positive) and E0 its eigenvalue.
    """
    import workloads as W
    from oracle import fock
    h1, eri, ec = W.hubbard_ring(norb, t, U)
    ints = oracle.Ints(h1, eri, ec)
    A, B = fock.sector(norb, na, nb)          # already key ascending
    hii = np.array([oracle.diag(ints, (a, b)) for a, b in zip(A, B)])
    order = np.lexsort((np.arange(len(A)), hii))   # stable: key order among equal H_ii
    sel = order[:ndets]
    pa, pb = A[sel], B[sel]
    E0, c = oracle.ground_state(ints, pa, pb)
    return pa, pb, c, E0


def main():
    import oracle
    pa, pb, c, E0 = hubbard_start(oracle)
    out = {
        "_about": "Start wavefunction of the (8e,8o) periodic Hubbard ring (t=1, U=4): the 100 "
                  "lowest-H_ii determinants (ties by key ascending), CI ground vector and energy. "
                  "Written by tests/golden/make_golden.py from the CPU oracle.",
        "alpha": [int(x) for x in pa], "beta": [int(x) for x in pb],
        "c": [float(x) for x in c], "E0": float(E0),
    }
    with open(os.path.join(HERE, "hubbard_8e8o_psi.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
