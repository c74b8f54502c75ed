"""Writes workloads/e0.json: the E0 input of each random workload.

E0 is an input of the search (Eq. 1's E_k = <psi|H psi>).  For the random
workloads it is the variational energy of the leading K = min(|psi|, 2000)
determinants of the seeded wavefunction, with their coefficients, computed by
the CPU oracle.  Run from the repository root:  python -m workloads.make_e0
"""
from __future__ import annotations

import json
import os

import workloads as W

K = 2000


def main():
    import oracle
    out = {"_about": "E0 per random workload: <psi_K|H|psi_K>/<psi_K|psi_K> over the leading "
                     f"K = min(|psi|, {K}) determinants, from the CPU oracle (workloads/make_e0.py)."}
    for name, w in W.WORKLOADS.items():
        if w.kind != "random":
            continue
        h1, eri, ec = w.integrals()
        A, B, c = w.psi()
        k = min(K, len(A))
        E0 = oracle.variational_energy(oracle.Ints(h1, eri, ec), A[:k], B[:k], c[:k])
        out[name] = {"E0": E0, "K": k}
        print(name, E0)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "e0.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
