"""Writes tests/golden/chain64_oracle.json from the FP64 oracle only.

Run from the repository root:  python tests/golden/make_golden.py
The stored values are the oracle's (recursion-exact function, 12 steps, and
Fermi-Dirac) for the seeded 64-site chain; no value comes from the CUDA path.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthetic  # noqa: E402


def main():
    p = synthetic.workload("chain64")
    out = {"workload": "chain64", "N": p.N, "beta": p.beta, "nocc": p.nocc, "n": p.n}
    for kind, n in (("rec", p.n), ("fd", None)):
        r = oracle.solve(p.H0, p.H1, p.beta, p.nocc, n=n, kind=kind)
        out[kind] = {
            "mu": r["mu"],
            "mu1": float(r["mu1"][0]),
            "alpha": float(r["alpha"][0]),
            "omega": r["omega"],
            "P0_fro": float(np.linalg.norm(r["P0"])),
            "P1_fro": float(np.linalg.norm(r["P1"][0])),
            "P0_diag_head": [float(v) for v in np.diag(r["P0"])[:8]],
            "P1_diag_head": [float(v) for v in np.diag(r["P1"][0])[:8]],
        }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "chain64_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
