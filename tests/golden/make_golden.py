"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run:  python tests/golden/make_golden.py
Each value is the lowest part of the discrete spectrum of the same Q1
operator the CUDA path applies, computed from the oracle's assembled matrices
by shift-invert Lanczos (scipy ARPACK) -- brute force, independent of ParO.
"""
import json
import os
import sys

import numpy as np
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import paro as O  # noqa: E402
from paper_1405_0260_gb300 import workloads as W  # noqa: E402


def lowest(p, k, shift):
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, 0.0)
    vals = spla.eigsh(ops.H, k=k, M=ops.M, sigma=shift, which="LM", tol=1e-14,
                      return_eigenvectors=False)
    return sorted(float(v) for v in vals)


def main():
    out = {}
    p = W.hydrogen(nc=32, L=10.0, N=5, seed=1000)
    out["hydrogen_32_L10"] = {
        "what": "lowest 6 discrete eigenvalues, H = K/2 + M_V, V=-1/r from a nucleus at (h/2,h/2,h/2), "
                "[-10,10]^3, 32^3 Q1 cells, Dirichlet",
        "values": lowest(p, 6, -0.6),
    }
    p = W.harmonic(nc=32, L=8.0, N=1, seed=1)
    out["harmonic_32_L8"] = {
        "what": "lowest 20 discrete eigenvalues, V=r^2/2, [-8,8]^3, 32^3 Q1 cells, Dirichlet",
        "values": lowest(p, 20, 1.0),
    }
    p = W.harmonic(nc=64, L=8.0, N=1, seed=1)
    out["harmonic_64_L8"] = {
        "what": "lowest 20 discrete eigenvalues, V=r^2/2, [-8,8]^3, 64^3 Q1 cells, Dirichlet",
        "values": lowest(p, 20, 1.0),
    }
    with open(os.path.join(HERE, "discrete_spectra.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
