"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run:  python tests/golden/make_golden.py [--modes-only]
Each value is the lowest part of the discrete spectrum of the same Q1
operator the CUDA path applies, computed from the oracle's assembled matrices
by shift-invert Lanczos (scipy ARPACK) -- brute force, independent of ParO.
The oscillator's exact eigenvectors are stored as their 1-D factors
(oracle.separable).
"""
import json
import os
import sys

import numpy as np
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import paro as O  # noqa: E402
from oracle import separable as S  # noqa: E402
from paper_1405_0260_gb300 import workloads as W  # noqa: E402


def lowest(p, k, shift):
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, 0.0)
    vals = spla.eigsh(ops.H, k=k, M=ops.M, sigma=shift, which="LM", tol=1e-14,
                      return_eigenvectors=False)
    return sorted(float(v) for v in vals)


def main(modes_only=False):
    path = os.path.join(HERE, "discrete_spectra.json")
    if modes_only:  # keep the stored Lanczos spectra (about 30 min of ARPACK on 8 cores)
        with open(path) as f:
            out = json.load(f)
        out.pop("harmonic_64_L8_modes", None)
        return _write(path, _modes(out))
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
    _write(path, _modes(out))


def _modes(out):
    # exact eigenvectors of the 64^3 oscillator as Kronecker products of 1-D modes
    # (oracle.separable): the 1-D eigenpairs, the index triple of each of the 20
    # lowest 3-D modes and their shell clusters
    mu, V = S.modes_1d(64, 8.0, 6)
    vals, _ = S.oscillator_modes(64, 8.0, 20)
    out["harmonic_64_L8_modes"] = {
        "what": "1-D generalized eigenpairs (k/2 + m2, m) of the 64-cell axis on [-8,8] (m-orthonormal, "
                "interior nodes); 3-D mode j = v1d[c] (x) v1d[b] (x) v1d[a] for triples[j] = (a, b, c) "
                "(x fastest); clusters: index ranges of the oscillator shells",
        "mu": [float(v) for v in mu],
        "v1d": [[float(x) for x in V[:, j]] for j in range(V.shape[1])],
        "triples": [list(t) for t in S.oscillator_triples(mu, 20)],
        "clusters": [list(c) for c in S.clusters(vals, 0.25)],
    }
    return out


def _write(path, out):
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main(modes_only="--modes-only" in sys.argv)
