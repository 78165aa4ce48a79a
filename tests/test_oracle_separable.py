"""Pins of oracle.separable (exact discrete oscillator eigenpairs from 1-D problems).

The reference vectors of the headline parity test come from this module; these
CPU tests tie it to brute force on the oracle's own 3-D assembly and to the
stored shift-invert Lanczos spectrum, so a wrong 1-D matrix, a transposed
Kronecker order or a dropped potential term fails here.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import paro as O
from oracle import separable as S
from paper_1405_0260_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _ops(nc, L):
    p = W.harmonic(nc=nc, L=L, N=1, seed=1)
    return O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, 0.0)


def test_modes_match_dense_eigh_of_the_assembled_operator():
    # brute force: dense generalized eigh of the oracle's element-by-element 3-D assembly
    nc, L, count = 8, 4.0, 20
    ops = _ops(nc, L)
    w, V = sla.eigh(ops.H.toarray(), ops.M.toarray())
    vals, vecs = S.oscillator_modes(nc, L, count)
    assert np.max(np.abs(vals - w[:count]) / np.abs(w[:count])) < 1e-11
    # each cluster of (nearly) equal values spans the same subspace
    for a, b in S.clusters(vals, 1e-8):
        ang = O.subspace_angles_M(ops.M, vecs[:, a:b], V[:, a:b])
        assert np.max(ang) < 1e-7, (a, b, ang)


def test_modes_are_m_orthonormal_eigenvectors_at_the_headline_size():
    nc, L, count = 64, 8.0, 20
    ops = _ops(nc, L)
    vals, vecs = S.oscillator_modes(nc, L, count)
    MV = ops.M @ vecs
    assert np.max(np.abs(vecs.T @ MV - np.eye(count))) < 1e-12
    res = ops.H @ vecs - MV * vals[None, :]
    rel = np.linalg.norm(res, axis=0) / np.linalg.norm(MV, axis=0)
    assert np.max(rel) < 1e-10, rel
    # the spectrum stored from shift-invert Lanczos on the same assembly
    with open(os.path.join(HERE, "golden", "discrete_spectra.json")) as f:
        gold = np.array(json.load(f)["harmonic_64_L8"]["values"][:count])
    assert np.max(np.abs(vals - gold)) < 1e-9


def test_shell_clusters_of_the_headline_workload():
    # 20 orbitals fill the oscillator shells n <= 3 (1 + 3 + 6 + 10 states);
    # the shells w (n + 3/2) stay about 1 Ha apart, the mesh splits each by < 0.1
    vals, _ = S.oscillator_modes(64, 8.0, 21)
    cl = S.clusters(vals[:20], 0.25)
    assert cl == [(0, 1), (1, 4), (4, 10), (10, 20)]
    assert vals[20] - vals[19] > 0.9


def test_stored_modes_match_the_oracle():
    with open(os.path.join(HERE, "golden", "discrete_spectra.json")) as f:
        g = json.load(f)["harmonic_64_L8_modes"]
    mu, V = S.modes_1d(64, 8.0, len(g["mu"]))
    assert np.max(np.abs(np.array(g["mu"]) - mu)) < 1e-13
    V1 = np.array(g["v1d"]).T
    # eigenvectors are defined up to sign
    s = np.sign(np.sum(V1 * V, axis=0))
    assert np.max(np.abs(V1 - V * s[None, :])) < 1e-12
    vals, _ = S.oscillator_modes(64, 8.0, 20)
    trip = S.oscillator_triples(mu, 20)
    assert [list(t) for t in trip] == g["triples"]
    assert [list(c) for c in S.clusters(vals, 0.25)] == g["clusters"]


@pytest.mark.parametrize("count", [1, 4, 10])
def test_small_counts_are_prefixes(count):
    vals, vecs = S.oscillator_modes(16, 6.0, count)
    v20, _ = S.oscillator_modes(16, 6.0, 20)
    assert np.allclose(vals, v20[:count], rtol=0, atol=1e-12)
    assert vecs.shape == (15 ** 3, count)
