"""Exact discrete eigenpairs of the Q1 harmonic oscillator from 1-D problems.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain numpy/scipy,
float64.

The fixed-potential source problems of Algorithm A.1 (Appendix) converge to
eigenpairs of the discrete pencil (H, M), H = K/2 + M_V (eq. 2.7 with a fixed
potential).  For V = (x^2 + y^2 + z^2)/2 sampled at the tensor 2-point Gauss
points of a uniform box mesh, every matrix is a sum of Kronecker products of
1-D matrices on the interior nodes of one axis:

    M   = m (x) m (x) m
    H   = a (x) m (x) m + m (x) a (x) m + m (x) m (x) a,   a = k/2 + m2,

with k, m the 1-D Q1 stiffness and mass matrices and m2 the 1-D Gauss sums of
(x^2/2) phi_i phi_j (2-point Gauss integrates the Q1 mass exactly, so the
factor of an axis the potential term does not depend on is m itself).  If
a v = mu m v, then (H, M) has the eigenvector v_c (x) v_b (x) v_a with
eigenvalue mu_a + mu_b + mu_c: the whole discrete spectrum and an exact basis
of every eigenspace come from one small 1-D generalized eigenproblem.

This gives reference vectors at sizes where the ParO oracle itself is too slow
to run to convergence (the 64^3 x 20 headline workload).  Degenerate and
nearly degenerate eigenvalues (the cubic mesh splits the oscillator shells
w (n + 3/2) only slightly) are compared as subspaces of whole clusters.

Pins (tests/test_oracle_separable.py): dense generalized eigh of the oracle's
3-D assembly on a small mesh (values and cluster subspaces), eigen-residuals
with the oracle's assembled operators at 64^3, the stored shift-invert Lanczos
spectrum, and M-orthonormality.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


def _gauss01():
    """2-point Gauss rule on [0, 1]: abscissae (1 -/+ 1/sqrt 3)/2, weights 1/2."""
    t = np.array([(1.0 - 1.0 / math.sqrt(3.0)) / 2.0, (1.0 + 1.0 / math.sqrt(3.0)) / 2.0])
    return t, np.array([0.5, 0.5])


def matrices_1d(nc: int, L: float):
    """1-D Q1 matrices on [-L, L] with nc cells, restricted to the nc-1 interior nodes.

    Element by element with the 2-point Gauss rule (l0 = 1 - t, l1 = t):
      k[i, j]  = sum_e int phi_i' phi_j'
      m[i, j]  = sum_e int phi_i phi_j
      m2[i, j] = sum_e sum_q w_q h (x_q^2 / 2) phi_i(x_q) phi_j(x_q)
    Returns (k, m, m2) as dense arrays.
    """
    h = 2.0 * L / nc
    t, w = _gauss01()
    lq = np.stack([1.0 - t, t])  # lq[a, q]
    dl = np.array([-1.0, 1.0]) / h  # derivative of l_a in x
    k = np.zeros((nc + 1, nc + 1))
    m = np.zeros((nc + 1, nc + 1))
    m2 = np.zeros((nc + 1, nc + 1))
    for e in range(nc):
        xq = -L + h * (e + t)
        for a in range(2):
            for b in range(2):
                k[e + a, e + b] += h * np.sum(w) * dl[a] * dl[b]
                m[e + a, e + b] += h * np.sum(w * lq[a] * lq[b])
                m2[e + a, e + b] += h * np.sum(w * 0.5 * xq ** 2 * lq[a] * lq[b])
    s = slice(1, nc)
    return k[s, s], m[s, s], m2[s, s]


def modes_1d(nc: int, L: float, k: int):
    """Lowest k generalized eigenpairs of (k/2 + m2, m): values ascending, vectors m-orthonormal."""
    k1, m1, m2 = matrices_1d(nc, L)
    mu, V = sla.eigh(0.5 * k1 + m2, m1)
    return mu[:k], V[:, :k]


def oscillator_triples(mu: np.ndarray, count: int):
    """The `count` lowest index triples (a, b, c) by mu_a + mu_b + mu_c (ties: lexicographic)."""
    n = mu.size
    cand = [(mu[a] + mu[b] + mu[c], (a, b, c)) for a in range(n) for b in range(n) for c in range(n)]
    cand.sort(key=lambda v: (v[0], v[1]))
    return [abc for _, abc in cand[:count]]


def oscillator_modes(nc: int, L: float, count: int):
    """Lowest `count` eigenpairs of the discrete 3-D oscillator on [-L, L]^3 with nc^3 cells.

    Returns (values, vectors): vectors (n_interior, count), interior nodes with x
    fastest (the unknown order of ``oracle.paro.Mesh``), M-orthonormal; column j
    is v_c (x) v_b (x) v_a for triple (a, b, c) = (x, y, z) mode indices.
    """
    nmode = 1
    while nmode ** 3 < count or (nmode * (nmode + 1) * (nmode + 2)) // 6 < count:
        nmode += 1
    nmode = min(nmode + 2, nc - 1)
    mu, V = modes_1d(nc, L, nmode)
    trip = oscillator_triples(mu, count)
    vals = np.array([mu[a] + mu[b] + mu[c] for a, b, c in trip])
    vecs = np.stack([np.kron(V[:, c], np.kron(V[:, b], V[:, a])) for a, b, c in trip], axis=1)
    return vals, vecs


def clusters(values: np.ndarray, gap: float):
    """Consecutive index ranges [lo, hi) of sorted values, split where neighbours differ by more than gap."""
    out = []
    lo = 0
    for i in range(1, len(values) + 1):
        if i == len(values) or values[i] - values[i - 1] > gap:
            out.append((lo, i))
            lo = i
    return out
