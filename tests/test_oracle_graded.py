"""Pins of the oracle on graded tensor-product meshes (Section 2.1: finite element
spaces on locally refined meshes; here the refinement is along each axis).

The assembly of a graded mesh is pinned to an independent construction: the
Kronecker form of the non-uniform 1-D Q1 matrices (written out below from the
1-D element integrals), exact integrals of a linear potential, the separable
oscillator spectrum from 1-D generalized eigenproblems, the uniform mesh as the
special case of equal spacing, Gauss points that integrate cubics exactly, and
the reason for grading at all: at the same number of unknowns, a mesh refined
toward a Coulomb nucleus gives a lower (better) ground-state Ritz value.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import paro as O
from paper_1405_0260_gb300 import workloads as W


def _tri1d(hc, lower, diag_fn, upper):
    """Interior-node matrix of a 1-D Q1 form from the cell sizes hc (len n)."""
    n = hc.size
    d = np.array([diag_fn(hc[i - 1], hc[i]) for i in range(1, n)])
    off = np.array([lower(hc[i]) for i in range(1, n - 1)])
    return sp.diags([off, d, off], [-1, 0, 1]).tocsr()


def k1d(hc):
    return _tri1d(hc, lambda h: -1.0 / h, lambda a, b: 1.0 / a + 1.0 / b, None)


def m1d(hc):
    return _tri1d(hc, lambda h: h / 6.0, lambda a, b: (a + b) / 3.0, None)


def xm1d(nodes):
    """Exact int x phi_i phi_j on the interior nodes (linear weight, non-uniform cells)."""
    n = nodes.size - 1
    A = np.zeros((n + 1, n + 1))
    for e in range(n):
        xe, h = nodes[e], nodes[e + 1] - nodes[e]
        A[e, e] += h * (xe / 3 + h / 12)
        A[e, e + 1] += h * (xe / 6 + h / 12)
        A[e + 1, e] += h * (xe / 6 + h / 12)
        A[e + 1, e + 1] += h * (xe / 3 + h / 4)
    return sp.csr_matrix(A[1:n, 1:n])


def kron3(az, ay, ax):
    return sp.kron(az, sp.kron(ay, ax)).tocsr()


def _graded_mesh(n, L, beta):
    ax = [W.graded_axis(n[d], L[d], beta[d]) for d in range(3)]
    return O.Mesh(n, None, None, coords=tuple(ax))


@pytest.mark.parametrize("n,L,beta", [((6, 5, 7), (2.0, 1.5, 3.0), (1.5, 0.8, 2.5)), ((8, 8, 8), (4.0, 4.0, 4.0),
                                                                                        (2.0, 2.0, 2.0))])
def test_graded_stiffness_and_mass_are_kronecker_products(n, L, beta):
    mesh = _graded_mesh(n, L, beta)
    ops = O.assemble(mesh, np.zeros(8 * n[0] * n[1] * n[2]), 0.0)
    hx, hy, hz = mesh.hc
    K = kron3(m1d(hz), m1d(hy), k1d(hx)) + kron3(m1d(hz), k1d(hy), m1d(hx)) + kron3(k1d(hz), m1d(hy), m1d(hx))
    M = kron3(m1d(hz), m1d(hy), m1d(hx))
    assert abs(ops.K - K).max() < 1e-12 * abs(K).max()
    assert abs(ops.M - M).max() < 1e-14 * abs(M).max()


def test_equal_spacing_is_the_uniform_mesh():
    n, L = (5, 6, 7), (1.0, 2.0, 1.5)
    u = O.Mesh(n, tuple(-v for v in L), L)
    g = O.Mesh(n, None, None, coords=tuple(u.nodes))
    rng = np.random.default_rng(11)
    Vq = rng.standard_normal(8 * n[0] * n[1] * n[2])
    a, b = O.assemble(u, Vq, 0.3), O.assemble(g, Vq, 0.3)
    for A, Bm in ((a.K, b.K), (a.M, b.M), (a.MV, b.MV)):
        assert abs(A - Bm).max() < 1e-13 * abs(A).max()
    assert np.allclose(O.gauss_points(u), O.gauss_points(g), rtol=0, atol=1e-14)


def test_linear_potential_is_the_exact_integral_on_a_graded_mesh():
    n, L, beta = (7, 5, 6), (3.0, 2.0, 2.5), (2.0, 1.0, 1.5)
    mesh = _graded_mesh(n, L, beta)
    X = O.gauss_points(mesh)
    ops = O.assemble(mesh, X[..., 0].ravel(), 0.0)
    hx, hy, hz = mesh.hc
    ref = kron3(m1d(hz), m1d(hy), xm1d(mesh.nodes[0]))
    assert abs(ops.MV - ref).max() < 1e-13 * abs(ref).max()


def test_gauss_points_integrate_cubics_exactly_on_a_graded_mesh():
    mesh = _graded_mesh((6, 5, 4), (2.0, 1.0, 1.5), (1.5, 0.5, 2.0))
    X = O.gauss_points(mesh)
    hz, hy, hx = np.meshgrid(mesh.hc[2], mesh.hc[1], mesh.hc[0], indexing="ij")
    wq = (hx * hy * hz / 8.0)[..., None, None, None]
    f = X[..., 0] ** 3 * X[..., 1] ** 2 + X[..., 2] ** 3
    Lx, Ly, Lz = 2.0, 1.0, 1.5
    exact = 0.0 * (2 * Ly ** 3 / 3) * (2 * Lz) + 0.0  # odd powers of x and z integrate to zero on a symmetric box
    assert abs(np.sum(wq * f) - exact) < 1e-12
    g = X[..., 0] ** 2 * X[..., 1] ** 2 * X[..., 2] ** 2
    exact = (2 * Lx ** 3 / 3) * (2 * Ly ** 3 / 3) * (2 * Lz ** 3 / 3)
    assert abs(np.sum(wq * g) - exact) < 1e-12 * exact


def test_graded_oscillator_spectrum_is_separable():
    # V = r^2 / 2 at the Gauss points: H = a x m x m + m x a x m + m x m x a with
    # non-uniform 1-D matrices a = k / 2 + m2, so the spectrum is every sum of
    # three 1-D generalized eigenvalues (one per axis)
    n, L, beta = (8, 7, 9), (4.0, 3.5, 4.5), (1.5, 1.0, 2.0)
    mesh = _graded_mesh(n, L, beta)
    X = O.gauss_points(mesh)
    Vq = 0.5 * (X ** 2).sum(axis=-1).ravel()
    ops = O.assemble(mesh, Vq, 0.0)
    dense = sla.eigh(ops.H.toarray(), ops.M.toarray(), eigvals_only=True)
    g = (1 - 1 / np.sqrt(3)) / 2, (1 + 1 / np.sqrt(3)) / 2
    mu = []
    for d in range(3):
        nodes = mesh.nodes[d]
        nc = nodes.size - 1
        m2 = np.zeros((nc + 1, nc + 1))
        for e in range(nc):
            h = nodes[e + 1] - nodes[e]
            for q in range(2):
                xq = nodes[e] + h * g[q]
                l = (1 - g[q], g[q])
                for a in range(2):
                    for b in range(2):
                        m2[e + a, e + b] += 0.5 * h * 0.5 * xq ** 2 * l[a] * l[b]
        a1 = 0.5 * k1d(mesh.hc[d]).toarray() + m2[1:nc, 1:nc]
        mu.append(sla.eigh(a1, m1d(mesh.hc[d]).toarray(), eigvals_only=True))
    sums = np.sort((mu[0][:, None, None] + mu[1][None, :, None] + mu[2][None, None, :]).ravel())
    assert np.max(np.abs(dense[:30] - sums[:30]) / sums[:30]) < 1e-11


def test_grading_toward_the_nucleus_lowers_the_ground_state():
    # the point of an adapted mesh: with the same 15^3 unknowns, cells graded toward
    # a Coulomb nucleus give a lower Ritz value (closer to the exact -1/2) than
    # uniform cells; the discrete value stays above -1/2 (conforming)
    def ground(p):
        mesh = O.Mesh(p.n, p.lo, p.hi, coords=p.coords)
        ops = O.assemble(mesh, p.Vq, 0.0)
        return spla.eigsh(ops.H, k=1, M=ops.M, sigma=-0.6, which="LM", return_eigenvectors=False)[0]

    e_graded = ground(W.graded_hydrogen(nc=16, L=10.0, beta=2.5))
    e_uniform = ground(W.graded_hydrogen(nc=16, L=10.0, beta=0.0))
    assert -0.5 < e_graded < e_uniform, (e_graded, e_uniform)
    assert (e_graded + 0.5) < 0.5 * (e_uniform + 0.5)
