"""Pins of the oracle's adaptive loop (Section 2.1: Solve -> Estimate -> Mark ->
Refine) on tensor-product meshes, each against something other than itself:

- the indicators of one Q1 hat function against hand-computed integrals (the
  element term (lambda - V)^2 int phi^2 = (lambda - V)^2 prod h_d / 3 per cell;
  the normal-derivative jumps (1/h_l + 1/h_r) on the node's planes and 1/h on
  the neighbouring planes, times int phi_y^2 int phi_z^2 per face cell), on a
  uniform and a graded mesh, and zero away from the hat's support;
- Doerfler marking (eq. 2.2) against brute force over all subsets of small
  random indicator sets (least cardinality reaching theta of the total),
  maximum marking (eq. 2.3) against its definition with theta on eta (not
  eta^2);
- refinement: every marked cell is bisected along all three axes, old nodes
  are kept, unmarked intervals are not split;
- transfer: nested spaces make it exact (coarse -> fine -> finer equals
  coarse -> finer, and old nodes keep their values);
- the loop: on nested meshes the lowest discrete eigenvalue never increases
  (Rayleigh-Ritz on a larger space), and Doerfler marking on a Coulomb problem
  marks the cells at the nucleus first.
"""
import itertools

import numpy as np
import scipy.linalg as sla

from oracle import adapt as A
from oracle import paro as O
from paper_1405_0260_gb300 import workloads as W


def _hat_case(coords):
    mesh = O.Mesh((len(coords[0]) - 1, len(coords[1]) - 1, len(coords[2]) - 1), None, None, coords=coords)
    nx, ny, nz = mesh.n
    # hat at interior node (i, j, k)
    i, j, k = 2, 2, 3
    U = np.zeros((mesh.n_interior, 1))
    U[mesh.interior_index(i, j, k), 0] = 1.0
    c, lam = 0.7, 1.9
    Vq = np.full(nx * ny * nz * 8, c)
    eta2 = A.indicators(mesh, Vq, np.array([lam]), U)
    hx, hy, hz = mesh.hc
    return mesh, (i, j, k), c, lam, eta2, hx, hy, hz


def _expected_hat(mesh, node, c, lam, hx, hy, hz):
    """Per-cell indicators of the hat, from hand integrals."""
    nx, ny, nz = mesh.n
    i, j, k = node
    out = np.zeros((nz, ny, nx))
    # element terms on the 8 cells around the node
    for cz in (k - 1, k):
        for cy in (j - 1, j):
            for cx in (i - 1, i):
                diam2 = hx[cx] ** 2 + hy[cy] ** 2 + hz[cz] ** 2
                out[cz, cy, cx] += diam2 * (lam - c) ** 2 * hx[cx] * hy[cy] * hz[cz] / 27.0

    def add_face(axis, plane, jump_coef):
        # the jump is jump_coef * phi_a * phi_b on each face cell around the node's
        # line; int (phi_a phi_b)^2 = h_a / 3 * h_b / 3 over a face cell touching it
        if axis == 0:
            la, lb, ha, hb = (j - 1, j), (k - 1, k), hy, hz
        elif axis == 1:
            la, lb, ha, hb = (i - 1, i), (k - 1, k), hx, hz
        else:
            la, lb, ha, hb = (i - 1, i), (j - 1, j), hx, hy
        for a in la:
            for b in lb:
                integral = jump_coef ** 2 * ha[a] * hb[b] / 9.0
                hF = np.sqrt(ha[a] ** 2 + hb[b] ** 2)
                share = 0.5 * hF * 0.25 * integral
                for cell in (plane - 1, plane):  # the two cells sharing the face
                    if axis == 0:
                        out[b, a, cell] += share
                    elif axis == 1:
                        out[b, cell, a] += share
                    else:
                        out[cell, b, a] += share

    for axis, (p, h) in enumerate(((i, hx), (j, hy), (k, hz))):
        add_face(axis, p, 1.0 / h[p - 1] + 1.0 / h[p])  # the node's own plane
        add_face(axis, p - 1, 1.0 / h[p - 1])             # the plane before
        add_face(axis, p + 1, 1.0 / h[p])                 # the plane after
    return out


def test_indicators_of_a_hat_function_uniform():
    ax = np.linspace(-2.0, 2.0, 7)
    mesh, node, c, lam, eta2, hx, hy, hz = _hat_case((ax, ax, np.linspace(-2.0, 2.0, 8)))
    exp = _expected_hat(mesh, node, c, lam, hx, hy, hz)
    assert np.allclose(eta2, exp, rtol=1e-13, atol=1e-15), np.max(np.abs(eta2 - exp))
    assert np.count_nonzero(eta2) == np.count_nonzero(exp)


def test_indicators_of_a_hat_function_graded():
    cx = np.array([-3.0, -1.5, -0.6, 0.0, 0.4, 1.5, 3.0])
    cy = np.array([-2.0, -0.9, -0.2, 0.5, 1.1, 2.5])
    cz = np.array([-1.0, -0.7, -0.3, 0.1, 0.2, 0.8, 1.6])
    mesh, node, c, lam, eta2, hx, hy, hz = _hat_case((cx, cy, cz))
    exp = _expected_hat(mesh, node, c, lam, hx, hy, hz)
    assert np.allclose(eta2, exp, rtol=1e-13, atol=1e-15), np.max(np.abs(eta2 - exp))


def test_dorfler_marking_is_a_least_cardinality_set():
    rng = np.random.default_rng(8100)
    for trial in range(40):
        n = int(rng.integers(1, 9))
        e = rng.random(n) ** 3
        if trial % 5 == 0:
            e[: n // 2] = e[0]  # ties
        theta = float(rng.uniform(0.05, 0.95))
        m = A.mark_dorfler(e, theta)
        assert e[m].sum() >= theta * e.sum()
        best = min(len(S) for r in range(n + 1) for S in itertools.combinations(range(n), r)
                   if e[list(S)].sum() >= theta * e.sum())
        assert m.sum() == best, (e, theta, m)


def test_maximum_marking_uses_theta_on_eta():
    eta = np.array([1.0, 0.7, 0.5, 0.3, 0.05])
    m = A.mark_maximum(eta ** 2, 0.6)
    assert m.tolist() == [True, True, False, False, False]  # eta >= 0.6 (theta on eta^2 would drop 0.7)
    m = A.mark_maximum(eta ** 2, 0.45)
    assert m.tolist() == [True, True, True, False, False]


def test_refinement_bisects_the_marked_cells_and_keeps_old_nodes():
    ax = np.linspace(0.0, 1.0, 5)
    mesh = O.Mesh((4, 4, 4), None, None, coords=(ax, ax ** 1.5, np.sqrt(ax)))
    marked = np.zeros((4, 4, 4), dtype=bool)
    marked[1, 2, 3] = True  # [cz][cy][cx]
    marked[3, 2, 0] = True
    xs, ys, zs = A.refine_coords(mesh, marked)
    assert len(xs) == 5 + 2 and len(ys) == 5 + 1 and len(zs) == 5 + 2
    for new, old, hit in ((xs, mesh.nodes[0], (0, 3)), (ys, mesh.nodes[1], (2,)), (zs, mesh.nodes[2], (1, 3))):
        assert set(old.tolist()) <= set(new.tolist())
        for k in range(len(old) - 1):
            inside = new[(new > old[k]) & (new < old[k + 1])]
            if k in hit:
                assert inside.tolist() == [0.5 * (old[k] + old[k + 1])]
            else:
                assert inside.size == 0


def test_transfer_is_exact_between_nested_spaces():
    rng = np.random.default_rng(8200)
    ax = np.linspace(-1.0, 1.0, 6)
    coarse = O.Mesh((5, 5, 5), None, None, coords=(ax, ax, ax))
    U = rng.standard_normal((coarse.n_interior, 3))
    m1 = rng.random((5, 5, 5)) < 0.2
    c1 = A.refine_coords(coarse, m1)
    fine = O.Mesh((len(c1[0]) - 1, len(c1[1]) - 1, len(c1[2]) - 1), None, None, coords=c1)
    m2 = rng.random((fine.n[2], fine.n[1], fine.n[0])) < 0.3
    c2 = A.refine_coords(fine, m2)
    finer = O.Mesh((len(c2[0]) - 1, len(c2[1]) - 1, len(c2[2]) - 1), None, None, coords=c2)
    direct = A.transfer(coarse, finer, U)
    twice = A.transfer(fine, finer, A.transfer(coarse, fine, U))
    assert np.max(np.abs(direct - twice)) < 1e-13
    # old nodes keep their values
    Uf = A.transfer(coarse, fine, U)
    Wc, Wf = A.nodal(coarse, U), A.nodal(fine, Uf)
    ix = [np.searchsorted(fine.nodes[d], coarse.nodes[d]) for d in range(3)]
    assert np.max(np.abs(Wf[np.ix_(ix[2], ix[1], ix[0])] - Wc)) < 1e-14


def _lowest(mesh, Vq):
    ops = O.assemble(mesh, Vq, 0.0)
    return sla.eigh(ops.H.toarray(), ops.M.toarray(), eigvals_only=True, subset_by_index=[0, 0])[0], ops


def _coulomb_vq(mesh, R):
    x, y, z = W.gauss_point_coords(mesh.n, mesh.lo, mesh.hi, tuple(mesh.nodes))
    return np.ascontiguousarray((-1.0 / np.sqrt((x - R[0]) ** 2 + (y - R[1]) ** 2 + (z - R[2]) ** 2)).ravel())


def test_adaptive_loop_lowers_the_ground_state_on_nested_spaces():
    """A linear potential (2-point Gauss integrates V phi_i phi_j exactly, so every
    mesh discretises the same form): refined meshes contain the coarse space and
    the lowest discrete eigenvalue cannot rise."""
    ax = np.linspace(-3.0, 3.0, 7)
    mesh = O.Mesh((6, 6, 6), None, None, coords=(ax, ax, ax))
    prev = np.inf
    for step in range(4):
        x, y, z = W.gauss_point_coords(mesh.n, mesh.lo, mesh.hi, tuple(mesh.nodes))
        Vq = np.ascontiguousarray((0.8 * x - 0.3 * y + 0.5 * z).ravel())
        lam, ops = _lowest(mesh, Vq)
        assert lam <= prev + 1e-12, (step, lam, prev)
        prev = lam
        w, V = sla.eigh(ops.H.toarray(), ops.M.toarray(), subset_by_index=[0, 0])
        eta2 = A.indicators(mesh, Vq, w, V)
        marked = A.mark_dorfler(eta2, 0.4)
        assert 0 < marked.sum() < marked.size
        c = A.refine_coords(mesh, marked)
        mesh = O.Mesh((len(c[0]) - 1, len(c[1]) - 1, len(c[2]) - 1), None, None, coords=c)


def test_indicators_peak_at_the_nucleus():
    """Coulomb potential off the nodes: the largest indicator of the ground state
    sits in the cell holding the nucleus or next to it."""
    R = (0.3, -0.2, 0.1)
    ax = np.linspace(-6.0, 6.0, 9)
    mesh = O.Mesh((8, 8, 8), None, None, coords=(ax, ax, ax))
    Vq = _coulomb_vq(mesh, R)
    _, ops = _lowest(mesh, Vq)
    w, V = sla.eigh(ops.H.toarray(), ops.M.toarray(), subset_by_index=[0, 0])
    eta2 = A.indicators(mesh, Vq, w, V)
    top = np.unravel_index(np.argmax(eta2), eta2.shape)  # (cz, cy, cx)
    for d, (cidx, coord) in enumerate(zip(top[::-1], R)):
        near = np.searchsorted(mesh.nodes[d], coord) - 1
        assert abs(cidx - near) <= 1, (top, R)
