"""The seeded input recipes (CPU only).

Every GPU test, the bench and the oracle consume the arrays of
paper_1405_0260_gb300/workloads.py.  These tests pin that module to the
workload definitions it states, by properties that do not retype its code:
exact Gauss quadrature of polynomials (2-point Gauss is exact to degree 3 per
axis), the distance of the Gauss points from a cell centre, the stated node
order, the seeded draw order, and the ranges and separations of the nuclei.
"""
import math

import numpy as np
import pytest

from paper_1405_0260_gb300 import workloads as W


def _cell_weight(p):
    return float(np.prod(p.h)) / 8.0


def test_gauss_points_integrate_cubic_polynomials_exactly():
    n, lo, hi = (3, 4, 5), (-1.0, 0.0, -2.0), (2.0, 1.5, 0.5)
    x, y, z = W.gauss_point_coords(n, lo, hi)
    w = np.prod([(hi[d] - lo[d]) / n[d] for d in range(3)]) / 8.0
    f = x ** 3 * y ** 2 * z + 2.0 * x * z ** 3 - y ** 3 + 1.0

    def I(a, b, k):  # integral of t^k over [a, b]
        return (b ** (k + 1) - a ** (k + 1)) / (k + 1)

    exact = (I(lo[0], hi[0], 3) * I(lo[1], hi[1], 2) * I(lo[2], hi[2], 1)
             + 2.0 * I(lo[0], hi[0], 1) * I(lo[1], hi[1], 0) * I(lo[2], hi[2], 3)
             - I(lo[0], hi[0], 0) * I(lo[1], hi[1], 3) * I(lo[2], hi[2], 0)
             + I(lo[0], hi[0], 0) * I(lo[1], hi[1], 0) * I(lo[2], hi[2], 0))
    assert abs(w * f.sum() - exact) < 1e-12 * max(1.0, abs(exact))


def test_gauss_point_order_is_cell_major_then_qz_qy_qx():
    n, lo, hi = (3, 4, 5), (0.0, 0.0, 0.0), (3.0, 4.0, 5.0)  # unit cells
    x, y, z = W.gauss_point_coords(n, lo, hi)
    a, b = (1 - 1 / math.sqrt(3)) / 2, (1 + 1 / math.sqrt(3)) / 2
    # flat index ((((cz*ny + cy)*nx + cx)*2 + qz)*2 + qy)*2 + qx
    X, Y, Z = x.ravel(), y.ravel(), z.ravel()
    for cz, cy, cx, qz, qy, qx in [(0, 0, 0, 0, 0, 1), (4, 3, 2, 1, 0, 1), (2, 1, 0, 0, 1, 0)]:
        k = ((((cz * 4 + cy) * 3 + cx) * 2 + qz) * 2 + qy) * 2 + qx
        assert X[k] == pytest.approx(cx + (a, b)[qx], abs=1e-15)
        assert Y[k] == pytest.approx(cy + (a, b)[qy], abs=1e-15)
        assert Z[k] == pytest.approx(cz + (a, b)[qz], abs=1e-15)


def test_interior_node_order_matches_the_stated_row_formula():
    n, lo, hi = (3, 4, 5), (0.0, 0.0, 0.0), (3.0, 4.0, 5.0)
    xyz = W.interior_node_coords(n, lo, hi)
    nx, ny, nz = n
    assert xyz.shape == ((nx - 1) * (ny - 1) * (nz - 1), 3)
    for i in range(1, nx):
        for j in range(1, ny):
            for k in range(1, nz):
                row = ((k - 1) * (ny - 1) + (j - 1)) * (nx - 1) + (i - 1)
                assert tuple(xyz[row]) == (float(i), float(j), float(k))


def test_gaussian_orbitals_draw_widths_then_centres():
    n, lo, hi, N = (6, 6, 6), (-3.0,) * 3, (3.0,) * 3, 4
    U = W.gaussian_orbitals(n, lo, hi, N, np.random.default_rng(11))
    rng = np.random.default_rng(11)
    w = rng.uniform(0.5, 3.0, size=N)
    c = rng.uniform(-1.0, 1.0, size=(N, 3))
    assert np.all((w >= 0.5) & (w <= 3.0)) and np.all(np.abs(c) <= 1.0)
    xyz = W.interior_node_coords(n, lo, hi)
    for row in (0, 17, 62, xyz.shape[0] - 1):
        for i in range(N):
            d2 = sum((xyz[row, a] - c[i, a]) ** 2 for a in range(3))
            assert U[row, i] == pytest.approx(math.exp(-d2 / (2 * w[i] ** 2)), rel=1e-14)
    assert np.all(U > 0) and np.all(U <= 1)


def test_hydrogen_nucleus_sits_at_a_cell_centre():
    p = W.hydrogen()
    assert p.n == (32, 32, 32) and p.lo == (-10.0,) * 3 and p.hi == (10.0,) * 3
    assert p.N == 5 and p.sigma == 2.0 and p.tol == 1e-8
    h = 20.0 / 32
    assert np.allclose(p.nuclei[0, :3], [h / 2] * 3) and p.nuclei[0, 3] == 1.0
    # the eight Gauss points of the nucleus's cell are the nearest ones, each h/2 away
    assert np.min(p.Vq) == pytest.approx(-2.0 / h, rel=1e-13)
    assert np.sum(np.isclose(p.Vq, -2.0 / h, rtol=1e-12)) == 8
    assert np.all(p.Vq < 0) and np.all(np.isfinite(p.Vq))
    assert np.max(p.Vq) == pytest.approx(-1.0 / np.max(np.linalg.norm(
        np.stack([c.ravel() for c in W.gauss_point_coords(p.n, p.lo, p.hi)], 1) - h / 2, axis=1)))


def test_harmonic_potential_integrates_to_the_closed_form():
    p = W.harmonic(nc=16, L=8.0, N=3)
    # int over [-L, L]^3 of r^2 / 2 = 4 L^5 (2-point Gauss is exact for quadratics)
    assert _cell_weight(p) * p.Vq.sum() == pytest.approx(4.0 * 8.0 ** 5, rel=1e-13)
    d = W.harmonic()
    assert d.n == (64, 64, 64) and d.N == 20 and d.sigma == 0.0 and d.lo == (-8.0,) * 3
    assert d.U0.shape == (63 ** 3, 20)


def test_cluster_recipe():
    p = W.cluster(nc=16)  # the nuclei are drawn before anything depends on the mesh
    nuc = p.nuclei
    assert nuc.shape == (8, 4)
    assert np.all(np.abs(nuc[:, :3]) <= 6.0)
    assert set(np.unique(nuc[:, 3])).issubset({1.0, 2.0, 3.0, 4.0})
    d = np.linalg.norm(nuc[:, None, :3] - nuc[None, :, :3], axis=2) + np.eye(8) * 1e9
    assert np.min(d) >= 2.0
    assert p.n_occ == math.ceil(nuc[:, 3].sum() / 2) and p.N == p.n_occ + 8
    assert p.lo == (-12.0,) * 3 and p.hi == (12.0,) * 3
    assert np.array_equal(W.cluster(nc=24).nuclei, nuc)
    # softened wells: at every Gauss point V is below the deepest single well there
    # and above -sum_k Z_k / 0.5 (the softening caps each well at 2 Z_k)
    assert np.all(p.Vq > -2.0 * nuc[:, 3].sum() - 1e-12)
    x, y, z = (c.ravel() for c in W.gauss_point_coords(p.n, p.lo, p.hi))
    single = np.max([Zk / np.sqrt((x - a) ** 2 + (y - b) ** 2 + (z - c) ** 2 + 0.25)
                     for a, b, c, Zk in nuc], axis=0)
    assert np.all(p.Vq <= -single + 1e-12)


def test_batch_recipe_ranges_and_determinism():
    meshes = (4, 6, 8)
    S = W.batch_systems(count=12, seed=4000, meshes=meshes)
    assert len(S) == 12
    for p in S:
        assert p.n[0] in meshes and p.n[0] == p.n[1] == p.n[2]
        assert 4 <= p.N <= 48 and 1 <= p.nuclei.shape[0] <= 6
        assert np.all(np.abs(p.nuclei[:, :3]) <= 4.0)
        assert set(np.unique(p.nuclei[:, 3])).issubset({1.0, 2.0, 3.0})
        M = p.nuclei.shape[0]
        if M > 1:
            d = np.linalg.norm(p.nuclei[:, None, :3] - p.nuclei[None, :, :3], axis=2) + np.eye(M) * 1e9
            assert np.min(d) >= 1.5
        assert p.lo == (-10.0,) * 3 and p.U0.shape == (p.n_interior, p.N)
    again = W.batch_systems(count=12, seed=4000, meshes=meshes)
    assert all(np.array_equal(a.U0, b.U0) and np.array_equal(a.Vq, b.Vq) for a, b in zip(S, again))
    other = W.batch_systems(count=12, seed=4001, meshes=meshes)
    assert any(a.N != b.N or not np.array_equal(a.nuclei, b.nuclei) for a, b in zip(S, other))


def test_large_cluster_recipe():
    p = W.large_cluster(nc=8, N=6)
    nuc = p.nuclei
    assert nuc.shape == (40, 4) and np.all(np.abs(nuc[:, :3]) <= 14.0)
    d = np.linalg.norm(nuc[:, None, :3] - nuc[None, :, :3], axis=2) + np.eye(40) * 1e9
    assert np.min(d) >= 1.8
    assert set(np.unique(nuc[:, 3])).issubset({1.0, 2.0, 3.0, 4.0})
    assert p.lo == (-20.0,) * 3 and p.U0.shape == (7 ** 3, 6)


def test_place_nuclei_gives_up_when_the_separation_cannot_be_met():
    with pytest.raises(RuntimeError):
        W.place_nuclei(np.random.default_rng(0), 10, 3, 0.1, 1.0, max_tries=1000)
