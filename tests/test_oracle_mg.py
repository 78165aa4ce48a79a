"""Pins of the multigrid preconditioner of the oracle (no GPU).

The V-cycle is pinned to what the finite-element setting fixes independently
of it: nested Q1 spaces (prolongation = evaluation of the coarse function at
the fine nodes; Galerkin products = the matrices assembled directly on the
coarse mesh), the symmetry and definiteness a preconditioner for CG needs,
contraction of the error propagator in the energy norm, and a direct sparse
solve.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import mg as MG
from oracle import paro as O
from paper_1405_0260_gb300 import workloads as W


def _coarse_q1_at(mesh_c, vals_c, pts):
    """Coarse Q1 function (interior nodal values vals_c, zero on the boundary) at points.

    Cell lookup and the 8-corner trilinear formula: independent of the Kronecker
    construction of the prolongation."""
    nx, ny, nz = mesh_c.n
    full = np.zeros((nz + 1, ny + 1, nx + 1))
    full[1:nz, 1:ny, 1:nx] = vals_c.reshape(nz - 1, ny - 1, nx - 1)
    out = np.zeros(len(pts))
    for q, x in enumerate(pts):
        t = (x - np.array(mesh_c.lo)) / mesh_c.h
        c = np.minimum(np.floor(t).astype(int), np.array([nx, ny, nz]) - 1)
        f = t - c
        s = 0.0
        for az in range(2):
            for ay in range(2):
                for ax in range(2):
                    w = (f[0] if ax else 1 - f[0]) * (f[1] if ay else 1 - f[1]) * (f[2] if az else 1 - f[2])
                    s += w * full[c[2] + az, c[1] + ay, c[0] + ax]
        out[q] = s
    return out


@pytest.mark.parametrize("n", [(4, 4, 4), (8, 6, 4), (6, 8, 10)])
def test_prolongation_evaluates_the_coarse_function(n):
    mesh = O.Mesh(n, (-1.0, -2.0, 0.0), (2.0, 1.0, 3.5))
    mc = MG.coarse_mesh(mesh)
    rng = np.random.default_rng(11)
    vc = rng.standard_normal(mc.n_interior)
    fine = MG.prolongation(mesh) @ vc
    ref = _coarse_q1_at(mc, vc, mesh.interior_coords())
    assert np.max(np.abs(fine - ref)) < 1e-13


def test_galerkin_products_equal_coarse_assembly():
    n = (8, 6, 10)
    mesh = O.Mesh(n, (-3.0, -2.0, -4.0), (3.0, 2.5, 4.0))
    mc = MG.coarse_mesh(mesh)
    c = 0.7
    fine = O.assemble(mesh, np.full(8 * np.prod(n), c), 0.0)
    coarse = O.assemble(mc, np.full(8 * np.prod(mc.n), c), 0.0)
    P = MG.prolongation(mesh)
    for F, C in ((fine.K, coarse.K), (fine.M, coarse.M), (fine.MV, coarse.MV)):
        G = (P.T @ F @ P).toarray()
        assert np.max(np.abs(G - C.toarray())) < 1e-12 * np.max(np.abs(C.toarray()))


def test_hierarchy_shapes_and_jacobi_weights():
    p = W.harmonic(nc=16, L=6.0, N=2, seed=1, sigma=0.0)
    mesh = O.Mesh(p.n, p.lo, p.hi)
    ops = O.assemble(mesh, p.Vq, 0.0)
    lev = MG.hierarchy((0.5 * ops.K).tocsr(), mesh)
    assert [l.mesh.n for l in lev] == [(16,) * 3, (8,) * 3, (4,) * 3, (2,) * 3]
    # the Q1 Laplacian: sum_j |A_ij| / A_ii = 2 away from the boundary on every level
    # (a Galerkin product of the Q1 Laplacian is the coarse Q1 Laplacian) -> w = 2/3;
    # a single interior node -> w = 1 (one sweep is the exact solve)
    assert all(abs(l.omega - 2.0 / 3.0) < 1e-12 for l in lev[:-1])
    assert lev[-1].A.shape == (1, 1) and lev[-1].omega == 1.0
    # odd cell counts do not coarsen
    assert len(MG.hierarchy(ops.A, O.Mesh((9, 8, 8), p.lo, p.hi))) == 1


def _problem(nc, kind):
    if kind == "poisson":
        p = W.harmonic(nc=nc, L=8.0, N=2, seed=3, sigma=0.0)
        mesh = O.Mesh(p.n, p.lo, p.hi)
        ops = O.assemble(mesh, 0.0 * p.Vq, 0.0)
        return mesh, (0.5 * ops.K).tocsr(), ops.M
    p = W.cluster(nc=nc, L=12.0)
    mesh = O.Mesh(p.n, p.lo, p.hi)
    ops = O.assemble(mesh, p.Vq, 6.0)
    return mesh, ops.A, ops.M


@pytest.mark.parametrize("kind", ["poisson", "cluster"])
def test_vcycle_is_symmetric_positive_definite(kind):
    mesh, A, _ = _problem(16, kind)
    lev = MG.hierarchy(A, mesh)
    rng = np.random.default_rng(5)
    x, y = rng.standard_normal((2, A.shape[0]))
    for nu in (1, 2):
        Bx, By = MG.vcycle(lev, x, nu), MG.vcycle(lev, y, nu)
        assert abs(x @ By - y @ Bx) < 1e-12 * abs(x @ Bx)
        Z = rng.standard_normal((A.shape[0], 6))
        assert np.all(np.einsum("ij,ij->j", Z, MG.vcycle(lev, Z, nu)) > 0)


@pytest.mark.parametrize("kind,bound", [("poisson", 0.5), ("cluster", 0.8)])
def test_vcycle_error_propagator_contracts_in_energy_norm(kind, bound):
    """||I - B A||_A by power iteration on E = I - B A (self-adjoint in the A inner product)."""
    mesh, A, _ = _problem(16, kind)
    lev = MG.hierarchy(A, mesh)
    rng = np.random.default_rng(9)
    e = rng.standard_normal(A.shape[0])
    rho = 0.0
    for _ in range(40):
        e = e / np.sqrt(e @ (A @ e))
        e2 = e - MG.vcycle(lev, A @ e)
        rho = np.sqrt(e2 @ (A @ e2))
        e = e2
    assert 0.0 < rho < bound


def test_mg_pcg_matches_direct_solve_and_is_mesh_independent():
    iters_mg, iters_jac = [], []
    for nc in (8, 16, 32):
        mesh, A, M = _problem(nc, "poisson")
        rng = np.random.default_rng(nc)
        b = M @ rng.standard_normal((A.shape[0], 2))
        lev = MG.hierarchy(A, mesh)
        r = MG.mg_pcg(lev, b, None, 1e-10, 100)
        assert r.converged.all()
        x = np.column_stack([spla.spsolve(A.tocsc(), b[:, i]) for i in range(2)])
        assert np.max(np.abs(r.X - x)) < 1e-8 * np.max(np.abs(x))
        iters_mg.append(int(r.iters.max()))
        iters_jac.append(int(O.pcg(A, b, np.zeros_like(b), 1e-10, 5000).iters.max()))
    # V(1,1) as a preconditioner: iteration counts stay flat under refinement,
    # Jacobi's roughly double with each halving of h
    assert max(iters_mg) - min(iters_mg) <= 3 and max(iters_mg) <= 16
    assert iters_jac[2] > 3 * iters_jac[0] and iters_jac[2] > 4 * iters_mg[2]


def test_mg_pcg_warm_start_and_masks():
    mesh, A, M = _problem(16, "cluster")
    lev = MG.hierarchy(A, mesh)
    rng = np.random.default_rng(2)
    b = M @ rng.standard_normal((A.shape[0], 3))
    x = np.column_stack([spla.spsolve(A.tocsc(), b[:, i]) for i in range(3)])
    X0 = x.copy()
    X0[:, 1] += 1e-3 * rng.standard_normal(A.shape[0])  # only column 1 is off
    r = MG.mg_pcg(lev, b, X0, 1e-9, 100)
    assert r.iters[0] == 0 and r.iters[2] == 0 and r.iters[1] > 0
    assert np.max(np.abs(r.X - x)) < 1e-7 * np.max(np.abs(x))
