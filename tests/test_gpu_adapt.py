"""The adaptive loop of Section 2.1 on the GPU (paro_estimate, paro_mark,
paro_refine_coords, paro_transfer) against the oracle's adaptive loop
(oracle/adapt.py): the error indicators of the same orbitals on uniform and
graded meshes, the transfer to a refined mesh, and three adaptive steps of the whole loop (Solve with
paro_iterate on each mesh, float64 handles) against the oracle's loop on the
same meshes."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import adapt as A
from oracle import paro as O
from paper_1405_0260_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_0260_gb300 import binding

    binding.lib()
    return binding


def _coulomb(n, coords, R):
    x, y, z = W.gauss_point_coords(n, None, None, coords)
    return np.ascontiguousarray((-1.0 / np.sqrt((x - R[0]) ** 2 + (y - R[1]) ** 2 + (z - R[2]) ** 2)).ravel())


def _mesh(B, coords, prec=None):
    n = tuple(len(c) - 1 for c in coords)
    return B.Mesh(n, None, None, prec if prec is not None else B.PARO_FP64, coords=coords)


@pytest.mark.parametrize("graded", [False, True])
def test_indicators_match_the_oracle(B, graded):
    if graded:
        coords = (np.array([-5.0, -3.0, -1.6, -0.7, -0.2, 0.3, 1.1, 2.4, 5.0]),
                  np.array([-4.0, -2.0, -0.8, 0.1, 0.9, 2.0, 4.0]),
                  np.array([-6.0, -3.5, -1.5, -0.4, 0.2, 0.9, 2.2, 3.6, 6.0]))
    else:
        ax = np.linspace(-5.0, 5.0, 10)
        coords = (ax, np.linspace(-4.0, 4.0, 8), np.linspace(-6.0, 6.0, 11))
    n = tuple(len(c) - 1 for c in coords)
    mesh = O.Mesh(n, None, None, coords=coords)
    rng = np.random.default_rng(8300)
    N = 6
    U = rng.standard_normal((mesh.n_interior, N))
    lam = rng.uniform(-1.0, 1.0, N)
    Vq = _coulomb(n, coords, (0.37, -0.21, 0.13))
    ref = A.indicators(mesh, Vq, lam, U)
    m = _mesh(B, coords)
    Vd = torch.from_numpy(Vq).cuda()
    m.set_potential(Vd, 0.0)
    eta2 = torch.empty(n[0] * n[1] * n[2], dtype=torch.float64, device="cuda")
    m.estimate(torch.from_numpy(U).cuda(), lam, Vd, eta2)
    got = eta2.cpu().numpy().reshape(ref.shape)
    assert np.max(np.abs(got - ref) / np.maximum(ref, 1e-300)) < 1e-12, np.max(np.abs(got - ref) / ref)
    m.close()


def test_transfer_matches_the_oracle(B):
    rng = np.random.default_rng(8500)
    coords = (np.linspace(-3, 3, 8), np.linspace(-2, 2, 6) ** 3 / 4.0, np.linspace(-3, 3, 9))
    n = tuple(len(c) - 1 for c in coords)
    coarse = O.Mesh(n, None, None, coords=coords)
    marked = rng.random((n[2], n[1], n[0])) < 0.2
    fc = A.refine_coords(coarse, marked)
    fine = O.Mesh(tuple(len(c) - 1 for c in fc), None, None, coords=fc)
    U = rng.standard_normal((coarse.n_interior, 5))
    ref = A.transfer(coarse, fine, U)
    mc, mf = _mesh(B, coords), _mesh(B, fc)
    Ud = torch.from_numpy(U).cuda()
    out = torch.empty((fine.n_interior, 5), dtype=torch.float64, device="cuda")
    mc.transfer_to(mf, Ud, out)
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-14 * np.max(np.abs(U))
    mc.close()
    mf.close()


def test_two_adaptive_steps_match_the_oracle(B):
    """Solve -> Estimate -> Mark -> Refine twice on a hydrogen-like problem with
    the nucleus off the nodes: the ground level on each mesh against dense
    diagonalisation of the oracle's operators, the indicators and
    marks against the oracle's on the GPU's orbitals, and the refined meshes
    identical to the oracle's."""
    R = (0.31, -0.23, 0.17)
    ax = np.linspace(-8.0, 8.0, 9)
    coords = (ax, ax, ax)
    N = 1
    U = None
    prev = None
    for step in range(3):
        n = tuple(len(c) - 1 for c in coords)
        mesh = O.Mesh(n, None, None, coords=coords)
        Vq = _coulomb(n, coords, R)
        ops = O.assemble(mesh, Vq, 2.0)
        exact = sla.eigh(ops.H.toarray(), ops.M.toarray(), eigvals_only=True, subset_by_index=[0, N - 1])
        m = _mesh(B, coords)
        Vd = torch.from_numpy(Vq).cuda()
        m.set_potential(Vd, 2.0)
        if U is None:
            p = W.hydrogen(nc=n[0], L=8.0, N=N, seed=8600, sigma=2.0)
            Ud = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
        else:
            Ud = torch.empty((mesh.n_interior, N), dtype=torch.float64, device="cuda")
            prev.transfer_to(m, U, Ud)
            assert np.max(np.abs(Ud.cpu().numpy() - A.transfer(prev_mesh, mesh, U.cpu().numpy()))) < 1e-13
        rc, lam, st = m.iterate(Ud, None, B.paro_default_params(tol=1e-12, max_outer=2000, solve_tol=1e-12))
        assert rc == 0
        assert np.max(np.abs(lam - exact)) < 1e-8, (step, lam, exact)
        eta2 = torch.empty(n[0] * n[1] * n[2], dtype=torch.float64, device="cuda")
        m.estimate(Ud, lam, Vd, eta2)
        e_gpu = eta2.cpu().numpy().reshape(n[2], n[1], n[0])
        e_ref = A.indicators(mesh, Vq, lam, Ud.cpu().numpy())
        assert np.max(np.abs(e_gpu - e_ref) / np.maximum(e_ref, 1e-300)) < 1e-12
        marked = B.mark(e_gpu, B.PARO_MARK_DORFLER, 0.5)
        assert np.array_equal(marked, A.mark_dorfler(e_ref, 0.5))
        new = B.refine_coords(n, coords, marked)
        for d, c in enumerate(A.refine_coords(mesh, marked)):
            assert np.array_equal(new[d], c)
        if prev is not None:
            prev.close()
        prev, prev_mesh, U = m, mesh, Ud
        coords = new
    prev.close()
