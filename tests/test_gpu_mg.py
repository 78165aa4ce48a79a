"""Parity of the multigrid preconditioner (through the C ABI) with the oracle's
V-cycle (oracle/mg.py), and of the MG-preconditioned solves with direct solves.

Tolerances: the V-cycle runs in float32 on every level (float32 operator
weights, transfers and sweeps) against the float64 oracle: 3e-5 of max |B r|;
MG-PCG solves inside float64-accurate refinement reach the same solve tolerance
as the Jacobi path, so they are held to the same bounds (1e-9 relative against a
sparse direct solve, eigenvalues 1e-7 against dense diagonalisation).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import ks as KS
from oracle import mg as MG
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


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


CASES = [
    # (problem, N): 4 levels down to one interior node; 12 -> 6 -> 3 (8 coarse
    # nodes); uneven axes (8, 12, 16) -> (4, 6, 8) -> (2, 3, 4); odd counts: no
    # coarsening (the smoother alone)
    ("harmonic16", 3),
    ("cluster12", 20),
    ("uneven", 6),
    ("odd", 4),
]


def problem(name):
    if name == "harmonic16":
        return W.harmonic(nc=16, L=6.0, N=3, seed=7100, sigma=0.5)
    if name == "cluster12":
        p = W.cluster(nc=12, L=8.0)
        p.sigma = 6.0
        return p
    if name == "uneven":
        p = W.harmonic(nc=8, L=5.0, N=6, seed=7200, sigma=1.0)
        n = (8, 12, 16)
        mesh = O.Mesh(n, (-4.0, -5.0, -6.0), (4.0, 5.0, 6.0))
        X = O.gauss_points(mesh).reshape(-1, 3)
        p.n, p.lo, p.hi = n, mesh.lo, mesh.hi
        p.Vq = np.ascontiguousarray(0.5 * (X ** 2).sum(1))
        return p
    return W.harmonic(nc=9, L=5.0, N=4, seed=7300, sigma=1.0)


@pytest.mark.parametrize("name,N", CASES)
@pytest.mark.parametrize("nu,nu_c", [(1, 4), (2, 3)])
def test_vcycle_matches_oracle(B, name, N, nu, nu_c):
    p = problem(name)
    mesh = O.Mesh(p.n, p.lo, p.hi)
    ops = O.assemble(mesh, p.Vq, p.sigma)
    levels = MG.hierarchy(ops.A, mesh)
    rng = np.random.default_rng(7000 + N)
    R = rng.standard_normal((mesh.n_interior, N)).astype(np.float32)
    ref = MG.vcycle(levels, R.astype(np.float64), nu, nu_c)
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED)
    vq = dev(p.Vq)
    m.set_potential(vq, p.sigma)
    Z = torch.empty((mesh.n_interior, N), dtype=torch.float32, device="cuda")
    m.mg_vcycle(dev(R, torch.float32), Z, B.paro_default_params(mg_nu=nu, mg_coarse_sweeps=nu_c))
    err = np.max(np.abs(host(Z) - ref))
    assert err < 3e-5 * np.max(np.abs(ref)), (name, err, np.max(np.abs(ref)))
    # a second potential on the same handle rebuilds the hierarchy
    m.set_potential(vq, p.sigma + 1.0)
    levels2 = MG.hierarchy(O.assemble(mesh, p.Vq, p.sigma + 1.0).A, mesh)
    m.mg_vcycle(dev(R, torch.float32), Z, B.paro_default_params(mg_nu=nu, mg_coarse_sweeps=nu_c))
    ref2 = MG.vcycle(levels2, R.astype(np.float64), nu, nu_c)
    assert np.max(np.abs(host(Z) - ref2)) < 3e-5 * np.max(np.abs(ref2))
    m.close()


def test_mg_orbital_solve_matches_direct_solve_with_fewer_iterations(B):
    # a weakly shifted free box: Jacobi-PCG iterations grow like 1/h, the V-cycle's do not
    p = W.harmonic(nc=32, L=8.0, N=5, seed=7400, sigma=0.05)
    p.Vq = np.zeros_like(p.Vq)
    mesh = O.Mesh(p.n, p.lo, p.hi)
    ops = O.assemble(mesh, p.Vq, p.sigma)
    lam = np.linspace(0.1, 0.5, p.N)
    rhs = (ops.M @ p.U0) * (lam + p.sigma)[None, :]
    ref = np.column_stack([spla.spsolve(ops.A.tocsc(), rhs[:, i]) for i in range(p.N)])
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED)
    vq = dev(p.Vq)
    m.set_potential(vq, p.sigma)
    U = dev(p.U0)
    its = {}
    for pc in (B.PARO_PRECOND_JACOBI, B.PARO_PRECOND_MG):
        X = torch.empty_like(U)
        rc, st = m.orbital_solve(lam, U, X, B.paro_default_params(solve_tol=1e-11, precond=pc))
        assert rc == 0
        assert np.max(np.abs(host(X) - ref)) < 1e-9 * np.max(np.abs(ref)), pc
        its[pc] = st.cg_iters_f32
    assert its[B.PARO_PRECOND_MG] * 3 < its[B.PARO_PRECOND_JACOBI], its
    m.close()


def test_mg_iterate_reaches_the_dense_spectrum(B):
    p = W.harmonic(nc=16, L=6.0, N=4, seed=7500, sigma=0.0)
    mesh = O.Mesh(p.n, p.lo, p.hi)
    ops = O.assemble(mesh, p.Vq, 0.0)
    exact = sla.eigh(ops.H.toarray(), ops.M.toarray(), eigvals_only=True, subset_by_index=[0, 3])
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED)
    vq = dev(p.Vq)
    m.set_potential(vq, 0.0)
    U = dev(p.U0)
    rc, lam, st = m.iterate(U, None, B.paro_default_params(tol=1e-10, max_outer=400, solve_tol=1e-11,
                                                           precond=B.PARO_PRECOND_MG))
    assert rc == 0
    assert np.max(np.abs(lam - exact)) < 1e-7, (lam, exact)
    m.close()


def test_mg_hartree_matches_oracle(B):
    nc, L = 12, 5.0
    mesh = O.Mesh((nc, nc, nc), (-L, -L, -L), (L, L, L))
    X = O.gauss_points(mesh).reshape(-1, 3)
    Vext = np.ascontiguousarray(-2.0 / np.sqrt((X ** 2).sum(1) + 0.25))
    p = W.harmonic(nc=nc, L=L, N=4, seed=7600)
    occ = KS.occupations(4, 3)
    rho = KS.density_gauss(mesh, O.rayleigh_ritz(O.assemble(mesh, Vext, 3.0), p.U0).U, occ)
    ref = KS.hartree(mesh, rho).VH_q
    vq = dev(Vext)
    for hp in (B.PARO_PRECOND_MG, B.PARO_PRECOND_JACOBI, B.PARO_PRECOND_AUTO):
        # a fresh handle each time: the Hartree solve starts from the previous solution
        m = B.Mesh(mesh.n, mesh.lo, mesh.hi, B.PARO_MIXED)
        m.set_potential(vq, 3.0)
        v = torch.empty_like(vq)
        vh = torch.empty_like(vq)
        m.ks_potential(dev(rho), vq, v, vh, B.paro_default_params(solve_tol=1e-12, hartree_precond=hp))
        assert np.max(np.abs(host(vh) - ref)) < 1e-9 * np.max(np.abs(ref)), hp
        m.close()


def test_mg_needs_a_mixed_handle_and_valid_sweeps(B):
    p = W.harmonic(nc=8, L=4.0, N=4, seed=7700, sigma=0.5)
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_FP64)
    vq = dev(p.Vq)
    m.set_potential(vq, p.sigma)
    U = dev(p.U0)
    X = torch.empty_like(U)
    with pytest.raises(B.ParoError):
        m.orbital_solve(np.ones(4), U, X, B.paro_default_params(precond=B.PARO_PRECOND_MG))
    rho = torch.full_like(vq, 0.01)
    with pytest.raises(B.ParoError):
        m.ks_potential(rho, vq, torch.empty_like(vq), None, B.paro_default_params(hartree_precond=B.PARO_PRECOND_MG))
    m.close()
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED)
    m.set_potential(vq, p.sigma)
    Z = torch.empty((U.shape[0], 4), dtype=torch.float32, device="cuda")
    with pytest.raises(B.ParoError):
        m.mg_vcycle(U.float(), Z, B.paro_default_params(mg_nu=0))
    m.close()
