"""Graded tensor-product meshes on the GPU (Section 2.1's locally refined spaces,
refined along each axis), against the CPU FP64 oracle's graded assembly.

  * operator applies (float64, float-float, float32) against the oracle's
    element-by-element matrices, with the bounds of the uniform-mesh tests;
  * the float64 ParO loop iterate by iterate against the oracle (1e-10 relative);
  * the mixed path converged on a mesh graded toward a Coulomb nucleus reaches the
    discrete spectrum of that mesh (dense generalized eigh of the oracle's assembly)
    within 1e-6 Ha, and its ground state lies below the uniform mesh's;
  * the calls a graded handle does not support report PARO_ERR_ARG.
"""
import numpy as np
import pytest
import scipy.linalg as sla

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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def graded_problem(n, L, beta, N, seed, sigma):
    ax = tuple(W.graded_axis(n[d], L[d], beta[d]) for d in range(3))
    lo, hi = tuple(-v for v in L), tuple(L)
    x, y, z = W.gauss_point_coords(n, lo, hi, ax)
    rng = np.random.default_rng(seed)
    V = 0.3 * (x ** 2 + y ** 2 + z ** 2) - 1.0 / np.sqrt(x ** 2 + y ** 2 + z ** 2 + 0.3)
    V = np.ascontiguousarray((V + 0.2 * rng.standard_normal(V.shape)).ravel())
    nI = (n[0] - 1) * (n[1] - 1) * (n[2] - 1)
    return W.Problem("graded", n, lo, hi, V, sigma, rng.standard_normal((nI, N)), 0, coords=ax)


def oracle_ops(p):
    return O.assemble(O.Mesh(p.n, p.lo, p.hi, coords=p.coords), p.Vq, p.sigma)


def make_mesh(B, p, precision):
    m = B.Mesh(p.n, p.lo, p.hi, precision, coords=p.coords)
    Vq = dev(p.Vq)
    m.set_potential(Vq, p.sigma)
    m._vq = Vq
    return m


CASES = [((7, 6, 9), (1.5, 2.0, 1.25), (1.5, 0.7, 2.0), 5), ((12, 10, 13), (3.0, 2.5, 3.5), (2.5, 2.0, 1.0), 13)]


@pytest.mark.parametrize("n,L,beta,N", CASES)
def test_graded_applies_match_the_oracle(B, n, L, beta, N):
    p = graded_problem(n, L, beta, N, 700 + N, 0.7)
    ops = oracle_ops(p)
    X = dev(p.U0)
    Y = torch.empty_like(X)
    for prec, ff, tol in ((B.PARO_FP64, False, 1e-13), (B.PARO_MIXED, True, 100 * 2.0 ** -48)):
        m = make_mesh(B, p, prec)
        for op, A in ((B.PARO_OP_A, ops.A), (B.PARO_OP_H, ops.H), (B.PARO_OP_M, ops.M)):
            m.apply(op, X, Y, float_float=ff)
            err = np.abs(host(Y) - A @ p.U0)
            bound = abs(A) @ np.abs(p.U0)
            assert np.all(err <= tol * bound + 1e-300), (prec, op, (err / bound).max())
        if prec == B.PARO_MIXED:  # the float32 weights of the CG kernels
            U32 = p.U0.astype(np.float32).astype(np.float64)
            X32 = dev(U32, torch.float32)
            Y32 = torch.empty_like(X32)
            m.apply(B.PARO_OP_A, X32, Y32)
            err = np.abs(host(Y32) - ops.A @ U32)
            assert np.all(err <= 4e-6 * (abs(ops.A) @ np.abs(U32))), err.max()
        m.close()


def test_graded_fp64_iterate_matches_the_oracle_iterate_by_iterate(B):
    p = W.graded_hydrogen(nc=12, L=8.0, beta=2.0, N=5, seed=1201, sigma=2.0)
    ops = oracle_ops(p)
    ref = O.paro(ops, p.U0, pcg_tol=1e-12, fixed_outer=5)
    m = make_mesh(B, p, B.PARO_FP64)
    U = dev(p.U0)
    rc, lam, st = m.iterate(U, None, B.paro_default_params(fixed_outer=5, solve_tol=1e-12))
    assert rc == 0 and st.outer_iters == 5
    assert np.max(np.abs(lam - ref.lam) / np.abs(ref.lam)) < 1e-10
    u = host(U)
    assert np.max(np.abs(u.T @ (ops.M @ u) - np.eye(p.N))) < 1e-12
    assert np.max(O.subspace_angles_M(ops.M, u, ref.U)) < 1e-7
    m.close()


def test_graded_mixed_path_reaches_the_discrete_spectrum_and_beats_uniform(B):
    lams = {}
    for beta in (2.5, 0.0):
        p = W.graded_hydrogen(nc=16, L=10.0, beta=beta, N=5, seed=1300, sigma=2.0)
        ops = O.assemble(O.Mesh(p.n, p.lo, p.hi, coords=p.coords), p.Vq, 0.0)
        # dense generalized eigh of the oracle's assembly: the symmetric graded mesh keeps
        # the cubic symmetry about the nucleus, so 2p is an exact triplet (Lanczos can
        # miss a copy of a multiple eigenvalue)
        disc = sla.eigh(ops.H.toarray(), ops.M.toarray(), eigvals_only=True, subset_by_index=[0, 4])
        m = make_mesh(B, p, B.PARO_MIXED)
        U = dev(p.U0)
        rc, lam, st = m.iterate(U, None, B.paro_default_params(tol=1e-9, max_outer=600, solve_tol=1e-10))
        assert rc == 0, B.paro_last_error(m.h)
        assert st.cg_iters_f32 > 0
        assert np.max(np.abs(lam - disc)) < 1e-6, (beta, lam, disc)
        lams[beta] = lam
        m.close()
    # the mesh graded toward the nucleus gives the better (lower) ground state
    assert -0.5 < lams[2.5][0] < lams[0.0][0] - 0.01


def test_graded_handles_refuse_the_uniform_only_calls(B):
    p = W.graded_hydrogen(nc=8, L=6.0, beta=1.5, N=4, seed=1400, sigma=2.0)
    m = make_mesh(B, p, B.PARO_MIXED)
    U = dev(p.U0)
    rc, _, _ = m.iterate(U, None, B.paro_default_params(fixed_outer=1, precond=B.PARO_PRECOND_MG), allow=(-1,))
    assert rc == -1 and "uniform" in B.paro_last_error(m.h)
    rho = torch.zeros(8 * 8 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(B.ParoError):
        m.density(U, np.full(4, 2.0), rho)
    m.close()
