"""Failure detection on the GPU without a GPU fault.

Every device-side wait of the float32 CG kernel (TMA completion, the cross-CTA
reduction) is bounded.  A wait limit of one poll makes the waits run out on
purpose: the kernel records the timeout, lets its copies in flight land and
returns, so the call reports PARO_ERR_TIMEOUT and the same handle then solves
normally.  Iteration limits cut short on purpose report PARO_ERR_NOT_CONVERGED
with the outputs written.  Nothing here traps, faults or hangs the device.
"""
import numpy as np
import pytest

from oracle import paro as O
from paper_1405_0260_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TIMEOUT, NOT_CONVERGED = -6, -4


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_0260_gb300 import binding

    binding.lib()
    return binding


def _setup(B, prec, nc=12, N=8, seed=6100):
    p = W.harmonic(nc=nc, L=5.0, N=N, seed=seed, sigma=0.0)
    m = B.Mesh(p.n, p.lo, p.hi, prec)
    Vq = torch.from_numpy(p.Vq).cuda()
    m.set_potential(Vq, p.sigma)
    U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
    Urr = torch.empty_like(U)
    lam, _ = m.rayleigh_ritz(U, Urr)
    return p, m, Vq, lam, Urr


def test_a_bounded_wait_that_runs_out_is_reported_and_the_handle_stays_usable(B):
    p, m, Vq, lam, U = _setup(B, B.PARO_MIXED)
    X = torch.empty_like(U)
    rc, _ = m.orbital_solve(lam, U, X, B.paro_default_params(solve_tol=1e-10, wait_polls=1), allow=(TIMEOUT,))
    assert rc == TIMEOUT, rc
    assert "wait ran out" in B.paro_last_error(m.h)
    # the same handle, the default wait limit: a normal solve, checked against the oracle's residual
    rc, st = m.orbital_solve(lam, U, X, B.paro_default_params(solve_tol=1e-10))
    assert rc == 0 and st.refine_sweeps >= 1
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)
    u, x = U.cpu().numpy(), X.cpu().numpy()
    b = (ops.M @ u) * (lam + p.sigma)[None, :]
    rel = np.linalg.norm(b - ops.A @ x, axis=0) / np.linalg.norm(b, axis=0)
    assert np.all(rel < 1.5e-10), rel
    m.close()


def test_cg_iteration_limit_reports_not_converged_with_the_iterate_written(B):
    p, m, Vq, lam, U = _setup(B, B.PARO_FP64)
    X = torch.full_like(U, float("nan"))
    rc, st = m.orbital_solve(lam, U, X, B.paro_default_params(solve_tol=1e-12, pcg_maxit=3),
                             allow=(NOT_CONVERGED,))
    assert rc == NOT_CONVERGED
    x = X.cpu().numpy()
    assert np.all(np.isfinite(x))
    # three CG steps from the warm start x0 = u reduce the residual, but not to 1e-12
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)
    u = U.cpu().numpy()
    b = (ops.M @ u) * (lam + p.sigma)[None, :]
    r0 = np.linalg.norm(b - ops.A @ u, axis=0)
    r3 = np.linalg.norm(b - ops.A @ x, axis=0)
    assert np.all(r3 < r0) and np.max(r3 / np.linalg.norm(b, axis=0)) > 1e-12
    m.close()


def test_refinement_sweep_limit_reports_not_converged(B):
    p, m, Vq, lam, U = _setup(B, B.PARO_MIXED)
    X = torch.empty_like(U)
    rc, st = m.orbital_solve(lam, U, X, B.paro_default_params(solve_tol=1e-12, max_refine=1),
                             allow=(NOT_CONVERGED,))
    assert rc == NOT_CONVERGED and st.refine_sweeps == 1
    assert np.all(np.isfinite(X.cpu().numpy()))
    m.close()


def test_outer_iteration_limit_reports_not_converged_with_the_state_written(B):
    for prec in (B.PARO_FP64, B.PARO_MIXED):
        p, m, Vq, lam, U = _setup(B, prec)
        rc, lam2, st = m.iterate(U, lam, B.paro_default_params(tol=1e-14, max_outer=2, solve_tol=1e-10),
                                 allow=(NOT_CONVERGED,))
        assert rc == NOT_CONVERGED and st.outer_iters == 2
        # the state after the two iterations is returned: Ritz values still decrease
        # and the orbitals are M-orthonormal, so the loop can be resumed from it
        # (mixed handles: tensor-core Grams, ~1e-9 of |x||y| per entry at this size)
        slack = 1e-9 if prec == B.PARO_FP64 else 1e-7
        assert np.all(np.isfinite(lam2)) and np.all(lam2 <= lam + slack)
        ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)
        u = U.cpu().numpy()
        assert np.max(np.abs(u.T @ (ops.M @ u) - np.eye(p.N))) < slack * 10
        m.close()
