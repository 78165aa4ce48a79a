"""Parity at the full size of the headline workload, in the configuration bench.py
times: harmonic oscillator, 64^3 cells (250 047 unknowns), N = 20, mixed
precision, one outer iteration per call with the source problems to 1e-10.

At this size the oracle does not run the method; it checks properties that hold
at any size with its own assembled operators: the source-problem residuals
||b_i - A x_i|| / ||b_i|| of every orbital, the M-orthonormality of the Ritz
vectors, their eigen-residuals, the discrete spectrum stored by
tests/golden/make_golden.py (shift-invert Lanczos on the oracle's assembly), and
the exact discrete eigenvectors of this separable operator (oracle.separable,
Kronecker products of 1-D modes): the orbitals of every oscillator shell are
compared with them as subspaces, by M-principal angles.
"""
import json
import os

import numpy as np
import pytest

from gram_budget import gram_tc_error, rotation_tc_error
from oracle import paro as O
from oracle import separable as S
from paper_1405_0260_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_0260_gb300 import binding

    binding.lib()
    return binding


@pytest.fixture(scope="module")
def case():
    p = W.harmonic(nc=64, L=8.0, N=20, seed=2000, sigma=0.0)  # the bench problem of rank 0
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)
    with open(os.path.join(HERE, "golden", "discrete_spectra.json")) as f:
        gold = np.array(json.load(f)["harmonic_64_L8"]["values"][: p.N])
    return p, ops, gold


def test_fullsize_source_problems_meet_the_tolerance(B, case):
    p, ops, _ = case
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED)
    vq = torch.from_numpy(p.Vq).cuda()
    m.set_potential(vq, p.sigma)
    U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
    Urr = torch.empty_like(U)
    lam, _ = m.rayleigh_ritz(U, Urr)
    X = torch.empty_like(U)
    rc, st = m.orbital_solve(lam, Urr, X, B.paro_default_params(solve_tol=1e-10))
    assert rc == 0 and st.refine_sweeps <= 3
    u, x = Urr.cpu().numpy(), X.cpu().numpy()
    b = (ops.M @ u) * (lam + p.sigma)[None, :]
    rel = np.linalg.norm(b - ops.A @ x, axis=0) / np.linalg.norm(b, axis=0)
    # the mixed path tests its own float-float residual against 1e-10; the oracle's
    # float64 residual of the returned float64 solution agrees to rounding
    assert np.all(rel < 1.5e-10), rel
    m.close()


def test_fullsize_iteration_reaches_the_discrete_spectrum(B, case):
    p, ops, gold = case
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED)
    vq = torch.from_numpy(p.Vq).cuda()
    m.set_potential(vq, p.sigma)
    U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
    params = B.paro_default_params(fixed_outer=1, solve_tol=1e-10)
    lam, err, outer = None, np.inf, 0
    while outer < 400 and not err < 1e-6:
        _, lam, _ = m.iterate(U, lam, params)
        outer += 1
        err = float(np.max(np.abs(lam - gold)))
    assert err < 1e-6, (outer, lam, gold)
    u = U.cpu().numpy()
    # M-orthonormal to the accuracy of the Gram matrices the last Rayleigh-Ritz step
    # used: one call per outer iteration keeps the tensor-core Grams, which round
    # every input to 24 bits below its chunk's column maximum; bound: 10x the
    # expected largest entry error of tests/gram_budget.py (~6.5e-9 here; measured 3e-9 to 2.3e-8
    # with the float-float rotation)
    # plus the rounding of the tensor-core rotation U = X C (near convergence C is
    # close to the identity, X close to U)
    G = u.T @ (ops.M @ u)
    Mu = ops.M @ u
    budget = gram_tc_error(p.n, u, Mu) + rotation_tc_error(u, np.eye(p.N), Mu)
    assert np.max(np.abs(G - np.eye(p.N))) < 10 * budget
    # eigen-residuals relative to ||M u||: an eigenvalue within 1e-6 Ha leaves a
    # residual of order sqrt(1e-6 * gap); a wrong vector leaves O(1)
    res = O.eigen_residuals(ops, u, lam) / np.linalg.norm(ops.M @ u, axis=0)
    assert np.max(res) < 2e-2, res
    m.close()


def test_fullsize_orbitals_span_the_exact_eigenspaces(B, case):
    # one call to a tight stop, as a user would run it: the loop switches to the
    # float-float Grams once max |delta lambda| < 1e-6, so |delta lambda| can fall
    # to 1e-12.  The vector error goes like the square root of the eigenvalue
    # error (an eigenvalue within e of its limit leaves a vector error of about
    # sqrt(e / gap)), so angles below 1e-5 need the eigenvalues to ~1e-11.
    p, ops, gold = case
    vals, V = S.oscillator_modes(64, 8.0, p.N)
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED)
    vq = torch.from_numpy(p.Vq).cuda()
    m.set_potential(vq, p.sigma)
    U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
    rc, lam, st = m.iterate(U, None, B.paro_default_params(tol=1e-12, max_outer=300, solve_tol=1e-11))
    assert rc == 0, B.paro_last_error(m.h)
    assert np.max(np.abs(lam - vals)) < 1e-10, (lam - vals)
    u = U.cpu().numpy()
    # the last Rayleigh-Ritz steps use float-float Grams: M-orthonormal to ~1e-14
    assert np.max(np.abs(u.T @ (ops.M @ u) - np.eye(p.N))) < 1e-12
    for a, b in S.clusters(vals, 0.25):  # the shells n = 0..3: 1, 3, 6 and 10 orbitals
        ang = O.subspace_angles_M(ops.M, u[:, a:b], V[:, a:b])
        assert np.max(ang) < 1e-5, (a, b, ang)
    m.close()
