"""Parity at the full size of the headline workload, in the configuration bench.py
times: harmonic oscillator, 64^3 cells (250 047 unknowns), N = 20, mixed
precision, one outer iteration per call with the source problems to 1e-10.

At this size the oracle does not run the method; it checks properties that hold
at any size with its own assembled operators: the source-problem residuals
||b_i - A x_i|| / ||b_i|| of every orbital, the M-orthonormality of the Ritz
vectors, their eigen-residuals, and the discrete spectrum stored by
tests/golden/make_golden.py (shift-invert Lanczos on the oracle's assembly).
"""
import json
import os

import numpy as np
import pytest

from oracle import paro as O
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
    # used: until max |delta lambda| < 1e-6 those are the tensor-core Grams, which
    # round every input 24 bits below its chunk's column maximum (at most ~6e-8
    # relative on one product; about 5e-10 on a Gram entry at this size, where the
    # rounding errors of many nodes partly cancel); the bound leaves room for both
    G = u.T @ (ops.M @ u)
    assert np.max(np.abs(G - np.eye(p.N))) < 2e-7
    # eigen-residuals relative to ||M u||: an eigenvalue within 1e-6 Ha leaves a
    # residual of order sqrt(1e-6 * gap); a wrong vector leaves O(1)
    res = O.eigen_residuals(ops, u, lam) / np.linalg.norm(ops.M @ u, axis=0)
    assert np.max(res) < 2e-2, res
    m.close()
