"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every case runs the same seeded inputs through both sides.  Tolerances:
  * float64 operator applies: rounding of a 27-term sum, |err| <= 1e-13 (|A| |x|)
  * float32 applies: 27 float32 products and sums, |err| <= 4e-6 (|A| |x|)
  * source problems (both sides CG to ||r|| <= 1e-12 ||b||): solutions agree
    within the solve tolerance times the condition number the mesh gives
  * eigenvalues of the float64 path: 1e-10 relative to the oracle, taken
    iterate by iterate for a fixed number of outer iterations
  * eigenvalues of the mixed path: 1e-6 Ha, orbital subspace angles < 1e-5
"""
import json
import math
import os

import numpy as np
import pytest

from gram_budget import gram_tc_error, rotation_tc_error
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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def make_mesh(B, p, precision=None):
    prec = B.PARO_FP64 if precision is None else precision
    m = B.Mesh(p.n, p.lo, p.hi, prec)
    Vq = dev(p.Vq)
    m.set_potential(Vq, p.sigma)
    m._vq = Vq
    return m


def oracle_ops(p):
    return O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)


def rough_potential(n, lo, hi, seed):
    """A smooth well plus seeded noise at the Gauss points (exercises every weight)."""
    x, y, z = W.gauss_point_coords(n, lo, hi)
    rng = np.random.default_rng(seed)
    V = 0.3 * (x ** 2 + y ** 2 + z ** 2) - 1.0 / np.sqrt(x ** 2 + y ** 2 + z ** 2 + 0.3)
    return np.ascontiguousarray((V + 0.2 * rng.standard_normal(V.shape)).ravel())


APPLY_CASES = [((2, 2, 2), 1), ((5, 4, 6), 3), ((7, 6, 9), 4), ((9, 11, 8), 5), ((12, 10, 13), 13),
               ((17, 9, 11), 40)]


@pytest.mark.parametrize("n,N", APPLY_CASES)
def test_apply_fp64_matches_assembled_operators(B, n, N):
    lo, hi = (-1.5, -2.0, -1.0), (2.5, 1.0, 1.75)
    rng = np.random.default_rng(100 + N)
    nI = (n[0] - 1) * (n[1] - 1) * (n[2] - 1)
    p = W.Problem("apply", n, lo, hi, rough_potential(n, lo, hi, N), 0.7, rng.standard_normal((nI, N)), 0)
    ops = oracle_ops(p)
    m = make_mesh(B, p)
    X = dev(p.U0)
    Y = torch.empty_like(X)
    for op, A in ((B.PARO_OP_A, ops.A), (B.PARO_OP_H, ops.H), (B.PARO_OP_M, ops.M)):
        m.apply(op, X, Y)
        ref = A @ p.U0
        bound = abs(A) @ np.abs(p.U0)
        err = np.abs(host(Y) - ref)
        assert np.all(err <= 1e-13 * bound + 1e-300), (op, err.max(), bound.max())
    m.close()


@pytest.mark.parametrize("n,N", APPLY_CASES)
def test_apply_float_float_matches_assembled_operators(B, n, N):
    # Float-float arithmetic (the mixed path's float64-accurate applies).  Bound:
    # values and weights are split to ~48 bits (2^-48 relative); every product
    # drops lo*lo and rounds its cross terms to float32 (2^-48 of |w x|); the lo
    # accumulator rounds at 2^-24 of itself, itself <= 2^-24 of the sum; 27 terms
    # and a handful of roundings each give |err| <= ~100 * 2^-48 * (|A| |x|).
    lo, hi = (-1.5, -2.0, -1.0), (2.5, 1.0, 1.75)
    rng = np.random.default_rng(300 + N)
    nI = (n[0] - 1) * (n[1] - 1) * (n[2] - 1)
    p = W.Problem("apply_ff", n, lo, hi, rough_potential(n, lo, hi, 11 + N), 0.7, rng.standard_normal((nI, N)), 0)
    ops = oracle_ops(p)
    m = make_mesh(B, p, B.PARO_MIXED)
    X = dev(p.U0)
    Y = torch.empty_like(X)
    for op, A in ((B.PARO_OP_A, ops.A), (B.PARO_OP_H, ops.H), (B.PARO_OP_M, ops.M)):
        m.apply(op, X, Y, float_float=True)
        ref = A @ p.U0
        bound = abs(A) @ np.abs(p.U0)
        err = np.abs(host(Y) - ref)
        assert np.all(err <= 100 * 2.0 ** -48 * bound + 1e-300), (op, (err / bound).max())
    m.close()


@pytest.mark.parametrize("n,N", APPLY_CASES[1:])
def test_apply_fp32_matches_assembled_operator(B, n, N):
    lo, hi = (-2.0, -2.0, -2.0), (2.0, 2.0, 2.0)
    rng = np.random.default_rng(200 + N)
    nI = (n[0] - 1) * (n[1] - 1) * (n[2] - 1)
    U = rng.standard_normal((nI, N)).astype(np.float32).astype(np.float64)
    p = W.Problem("apply32", n, lo, hi, rough_potential(n, lo, hi, 7 + N), 1.3, U, 0)
    ops = oracle_ops(p)
    m = make_mesh(B, p, B.PARO_MIXED)
    X = dev(U, torch.float32)
    Y = torch.empty_like(X)
    m.apply(B.PARO_OP_A, X, Y)
    ref = ops.A @ U
    bound = abs(ops.A) @ np.abs(U)
    err = np.abs(host(Y) - ref)
    assert np.all(err <= 4e-6 * bound), err.max()
    m.close()


def test_apply_free_box_sine_mode_is_exact_eigenvector(B):
    # closed form: the discrete (K/2, M) eigenpairs are products of sine modes
    n, L = (16, 12, 10), (1.0, 0.75, 0.6)
    lo, hi = tuple(-v for v in L), L
    p = W.Problem("box", n, lo, hi, np.zeros(8 * 16 * 12 * 10), 0.0, np.zeros((1, 1)), 0)
    xyz = W.interior_node_coords(n, lo, hi)
    modes = [(1, 1, 1), (2, 1, 3), (5, 4, 2)]
    U = np.stack([np.sin(a * math.pi * (xyz[:, 0] + L[0]) / (2 * L[0])) *
                  np.sin(b * math.pi * (xyz[:, 1] + L[1]) / (2 * L[1])) *
                  np.sin(c * math.pi * (xyz[:, 2] + L[2]) / (2 * L[2])) for a, b, c in modes], axis=1)
    m = make_mesh(B, p)
    X = dev(U)
    HX = torch.empty_like(X)
    MX = torch.empty_like(X)
    m.apply(B.PARO_OP_H, X, HX)
    m.apply(B.PARO_OP_M, X, MX)
    hx = [2 * L[d] / n[d] for d in range(3)]
    for j, mode in enumerate(modes):
        mu = [6 * (1 - math.cos(k * math.pi / n[d])) / (hx[d] ** 2 * (2 + math.cos(k * math.pi / n[d])))
              for d, k in enumerate(mode)]
        lam = 0.5 * sum(mu)
        r = host(HX)[:, j] - lam * host(MX)[:, j]
        assert np.linalg.norm(r) < 1e-12 * np.linalg.norm(host(HX)[:, j])
    m.close()


def test_orbital_solve_fp64_matches_oracle(B):
    p = W.hydrogen(nc=12, L=6.0, N=5, seed=1100, sigma=2.0)
    ops = oracle_ops(p)
    rr = O.rayleigh_ritz(ops, p.U0)
    ref = O.source_problems(ops, rr.U, rr.lam, 1e-12, 5000)
    m = make_mesh(B, p)
    U = dev(rr.U)
    X = torch.empty_like(U)
    params = B.paro_default_params(solve_tol=1e-12, pcg_maxit=5000, check_every=4)
    rc, st = m.orbital_solve(rr.lam, U, X, params)
    x = host(X)
    assert rc == 0
    assert np.max(np.abs(x - ref.X)) < 1e-9 * np.max(np.abs(ref.X))
    # same recurrences in the same precision: iteration counts agree up to rounding
    assert abs(st.cg_iters - int(ref.iters.sum())) <= 2 * p.N
    assert st.max_relres < 1e-11
    assert st.kernel_launches > 0
    m.close()


def test_orbital_solve_mixed_refinement_reaches_fp64_tolerance(B):
    p = W.harmonic(nc=14, L=6.0, N=7, seed=2100, sigma=0.0)
    ops = oracle_ops(p)
    rr = O.rayleigh_ritz(ops, p.U0)
    ref = O.source_problems(ops, rr.U, rr.lam, 1e-12, 5000)
    m = make_mesh(B, p, B.PARO_MIXED)
    U = dev(rr.U)
    X = torch.empty_like(U)
    params = B.paro_default_params(solve_tol=1e-11, inner_tol=1e-4)
    rc, st = m.orbital_solve(rr.lam, U, X, params)
    assert rc == 0 and st.refine_sweeps >= 2 and st.cg_iters_f32 > 0
    assert st.max_relres <= 1e-11
    assert np.max(np.abs(host(X) - ref.X)) < 1e-8 * np.max(np.abs(ref.X))
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_orbital_solve_many_orbital_blocks_ragged_mesh(B, prec):
    # N = 41 orbitals (padded to 44): the tiled CG kernel splits them into several
    # orbital blocks, the last one ragged; a non-cubic mesh leaves ragged x, y and z tiles
    n, lo, hi = (19, 11, 9), (-4.0, -3.0, -2.5), (4.5, 2.0, 2.0)
    rng = np.random.default_rng(4100)
    x, y, z = W.gauss_point_coords(n, lo, hi)
    Vq = np.ascontiguousarray((0.5 * (x ** 2 + y ** 2 + z ** 2)).ravel())
    ops = O.assemble(O.Mesh(n, lo, hi), Vq, 0.5)
    nI = (n[0] - 1) * (n[1] - 1) * (n[2] - 1)
    U0 = rng.standard_normal((nI, 41))
    rr = O.rayleigh_ritz(ops, U0)
    ref = O.source_problems(ops, rr.U, rr.lam, 1e-12, 5000)
    m = B.Mesh(n, lo, hi, B.PARO_FP64 if prec == "fp64" else B.PARO_MIXED)
    Vd = dev(Vq)
    m.set_potential(Vd, 0.5)
    U = dev(rr.U)
    X = torch.empty_like(U)
    params = B.paro_default_params(solve_tol=1e-11, pcg_maxit=5000, inner_tol=1e-4)
    rc, st = m.orbital_solve(rr.lam, U, X, params)
    assert rc == 0, B.paro_last_error(m.h)
    assert st.max_relres <= 1e-11
    assert np.max(np.abs(host(X) - ref.X)) < 1e-8 * np.max(np.abs(ref.X))
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_orbital_solve_wide_blocks(B, prec):
    # N = 90 (Np = 92): three orbital blocks of the tiled CG, the last one ragged,
    # and reductions over 3 Np > the streaming kernels' thread count
    p = W.harmonic(nc=10, L=5.0, N=90, seed=4200, sigma=1.0)
    ops = oracle_ops(p)
    rr = O.rayleigh_ritz(ops, p.U0)
    ref = O.source_problems(ops, rr.U, rr.lam, 1e-12, 5000)
    m = make_mesh(B, p, B.PARO_FP64 if prec == "fp64" else B.PARO_MIXED)
    U = dev(rr.U)
    X = torch.empty_like(U)
    rc, st = m.orbital_solve(rr.lam, U, X, B.paro_default_params(solve_tol=1e-11, pcg_maxit=5000))
    assert rc == 0, B.paro_last_error(m.h)
    assert st.max_relres <= 1e-11
    assert np.max(np.abs(host(X) - ref.X)) < 1e-8 * np.max(np.abs(ref.X))
    m.close()


@pytest.mark.parametrize("N", [1, 6, 11])
def test_rayleigh_ritz_matches_oracle(B, N):
    p = W.harmonic(nc=10, L=5.0, N=N, seed=3100 + N)
    ops = oracle_ops(p)
    ref = O.rayleigh_ritz(ops, p.U0)
    m = make_mesh(B, p)
    X = dev(p.U0)
    U = torch.empty_like(X)
    lam, st = m.rayleigh_ritz(X, U)
    assert np.max(np.abs(lam - ref.lam) / np.abs(ref.lam)) < 1e-11
    u = host(U)
    G = u.T @ (ops.M @ u)
    assert np.max(np.abs(G - np.eye(N))) < 1e-12
    assert np.max(O.subspace_angles_M(ops.M, u, ref.U)) < 1e-8
    # column by column (Ritz values are simple here): same vector up to sign
    for j in range(N):
        s = np.sign(u[:, j] @ (ops.M @ ref.U[:, j]))
        assert np.max(np.abs(s * u[:, j] - ref.U[:, j])) < 1e-7 * np.max(np.abs(ref.U[:, j]))
    # rotation in place: X and U_out may alias
    lam2, _ = m.rayleigh_ritz(X, X)
    assert np.max(np.abs(lam2 - lam)) < 1e-13 * np.max(np.abs(lam))
    assert np.max(np.abs(host(X) - u)) < 1e-13 * np.max(np.abs(u))
    m.close()


def test_rayleigh_ritz_of_ill_conditioned_guesses_on_a_mixed_handle(B):
    """48 raw Gaussian guesses on a 12^3 mesh (overlap condition ~7e7): the fast
    Rayleigh-Ritz of a mixed handle (tensor-core Grams from 24-bit inputs,
    float-float eigensolve) cannot resolve them, so the step falls back to float64
    Grams and eigensolve; the Ritz values match the oracle's float64 step."""
    p = W.harmonic(nc=12, L=5.0, N=48, seed=7100, sigma=0.0)
    ops = oracle_ops(p)
    ref = O.rayleigh_ritz(ops, p.U0)
    m = make_mesh(B, p, B.PARO_MIXED)
    X = dev(p.U0)
    U = torch.empty_like(X)
    lam, st = m.rayleigh_ritz(X, U)
    # float64 arithmetic on an overlap of condition ~7e7: agreement to ~1e-16 x cond
    assert np.max(np.abs(lam - ref.lam) / np.abs(ref.lam)) < 1e-7, np.max(np.abs(lam - ref.lam) / np.abs(ref.lam))
    u = host(U)
    assert np.max(np.abs(u.T @ (ops.M @ u) - np.eye(48))) < 1e-7
    m.close()


@pytest.mark.parametrize("N", [3, 20, 33, 64, 90, 128, 200])
def test_rayleigh_ritz_tensor_core_grams_match_oracle(B, N):
    # mixed handles form both Gram matrices on the tensor cores (tcgen05, exact
    # products of BF16 digits of the inputs rounded to 24 bits below their chunk's
    # column maximum, float-float across 128-node chunks); 128 x 64 blocks for
    # N > 32.  Input as inside the ParO loop: near M-orthonormal (Ritz vectors of
    # the guesses plus a 1e-2 perturbation; the error of any Gram is amplified by
    # cond(X^T M X)).  Bounds: 10x the budget of tests/gram_budget.py.
    p = W.harmonic(nc=20, L=6.0, N=N, seed=3400 + N, sigma=1.0)
    ops = oracle_ops(p)
    rng = np.random.default_rng(3500 + N)
    X0 = O.rayleigh_ritz(ops, p.U0).U
    X0 = X0 + 1e-2 * np.max(np.abs(X0)) * rng.standard_normal(X0.shape)
    ref = O.rayleigh_ritz(ops, X0)
    m = make_mesh(B, p, B.PARO_MIXED)
    X = dev(X0)
    U = torch.empty_like(X)
    lam, st = m.rayleigh_ritz(X, U)
    assert st.rr_tc_steps == (1 if N <= 256 else 0)
    # the Grams' error, and how the small eigenproblem passes it on: with C the
    # G_B-orthonormal eigenvectors (||C||^2 = 1 / lambda_min(G_B)), U^T M U - I =
    # -C^T dG_B C and a Ritz value moves by about (||dG_A|| + |theta| ||dG_B||) ||C||^2
    GB = X0.T @ (ops.M @ X0)
    lmin = np.linalg.eigvalsh(0.5 * (GB + GB.T))[0]
    eB = gram_tc_error(p.n, X0, ops.M @ X0)
    eA = gram_tc_error(p.n, X0, ops.H @ X0)
    scale = np.max(np.abs(ref.lam))
    err = np.max(np.abs(lam - ref.lam))
    assert err < 10 * (eA + scale * eB) / lmin, (err, (eA + scale * eB) / lmin)
    assert err < 1e-6  # the mixed path's eigenvalue target
    u = host(U)
    orth = np.max(np.abs(u.T @ (ops.M @ u) - np.eye(N)))
    # the rotation U = X C runs on the tensor cores too (in 128-orbital K and column
    # blocks above 128), from the same 24-bit inputs; its rounding adds rotation_tc_error
    eR = rotation_tc_error(X0, ref.C, ops.M @ ref.U)
    assert orth < 10 * (eB / lmin + eR), (orth, eB / lmin, eR)
    # single Ritz vectors whose Ritz value is separated from its neighbours (M-principal
    # angles: normalisation errors of the size bounded above do not count as angles)
    gaps = np.minimum(np.diff(ref.lam, prepend=-np.inf), np.diff(ref.lam, append=np.inf))
    sep = np.flatnonzero(gaps > 1e-2 * scale)
    assert sep.size > 0
    for i in sep:
        assert O.subspace_angles_M(ops.M, u[:, [i]], ref.U[:, [i]])[0] < 1e-5
    m.close()


def test_iterate_fp64_iterate_by_iterate(B):
    # fixed number of outer iterations from identical inputs, both sides in float64
    p = W.hydrogen(nc=12, L=8.0, N=5, seed=1200, sigma=2.0)
    ops = oracle_ops(p)
    ref = O.paro(ops, p.U0, pcg_tol=1e-12, fixed_outer=6)
    m = make_mesh(B, p)
    U = dev(p.U0)
    params = B.paro_default_params(fixed_outer=6, solve_tol=1e-12, check_every=8)
    rc, lam, st = m.iterate(U, None, params)
    assert rc == 0 and st.outer_iters == 6
    assert np.max(np.abs(lam - ref.lam) / np.abs(ref.lam)) < 1e-10
    u = host(U)
    assert np.max(np.abs(u.T @ (ops.M @ u) - np.eye(5))) < 1e-12
    assert np.max(O.subspace_angles_M(ops.M, u, ref.U)) < 1e-7
    m.close()


def test_hydrogen_32_converges_to_discrete_spectrum(B):
    # full 32^3 hydrogen workload: tol 1e-8 on |delta lambda|, sigma = 2
    with open(os.path.join(HERE, "golden", "discrete_spectra.json")) as f:
        gold = np.array(json.load(f)["hydrogen_32_L10"]["values"][:5])
    p = W.hydrogen(nc=32, L=10.0, N=5, seed=1000, sigma=2.0)
    m = make_mesh(B, p)
    U = dev(p.U0)
    params = B.paro_default_params(tol=1e-8, max_outer=400, solve_tol=1e-12)
    rc, lam, st = m.iterate(U, None, params)
    assert rc == 0, B.paro_last_error(m.h)
    # stopping at |delta lambda| < 1e-8 leaves ~1e-7 on the slowest level
    assert np.max(np.abs(lam - gold)) < 1e-6, (lam, gold)
    assert np.all(lam >= gold - 1e-9)  # Ritz values bound the discrete ones from above
    u = host(U)
    ops = oracle_ops(p)
    assert np.max(np.abs(u.T @ (ops.M @ u) - np.eye(5))) < 1e-12
    m.close()


def test_mixed_iterate_matches_oracle_to_1e6(B):
    p = W.harmonic(nc=16, L=6.0, N=10, seed=2200, sigma=0.0)
    ops = oracle_ops(p)
    ref = O.paro(ops, p.U0, tol=1e-12, max_outer=300, pcg_tol=1e-12)
    m = make_mesh(B, p, B.PARO_MIXED)
    U = dev(p.U0)
    # the vector error is about the square root of the eigenvalue change at the
    # stop, so angles below 1e-5 need |delta lambda| well below 1e-10
    params = B.paro_default_params(tol=1e-12, max_outer=400, solve_tol=1e-11)
    rc, lam, st = m.iterate(U, None, params)
    assert rc == 0
    assert np.max(np.abs(lam - ref.lam)) < 1e-6
    assert st.cg_iters_f32 > 0
    u = host(U)
    # clusters of (numerically) equal values are compared as subspaces
    for a, b in ((0, 1), (1, 4), (4, 10)):
        assert np.max(O.subspace_angles_M(ops.M, u[:, a:b], ref.U[:, a:b])) < 1e-5
    m.close()


def test_mixed_iterate_with_extra_refinement_sweeps_matches_oracle(B):
    # a loose inner tolerance leaves the first two refinement sweeps short of
    # solve_tol, so the outer iterations take further sweeps after the closing
    # check (which writes H x over the right-hand side; the sweeps after it form
    # the right-hand side again): the same Ritz values and subspaces as the oracle
    p = W.harmonic(nc=12, L=6.0, N=10, seed=2300, sigma=0.0)
    ops = oracle_ops(p)
    ref = O.paro(ops, p.U0, tol=1e-12, max_outer=300, pcg_tol=1e-12)
    m = make_mesh(B, p, B.PARO_MIXED)
    U = dev(p.U0)
    loose = dict(solve_tol=1e-11, inner_tol=1e-2, max_refine=40)
    rc, lam, st = m.iterate(U, None, B.paro_default_params(fixed_outer=1, **loose))
    assert rc == 0
    assert st.refine_sweeps > 2  # the first outer iteration from the initial guesses
    rc, lam, st = m.iterate(U, lam, B.paro_default_params(tol=1e-12, max_outer=400, **loose))
    assert rc == 0
    assert np.max(np.abs(lam - ref.lam)) < 1e-6
    u = host(U)
    for a, b in ((0, 1), (1, 4), (4, 10)):
        assert np.max(O.subspace_angles_M(ops.M, u[:, a:b], ref.U[:, a:b])) < 1e-5
    m.close()


def test_harmonic_32_mixed_converges_to_discrete_spectrum(B):
    with open(os.path.join(HERE, "golden", "discrete_spectra.json")) as f:
        gold = np.array(json.load(f)["harmonic_32_L8"]["values"][:10])
    p = W.harmonic(nc=32, L=8.0, N=10, seed=2300, sigma=0.0)
    m = make_mesh(B, p, B.PARO_MIXED)
    U = dev(p.U0)
    params = B.paro_default_params(tol=1e-9, max_outer=400, solve_tol=1e-10)
    rc, lam, st = m.iterate(U, None, params)
    assert rc == 0
    assert np.max(np.abs(lam - gold)) < 1e-6
    m.close()


def test_mixed_iterate_with_tensor_core_grams_converges_to_discrete_spectrum(B):
    # N = 40 > 32: the loop's Rayleigh-Ritz takes both Grams on the tensor cores; the
    # start on the (ill-conditioned) guesses uses float64 Grams.  The lowest 35
    # values (shells n <= 4) are checked against dense diagonalisation, 5 are buffer.
    import scipy.linalg as sla
    p = W.harmonic(nc=12, L=6.0, N=40, seed=2400, sigma=0.0)
    ops = oracle_ops(p)
    exact = sla.eigh(ops.H.toarray(), ops.M.toarray(), eigvals_only=True, subset_by_index=[0, 34])
    m = make_mesh(B, p, B.PARO_MIXED)
    U = dev(p.U0)
    params = B.paro_default_params(tol=1e-9, max_outer=800, solve_tol=1e-10, n_check=35)
    rc, lam, st = m.iterate(U, None, params)
    assert rc == 0, (st.outer_iters, st.max_dlambda)
    # tensor-core Grams until |delta lambda| < 1e-6 max |lambda|, accurate ones after
    assert 0 < st.rr_tc_steps < st.outer_iters
    assert np.max(np.abs(lam[:35] - exact)) < 1e-6, np.max(np.abs(lam[:35] - exact))
    u = host(U)
    assert np.max(np.abs(u.T @ (ops.M @ u) - np.eye(40))) < 1e-7
    m.close()


def test_errors_are_reported_not_raised_on_device(B):
    p = W.hydrogen(nc=8, L=6.0, N=3, seed=1300, sigma=-3.0)  # A = H - 3M is indefinite
    m = make_mesh(B, p)
    U = dev(p.U0)
    X = torch.empty_like(U)
    rc, _ = m.orbital_solve(np.array([-0.4, -0.1, -0.1]), U, X, allow=(-3, -4))
    assert rc == -3  # PARO_ERR_NOT_SPD
    with pytest.raises(B.ParoError):
        m.orbital_solve(np.zeros(3), U, U)  # X aliases U
    # the handle stays usable after an error
    m.set_potential(m._vq, 2.0)
    rc, _ = m.orbital_solve(np.array([-0.4, -0.1, -0.1]), U, X)
    assert rc == 0
    Ubad = U.clone()
    Ubad[3, 1] = float("nan")
    rc, _ = m.orbital_solve(np.zeros(3), Ubad, X, allow=(-5,))
    assert rc == -5  # PARO_ERR_NONFINITE
    m.close()
    m2 = B.Mesh(p.n, p.lo, p.hi)
    with pytest.raises(B.ParoError) as e:
        m2.rayleigh_ritz(U, X)
    assert e.value.code == -8  # no potential yet
    m2.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_256_orbitals_solve_and_rayleigh_ritz(B, prec):
    # the widest orbital count of the large workload on a small mesh: 8 CG orbital
    # blocks, tensor-core Grams in 2 x 4 blocks and the tensor-core rotation in 2 x 2
    # blocks of 128 (mixed; float64 rotation on float64 handles), the small
    # eigensolve at N = 256 with its work matrices in global memory
    N = 256
    p = W.harmonic(nc=12, L=6.0, N=N, seed=4300, sigma=1.0)
    ops = oracle_ops(p)
    rng = np.random.default_rng(4301)
    # an M-orthonormal block of random vectors (256 Gaussians on 1331 unknowns are
    # numerically dependent)
    Gr = rng.standard_normal((p.n_interior, N))
    Lc = np.linalg.cholesky(Gr.T @ (ops.M @ Gr))
    U0 = np.linalg.solve(Lc, Gr.T).T
    m = make_mesh(B, p, B.PARO_FP64 if prec == "fp64" else B.PARO_MIXED)
    # Step 3 on the Ritz vectors of the guesses
    lam0 = np.linspace(1.5, 8.0, N)
    ref = O.source_problems(ops, U0, lam0, 1e-12, 5000)
    U = dev(U0)
    X = torch.empty_like(U)
    rc, st = m.orbital_solve(lam0, U, X, B.paro_default_params(solve_tol=1e-11, pcg_maxit=5000))
    assert rc == 0 and st.max_relres <= 1e-11
    assert np.max(np.abs(host(X) - ref.X)) < 1e-8 * np.max(np.abs(ref.X))
    # Step 4 on a near-orthonormal block
    X0 = U0 + 1e-2 * np.max(np.abs(U0)) * rng.standard_normal(U0.shape)
    rr = O.rayleigh_ritz(ops, X0)
    Xd = dev(X0)
    Ud = torch.empty_like(Xd)
    lam, st = m.rayleigh_ritz(Xd, Ud)
    scale = np.max(np.abs(rr.lam))
    tol = 1e-10 if prec == "fp64" else 3e-8
    assert np.max(np.abs(lam - rr.lam)) < tol * scale, np.max(np.abs(lam - rr.lam)) / scale
    u = host(Ud)
    assert np.max(np.abs(u.T @ (ops.M @ u) - np.eye(N))) < (1e-10 if prec == "fp64" else 1e-6)
    assert st.rr_tc_steps == (1 if prec == "mixed" else 0)
    m.close()


@pytest.mark.parametrize("N,sizes", [(10, [1, 3, 6]), (70, [1, 3, 6, 10, 15, 21, 14])])
def test_cluster_separated_iterate_matches_oracle(B, N, sizes):
    # eigenvalue separation: one small eigenproblem per shell of the oscillator
    # (after block Gram-Schmidt), iterate by iterate against the oracle; N = 70
    # runs the whole-GPU eigensolve
    p = W.harmonic(nc=10, L=6.0, N=N, seed=4400 + N, sigma=0.5)
    # a well-conditioned start (70 Gaussians on 729 unknowns have cond(X^T M X) ~ 1e9,
    # which the initial float64 Rayleigh-Ritz turns into ~1e-7 differences)
    p.U0 = np.random.default_rng(4500 + N).standard_normal(p.U0.shape)
    ops = oracle_ops(p)
    ref = O.paro(ops, p.U0, pcg_tol=1e-12, fixed_outer=3, clusters=sizes)
    m = make_mesh(B, p)
    U = dev(p.U0)
    params = B.paro_default_params(fixed_outer=3, solve_tol=1e-12).set_clusters(sizes)
    rc, lam, st = m.iterate(U, None, params)
    assert rc == 0
    assert np.max(np.abs(lam - ref.lam) / np.abs(ref.lam)) < 1e-9, np.max(np.abs(lam - ref.lam))
    u = host(U)
    assert np.max(np.abs(u.T @ (ops.M @ u) - np.eye(N))) < 1e-10
    o = 0
    for q in sizes:  # each cluster's span, compared with the oracle's
        assert np.max(O.subspace_angles_M(ops.M, u[:, o:o + q], ref.U[:, o:o + q])) < 1e-6
        o += q
    # sizes that do not add up to N are rejected
    with pytest.raises(B.ParoError):
        m.iterate(dev(p.U0), None, B.paro_default_params(fixed_outer=1).set_clusters(sizes[:-1]))
    m.close()
