"""Pins of the CPU oracle against what the mathematics fixes (no GPU).

Each test pins one oracle function to something other than itself:
closed forms of the discrete Q1 operators, exact integrals, the discrete
sine spectrum of the free box, textbook harmonic-oscillator and hydrogen
levels, a direct sparse solve, dense brute-force eigenvalues and the
invariants of the Rayleigh-Ritz step.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import paro as O
from paper_1405_0260_gb300 import workloads as W


def _tri(n, d, o):
    """(n x n) tridiagonal with diagonal d and off-diagonals o."""
    return sp.diags([np.full(n - 1, o), np.full(n, d), np.full(n - 1, o)], [-1, 0, 1]).tocsr()


def _k1(n, h):
    return _tri(n - 1, 2.0 / h, -1.0 / h)


def _m1(n, h):
    return _tri(n - 1, 4.0 * h / 6.0, h / 6.0)


def _xm1(n, lo, h):
    """1-D matrix of the exact integrals int x phi_i phi_j over [lo, lo + n h] (interior nodes).

    On the element [x_e, x_e + h] with x = x_e + h t, l0 = 1 - t, l1 = t:
      int x l0 l0 = h (x_e/3 + h/12), int x l0 l1 = h (x_e/6 + h/12), int x l1 l1 = h (x_e/3 + h/4).
    """
    A = np.zeros((n + 1, n + 1))
    for e in range(n):
        xe = lo + e * h
        A[e, e] += h * (xe / 3 + h / 12)
        A[e, e + 1] += h * (xe / 6 + h / 12)
        A[e + 1, e] += h * (xe / 6 + h / 12)
        A[e + 1, e + 1] += h * (xe / 3 + h / 4)
    return sp.csr_matrix(A[1:n, 1:n])


def _kron3(az, ay, ax):
    """Matrix on the interior nodes (x fastest) of a separable operator."""
    return sp.kron(az, sp.kron(ay, ax)).tocsr()


def _mesh(n, L):
    return O.Mesh(n, tuple(-v for v in L), tuple(L))


@pytest.mark.parametrize("n,L", [((4, 5, 6), (1.0, 1.5, 2.0)), ((7, 3, 4), (2.0, 1.0, 0.5))])
def test_stiffness_and_mass_are_kronecker_products(n, L):
    mesh = _mesh(n, L)
    ops = O.assemble(mesh, np.zeros(8 * n[0] * n[1] * n[2]), 0.0)
    hx, hy, hz = mesh.h
    kx, ky, kz = _k1(n[0], hx), _k1(n[1], hy), _k1(n[2], hz)
    mx, my, mz = _m1(n[0], hx), _m1(n[1], hy), _m1(n[2], hz)
    K = _kron3(mz, my, kx) + _kron3(mz, ky, mx) + _kron3(kz, my, mx)
    M = _kron3(mz, my, mx)
    assert abs(ops.K - K).max() < 1e-13 * abs(K).max()
    assert abs(ops.M - M).max() < 1e-15 * abs(M).max() + 1e-300
    assert ops.MV.nnz == 0 or abs(ops.MV).max() == 0.0


def test_constant_potential_is_scaled_mass():
    # two-point Gauss integrates the Q1 mass exactly, so V = c gives c M
    n, L = (5, 4, 6), (1.0, 2.0, 1.5)
    mesh = _mesh(n, L)
    ops = O.assemble(mesh, np.full(8 * 5 * 4 * 6, 2.75), 0.0)
    assert abs(ops.MV - 2.75 * ops.M).max() < 1e-14 * abs(ops.M).max()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_linear_potential_is_exact_integral(axis):
    # V = coordinate along `axis`: degree 3 per axis, integrated exactly by 2-point Gauss.
    n, L = (5, 6, 7), (1.0, 1.25, 0.75)
    mesh = _mesh(n, L)
    x, y, z = W.gauss_point_coords(n, mesh.lo, mesh.hi)
    V = [x, y, z][axis].ravel()
    ops = O.assemble(mesh, V, 0.0)
    m = [_m1(n[d], mesh.h[d]) for d in range(3)]
    m[axis] = _xm1(n[axis], mesh.lo[axis], mesh.h[axis])
    ref = _kron3(m[2], m[1], m[0])
    assert abs(ops.MV - ref).max() < 1e-14 * abs(ref).max()


def test_product_potential_is_exact_integral():
    n, L = (4, 5, 6), (1.0, 1.5, 2.0)
    mesh = _mesh(n, L)
    x, y, z = W.gauss_point_coords(n, mesh.lo, mesh.hi)
    ops = O.assemble(mesh, (x * y * z).ravel(), 0.0)
    ref = _kron3(*[_xm1(n[d], mesh.lo[d], mesh.h[d]) for d in (2, 1, 0)])
    assert abs(ops.MV - ref).max() < 1e-14 * abs(ref).max()


def _box_spectrum(n, h):
    """Closed-form generalized eigenvalues of (K/2, M): 1/2 (mu_a + mu_b + mu_c),
    mu(j) = 6 (1 - cos t) / (h^2 (2 + cos t)), t = j pi / n."""
    mus = []
    for d in range(3):
        t = np.arange(1, n[d]) * math.pi / n[d]
        mus.append(6.0 * (1.0 - np.cos(t)) / (h[d] ** 2 * (2.0 + np.cos(t))))
    lam = 0.5 * (mus[0][None, None, :] + mus[1][None, :, None] + mus[2][:, None, None])
    return np.sort(lam.ravel())


def test_free_box_discrete_spectrum_dense():
    n, L = (6, 5, 7), (1.0, 0.8, 1.3)
    mesh = _mesh(n, L)
    ops = O.assemble(mesh, np.zeros(8 * 6 * 5 * 7), 0.0)
    lam = sla.eigh(ops.H.toarray(), ops.M.toarray(), eigvals_only=True)
    ref = _box_spectrum(n, mesh.h)
    assert np.max(np.abs(lam - ref) / ref) < 1e-12


def test_free_box_sine_mode_fixed_point():
    # an exact discrete eigenpair is a fixed point of the shifted source problem
    n, L = (8, 8, 8), (1.0, 1.0, 1.0)
    mesh = _mesh(n, L)
    sigma = 1.5
    ops = O.assemble(mesh, np.zeros(8 * 512), sigma)
    xyz = mesh.interior_coords()
    u = (np.sin(math.pi * (xyz[:, 0] + 1) / 2) * np.sin(2 * math.pi * (xyz[:, 1] + 1) / 2)
         * np.sin(math.pi * (xyz[:, 2] + 1) / 2))
    lam = _box_spectrum(n, mesh.h)
    h = mesh.h
    mu = [6.0 * (1.0 - math.cos(j * math.pi / 8)) / (h[0] ** 2 * (2.0 + math.cos(j * math.pi / 8))) for j in (1, 2, 1)]
    lam_u = 0.5 * sum(mu)
    assert np.min(np.abs(lam - lam_u)) < 1e-12 * lam_u
    r = ops.H @ u - lam_u * (ops.M @ u)
    assert np.linalg.norm(r) < 1e-13 * np.linalg.norm(ops.H @ u)
    sol = O.source_problems(ops, u[:, None], np.array([lam_u]), 1e-13, 2000)
    assert np.linalg.norm(sol.X[:, 0] - u) < 1e-11 * np.linalg.norm(u)
    assert sol.iters[0] == 0


def test_pcg_matches_direct_solve():
    p = W.hydrogen(nc=10, L=6.0, N=3, seed=11, sigma=2.0)
    mesh = O.Mesh(p.n, p.lo, p.hi)
    ops = O.assemble(mesh, p.Vq, p.sigma)
    rng = np.random.default_rng(5)
    B = rng.standard_normal((mesh.n_interior, 3))
    res = O.pcg(ops.A, B, np.zeros_like(B), 1e-13, 5000)
    Xd = spla.spsolve(ops.A.tocsc(), B)
    assert res.converged.all()
    assert np.max(np.abs(res.X - Xd)) < 1e-10 * np.max(np.abs(Xd))
    # the shifted operator must be SPD at this sigma; a negative shift breaks it
    bad = O.Operators(ops.mesh, ops.K, ops.M, ops.MV, -5.0)
    with pytest.raises(FloatingPointError):
        O.pcg(bad.A, B, np.zeros_like(B), 1e-13, 5000)


def test_rayleigh_ritz_conditions_and_interlacing():
    p = W.harmonic(nc=6, L=4.0, N=5, seed=3)
    mesh = O.Mesh(p.n, p.lo, p.hi)
    ops = O.assemble(mesh, p.Vq, 0.0)
    rr = O.rayleigh_ritz(ops, p.U0)
    N = p.N
    # M-orthonormal Ritz vectors, diagonal projected operator
    G = rr.U.T @ (ops.M @ rr.U)
    assert np.max(np.abs(G - np.eye(N))) < 1e-13
    T = rr.U.T @ (ops.H @ rr.U)
    assert np.max(np.abs(T - np.diag(rr.lam))) < 1e-12 * np.max(np.abs(rr.lam))
    # Ritz conditions on the original pencil
    assert np.max(np.abs(rr.GA @ rr.C - rr.GB @ rr.C * rr.lam[None, :])) < 1e-11 * np.max(np.abs(rr.GA))
    assert np.all(np.diff(rr.lam) >= 0)
    # Cauchy interlacing: Ritz values bound the discrete eigenvalues from above
    lam = sla.eigh(ops.H.toarray(), ops.M.toarray(), eigvals_only=True)
    assert np.all(rr.lam >= lam[:N] - 1e-12)
    assert np.all(rr.lam <= lam[-N:] + 1e-12)


def test_paro_converges_to_dense_spectrum():
    # brute force on a tiny mesh: ParO's converged values are the lowest discrete eigenvalues
    p = W.harmonic(nc=8, L=5.0, N=4, seed=21, sigma=0.0)
    mesh = O.Mesh(p.n, p.lo, p.hi)
    ops = O.assemble(mesh, p.Vq, p.sigma)
    res = O.paro(ops, p.U0, tol=1e-13, max_outer=400, pcg_tol=1e-13)
    lam, vec = sla.eigh(ops.H.toarray(), ops.M.toarray())
    assert np.max(np.abs(res.lam - lam[:4])) < 1e-9
    # eigenvalue error is quadratic in the vector error: vectors are checked at ~sqrt(tol)
    assert np.max(O.eigen_residuals(ops, res.U, res.lam)) < 2e-6
    # {1} and {3}: the lowest four span two complete shells
    assert np.max(O.subspace_angles_M(ops.M, res.U, vec[:, :4])) < 1e-6
    # Ritz values decrease (up to rounding) along the iteration
    hist = np.array(res.history)
    assert np.all(np.diff(hist, axis=0) <= 1e-12)


def test_paro_free_box_lowest_modes():
    p = W.free_box(n=(8, 8, 8), L=(1.0, 1.0, 1.0), N=4, seed=9, sigma=0.5)
    mesh = O.Mesh(p.n, p.lo, p.hi)
    ops = O.assemble(mesh, p.Vq, p.sigma)
    res = O.paro(ops, p.U0, tol=1e-12, max_outer=400, pcg_tol=1e-13)
    ref = _box_spectrum(p.n, mesh.h)[:4]
    assert np.max(np.abs(res.lam - ref) / ref) < 1e-9


def _lowest(ops, k, shift):
    vals = spla.eigsh(ops.H, k=k, M=ops.M, sigma=shift, which="LM", return_eigenvectors=False)
    return np.sort(vals)


def test_harmonic_oscillator_levels_and_rate():
    # w(n + 3/2) with shells 1, 3, 6; the Q1 error falls as h^2 under mesh halving
    errs = []
    for nc in (10, 20):
        p = W.harmonic(nc=nc, L=6.0, N=1, seed=1)
        ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, 0.0)
        lam = _lowest(ops, 10, 1.0)
        errs.append(lam[0] - 1.5)
        if nc == 20:
            assert abs(lam[0] - 1.5) < 0.04
            assert np.all(np.abs(lam[1:4] - 2.5) < 0.12)
            assert np.all(np.abs(lam[4:10] - 3.5) < 0.25)
    ratio = errs[0] / errs[1]
    assert 3.5 < ratio < 4.6, ratio


def _separable_oscillator_spectrum(nc, L, k):
    """Lowest k eigenvalues of the discrete Q1 harmonic oscillator from 1-D problems.

    With V = (x^2 + y^2 + z^2)/2 sampled at the tensor 2-point Gauss points, the
    potential mass matrix splits into (m2/2) x m x m + ... , where m2 is the 1-D
    matrix of the Gauss sums of x^2 phi_i phi_j.  So H = K/2 + M_V = a x m x m +
    m x a x m + m x m x a with a = k/2 + m2/2, and the generalized eigenvalues
    of (H, m x m x m) are all sums mu_a + mu_b + mu_c of the 1-D ones of (a, m).
    """
    h = 2.0 * L / nc
    t = np.array([(1 - 1 / math.sqrt(3)) / 2, (1 + 1 / math.sqrt(3)) / 2])
    m2 = np.zeros((nc + 1, nc + 1))
    for e in range(nc):
        xq = -L + h * (e + t)
        lq = np.stack([1 - t, t])  # basis values at the Gauss points
        for a in range(2):
            for b in range(2):
                m2[e + a, e + b] += np.sum(0.5 * h * xq ** 2 * lq[a] * lq[b])
    a1 = 0.5 * _k1(nc, h).toarray() + 0.5 * m2[1:nc, 1:nc]
    mu = sla.eigh(a1, _m1(nc, h).toarray(), eigvals_only=True)
    mu = np.sort(mu)[: k + 2]
    sums = np.sort((mu[:, None, None] + mu[None, :, None] + mu[None, None, :]).ravel())
    return sums[:k]


def test_harmonic_oscillator_separable_spectrum_dense():
    # the oracle's assembled 3-D operator against the 1-D separable construction
    p = W.harmonic(nc=8, L=4.0, N=1, seed=1)
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, 0.0)
    dense = sla.eigh(ops.H.toarray(), ops.M.toarray(), eigvals_only=True)
    sep = _separable_oscillator_spectrum(8, 4.0, 30)
    assert np.max(np.abs(dense[:30] - sep) / np.abs(sep)) < 1e-11


@pytest.mark.parametrize("key,nc", [("harmonic_32_L8", 32), ("harmonic_64_L8", 64)])
def test_stored_oscillator_spectra_match_separable_form(key, nc):
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "discrete_spectra.json")) as f:
        gold = np.array(json.load(f)[key]["values"])
    sep = _separable_oscillator_spectrum(nc, 8.0, len(gold))
    assert np.max(np.abs(gold - sep)) < 1e-9


def test_hydrogen_ground_state_trend():
    # -Z^2/(2 n^2): the n = 1 level approaches -1/2 and the four n = 2 levels
    # (2s and the 2p triplet, split by the cubic mesh) approach -1/8 from above
    # as the mesh is refined
    vals = []
    for nc in (16, 32):
        p = W.hydrogen(nc=nc, L=10.0, N=1, seed=1)
        ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, 0.0)
        vals.append(_lowest(ops, 5, -0.6))
    exact = np.array([-0.5, -0.125, -0.125, -0.125, -0.125])
    assert -0.5 < vals[1][0] < -0.4
    assert np.all((vals[1][1:] > -0.125) & (vals[1][1:] < -0.1))
    assert np.all(np.abs(vals[1] - exact) < np.abs(vals[0] - exact))


@pytest.mark.slow
def test_paro_on_the_full_hydrogen_workload_reaches_its_discrete_spectrum():
    # the 32^3, N = 5 hydrogen workload as specified (sigma = 2, stop at
    # max |delta lambda| < 1e-8) against the spectrum that shift-invert Lanczos
    # finds for the same assembly (tests/golden/make_golden.py)
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "discrete_spectra.json")) as f:
        gold = np.array(json.load(f)["hydrogen_32_L10"]["values"][:5])
    p = W.hydrogen()
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)
    res = O.paro(ops, p.U0, tol=p.tol, max_outer=400, pcg_tol=1e-12)
    assert res.outer < 400
    # the slowest level (the top of the nearly degenerate 2p shell) is still
    # ~1e-7 above its limit when the change per iteration falls below 1e-8
    assert np.max(np.abs(res.lam - gold)) < 1e-6, (res.lam, gold)
    assert np.all(res.lam >= gold - 1e-10)  # Ritz values bound the discrete ones from above
    assert np.max(np.abs(res.U.T @ (ops.M @ res.U) - np.eye(5))) < 1e-12


def test_subspace_angles_of_same_span_are_zero():
    p = W.harmonic(nc=6, L=4.0, N=4, seed=2)
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, 0.0)
    rng = np.random.default_rng(0)
    T = rng.standard_normal((4, 4))
    ang = O.subspace_angles_M(ops.M, p.U0, p.U0 @ T)
    assert np.max(ang) < 1e-6


def test_subspace_angles_of_known_rotation():
    # span{e1, e2} against span{e1, cos t e2 + sin t e3} in the Euclidean (M = I) product:
    # one zero angle and one angle t, resolved down to tiny t by the sine form
    M = sp.identity(5, format="csr")
    U = np.eye(5)[:, :2]
    for t in (0.3, 1e-6, 1e-10):
        W = np.stack([np.eye(5)[:, 0], math.cos(t) * np.eye(5)[:, 1] + math.sin(t) * np.eye(5)[:, 2]], axis=1)
        ang = O.subspace_angles_M(M, U, W)
        assert abs(ang[0]) < 1e-15 and abs(ang[1] - t) < 1e-6 * t


def test_cluster_separated_rayleigh_ritz_nested_spans_and_block_ritz_conditions():
    # eigenvalue separation (Section 3) with block Gram-Schmidt: the first k clusters'
    # Ritz vectors span exactly the first k clusters' columns of X, all of them are
    # M-orthonormal, and the Ritz conditions hold inside each block (not across)
    p = W.harmonic(nc=8, L=5.0, N=7, seed=31, sigma=0.0)
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, 0.0)
    X = O.rayleigh_ritz(ops, p.U0).U + 0.05 * np.random.default_rng(32).standard_normal((p.n_interior, 7))
    sizes = [1, 3, 3]
    rr = O.rayleigh_ritz_clusters(ops, X, sizes)
    assert np.max(np.abs(rr.U.T @ (ops.M @ rr.U) - np.eye(7))) < 1e-12
    o = 0
    for q in sizes:
        assert np.max(O.subspace_angles_M(ops.M, rr.U[:, :o + q], X[:, :o + q])) < 1e-10
        U = rr.U[:, o:o + q]
        assert np.max(np.abs(U.T @ (ops.H @ U) - np.diag(rr.lam[o:o + q]))) < 1e-11 * np.max(np.abs(rr.lam))
        o += q
    # across blocks H is not diagonalised: the separation leaves the coupling in place
    assert np.max(np.abs(rr.U[:, :1].T @ (ops.H @ rr.U[:, 1:4]))) > 1e-6
    # a single cluster is the full problem
    full = O.rayleigh_ritz(ops, X)
    one = O.rayleigh_ritz_clusters(ops, X, [7])
    assert np.max(np.abs(full.lam - one.lam)) < 1e-12 * np.max(np.abs(full.lam))


def test_cluster_separated_paro_reaches_the_box_spectrum():
    # well-posed initial data (each cluster's guesses near its own eigenspace): ParO with
    # one Rayleigh-Ritz problem per degenerate shell {1}, {3} converges to the closed form
    n, L = (8, 8, 8), (1.0, 1.0, 1.0)
    mesh = _mesh(n, L)
    ops = O.assemble(mesh, np.zeros(8 * 512), 0.5)
    xyz = mesh.interior_coords()

    def mode(a, b, c):
        return (np.sin(a * math.pi * (xyz[:, 0] + 1) / 2) * np.sin(b * math.pi * (xyz[:, 1] + 1) / 2)
                * np.sin(c * math.pi * (xyz[:, 2] + 1) / 2))

    exact = np.stack([mode(1, 1, 1), mode(2, 1, 1), mode(1, 2, 1), mode(1, 1, 2)], axis=1)
    rng = np.random.default_rng(33)
    U0 = exact + 0.05 * rng.standard_normal(exact.shape)
    res = O.paro(ops, U0, tol=1e-12, max_outer=400, pcg_tol=1e-13, clusters=[1, 3])
    ref = _box_spectrum(n, mesh.h)[:4]
    assert np.max(np.abs(res.lam - ref) / ref) < 1e-9


@pytest.mark.parametrize("n", [(2, 2, 2), (2, 3, 4), (3, 3, 3)])
def test_tiny_meshes_have_the_closed_form_spectrum(n):
    # the smallest meshes: one interior node at 2^3; every mode of the box
    L = (1.0, 0.7, 1.3)
    mesh = _mesh(n, L)
    ops = O.assemble(mesh, np.zeros(8 * n[0] * n[1] * n[2]), 0.0)
    lam = sla.eigh(ops.H.toarray(), ops.M.toarray(), eigvals_only=True)
    assert np.max(np.abs(lam - _box_spectrum(n, mesh.h)) / lam) < 1e-13


def test_single_orbital_rayleigh_ritz_is_the_rayleigh_quotient():
    p = W.harmonic(nc=5, L=3.0, N=1, seed=4)
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, 0.0)
    x = p.U0[:, 0]
    rr = O.rayleigh_ritz(ops, p.U0)
    q = (x @ (ops.H @ x)) / (x @ (ops.M @ x))
    assert abs(rr.lam[0] - q) < 1e-14 * abs(q)
    assert abs(rr.U[:, 0] @ (ops.M @ rr.U[:, 0]) - 1.0) < 1e-14


def test_paro_resumes_from_its_state_bit_for_bit():
    # the state of the loop is (U, lambda): two outer iterations, then two more
    # from that state, equal four in one run exactly
    p = W.hydrogen(nc=6, L=5.0, N=3, seed=31, sigma=2.0)
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)
    full = O.paro(ops, p.U0, pcg_tol=1e-12, fixed_outer=4)
    half = O.paro(ops, p.U0, pcg_tol=1e-12, fixed_outer=2)
    rest = O.paro(ops, half.U, pcg_tol=1e-12, fixed_outer=2, lam0=half.lam)
    assert np.array_equal(rest.lam, full.lam) and np.array_equal(rest.U, full.U)


def test_buffer_orbitals_converge_the_occupied_ones_in_fewer_iterations():
    # Algorithm 3.2: iterating N + m orbitals and testing the lowest N converges
    # those N to the same values, faster: the source problems damp the error in
    # orbital i by about (lambda_i + sigma) / (lambda_(N+m+1) + sigma) per step
    outer = []
    for N in (4, 7, 10):
        p = W.harmonic(nc=10, L=5.0, N=N, seed=21, sigma=0.0)
        ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)
        res = O.paro(ops, p.U0, tol=1e-10, max_outer=500, pcg_tol=1e-12, n_check=4)
        lam = _lowest(ops, 4, 1.0)
        assert np.max(np.abs(res.lam[:4] - lam)) < 1e-8
        outer.append(res.outer)
    assert outer[0] > outer[1] > outer[2], outer


@pytest.mark.parametrize("sigma", [0.0, 2.0])
def test_eigenvalue_error_contracts_at_the_shifted_inverse_iteration_rate(sigma):
    # one outer step applies (H + sigma M)^-1 (Lambda + sigma) M to the orbitals and
    # projects: the vector error of the highest tested level falls by about
    # (lambda_N + sigma) / (lambda_(N+1) + sigma) per step, its eigenvalue error by
    # the square of that
    p = W.harmonic(nc=10, L=5.0, N=4, seed=21, sigma=sigma)
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)
    lam = _lowest(ops, 5, 1.0)
    res = O.paro(ops, p.U0, tol=1e-13, max_outer=200, pcg_tol=1e-13)
    err = np.abs(np.array(res.history)[:, 3] - lam[3])
    mid = (err[:-1] < 1e-4) & (err[1:] > 1e-11)
    observed = np.median(err[1:][mid] / err[:-1][mid])
    predicted = ((lam[3] + sigma) / (lam[4] + sigma)) ** 2
    assert mid.sum() >= 5 and abs(observed / predicted - 1) < 0.06, (observed, predicted)
