"""Batches of independent systems (paro_batch_*): several meshes, orbital counts,
potentials and precisions advanced together.  In batched mode the float32
correction solves of the mixed-precision systems run as one cooperative launch
per refinement sweep (k_cg2b over every system still iterating); in pool mode
each system runs alone from a pool of host threads.  Each system must reach what
it reaches alone (the same algorithm; only the order of the floating-point sums
differs), and one of them the discrete spectrum of dense diagonalisation."""
import os

import numpy as np
import pytest

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


def systems():
    """(problem, precision) pairs: uneven meshes, N and potentials."""
    # whole shells (harmonic: 1 + 3 (+ 6); hydrogen-like: 1 + 4), so that no
    # (near-)degenerate cluster is cut by N
    return [
        (W.harmonic(nc=12, L=6.0, N=10, seed=6100, sigma=0.0), 1),
        (W.hydrogen(nc=10, L=6.0, N=5, seed=6200, sigma=2.0), 0),
        (W.harmonic(nc=9, L=5.0, N=4, seed=6300, sigma=0.0), 1),
        (W.hydrogen(nc=14, L=8.0, N=5, seed=6400, sigma=2.0), 1),
        (W.harmonic(nc=8, L=4.0, N=4, seed=6500, sigma=0.5), 0),
    ]


def run_alone(B, p, prec, params):
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED if prec else B.PARO_FP64, stream=stream)
        vq = torch.from_numpy(np.ascontiguousarray(p.Vq)).cuda()
        m.set_potential(vq, p.sigma)
        U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
        rc, lam, st = m.iterate(U, None, params)
    stream.synchronize()
    m.close()
    return rc, lam


@pytest.mark.parametrize("fused", [True, False])
def test_batch_matches_systems_run_alone(B, fused):
    params = B.paro_default_params(tol=1e-9, max_outer=600, solve_tol=1e-11)
    batch = B.Batch(workers=3, fused=fused)
    keep = []
    for p, prec in systems():
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED if prec else B.PARO_FP64, stream=stream)
            vq = torch.from_numpy(np.ascontiguousarray(p.Vq)).cuda()
            m.set_potential(vq, p.sigma)
            U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
        torch.cuda.synchronize()
        batch.add(m, U, None, params)
        keep.append((m, vq, U, stream))
    rcs, lams, stats = batch.iterate()
    torch.cuda.synchronize()
    assert all(rc == 0 for rc in rcs), rcs
    assert all(st.outer_iters > 0 for st in stats)
    # batched mode: the three mixed systems' correction solves ran as batched launches
    # (at least two refinement sweeps an outer iteration of the longest of them)
    nmix_outer = max(st.outer_iters for (p, prec), st in zip(systems(), stats) if prec)
    if fused:
        assert batch.fused_launches() >= 2 * nmix_outer, (batch.fused_launches(), nmix_outer)
    else:
        assert batch.fused_launches() == 0
    for (p, prec), lam in zip(systems(), lams):
        rc, ref = run_alone(B, p, prec, params)
        assert rc == 0
        # the stop leaves |delta lambda| < 1e-9; the two runs differ in rounding only
        assert np.max(np.abs(lam - ref)) < 1e-7 * max(1.0, np.max(np.abs(ref))), (p.name, lam, ref)
    # the harmonic-oscillator system against dense diagonalisation of the same operator
    p = systems()[2][0]
    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, 0.0)
    import scipy.linalg as sla

    exact = sla.eigh(ops.H.toarray(), ops.M.toarray(), eigvals_only=True, subset_by_index=[0, 3])
    assert np.max(np.abs(lams[2][:4] - exact)) < 1e-6
    batch.close()
    for m, *_ in keep:
        m.close()


def test_batch_rejects_a_handle_twice(B):
    p = W.harmonic(nc=8, L=4.0, N=4, seed=6600, sigma=0.0)
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_FP64)
    vq = torch.from_numpy(np.ascontiguousarray(p.Vq)).cuda()
    m.set_potential(vq, 0.0)
    U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
    batch = B.Batch(workers=2)
    batch.add(m, U)
    with pytest.raises(B.ParoError):
        batch.add(m, U.clone())
    batch.close()
    m.close()


def _mixed_systems():
    """Mixed-precision systems on ragged meshes (uneven tile columns and z-chunks),
    orbital counts that leave partial orbital blocks and groups."""
    return [
        W.harmonic(nc=13, L=6.0, N=10, seed=6710, sigma=0.0),
        W.hydrogen(nc=11, L=6.0, N=5, seed=6720, sigma=2.0),
        W.harmonic(nc=17, L=6.5, N=20, seed=6730, sigma=0.0),
        W.harmonic(nc=9, L=5.0, N=4, seed=6740, sigma=0.0),
    ]


def _make(B, p):
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED, stream=stream)
        vq = torch.from_numpy(np.ascontiguousarray(p.Vq)).cuda()
        m.set_potential(vq, p.sigma)
        U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
    torch.cuda.synchronize()
    return m, vq, U, stream


@pytest.mark.parametrize("geometry", [0, 1, 2, 3, 5, 9])
def test_batched_correction_solves_match_the_oracle_for_forced_geometries(B, geometry, monkeypatch):
    """A fixed number of outer iterations in one batch, every system against the
    oracle's ParO from the same start (the same iterates up to the solve
    tolerance): candidate geometries forced one by one (two-node and one-node
    tiles, several block widths)."""
    monkeypatch.setenv("PARO_CG2B_GEOMETRY", str(geometry))
    params = B.paro_default_params(fixed_outer=3, solve_tol=1e-10)
    batch = B.Batch()
    keep = []
    probs = _mixed_systems()
    for p in probs:
        m, vq, U, stream = _make(B, p)
        batch.add(m, U, None, params)
        keep.append((m, vq, U, stream))
    rcs, lams, stats = batch.iterate()
    torch.cuda.synchronize()
    assert all(rc == 0 for rc in rcs), rcs
    assert batch.fused_launches() >= 6
    for p, lam, (m, vq, U, stream) in zip(probs, lams, keep):
        ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)
        ref = O.paro(ops, p.U0, pcg_tol=1e-10, fixed_outer=3)
        # the mixed path's bar against the float64 oracle: 1e-6 Ha
        assert np.max(np.abs(lam - ref.lam)) < 1e-6, (p.name, lam, ref.lam)
        # the vectors: M-orthonormal, and spanning the oracle's iterate
        u = U.cpu().numpy()
        assert np.max(np.abs(u.T @ (ops.M @ u) - np.eye(u.shape[1]))) < 1e-6
    batch.close()
    for m, *_ in keep:
        m.close()


def test_batched_wait_that_runs_out_is_reported_to_every_system(B):
    """wait_polls = 1: the batched kernel's first ring wait runs out; every mixed
    system of the launch reports PARO_ERR_TIMEOUT, and the same handles then
    iterate normally in a new batch."""
    probs = _mixed_systems()[:3]
    keep = []
    batch = B.Batch()
    for p in probs:
        m, vq, U, stream = _make(B, p)
        batch.add(m, U, None, B.paro_default_params(fixed_outer=1, solve_tol=1e-10, wait_polls=1))
        keep.append((m, vq, U, stream))
    rcs, _, _ = batch.iterate()
    torch.cuda.synchronize()
    assert all(rc == -6 for rc in rcs), rcs
    batch.close()
    batch = B.Batch()
    for p, (m, vq, U, stream) in zip(probs, keep):
        U.copy_(torch.from_numpy(np.ascontiguousarray(p.U0)).cuda())
        batch.add(m, U, None, B.paro_default_params(fixed_outer=2, solve_tol=1e-10))
    torch.cuda.synchronize()
    rcs, lams, _ = batch.iterate()
    torch.cuda.synchronize()
    assert all(rc == 0 for rc in rcs), rcs
    for p, lam in zip(probs, lams):
        ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)
        ref = O.paro(ops, p.U0, pcg_tol=1e-10, fixed_outer=2)
        assert np.max(np.abs(lam - ref.lam)) < 1e-6
    batch.close()
    for m, *_ in keep:
        m.close()
