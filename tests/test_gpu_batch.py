"""Batches of independent systems (paro_batch_*): several meshes, orbital counts,
potentials and precisions advanced concurrently from a pool of host threads, one
CUDA stream per system.  Each system must reach what it reaches alone (the same
algorithm; only the interleaving on the GPU differs), and one of them the
discrete spectrum of dense diagonalisation."""
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


def test_batch_matches_systems_run_alone(B):
    params = B.paro_default_params(tol=1e-9, max_outer=600, solve_tol=1e-11)
    batch = B.Batch(workers=3)
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
