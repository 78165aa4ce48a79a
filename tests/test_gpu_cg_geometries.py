"""Every geometry of the single-pass CG kernel against the oracle (Step 3, the N
shifted source problems of eq. 3.2).

The autotuner keeps one geometry per (mesh, orbital count): tile shape, orbital
block width, one or two nodes per thread.  Here each candidate is forced in turn
(PARO_CG2_GEOMETRY=<i>, read when a handle plans its solver) on meshes whose node
counts leave ragged tiles in x, y and z, and the mixed-precision solve (float32
CG in float-float refinement) must reach the oracle's solution of the same
source problems.  The plan each handle used is read from its PARO_PRINT_PLAN line.
"""
import re

import numpy as np
import pytest

from oracle import paro as O
from paper_1405_0260_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

PLAN = re.compile(r"paro single-pass CG plan: tile (\d+)x(\d+), (\d) nodes a thread, block (\d+) orbitals.*geometry (\w+)")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_0260_gb300 import binding

    binding.lib()
    return binding


def problem(n, N, seed):
    lo, hi = (-4.0, -3.5, -2.5), (4.5, 3.0, 2.0)
    x, y, z = W.gauss_point_coords(n, lo, hi)
    Vq = np.ascontiguousarray((0.5 * (x ** 2 + y ** 2 + z ** 2)).ravel())
    ops = O.assemble(O.Mesh(n, lo, hi), Vq, 0.5)
    nI = (n[0] - 1) * (n[1] - 1) * (n[2] - 1)
    rr = O.rayleigh_ritz(ops, np.random.default_rng(seed).standard_normal((nI, N)))
    ref = O.source_problems(ops, rr.U, rr.lam, 1e-12, 5000)
    return lo, hi, Vq, rr, ref


@pytest.mark.parametrize("n,N", [((21, 19, 9), 20), ((35, 14, 7), 8), ((18, 17, 6), 41)])
def test_every_single_pass_geometry_solves_the_source_problems(B, capfd, monkeypatch, n, N):
    lo, hi, Vq, rr, ref = problem(n, N, 7000 + N)
    monkeypatch.setenv("PARO_PRINT_PLAN", "1")
    seen = set()
    for i in range(32):
        monkeypatch.setenv("PARO_CG2_GEOMETRY", str(i))
        capfd.readouterr()
        m = B.Mesh(n, lo, hi, B.PARO_MIXED)
        Vd = torch.from_numpy(Vq).cuda()
        m.set_potential(Vd, 0.5)
        U = torch.from_numpy(np.ascontiguousarray(rr.U)).cuda()
        X = torch.empty_like(U)
        rc, st = m.orbital_solve(rr.lam, U, X, B.paro_default_params(solve_tol=1e-11, inner_tol=1e-4))
        torch.cuda.synchronize()
        # the plan is made (and printed) when the handle first solves
        plans = [g for g in PLAN.findall(capfd.readouterr().err) if g[4] == "forced"]
        if not plans:  # past the last candidate: the autotuner ran instead
            m.close()
            break
        assert rc == 0, (plans[-1], B.paro_last_error(m.h))
        assert st.cg_iters_f32 > 0 and st.max_relres <= 1e-11, plans[-1]
        err = np.max(np.abs(X.cpu().numpy() - ref.X)) / np.max(np.abs(ref.X))
        assert err < 1e-8, (plans[-1], err)
        seen.add(plans[-1][:4])
        m.close()
    assert len(seen) >= 3, seen
    # the candidates include both thread layouts wherever a 128-node tile fits the limits
    if N <= 20:
        assert {g[2] for g in seen} == {"1", "2"}, seen
