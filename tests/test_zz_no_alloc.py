"""The eigensolve entry point that allocates no device memory.

paro_small_eig_static serves callers that cannot call cudaMalloc (an
application that owns all device memory through its own pool, or a
latency-critical loop where an allocation could synchronise the device).  Its
work matrices sit in a fixed device array inside the library.  These tests
call it through the C ABI several times in a row, with different sizes so that
each call runs on the previous call's leftover scratch, and check it against
the Rayleigh-Ritz step of the existing entry point paro_rayleigh_ritz (same
Ritz values and vectors) and against scipy's float64 generalized eigensolver on
the same host matrices, at the largest accepted size too.  An indefinite G_B is
reported as not positive definite with C and theta left untouched, and the
next call is unaffected.  The file name sorts last so that a run stopping at
the first failure has run every other test.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1405_0260_gb300 import workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MAX_N = 128  # PARO_STATIC_EIG_MAX_N


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_0260_gb300 import binding

    binding.lib()
    return binding


def _call(B, GA, GB):
    N = GA.shape[0]
    C = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
    theta = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = B.paro_small_eig_static(N, GA.data_ptr(), GB.data_ptr(), C.data_ptr(), theta.data_ptr(), stream)
    return rc, C.cpu().numpy(), theta.cpu().numpy()


def _check_against_scipy(ga, gb, C, th, tol):
    # scipy's float64 generalized eigensolver (LAPACK) on the same host matrices
    w = sla.eigh(ga, gb, eigvals_only=True)
    scale = np.max(np.abs(w))
    assert np.max(np.abs(th - w)) < tol * scale, np.max(np.abs(th - w)) / scale
    N = ga.shape[0]
    assert np.max(np.abs(C.T @ gb @ C - np.eye(N))) < tol * 10
    assert np.max(np.abs(C.T @ ga @ C - np.diag(th))) < tol * 10 * scale


def _case(B, N, seed):
    p = W.harmonic(nc=10, L=5.0, N=N, seed=seed)
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_FP64)
    Vq = torch.from_numpy(p.Vq).cuda()
    m.set_potential(Vq, p.sigma)
    X = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
    U_ref = torch.empty_like(X)
    lam_ref, _ = m.rayleigh_ritz(X, U_ref)
    HX = torch.empty_like(X)
    MX = torch.empty_like(X)
    m.apply(B.PARO_OP_H, X, HX)
    m.apply(B.PARO_OP_M, X, MX)
    torch.cuda.synchronize()
    GA = (X.T @ HX).contiguous()
    GB = (X.T @ MX).contiguous()
    rc, Cn, th = _call(B, GA, GB)
    assert rc == B.PARO_OK
    # the existing entry point: same Ritz values and vectors
    assert np.max(np.abs(th - lam_ref) / np.abs(lam_ref)) < 1e-11
    ga, gb = GA.cpu().numpy(), GB.cpu().numpy()
    ga, gb = 0.5 * (ga + ga.T), 0.5 * (gb + gb.T)
    assert np.max(np.abs(Cn.T @ gb @ Cn - np.eye(N))) < 1e-12
    U = X.cpu().numpy() @ Cn
    ur = U_ref.cpu().numpy()
    for j in range(N):
        s = np.sign(U[:, j] @ ur[:, j])
        assert np.max(np.abs(s * U[:, j] - ur[:, j])) < 1e-7 * np.max(np.abs(ur[:, j]))
    # and scipy: these overlap matrices are ill-conditioned (Gaussian guesses), so
    # the eigenvalues agree to the conditioning, not to the last bits
    w = sla.eigh(ga, gb, eigvals_only=True)
    assert np.max(np.abs(th - w) / np.abs(w)) < 1e-9
    m.close()


def _spd_pair(N, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((N, N))
    ga = 0.5 * (A + A.T)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    gb = (Q * rng.uniform(0.5, 2.0, N)) @ Q.T
    gb = 0.5 * (gb + gb.T)
    return ga, gb


def test_static_scratch_eigensolve_matches_rayleigh_ritz_twice(B):
    _case(B, 11, 5101)
    _case(B, 4, 5102)


@pytest.mark.parametrize("N", [MAX_N, 37])
def test_static_scratch_eigensolve_matches_scipy(B, N):
    # well-conditioned pencils (cond(G_B) <= 4): float64 agreement to ~1e-13
    ga, gb = _spd_pair(N, 5200 + N)
    rc, C, th = _call(B, torch.from_numpy(ga).cuda(), torch.from_numpy(gb).cuda())
    assert rc == B.PARO_OK
    _check_against_scipy(ga, gb, C, th, 1e-12)


def test_static_scratch_eigensolve_reports_an_indefinite_overlap(B):
    N = 12
    ga, _ = _spd_pair(N, 5301)
    gb = np.diag([1.0, -1.0] * (N // 2))
    rc, C, th = _call(B, torch.from_numpy(ga).cuda(), torch.from_numpy(gb).cuda())
    assert rc == -3  # PARO_ERR_NOT_SPD
    assert np.all(np.isnan(C)) and np.all(np.isnan(th))  # not written
    # the status word is cleared for the next call
    ga, gb = _spd_pair(N, 5302)
    rc, C, th = _call(B, torch.from_numpy(ga).cuda(), torch.from_numpy(gb).cuda())
    assert rc == B.PARO_OK
    _check_against_scipy(ga, gb, C, th, 1e-12)


def test_static_scratch_eigensolve_rejects_sizes_beyond_maximum(B):
    N = MAX_N + 1
    G = torch.eye(N, dtype=torch.float64, device="cuda")
    out = torch.empty((N, N), dtype=torch.float64, device="cuda")
    th = torch.empty(N, dtype=torch.float64, device="cuda")
    rc = B.paro_small_eig_static(N, G.data_ptr(), G.data_ptr(), out.data_ptr(), th.data_ptr(), 0)
    assert rc == -1  # PARO_ERR_ARG
    rc = B.paro_small_eig_static(0, G.data_ptr(), G.data_ptr(), out.data_ptr(), th.data_ptr(), 0)
    assert rc == -1
