"""The eigensolve entry point that allocates no device memory.

paro_small_eig_static serves callers that cannot call cudaMalloc (an
application that owns all device memory through its own pool, or a
latency-critical loop where an allocation could synchronise the device).  Its
work matrices sit in a fixed device array inside the library.  This test
calls it through the C ABI twice in a row, with different sizes so that the
second call runs on the first call's leftover scratch, and checks it against
the Rayleigh-Ritz step of the existing entry point paro_rayleigh_ritz, within
the tolerances of the other Rayleigh-Ritz parity tests.  The file name sorts
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

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
    C = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
    theta = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = B.paro_small_eig_static(N, GA.data_ptr(), GB.data_ptr(), C.data_ptr(), theta.data_ptr(), stream)
    assert rc == B.PARO_OK
    th = theta.cpu().numpy()
    assert np.max(np.abs(th - lam_ref) / np.abs(lam_ref)) < 1e-11
    Cn = C.cpu().numpy()
    gb = GB.cpu().numpy()
    assert np.max(np.abs(Cn.T @ gb @ Cn - np.eye(N))) < 1e-12
    U = (X @ C).cpu().numpy()
    ur = U_ref.cpu().numpy()
    for j in range(N):
        s = np.sign(U[:, j] @ ur[:, j])
        assert np.max(np.abs(s * U[:, j] - ur[:, j])) < 1e-7 * np.max(np.abs(ur[:, j]))
    m.close()


def test_static_scratch_eigensolve_matches_rayleigh_ritz_twice(B):
    _case(B, 11, 5101)
    _case(B, 4, 5102)


def test_static_scratch_eigensolve_rejects_sizes_beyond_maximum(B):
    N = 129
    G = torch.eye(N, dtype=torch.float64, device="cuda")
    out = torch.empty((N, N), dtype=torch.float64, device="cuda")
    th = torch.empty(N, dtype=torch.float64, device="cuda")
    rc = B.paro_small_eig_static(N, G.data_ptr(), G.data_ptr(), out.data_ptr(), th.data_ptr(), 0)
    assert rc == -1  # PARO_ERR_ARG
    rc = B.paro_small_eig_static(0, G.data_ptr(), G.data_ptr(), out.data_ptr(), th.data_ptr(), 0)
    assert rc == -1
