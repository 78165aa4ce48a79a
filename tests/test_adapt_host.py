"""The host logic of the adaptive loop (paro_mark, paro_refine_coords in
libparo.so) against the oracle (oracle/adapt.py), on the CPU: Doerfler and
maximum marking (eqs. 2.2-2.3) of random indicator sets give the same cells,
refinement of marked cells gives the same coordinates, and bad arguments are
refused."""
import ctypes

import numpy as np
import pytest

from oracle import adapt as A
from oracle import paro as O


@pytest.fixture(scope="module")
def B():
    from paper_1405_0260_gb300 import binding

    binding.lib()
    return binding


def test_marking_matches_the_oracle(B):
    rng = np.random.default_rng(8400)
    for shape in ((5, 6, 7), (1, 1, 9), (3, 3, 3)):
        eta2 = rng.random(shape) ** 4
        eta2.ravel()[::5] = eta2.ravel()[0]  # ties
        for theta in (0.05, 0.2, 0.5, 0.9, 0.99):
            assert np.array_equal(B.mark(eta2, B.PARO_MARK_DORFLER, theta), A.mark_dorfler(eta2, theta))
            assert np.array_equal(B.mark(eta2, B.PARO_MARK_MAXIMUM, theta), A.mark_maximum(eta2, theta))


def test_refinement_matches_the_oracle(B):
    rng = np.random.default_rng(8410)
    coords = (np.linspace(0, 1, 8), np.linspace(-1, 2, 7) ** 3, np.linspace(0, 3, 6))
    mesh = O.Mesh((7, 6, 5), None, None, coords=coords)
    for p in (0.02, 0.1, 0.5, 1.0):
        marked = rng.random((5, 6, 7)) < p
        got = B.refine_coords((7, 6, 5), coords, marked)
        ref = A.refine_coords(mesh, marked)
        for d in range(3):
            assert np.array_equal(got[d], ref[d])


def test_bad_arguments_are_refused(B):
    eta2 = np.ones((2, 2, 2))
    for theta in (0.0, 1.0, 1.5, -0.1):
        with pytest.raises(B.ParoError):
            B.mark(eta2, B.PARO_MARK_DORFLER, theta)
    with pytest.raises(B.ParoError):
        B.mark(eta2, 7, 0.5)
    bad = eta2.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(B.ParoError):
        B.mark(bad, B.PARO_MARK_MAXIMUM, 0.5)
    with pytest.raises(B.ParoError):  # coordinates not increasing
        B.refine_coords((2, 2, 2), (np.array([0.0, 1.0, 0.5]), np.arange(3.0), np.arange(3.0)),
                        np.zeros((2, 2, 2), dtype=bool))


def test_device_entry_points_refuse_null_handles_without_a_gpu(B):
    # paro_estimate and paro_transfer check their handles and sizes before any CUDA call
    lib = B.lib()
    lam = (ctypes.c_double * 1)(0.0)
    assert lib.paro_estimate(None, 1, None, lam, None, None) == -1  # PARO_ERR_ARG
    assert lib.paro_transfer(None, None, 1, None, None) == -1
    n = (ctypes.c_int * 3)(2, 2, 2)
    out = (ctypes.c_int * 3)()
    assert lib.paro_refine_coords(n, None, None, out, None) == -1
    assert lib.paro_mark(0, None, 0, 0.5, None) == -1
