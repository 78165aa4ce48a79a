"""Thin ctypes binding of ``libparo.so`` (declared in ``include/paro.h``).

Argument marshalling only: every arithmetic step runs in the CUDA kernels of
the library.  Device arrays are torch CUDA tensors passed by ``data_ptr()``;
host arrays are numpy float64.  The library is loaded from this package's
directory on first use; if it has not been built the call raises (there is no
CPU fallback).

Functions keep the C names: ``paro_mesh_create``, ``paro_set_potential``,
``paro_orbital_solve``, ``paro_rayleigh_ritz``, ``paro_iterate``,
``paro_apply``, ``paro_mesh_destroy``, ``paro_last_error``,
``paro_default_params``.  ``Mesh`` bundles a handle with its stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libparo.so")

PARO_OK = 0
STATUS = {
    0: "PARO_OK", -1: "PARO_ERR_ARG", -2: "PARO_ERR_CUDA", -3: "PARO_ERR_NOT_SPD",
    -4: "PARO_ERR_NOT_CONVERGED", -5: "PARO_ERR_NONFINITE", -6: "PARO_ERR_TIMEOUT",
    -7: "PARO_ERR_OOM", -8: "PARO_ERR_STATE",
}
PARO_FP64, PARO_MIXED = 0, 1
PARO_OP_A, PARO_OP_H, PARO_OP_M = 0, 1, 2
PARO_MARK_DORFLER, PARO_MARK_MAXIMUM = 0, 1
PARO_F64, PARO_F32, PARO_FF = 0, 1, 2
PARO_PRECOND_AUTO, PARO_PRECOND_JACOBI, PARO_PRECOND_MG = -1, 0, 1


class paro_params(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("max_outer", C.c_int), ("n_check", C.c_int),
        ("solve_tol", C.c_double), ("pcg_maxit", C.c_int), ("inner_tol", C.c_double),
        ("max_refine", C.c_int), ("check_every", C.c_int), ("fixed_outer", C.c_int),
        ("profile", C.c_int), ("n_clusters", C.c_int), ("cluster_size", C.POINTER(C.c_int)),
        ("precond", C.c_int), ("mg_nu", C.c_int), ("mg_coarse_sweeps", C.c_int), ("hartree_precond", C.c_int),
        ("wait_polls", C.c_int),
    ]

    def set_clusters(self, sizes):
        """Cluster-separated Rayleigh-Ritz with these consecutive group sizes (None: off)."""
        if not sizes:
            self.n_clusters, self.cluster_size, self._sizes = 0, None, None
            return self
        self._sizes = (C.c_int * len(sizes))(*[int(q) for q in sizes])  # kept alive with the params
        self.n_clusters = len(sizes)
        self.cluster_size = C.cast(self._sizes, C.POINTER(C.c_int))
        return self


class paro_stats(C.Structure):
    _fields_ = [
        ("outer_iters", C.c_int), ("refine_sweeps", C.c_int), ("cg_iters", C.c_longlong),
        ("cg_iters_f32", C.c_longlong), ("cg_iters_max", C.c_int), ("max_relres", C.c_double),
        ("max_dlambda", C.c_double), ("ms_solve", C.c_double), ("ms_rr", C.c_double),
        ("stencil_applies", C.c_longlong), ("kernel_launches", C.c_longlong),
        ("prof_launches", C.c_longlong), ("prof_ms", C.c_double), ("prof_dof_orb", C.c_longlong),
        ("prof_node_passes", C.c_longlong), ("rr_tc_steps", C.c_int),
        ("poisson_cg_iters", C.c_longlong), ("prof_dof_orb_active", C.c_longlong),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ParoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    L.paro_default_params.argtypes = [C.POINTER(paro_params)]
    L.paro_default_params.restype = None
    L.paro_mesh_create.argtypes = [C.POINTER(vp), ip, ip, ip, dp, dp, ip, vp]
    L.paro_mesh_destroy.argtypes = [vp]
    L.paro_set_potential.argtypes = [vp, vp, C.c_double]
    L.paro_orbital_solve.argtypes = [vp, ip, dp, vp, vp, C.POINTER(paro_params), C.POINTER(paro_stats)]
    L.paro_rayleigh_ritz.argtypes = [vp, ip, vp, vp, dp, C.POINTER(paro_stats)]
    L.paro_iterate.argtypes = [vp, ip, vp, dp, C.POINTER(paro_params), C.POINTER(paro_stats)]
    L.paro_apply.argtypes = [vp, ip, ip, ip, vp, vp]
    L.paro_mg_vcycle.argtypes = [vp, ip, vp, vp, C.POINTER(paro_params)]
    L.paro_density.argtypes = [vp, ip, vp, dp, vp]
    L.paro_ks_potential.argtypes = [vp, vp, vp, vp, vp, C.POINTER(paro_params)]
    L.paro_scf_iterate.argtypes = [vp, ip, dp, vp, C.c_double, vp, dp, C.POINTER(paro_params),
                                   C.POINTER(paro_stats)]
    L.paro_ks_density_in.argtypes = [vp, vp]
    L.paro_ks_energy.argtypes = [vp, ip, dp, dp, vp, C.POINTER(paro_params), dp]
    L.paro_last_error.argtypes = [vp]
    L.paro_last_error.restype = C.c_char_p
    L.paro_interior_nodes.argtypes = [vp]
    L.paro_interior_nodes.restype = C.c_longlong
    L.paro_batch_create.argtypes = [C.POINTER(vp), ip]
    L.paro_batch_add.argtypes = [vp, vp, ip, vp, dp, C.POINTER(paro_params)]
    L.paro_batch_size.argtypes = [vp]
    L.paro_batch_iterate.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(paro_stats)]
    L.paro_batch_destroy.argtypes = [vp]
    L.paro_estimate.argtypes = [vp, ip, vp, dp, vp, vp]
    L.paro_mark.argtypes = [C.c_longlong, dp, ip, C.c_double, C.POINTER(C.c_ubyte)]
    L.paro_refine_coords.argtypes = [C.POINTER(C.c_int), dp, C.POINTER(C.c_ubyte), C.POINTER(C.c_int), dp]
    L.paro_transfer.argtypes = [vp, vp, ip, vp, vp]
    L.paro_batch_set_fused.argtypes = [vp, ip]
    L.paro_batch_fused_launches.argtypes = [vp]
    L.paro_batch_fused_launches.restype = C.c_longlong
    L.paro_batch_last_error.argtypes = [vp]
    L.paro_batch_last_error.restype = C.c_char_p
    for f in ("paro_mesh_create", "paro_mesh_destroy", "paro_set_potential", "paro_orbital_solve",
              "paro_rayleigh_ritz", "paro_iterate", "paro_apply", "paro_mg_vcycle", "paro_density", "paro_ks_potential",
              "paro_scf_iterate", "paro_ks_density_in", "paro_ks_energy", "paro_batch_create", "paro_batch_add", "paro_batch_size",
              "paro_batch_iterate", "paro_batch_destroy", "paro_batch_set_fused", "paro_estimate", "paro_mark",
              "paro_refine_coords", "paro_transfer"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(rc, handle, allow=()):
    if rc != PARO_OK and rc not in allow:
        raise ParoError(rc, paro_last_error(handle))
    return rc


def paro_last_error(handle) -> str:
    s = lib().paro_last_error(handle)
    return s.decode() if s else ""


def paro_default_params(**over) -> paro_params:
    p = paro_params()
    lib().paro_default_params(C.byref(p))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def paro_mesh_create(n, lo, hi, precision=PARO_FP64, stream=0):
    h = C.c_void_p()
    lo_a = np.ascontiguousarray(lo, dtype=np.float64)
    hi_a = np.ascontiguousarray(hi, dtype=np.float64)
    rc = lib().paro_mesh_create(C.byref(h), int(n[0]), int(n[1]), int(n[2]), _dptr(lo_a), _dptr(hi_a),
                                int(precision), C.c_void_p(stream))
    _check(rc, None)
    return h


def paro_mesh_create_graded(n, coords, precision=PARO_FP64, stream=0):
    """A graded mesh: coords = three arrays of node coordinates (n_d + 1 each)."""
    h = C.c_void_p()
    ax = [np.ascontiguousarray(c, dtype=np.float64) for c in coords]
    L = lib()
    L.paro_mesh_create_graded.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, C.c_void_p]
    L.paro_mesh_create_graded.restype = C.c_int
    rc = L.paro_mesh_create_graded(C.byref(h), int(n[0]), int(n[1]), int(n[2]), _dptr(ax[0]), _dptr(ax[1]),
                                   _dptr(ax[2]), int(precision), C.c_void_p(stream))
    _check(rc, None)
    return h


def paro_mesh_destroy(h):
    return lib().paro_mesh_destroy(h)


def paro_set_potential(h, Vq_ptr: int, sigma: float):
    return _check(lib().paro_set_potential(h, C.c_void_p(Vq_ptr), float(sigma)), h)


def paro_orbital_solve(h, N, lam: np.ndarray, U_ptr, X_ptr, params=None, stats=None, allow=()):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    rc = lib().paro_orbital_solve(h, int(N), _dptr(lam), C.c_void_p(U_ptr), C.c_void_p(X_ptr),
                                  C.byref(params) if params is not None else None,
                                  C.byref(stats) if stats is not None else None)
    return _check(rc, h, allow)


def paro_rayleigh_ritz(h, N, X_ptr, U_ptr, lam_out: np.ndarray, stats=None):
    assert lam_out.dtype == np.float64 and lam_out.flags.c_contiguous and lam_out.size >= N
    rc = lib().paro_rayleigh_ritz(h, int(N), C.c_void_p(X_ptr), C.c_void_p(U_ptr), _dptr(lam_out),
                                  C.byref(stats) if stats is not None else None)
    return _check(rc, h)


def paro_iterate(h, N, U_ptr, lam: np.ndarray, params=None, stats=None, allow=()):
    assert lam.dtype == np.float64 and lam.flags.c_contiguous and lam.size >= N
    rc = lib().paro_iterate(h, int(N), C.c_void_p(U_ptr), _dptr(lam),
                            C.byref(params) if params is not None else None,
                            C.byref(stats) if stats is not None else None)
    return _check(rc, h, allow)


def mark(eta2: np.ndarray, strategy=PARO_MARK_DORFLER, theta=0.5) -> np.ndarray:
    """Marked cells (booleans, the shape of eta2) by paro_mark (host logic)."""
    e = np.ascontiguousarray(eta2, dtype=np.float64)
    out = np.zeros(e.size, dtype=np.uint8)
    rc = lib().paro_mark(e.size, _dptr(e), int(strategy), float(theta), out.ctypes.data_as(C.POINTER(C.c_ubyte)))
    if rc < 0:
        raise ParoError(rc, "paro_mark")
    return out.reshape(e.shape).astype(bool)


def refine_coords(n, coords, marked):
    """The node coordinates per axis after paro_refine_coords (host logic)."""
    cat = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64) for c in coords]))
    mk = np.ascontiguousarray(marked, dtype=np.uint8).ravel()
    nn = (C.c_int * 3)(*[int(v) for v in n])
    nout = (C.c_int * 3)()
    out = np.zeros(sum(2 * int(v) + 1 for v in n))
    rc = lib().paro_refine_coords(nn, _dptr(cat), mk.ctypes.data_as(C.POINTER(C.c_ubyte)), nout, _dptr(out))
    if rc != PARO_OK:
        raise ParoError(rc, "paro_refine_coords")
    res, o = [], 0
    for d in range(3):
        res.append(out[o:o + nout[d] + 1].copy())
        o += nout[d] + 1
    return tuple(res)


def paro_apply(h, N, op, dtype, X_ptr, Y_ptr):
    return _check(lib().paro_apply(h, int(N), int(op), int(dtype), C.c_void_p(X_ptr), C.c_void_p(Y_ptr)), h)


class Mesh:
    """A mesh handle bound to a torch CUDA stream (torch tensors in and out)."""

    def __init__(self, n, lo, hi, precision=PARO_FP64, stream=None, coords=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libparo needs a CUDA device (no CPU fallback)")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.n = tuple(int(v) for v in n)
        self.n_interior = (self.n[0] - 1) * (self.n[1] - 1) * (self.n[2] - 1)
        if coords is None:
            self.h = paro_mesh_create(self.n, lo, hi, precision, self.stream.cuda_stream)
        else:  # graded: node coordinates per axis (lo, hi unused)
            self.h = paro_mesh_create_graded(self.n, coords, precision, self.stream.cuda_stream)
        self._keep = []

    def close(self):
        if self.h is not None:
            paro_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _dev(self, t, dtype=None):
        import torch

        dtype = dtype or torch.float64
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
            raise ValueError(f"expected a contiguous CUDA {dtype} tensor")
        return t.data_ptr()

    def set_potential(self, Vq, sigma):
        self._keep = [Vq]
        paro_set_potential(self.h, self._dev(Vq), sigma)

    def orbital_solve(self, lam, U, X, params=None, allow=()):
        st = paro_stats()
        rc = paro_orbital_solve(self.h, U.shape[1], np.asarray(lam, dtype=np.float64), self._dev(U), self._dev(X),
                                params, st, allow)
        return rc, st

    def rayleigh_ritz(self, X, U_out):
        N = X.shape[1]
        lam = np.zeros(N)
        st = paro_stats()
        paro_rayleigh_ritz(self.h, N, self._dev(X), self._dev(U_out), lam, st)
        return lam, st

    def iterate(self, U, lam=None, params=None, allow=()):
        N = U.shape[1]
        lam = np.full(N, np.nan) if lam is None else np.array(lam, dtype=np.float64)
        st = paro_stats()
        rc = paro_iterate(self.h, N, self._dev(U), lam, params, st, allow)
        return rc, lam, st

    def estimate(self, U, lam, Vq, eta2):
        """eta2 (device, nx*ny*nz float64) = the error indicators of orbitals U (paro_estimate)."""
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        _check(lib().paro_estimate(self.h, U.shape[1], self._dev(U), _dptr(lam), self._dev(Vq), self._dev(eta2)),
               self.h)

    def transfer_to(self, other, U_from, U_to):
        """U_to (orbitals on `other`'s mesh) = U_from interpolated (paro_transfer)."""
        _check(lib().paro_transfer(self.h, other.h, U_from.shape[1], self._dev(U_from), self._dev(U_to)), other.h)

    def apply(self, op, X, Y, float_float=False):
        """Y = op X.  float32 tensors: float32 weights; float64 tensors: float64
        arithmetic, or float-float arithmetic when float_float (PARO_MIXED handles)."""
        import torch

        if X.dtype == torch.float32:
            dt = PARO_F32
        else:
            dt = PARO_FF if float_float else PARO_F64
        paro_apply(self.h, X.shape[1], op, dt, self._dev(X, X.dtype), self._dev(Y, X.dtype))

    def mg_vcycle(self, R, Z, params=None):
        """Z = B R, one multigrid V-cycle (float32 tensors, PARO_MIXED handles)."""
        import torch

        _check(lib().paro_mg_vcycle(self.h, R.shape[1], self._dev(R, torch.float32), self._dev(Z, torch.float32),
                                    C.byref(params) if params is not None else None), self.h)

    # Kohn-Sham (fields at the Gauss points, float64 device tensors of 8*nx*ny*nz values)
    def density(self, U, occ, rho):
        occ = np.ascontiguousarray(occ, dtype=np.float64)
        _check(lib().paro_density(self.h, U.shape[1], self._dev(U), _dptr(occ), self._dev(rho)), self.h)

    def ks_potential(self, rho, vext, v=None, vh=None, params=None):
        _check(lib().paro_ks_potential(self.h, self._dev(rho), self._dev(vext),
                                        None if v is None else self._dev(v), None if vh is None else self._dev(vh),
                                        C.byref(params) if params is not None else None), self.h)

    def scf_iterate(self, U, occ, vext, mix=0.3, params=None, allow=()):
        N = U.shape[1]
        occ = np.ascontiguousarray(occ, dtype=np.float64)
        lam = np.zeros(N)
        st = paro_stats()
        rc = lib().paro_scf_iterate(self.h, N, _dptr(occ), C.c_void_p(self._dev(vext)), float(mix),
                                     C.c_void_p(self._dev(U)), _dptr(lam),
                                     C.byref(params) if params is not None else None, C.byref(st))
        return _check(rc, self.h, allow), lam, st

    def ks_energy(self, U, occ, lam, params=None):
        """Kohn-Sham electronic energy (band-energy form) of the orbitals U."""
        N = U.shape[1]
        occ = np.ascontiguousarray(occ, dtype=np.float64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        e = np.zeros(1)
        _check(lib().paro_ks_energy(self.h, N, _dptr(occ), _dptr(lam), C.c_void_p(self._dev(U)),
                                    C.byref(params) if params is not None else None, _dptr(e)), self.h)
        return float(e[0])

    def ks_density_in(self, rho):
        _check(lib().paro_ks_density_in(self.h, self._dev(rho)), self.h)


class Batch:
    """Independent systems advanced together by paro_batch_iterate.

    fused=True (default): the correction solves of the mixed-precision systems
    run as one batched launch per refinement sweep; fused=False: a pool of
    `workers` host threads runs each system's loop on its own.
    add(mesh, U, lam=None, params=None): U a CUDA float64 tensor (n_interior x N)
    on the mesh's stream, updated in place; lam None starts with a Rayleigh-Ritz.
    iterate() returns the per-system status codes, eigenvalues and statistics;
    fused_launches() the batched launches of the last iterate.
    """

    def __init__(self, workers=4, fused=True):
        h = C.c_void_p()
        rc = lib().paro_batch_create(C.byref(h), int(workers))
        if rc != PARO_OK:
            raise ParoError(rc, "paro_batch_create")
        self.h = h
        self.items = []
        rc = lib().paro_batch_set_fused(self.h, 1 if fused else 0)
        if rc != PARO_OK:
            raise ParoError(rc, "paro_batch_set_fused")

    def fused_launches(self):
        return int(lib().paro_batch_fused_launches(self.h))

    def last_error(self):
        return lib().paro_batch_last_error(self.h).decode()

    def add(self, mesh, U, lam=None, params=None):
        N = U.shape[1]
        lam = np.full(N, np.nan) if lam is None else np.ascontiguousarray(lam, dtype=np.float64).copy()
        idx = lib().paro_batch_add(self.h, mesh.h, N, C.c_void_p(mesh._dev(U)), _dptr(lam),
                                   C.byref(params) if params is not None else None)
        if idx < 0:
            raise ParoError(idx, "paro_batch_add")
        self.items.append((mesh, U, lam, params))  # keeps U, lam and params alive
        return idx

    def iterate(self):
        n = len(self.items)
        rc = (C.c_int * max(n, 1))()
        st = (paro_stats * max(n, 1))()
        r = lib().paro_batch_iterate(self.h, rc, st)
        if r != PARO_OK and all(int(rc[i]) == PARO_OK for i in range(n)):
            raise ParoError(r, "paro_batch_iterate: " + self.last_error())
        return [int(rc[i]) for i in range(n)], [it[2] for it in self.items], [st[i] for i in range(n)]

    def close(self):
        if self.h is not None:
            lib().paro_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def paro_peak_fma(dtype, iters, out_ptr, stream=0):
    """float32 / float64 FMA rate of the SIMT pipes in TFLOP/s (a measurement aid)."""
    f = lib().paro_peak_fma
    f.argtypes = [C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]
    f.restype = C.c_int
    t = C.c_double(0.0)
    rc = f(int(dtype), int(iters), C.c_void_p(out_ptr), C.byref(t), C.c_void_p(stream))
    _check(rc, None)
    return t.value


def paro_small_eig_static(N, GA_ptr, GB_ptr, C_ptr, theta_ptr, stream=0):
    """Small generalized eigensolve with statically allocated scratch (allocates nothing).

    Returns the status code (0 = PARO_OK); there is no handle, so no message.
    """
    L = lib()
    f = L.paro_small_eig_static
    f.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f(int(N), C.c_void_p(GA_ptr), C.c_void_p(GB_ptr), C.c_void_p(C_ptr), C.c_void_p(theta_ptr),
             C.c_void_p(stream))
