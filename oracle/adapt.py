"""Adaptive loop on tensor-product meshes: Solve -> Estimate -> Mark -> Refine
(paper Section 2.1).  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Plain numpy, float64, written from the definitions:

Estimate (Section 2.1 names an a-posteriori error indicator per element,
eta_k(., tau), without a formula; the reading here is the standard residual
indicator of the eigenproblem -1/2 Lap u + V u = lambda u with Q1 elements,
summed over the orbitals):

    eta_tau^2 = sum_i [ h_tau^2 ||(lambda_i - V) u_i||^2_tau
                        + 1/2 sum_{F in d tau, F interior} h_F ||1/2 [d_n u_i]||^2_F ]

  * inside a trilinear element Lap u = 0 exactly, so the element residual is
    (lambda_i - V) u_i; its norm uses the 2x2x2 Gauss points of the cell, where
    V is given (exact for constant V: u^2 has degree 2 per axis);
  * [d_n u] is the jump of the normal derivative across an interior face
    (bilinear on the face, its square integrated exactly with the bilinear
    face mass matrix); each face is shared by two cells, hence the 1/2; faces
    on the Dirichlet boundary carry no jump term;
  * h_tau = diameter of the cell, h_F = diameter of the face.

Mark: Doerfler's strategy, eq. (2.2): a set M of least cardinality with
sum_{tau in M} eta_tau^2 >= theta sum_tau eta_tau^2 (largest indicators first,
ties by cell index); the maximum strategy, eq. (2.3): eta_tau >= theta max eta.

Refine: every marked element refined at least once (Section 2.1).  On a
tensor-product mesh an element is refined by bisecting its three axis
intervals; an interval is bisected once if any marked cell lies in it, so the
new mesh stays a tensor product (the cells sharing an interval are bisected too).

Transfer: the Q1 space of the coarse mesh is contained in that of the refined
mesh (every old node is a new node), so the coarse function is the trilinear
interpolant of its nodal values at the new nodes.

Pins: tests/test_oracle_adapt.py.
"""
from __future__ import annotations

import numpy as np

from .paro import Mesh, gauss_1d, q1_shape

# Bilinear mass matrix of the unit square, corners (0,0), (1,0), (0,1), (1,1).
_FACE_MASS = np.array([[4.0, 2.0, 2.0, 1.0], [2.0, 4.0, 1.0, 2.0], [2.0, 1.0, 4.0, 2.0], [1.0, 2.0, 2.0, 4.0]]) / 36.0


def nodal(mesh: Mesh, U: np.ndarray) -> np.ndarray:
    """Unknowns (n_interior, N) -> nodal values (nz+1, ny+1, nx+1, N), zero on the boundary."""
    nx, ny, nz = mesh.n
    N = U.shape[1]
    W = np.zeros((nz + 1, ny + 1, nx + 1, N))
    W[1:nz, 1:ny, 1:nx, :] = U.reshape(nz - 1, ny - 1, nx - 1, N)
    return W


def indicators(mesh: Mesh, Vq: np.ndarray, lam: np.ndarray, U: np.ndarray) -> np.ndarray:
    """eta_tau^2 of every cell, shape (nz, ny, nx) = [cz][cy][cx] (summed over orbitals)."""
    nx, ny, nz = mesh.n
    N = U.shape[1]
    W = nodal(mesh, U)
    hx, hy, hz = mesh.hc
    HX = hx[None, None, :]
    HY = hy[None, :, None]
    HZ = hz[:, None, None]
    eta2 = np.zeros((nz, ny, nx))
    # element term: (lambda - V) u at the 2x2x2 Gauss points of each cell
    g, gw = gauss_1d()
    l, _ = q1_shape(g)  # l[a][q]
    V = np.asarray(Vq, dtype=np.float64).reshape(nz, ny, nx, 2, 2, 2)
    vol = HX * HY * HZ
    diam2 = HX ** 2 + HY ** 2 + HZ ** 2
    for i in range(N):
        w = W[..., i]
        for qz in range(2):
            for qy in range(2):
                for qx in range(2):
                    uq = np.zeros((nz, ny, nx))
                    for az in range(2):
                        for ay in range(2):
                            for ax in range(2):
                                uq += (l[ax, qx] * l[ay, qy] * l[az, qz]) * w[az:nz + az, ay:ny + ay, ax:nx + ax]
                    wq = gw[qx] * gw[qy] * gw[qz] * vol
                    eta2 += diam2 * wq * ((lam[i] - V[:, :, :, qz, qy, qx]) * uq) ** 2
    # face terms: jumps of the normal derivative across the interior faces
    for i in range(N):
        w = W[..., i]
        # x-faces at node planes a = 1 .. nx-1 (between cells a-1 and a)
        dx = (w[:, :, 1:] - w[:, :, :-1]) / hx[None, None, :]  # (nz+1, ny+1, nx): d/dx in cell cx on its node lines
        jx = dx[:, :, 1:] - dx[:, :, :-1]  # (nz+1, ny+1, nx-1) at face corners
        c = np.stack([jx[:-1, :-1], jx[:-1, 1:], jx[1:, :-1], jx[1:, 1:]], axis=-1)  # corners (y, z) order (0,0),(1,0),(0,1),(1,1)
        area = HY * HZ  # (nz, ny, 1)
        fnorm = area * np.einsum("...a,ab,...b->...", c, _FACE_MASS, c)  # (nz, ny, nx-1)
        hF = np.sqrt(HY ** 2 + HZ ** 2)
        t = 0.5 * hF * 0.25 * fnorm  # 1/2 per cell, |1/2 [d_n u]|^2
        eta2[:, :, :-1] += t
        eta2[:, :, 1:] += t
        # y-faces at node planes b = 1 .. ny-1
        dy = (w[:, 1:, :] - w[:, :-1, :]) / hy[None, :, None]  # (nz+1, ny, nx+1)
        jy = dy[:, 1:, :] - dy[:, :-1, :]  # (nz+1, ny-1, nx+1)
        c = np.stack([jy[:-1, :, :-1], jy[:-1, :, 1:], jy[1:, :, :-1], jy[1:, :, 1:]], axis=-1)  # corners (x, z)
        area = HX * HZ
        fnorm = area * np.einsum("...a,ab,...b->...", c, _FACE_MASS, c)  # (nz, ny-1, nx)
        hF = np.sqrt(HX ** 2 + HZ ** 2)
        t = 0.5 * hF * 0.25 * fnorm
        eta2[:, :-1, :] += t
        eta2[:, 1:, :] += t
        # z-faces at node planes c = 1 .. nz-1
        dz = (w[1:, :, :] - w[:-1, :, :]) / hz[:, None, None]  # (nz, ny+1, nx+1)
        jz = dz[1:] - dz[:-1]  # (nz-1, ny+1, nx+1)
        c = np.stack([jz[:, :-1, :-1], jz[:, :-1, 1:], jz[:, 1:, :-1], jz[:, 1:, 1:]], axis=-1)  # corners (x, y)
        area = HX * HY
        fnorm = area * np.einsum("...a,ab,...b->...", c, _FACE_MASS, c)  # (nz-1, ny, nx)
        hF = np.sqrt(HX ** 2 + HY ** 2)
        t = 0.5 * hF * 0.25 * fnorm
        eta2[:-1] += t
        eta2[1:] += t
    return eta2


def mark_dorfler(eta2: np.ndarray, theta: float) -> np.ndarray:
    """Boolean mask (same shape): eq. (2.2), a least-cardinality set whose
    indicators reach theta of the total (largest first, ties by index)."""
    e = np.asarray(eta2, dtype=np.float64).ravel()
    order = np.argsort(-e, kind="stable")
    total = e.sum()
    mark = np.zeros(e.size, dtype=bool)
    acc = 0.0
    for k in order:
        if acc >= theta * total:
            break
        mark[k] = True
        acc += e[k]
    return mark.reshape(np.shape(eta2))


def mark_maximum(eta2: np.ndarray, theta: float) -> np.ndarray:
    """Boolean mask: eq. (2.3), eta >= theta max eta (on eta^2: >= theta^2 max)."""
    e = np.asarray(eta2, dtype=np.float64)
    return e >= theta * theta * e.max()


def refine_coords(mesh: Mesh, marked: np.ndarray):
    """Node coordinates per axis after bisecting every axis interval that holds a
    marked cell (marked: (nz, ny, nx) booleans)."""
    m = np.asarray(marked, dtype=bool)
    hit = [m.any(axis=(0, 1)), m.any(axis=(0, 2)), m.any(axis=(1, 2))]  # per x, y, z interval
    out = []
    for d in range(3):
        c = mesh.nodes[d]
        new = [c[0]]
        for k in range(len(c) - 1):
            if hit[d][k]:
                new.append(0.5 * (c[k] + c[k + 1]))
            new.append(c[k + 1])
        out.append(np.array(new))
    return tuple(out)


def transfer(coarse: Mesh, fine: Mesh, U: np.ndarray) -> np.ndarray:
    """Trilinear interpolation of the coarse Q1 function U (n_interior, N) at the
    interior nodes of the fine mesh."""
    W = nodal(coarse, U)
    N = U.shape[1]
    idx, t = [], []
    for d in range(3):
        c = coarse.nodes[d]
        p = fine.nodes[d][1:-1]
        k = np.clip(np.searchsorted(c, p, side="right") - 1, 0, len(c) - 2)
        idx.append(k)
        t.append((p - c[k]) / (c[k + 1] - c[k]))
    kx, ky, kz = idx
    tx, ty, tz = t
    out = np.zeros((len(kz), len(ky), len(kx), N))
    for az in range(2):
        wz = (1.0 - tz) if az == 0 else tz
        for ay in range(2):
            wy = (1.0 - ty) if ay == 0 else ty
            for ax in range(2):
                wx = (1.0 - tx) if ax == 0 else tx
                vals = W[np.ix_(kz + az, ky + ay, kx + ax)]
                out += (wz[:, None, None] * wy[None, :, None] * wx[None, None, :])[..., None] * vals
    return out.reshape(-1, N)
