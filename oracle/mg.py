"""FP64 CPU oracle: geometric multigrid preconditioner for the source problems.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 3's remark on two-level parallelisation: the N source problems are
independent (first level), and each one can itself be solved in parallel by
multigrid or domain decomposition (second level).  The paper names no
particular multigrid; the reading taken here, written out step by step:

  hierarchy     halve the cell counts while all three are even and >= 4; the
                coarse mesh covers the same box, its Q1 space is a subspace of
                the fine one
  prolongation  P: the coarse nodal basis written in the fine nodal basis
                (trilinear interpolation), P = P_z (x) P_y (x) P_x with the 1-D
                weights 1 at the coinciding node and 1/2 at the two fine
                neighbours
  coarse op     Galerkin A_c = P^T A P (SPD whenever A is)
  smoother      damped Jacobi x <- x + w D^-1 (b - A x) with
                w = min(1, 4 / (3 rho)), rho = max_i sum_j |A_ij| / A_ii (the
                Gershgorin bound of the spectrum of D^-1 A, so w rho <= 4/3 < 2)
  cycle         symmetric V(nu, nu): nu pre-sweeps (the first from x = 0),
                residual, restriction P^T, the coarse cycle, x += P e, nu
                post-sweeps; on the coarsest level nu_c sweeps from x = 0
  PCG           the textbook preconditioned CG with z = B r, B one V-cycle

Pins (tests/test_oracle_mg.py): P reproduces trilinear functions exactly;
P^T K_f P and P^T M_f P equal the stiffness and mass matrices assembled
directly on the coarse mesh (nested spaces, exact quadrature); B is symmetric
and positive definite; the two-grid and V-cycle error propagators contract in
the A-norm; MG-PCG reaches the sparse direct solution in a number of
iterations that stays bounded as the mesh is refined, while Jacobi-PCG's grows.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import paro as P_


def can_coarsen(n) -> bool:
    return all(v % 2 == 0 and v >= 4 for v in n)


def prolongation_1d(nf: int) -> sp.csr_matrix:
    """(nf-1) x (nf/2-1): fine interior node i (1..nf-1) from coarse interior J (1..nf/2-1).

    Fine node 2J coincides with coarse node J (weight 1); fine nodes 2J -/+ 1 sit
    halfway to the coarse neighbours (weight 1/2 each)."""
    nc = nf // 2
    rows, cols, vals = [], [], []
    for J in range(1, nc):
        for e, w in ((-1, 0.5), (0, 1.0), (1, 0.5)):
            i = 2 * J + e
            rows.append(i - 1)
            cols.append(J - 1)
            vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf - 1, nc - 1))


def prolongation(mesh: P_.Mesh) -> sp.csr_matrix:
    """Interior-node prolongation from the halved mesh (x fastest, as in Mesh)."""
    if mesh.graded:
        raise ValueError("the multigrid hierarchy is written for uniform meshes")
    nx, ny, nz = mesh.n
    return sp.kron(prolongation_1d(nz), sp.kron(prolongation_1d(ny), prolongation_1d(nx))).tocsr()


def coarse_mesh(mesh: P_.Mesh) -> P_.Mesh:
    return P_.Mesh(tuple(v // 2 for v in mesh.n), mesh.lo, mesh.hi)


def jacobi_weight(A: sp.csr_matrix) -> float:
    """w = min(1, 4 / (3 rho)), rho = max_i sum_j |A_ij| / A_ii."""
    d = A.diagonal()
    rho = float(np.max(np.asarray(abs(A).sum(axis=1)).ravel() / d))
    return min(1.0, 4.0 / (3.0 * rho))


@dataclass
class Level:
    mesh: P_.Mesh
    A: sp.csr_matrix
    dinv: np.ndarray
    omega: float
    P: sp.csr_matrix | None  # prolongation from the next (coarser) level, None on the coarsest


def hierarchy(A: sp.csr_matrix, mesh: P_.Mesh, max_levels: int = 32) -> list[Level]:
    """Levels 0 (the given operator) .. L-1 (coarsest), Galerkin coarse operators."""
    levels = []
    while True:
        last = not can_coarsen(mesh.n) or len(levels) + 1 >= max_levels
        P = None if last else prolongation(mesh)
        levels.append(Level(mesh, A, 1.0 / A.diagonal(), jacobi_weight(A), P))
        if last:
            return levels
        A = (P.T @ A @ P).tocsr()
        mesh = coarse_mesh(mesh)


def jacobi_sweeps(lev: Level, b: np.ndarray, x: np.ndarray | None, nu: int) -> np.ndarray:
    """nu damped Jacobi sweeps; x None means x = 0 (the first sweep is w D^-1 b)."""
    d = lev.dinv[:, None] if b.ndim == 2 else lev.dinv
    for _ in range(nu):
        if x is None:
            x = lev.omega * d * b
        else:
            x = x + lev.omega * d * (b - lev.A @ x)
    return x


def vcycle(levels: list[Level], b: np.ndarray, nu: int = 1, nu_c: int = 4, l: int = 0) -> np.ndarray:
    """One symmetric V(nu, nu)-cycle on level l from x = 0: returns B_l b."""
    lev = levels[l]
    if l == len(levels) - 1:
        return jacobi_sweeps(lev, b, None, nu_c)
    x = jacobi_sweeps(lev, b, None, nu)
    r = b - lev.A @ x
    e = vcycle(levels, lev.P.T @ r, nu, nu_c, l + 1)
    x = x + lev.P @ e
    return jacobi_sweeps(lev, b, x, nu)


def mg_pcg(levels: list[Level], B: np.ndarray, X0: np.ndarray | None, tol: float, maxit: int,
           nu: int = 1, nu_c: int = 4) -> P_.PCGResult:
    """Preconditioned CG with z = B r (one V-cycle), column by column semantics.

    Column i stops when ||r_i||_2 <= tol ||b_i||_2, tested before each update:
        z = B r, rz = (r, z), beta = rz / rz_old, p = z + beta p,
        q = A p, alpha = rz / (p, q), x += alpha p, r -= alpha q.
    """
    A = levels[0].A
    B = np.asarray(B, dtype=np.float64)
    one = B.ndim == 1
    if one:
        B = B[:, None]
    n, N = B.shape
    X = np.zeros((n, N)) if X0 is None else np.array(X0, dtype=np.float64, copy=True).reshape(n, N)
    R = B - A @ X
    bnorm = np.linalg.norm(B, axis=0)
    iters = np.zeros(N, dtype=np.int64)
    Pd = np.zeros((n, N))
    rz_old = np.ones(N)
    first = np.ones(N, dtype=bool)
    active = np.linalg.norm(R, axis=0) > tol * bnorm
    for _ in range(maxit):
        if not active.any():
            break
        Z = vcycle(levels, R, nu, nu_c)
        rz = np.einsum("ij,ij->j", R, Z)
        if np.any(rz[active] <= 0):
            raise FloatingPointError("(r, B r) <= 0: preconditioner not SPD")
        beta = np.where(first, 0.0, rz / np.where(active, rz_old, 1.0))
        Pd = np.where(active, Z + beta * Pd, Pd)
        Q = A @ Pd
        pq = np.einsum("ij,ij->j", Pd, Q)
        if np.any(pq[active] <= 0):
            raise FloatingPointError("p^T A p <= 0: operator not SPD")
        alpha = np.where(active, rz / np.where(active, pq, 1.0), 0.0)
        X += alpha * Pd
        R -= alpha * Q
        rz_old = np.where(active, rz, rz_old)
        first &= ~active
        iters += active
        active = active & (np.linalg.norm(R, axis=0) > tol * bnorm)
    relres = np.linalg.norm(R, axis=0) / np.where(bnorm > 0, bnorm, 1.0)
    if one:
        X = X[:, 0]
    return P_.PCGResult(X, iters, relres, relres <= tol)
