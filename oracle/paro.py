"""FP64 CPU oracle: Q1 discretisation, source problems, Rayleigh-Ritz, ParO loop.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain numpy/scipy,
float64 throughout, no blocking or fusion: every function is written so that
it can be checked against the paper by eye.

Notation (paper Section 2.2 and Appendix):
  a(w, v) = 1/2 (grad w, grad v) + (V w, v)           eq. (2.7), linear part
  (w, v)  = L2 inner product                          mass form
Discrete, on the interior nodes of a uniform nx x ny x nz Q1 hex mesh:
  K  stiffness  K_ij = (grad phi_i, grad phi_j)
  M  mass       M_ij = (phi_i, phi_j)
  MV potential  MV_ij = sum_cells sum_q w_q V(x_q) phi_i(x_q) phi_j(x_q)
                (2x2x2 Gauss points per cell, V given at those points)
  H = K/2 + MV                      the discrete a(., .)
  A = H + sigma M                   the shifted SPD operator of the source problems

Pins (tests/test_oracle_pins.py):
  assemble            -> Kronecker closed form of K and M, exact linear- and
                         trilinear-V integrals, constant-V == c*M, V=0 discrete
                         sine spectrum (down to one interior node)
  pcg                 -> direct sparse solve on the same system
  rayleigh_ritz       -> Ritz conditions, M-orthonormality, interlacing against
                         dense eigenvalues of the assembled pencil, the Rayleigh
                         quotient for one orbital
  paro                -> dense/ARPACK eigenvalues of the same pencil (the full
                         32^3 hydrogen workload included), harmonic-oscillator
                         levels w(n+3/2) with O(h^2) rate, hydrogen-like n = 1, 2
                         trends, fixed-point property, resume from (U, lambda)
tests/test_oracle_mutations.py plants plausible mistakes here and checks that
these pins catch them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------------------
# Mesh and reference element
# ---------------------------------------------------------------------------


@dataclass
class Mesh:
    """Hexahedral tensor-product mesh of the box [lo, hi] with n = (nx, ny, nz) cells.

    Uniform by default.  A graded mesh (Section 2.1: finite element spaces on
    locally refined meshes, here refined along each axis) gives the node
    coordinates of every axis in `coords` (n_d + 1 strictly increasing values
    each; lo and hi are then their end points).  Unknowns live on interior nodes
    only (homogeneous Dirichlet data on the whole boundary, the truncated domain
    of Section 2.2).  Interior node (i, j, k), 1 <= i <= nx-1 etc., has index
    ((k-1)(ny-1) + (j-1))(nx-1) + (i-1): x varies fastest.
    """

    n: tuple
    lo: tuple
    hi: tuple
    coords: tuple | None = None
    h: np.ndarray = field(init=False)

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        if self.coords is None:
            self.lo = tuple(float(v) for v in self.lo)
            self.hi = tuple(float(v) for v in self.hi)
            self.nodes = [self.lo[d] + (self.hi[d] - self.lo[d]) / self.n[d] * np.arange(self.n[d] + 1)
                          for d in range(3)]
            self.graded = False
        else:
            self.nodes = [np.asarray(c, dtype=np.float64) for c in self.coords]
            for d in range(3):
                if self.nodes[d].shape != (self.n[d] + 1,) or not np.all(np.diff(self.nodes[d]) > 0):
                    raise ValueError("coords: n_d + 1 strictly increasing node coordinates per axis")
            self.lo = tuple(float(c[0]) for c in self.nodes)
            self.hi = tuple(float(c[-1]) for c in self.nodes)
            self.graded = True
        self.hc = [np.diff(self.nodes[d]) for d in range(3)]  # cell sizes per axis
        self.h = np.array([(self.hi[d] - self.lo[d]) / self.n[d] for d in range(3)])  # mean cell size

    @property
    def n_interior(self) -> int:
        nx, ny, nz = self.n
        return (nx - 1) * (ny - 1) * (nz - 1)

    def interior_index(self, i, j, k):
        """Global unknown index of node (i, j, k), or -1 on the boundary."""
        nx, ny, nz = self.n
        i = np.asarray(i)
        j = np.asarray(j)
        k = np.asarray(k)
        inside = (i >= 1) & (i <= nx - 1) & (j >= 1) & (j <= ny - 1) & (k >= 1) & (k <= nz - 1)
        idx = ((k - 1) * (ny - 1) + (j - 1)) * (nx - 1) + (i - 1)
        return np.where(inside, idx, -1)

    def interior_coords(self) -> np.ndarray:
        """(n_interior, 3) coordinates in unknown order."""
        xs = [self.nodes[d][1:-1] for d in range(3)]
        Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def gauss_1d():
    """Two-point Gauss rule on [0, 1]: nodes (1 -/+ 1/sqrt 3)/2, weights 1/2."""
    t, w = np.polynomial.legendre.leggauss(2)  # on [-1, 1], ascending
    return (t + 1.0) / 2.0, w / 2.0


def q1_shape(t):
    """1-D linear Lagrange functions on [0, 1] and their derivatives at t.

    Returns (l, dl) with l[a] = value of l_a(t), a = 0 (1 - t) and a = 1 (t).
    """
    t = np.asarray(t, dtype=np.float64)
    l = np.stack([1.0 - t, t])
    dl = np.stack([-np.ones_like(t), np.ones_like(t)])
    return l, dl


def element_matrices(h):
    """Reference 8x8 element matrices by 2x2x2 Gauss quadrature.

    Local node a = (ax, ay, az) in {0,1}^3 has local index a = ax + 2 ay + 4 az;
    quadrature point q = (qx, qy, qz) has index qx + 2 qy + 4 qz.  Returns
      Ke[a, b] = sum_q w_q grad phi_a . grad phi_b    (exact: degree <= 2 per axis)
      Me[a, b] = sum_q w_q phi_a phi_b                 (exact: degree 2 per axis)
      P[q, a]  = phi_a(x_q)                            (to build the potential term)
      wq       = quadrature weight per point (h_x h_y h_z / 8)
    """
    g, gw = gauss_1d()
    l, dl = q1_shape(g)  # l[a, q1d]
    hx, hy, hz = h
    P = np.zeros((8, 8))
    G = np.zeros((8, 8, 3))
    wq = np.zeros(8)
    for qz in range(2):
        for qy in range(2):
            for qx in range(2):
                q = qx + 2 * qy + 4 * qz
                wq[q] = gw[qx] * gw[qy] * gw[qz] * hx * hy * hz
                for az in range(2):
                    for ay in range(2):
                        for ax in range(2):
                            a = ax + 2 * ay + 4 * az
                            P[q, a] = l[ax, qx] * l[ay, qy] * l[az, qz]
                            G[q, a, 0] = dl[ax, qx] / hx * l[ay, qy] * l[az, qz]
                            G[q, a, 1] = l[ax, qx] * dl[ay, qy] / hy * l[az, qz]
                            G[q, a, 2] = l[ax, qx] * l[ay, qy] * dl[az, qz] / hz
    Ke = np.einsum("q,qad,qbd->ab", wq, G, G)
    Me = np.einsum("q,qa,qb->ab", wq, P, P)
    return Ke, Me, P, wq


def gauss_points(mesh: Mesh) -> np.ndarray:
    """Physical Gauss points, shape (nz, ny, nx, 2, 2, 2, 3) = [cz][cy][cx][qz][qy][qx][xyz]."""
    g, _ = gauss_1d()
    nx, ny, nz = mesh.n
    out = np.zeros((nz, ny, nx, 2, 2, 2, 3))
    px = mesh.nodes[0][:-1, None] + mesh.hc[0][:, None] * g[None, :]  # [cell][q]
    py = mesh.nodes[1][:-1, None] + mesh.hc[1][:, None] * g[None, :]
    pz = mesh.nodes[2][:-1, None] + mesh.hc[2][:, None] * g[None, :]
    out[..., 0] = px[None, None, :, None, None, :]
    out[..., 1] = py[None, :, None, None, :, None]
    out[..., 2] = pz[:, None, None, :, None, None]
    return out


# ---------------------------------------------------------------------------
# Assembly (element by element, then drop boundary rows/cols: Dirichlet)
# ---------------------------------------------------------------------------


@dataclass
class Operators:
    mesh: Mesh
    K: sp.csr_matrix
    M: sp.csr_matrix
    MV: sp.csr_matrix
    sigma: float

    @property
    def H(self):
        """Discrete a(., .) of eq. (2.7) with a fixed potential: K/2 + MV."""
        return (0.5 * self.K + self.MV).tocsr()

    @property
    def A(self):
        """Shifted source-problem operator H + sigma M (SPD for a suitable sigma)."""
        return (0.5 * self.K + self.MV + self.sigma * self.M).tocsr()


def _cell_node_indices(mesh: Mesh) -> np.ndarray:
    """(n_cells, 8) global interior index of each local node, -1 on the boundary."""
    nx, ny, nz = mesh.n
    cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    idx = np.zeros((cx.size, 8), dtype=np.int64)
    for az in range(2):
        for ay in range(2):
            for ax in range(2):
                idx[:, ax + 2 * ay + 4 * az] = mesh.interior_index(cx + ax, cy + ay, cz + az)
    return idx


def _assemble(mesh: Mesh, cell_mats: np.ndarray) -> sp.csr_matrix:
    """Sum per-cell 8x8 matrices into the interior-node matrix."""
    idx = _cell_node_indices(mesh)
    rows = np.repeat(idx[:, :, None], 8, axis=2)
    cols = np.repeat(idx[:, None, :], 8, axis=1)
    keep = (rows >= 0) & (cols >= 0)
    n = mesh.n_interior
    return sp.coo_matrix((cell_mats[keep], (rows[keep], cols[keep])), shape=(n, n)).tocsr()


def assemble(mesh: Mesh, Vq: np.ndarray, sigma: float) -> Operators:
    """Assemble K, M and MV on the interior nodes.

    Vq: potential at the Gauss points, shape (nz, ny, nx, 2, 2, 2) or flat
    8*nx*ny*nz in the order [cz][cy][cx][qz][qy][qx].
    """
    nx, ny, nz = mesh.n
    Vq = np.asarray(Vq, dtype=np.float64).reshape(nz * ny * nx, 8)  # q = qx + 2qy + 4qz
    n_cells = nx * ny * nz
    if not mesh.graded:
        Ke, Me, P, wq = element_matrices(mesh.h)
        K = _assemble(mesh, np.broadcast_to(Ke, (n_cells, 8, 8)))
        M = _assemble(mesh, np.broadcast_to(Me, (n_cells, 8, 8)))
        # MV^e_ab = sum_q w_q V_cq phi_a(q) phi_b(q)
        MVe = np.einsum("q,cq,qa,qb->cab", wq, Vq, P, P)
    else:
        # every cell its own sizes: with the unit cell's per-direction stiffness parts
        # S_d (gradients along axis d only), Ke = sum_d (h_x h_y h_z / h_d^2) S_d,
        # Me = h_x h_y h_z Me(1), and the Gauss weights scale by h_x h_y h_z
        _, Me1, P, wq1 = element_matrices((1.0, 1.0, 1.0))
        Sd = _unit_stiffness_parts()
        hz, hy, hx = np.meshgrid(mesh.hc[2], mesh.hc[1], mesh.hc[0], indexing="ij")
        hx, hy, hz = hx.ravel(), hy.ravel(), hz.ravel()
        vol = hx * hy * hz
        Ke = ((vol / hx ** 2)[:, None, None] * Sd[0] + (vol / hy ** 2)[:, None, None] * Sd[1]
              + (vol / hz ** 2)[:, None, None] * Sd[2])
        K = _assemble(mesh, Ke)
        M = _assemble(mesh, vol[:, None, None] * Me1[None, :, :])
        MVe = np.einsum("c,q,cq,qa,qb->cab", vol, wq1, Vq, P, P)
    MV = _assemble(mesh, MVe)
    return Operators(mesh, K, M, MV, float(sigma))


def _unit_stiffness_parts() -> np.ndarray:
    """S[d][a, b] = sum_q w_q (d phi_a / d x_d)(d phi_b / d x_d) on the unit cell (2x2x2 Gauss)."""
    g, gw = gauss_1d()
    l, dl = q1_shape(g)
    S = np.zeros((3, 8, 8))
    for qz in range(2):
        for qy in range(2):
            for qx in range(2):
                w = gw[qx] * gw[qy] * gw[qz]
                for a in range(8):
                    ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
                    ga = (dl[ax, qx] * l[ay, qy] * l[az, qz], l[ax, qx] * dl[ay, qy] * l[az, qz],
                          l[ax, qx] * l[ay, qy] * dl[az, qz])
                    for b in range(8):
                        bx, by, bz = b & 1, (b >> 1) & 1, (b >> 2) & 1
                        gb = (dl[bx, qx] * l[by, qy] * l[bz, qz], l[bx, qx] * dl[by, qy] * l[bz, qz],
                              l[bx, qx] * l[by, qy] * dl[bz, qz])
                        for d in range(3):
                            S[d, a, b] += w * ga[d] * gb[d]
    return S


# ---------------------------------------------------------------------------
# Step 3: source problems by Jacobi PCG, one independent CG per column
# ---------------------------------------------------------------------------


@dataclass
class PCGResult:
    X: np.ndarray
    iters: np.ndarray  # CG updates performed per column
    relres: np.ndarray  # final ||r||_2 / ||b||_2 per column (recursive residual)
    converged: np.ndarray


def pcg(A: sp.csr_matrix, B: np.ndarray, X0: np.ndarray, tol: float, maxit: int) -> PCGResult:
    """Jacobi-preconditioned conjugate gradients, column by column semantics.

    Each column i solves A x_i = b_i from x_i = X0[:, i].  Column i stops when
    ||r_i||_2 <= tol ||b_i||_2 (tested before each update); an exhausted column
    is left as is.  The per-column recurrences are the textbook ones:
        q = A p, alpha = (r.z)/(p.q), x += alpha p, r -= alpha q,
        z = D^-1 r, beta = (r.z)_new/(r.z)_old, p = z + beta p.
    """
    B = np.asarray(B, dtype=np.float64)
    X = np.array(X0, dtype=np.float64, copy=True)
    if B.ndim == 1:
        B = B[:, None]
        X = X[:, None]
    n, N = B.shape
    dinv = 1.0 / A.diagonal()
    R = B - A @ X
    Z = dinv[:, None] * R
    P = Z.copy()
    rz = np.einsum("ij,ij->j", R, Z)
    bnorm = np.linalg.norm(B, axis=0)
    iters = np.zeros(N, dtype=np.int64)
    active = np.linalg.norm(R, axis=0) > tol * bnorm
    for _ in range(maxit):
        if not active.any():
            break
        Q = A @ P
        pq = np.einsum("ij,ij->j", P, Q)
        if np.any(pq[active] <= 0):
            raise FloatingPointError("p^T A p <= 0: operator not SPD (shift too small)")
        alpha = np.where(active, rz / np.where(active, pq, 1.0), 0.0)
        X += alpha * P
        R -= alpha * Q
        Z = dinv[:, None] * R
        rz_new = np.einsum("ij,ij->j", R, Z)
        beta = np.where(active, rz_new / np.where(active, rz, 1.0), 0.0)
        P = np.where(active, Z + beta * P, P)
        rz = np.where(active, rz_new, rz)
        iters += active
        active = active & (np.linalg.norm(R, axis=0) > tol * bnorm)
    relres = np.linalg.norm(R, axis=0) / np.where(bnorm > 0, bnorm, 1.0)
    return PCGResult(X, iters, relres, relres <= tol)


def source_problems(ops: Operators, U: np.ndarray, lam: np.ndarray, tol: float, maxit: int) -> PCGResult:
    """Step 3 (eq. alg-bvp) with the shift: (H + sigma M) x_i = (lambda_i + sigma) M u_i.

    Warm start x_i = u_i.  With sigma = 0 this is the paper's
    a(x_i, v) = lambda_i (u_i, v); the shift only rescales x_i by a factor
    for an exact eigenpair and keeps every system SPD.
    """
    B = (ops.M @ U) * (np.asarray(lam) + ops.sigma)[None, :]
    return pcg(ops.A, B, U, tol, maxit)


# ---------------------------------------------------------------------------
# Step 4: Rayleigh-Ritz on span{x_1 .. x_N}
# ---------------------------------------------------------------------------


@dataclass
class RRResult:
    U: np.ndarray  # M-orthonormal Ritz vectors, ascending Ritz values
    lam: np.ndarray
    GA: np.ndarray
    GB: np.ndarray
    C: np.ndarray


def rayleigh_ritz(ops: Operators, X: np.ndarray) -> RRResult:
    """Step 4 (eq. alg-evp): find (theta, c) with (X^T H X) c = theta (X^T M X) c.

    Cholesky G_B = L L^T, symmetric eigen of L^-1 G_A L^-T = Q Theta Q^T
    (ascending), C = L^-T Q, U = X C.  Then U^T M U = I and U^T H U = Theta.
    """
    X = np.asarray(X, dtype=np.float64)
    GA = X.T @ (ops.H @ X)
    GB = X.T @ (ops.M @ X)
    GA = 0.5 * (GA + GA.T)
    GB = 0.5 * (GB + GB.T)
    L = np.linalg.cholesky(GB)
    Linv = np.linalg.inv(L)
    S = Linv @ GA @ Linv.T
    theta, Q = np.linalg.eigh(0.5 * (S + S.T))
    C = Linv.T @ Q
    return RRResult(X @ C, theta, GA, GB, C)


def rayleigh_ritz_clusters(ops: Operators, X: np.ndarray, sizes) -> RRResult:
    """Step 4 separated by eigenvalue clusters (Section 3, "eigenvalue
    separation"): the columns of X are consecutive groups of sizes q_1, q_2, ...
    (one per cluster of the spectrum, ascending), and each group gets its own
    Rayleigh-Ritz problem of size q_i, so the small problems cost O(sum q_i^3)
    instead of O((sum q_i)^3).

    Reading: group c is first made M-orthogonal to the Ritz vectors of groups
    1 .. c-1 (block Gram-Schmidt).  Without it the source problems, which act as
    an inverse-iteration step, amplify every group's components along lower
    eigenvectors by lambda_i / lambda_j > 1 per iteration, and a higher cluster
    drifts onto a lower one; the separation the section assumes would not last.
    """
    X = np.asarray(X, dtype=np.float64)
    sizes = [int(q) for q in sizes]
    if sum(sizes) != X.shape[1] or min(sizes) < 1:
        raise ValueError("cluster sizes must be positive and add up to N")
    N = X.shape[1]
    U = np.zeros_like(X)
    theta = np.zeros(N)
    o = 0
    for q in sizes:
        Xc = X[:, o:o + q].copy()
        if o > 0:
            V = U[:, :o]
            Xc -= V @ (V.T @ (ops.M @ Xc))
        r = rayleigh_ritz(ops, Xc)
        U[:, o:o + q] = r.U
        theta[o:o + q] = r.lam
        o += q
    GA = X.T @ (ops.H @ X)
    GB = X.T @ (ops.M @ X)
    C = np.linalg.lstsq(X, U, rcond=None)[0]
    return RRResult(U, theta, GA, GB, C)


# ---------------------------------------------------------------------------
# Step 5: the ParO loop (Algorithm A.1 for a fixed potential; Algorithm 3.2
# when more orbitals are iterated than are tested for convergence)
# ---------------------------------------------------------------------------


@dataclass
class ParOResult:
    U: np.ndarray
    lam: np.ndarray
    outer: int
    history: list  # lambda after each outer iteration
    pcg_iters: list  # per outer iteration, per orbital


def paro(ops: Operators, U0: np.ndarray, tol: float = 1e-10, max_outer: int = 500,
         pcg_tol: float = 1e-12, pcg_maxit: int = 5000, n_check: int | None = None,
         lam0: np.ndarray | None = None, fixed_outer: int | None = None, clusters=None) -> ParOResult:
    """Run ParO from the initial orbitals U0.

    If lam0 is None the initial eigenvalue estimates (and orthonormal orbitals)
    come from one Rayleigh-Ritz step on span(U0): the paper asks for given
    initial data (lambda^(0), u^(0)) but does not say where lambda^(0) comes from.
    Stops when max_i |lambda_i^(n+1) - lambda_i^(n)| < tol over the lowest
    n_check values (all when None), or after fixed_outer iterations if given.
    clusters: sizes of consecutive orbital groups for the cluster-separated
    Rayleigh-Ritz of the outer iterations (the start is always a full one).
    """
    U = np.asarray(U0, dtype=np.float64)
    if lam0 is None:
        rr = rayleigh_ritz(ops, U)
        U, lam = rr.U, rr.lam
    else:
        lam = np.asarray(lam0, dtype=np.float64)
    N = U.shape[1]
    k = N if n_check is None else n_check
    history, pcg_iters = [], []
    outer = 0
    limit = fixed_outer if fixed_outer is not None else max_outer
    while outer < limit:
        sol = source_problems(ops, U, lam, pcg_tol, pcg_maxit)
        rr = rayleigh_ritz(ops, sol.X) if clusters is None else rayleigh_ritz_clusters(ops, sol.X, clusters)
        dl = np.max(np.abs(rr.lam[:k] - lam[:k]))
        U, lam = rr.U, rr.lam
        outer += 1
        history.append(lam.copy())
        pcg_iters.append(sol.iters.copy())
        if fixed_outer is None and dl < tol:
            break
    return ParOResult(U, lam, outer, history, pcg_iters)


# ---------------------------------------------------------------------------
# Checks used by tests: principal angles of M-orthonormal subspaces
# ---------------------------------------------------------------------------


def subspace_angles_M(M: sp.csr_matrix, U: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Principal angles between span(U) and span(W) (same dimension) in the M inner product.

    Taken from the sines: with M-orthonormal bases Qu, Qw, the singular values
    of the M-orthogonal residual Qw - Qu (Qu^T M Qw), measured in the M norm, are
    the sines of the angles.  The cosine form (arccos of the singular values of
    Qu^T M Qw) cannot resolve angles below sqrt(2 eps) ~ 1.5e-8.
    """
    GU = U.T @ (M @ U)
    GW = W.T @ (M @ W)
    LU = np.linalg.cholesky(GU)
    LW = np.linalg.cholesky(GW)
    Qu = U @ np.linalg.inv(LU).T
    Qw = W @ np.linalg.inv(LW).T
    R = Qw - Qu @ (Qu.T @ (M @ Qw))
    G = R.T @ (M @ R)
    s2 = np.clip(np.linalg.eigvalsh(0.5 * (G + G.T)), 0.0, 1.0)
    return np.sort(np.arcsin(np.sqrt(s2)))


def eigen_residuals(ops: Operators, U: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """||H u_i - lambda_i M u_i||_2 per column."""
    R = ops.H @ U - (ops.M @ U) * lam[None, :]
    return np.linalg.norm(R, axis=0)
