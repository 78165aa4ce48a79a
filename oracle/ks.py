"""FP64 CPU oracle: the Kohn-Sham pieces of the SCF workload.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain numpy/scipy,
float64 throughout.

Section 2.2 (Kohn-Sham equation, eq. (2.6) and the bilinear form (2.7)): the
effective potential is V_ext + V_H(rho) + V_xc(rho) with the density
rho = sum_i f_i |u_i|^2; the Hartree potential solves -Delta V_H = 4 pi rho
(the Poisson form the section gives); V_xc is a local-density approximation,
here the Slater exchange.  Everything is evaluated at the 2x2x2 Gauss points of
every cell, the points at which the operator takes its potential
(``oracle.paro.assemble``), in the order [cz][cy][cx][qz][qy][qx].

Readings (where Section 2.2 leaves a choice open):
  * occupations: f = 2 for the lowest floor(N_e/2) orbitals, 1 for an odd
    electron, 0 for the extra (buffer) orbitals of Algorithm 3.2;
  * the Hartree factor: -Delta V_H = 4 pi rho (the section's Poisson form; the
    1/2 written in front of its integral form contradicts it);
  * the Poisson problem lives on the truncated box with Dirichlet data of the
    monopole Q / |x - x_c| of the density (Q its charge, x_c its centre);
  * exchange: Slater, V_x = -(3 rho / pi)^(1/3), energy density
    e_x = -(3/4) (3/pi)^(1/3) rho^(4/3);
  * mixing: rho_in <- (1 - beta) rho_in + beta rho_out (beta = 0.3);
  * the potential of one outer iteration is built from rho_in and used in both
    Step 3 and Step 4.

Pins (tests/test_oracle_ks.py): the density integrates to sum f_i for
M-orthonormal orbitals (exact with the Gauss rule); the density of a trilinear
function equals its square at the Gauss points; the Hartree potential of a
Gaussian charge approaches Q erf(r / (sqrt 2 s)) / r at O(h^2); the Slater
energy of a Gaussian density matches its closed-form integral; SCF keeps the
charge and reaches self-consistency; at self-consistency the band-energy form of
the total energy equals its direct definition.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import paro as P


def occupations(N: int, n_electrons: int) -> np.ndarray:
    """f_i: 2 for the lowest floor(N_e/2) orbitals, 1 for an odd electron, else 0."""
    f = np.zeros(N)
    full = n_electrons // 2
    f[:full] = 2.0
    if n_electrons % 2:
        f[full] = 1.0
    return f


def _uniform(mesh: P.Mesh) -> None:
    if mesh.graded:
        raise ValueError("the Kohn-Sham pieces are written for uniform meshes")


def _cell_values(mesh: P.Mesh, U: np.ndarray) -> np.ndarray:
    """Orbital values at the Gauss points: (n_cells, 8, N), boundary nodes zero."""
    _uniform(mesh)
    _, _, Pq, _ = P.element_matrices(mesh.h)
    idx = P._cell_node_indices(mesh)  # (n_cells, 8), -1 on the boundary
    U = np.asarray(U, dtype=np.float64)
    Uext = np.vstack([U, np.zeros((1, U.shape[1]))])  # row -1 -> zeros
    nodal = Uext[idx]  # (n_cells, 8 nodes, N)
    return np.einsum("qa,can->cqn", Pq, nodal)


def density_gauss(mesh: P.Mesh, U: np.ndarray, occ: np.ndarray) -> np.ndarray:
    """rho at the Gauss points, flat (n_cells*8,): sum_i f_i u_i(x_q)^2."""
    vals = _cell_values(mesh, U)
    return np.einsum("cqn,n->cq", vals ** 2, np.asarray(occ, dtype=np.float64)).ravel()


def integrate(mesh: P.Mesh, fq: np.ndarray) -> float:
    """sum over cells and Gauss points of w_q f(x_q)."""
    _uniform(mesh)
    _, _, _, wq = P.element_matrices(mesh.h)
    return float(np.einsum("cq,q->", np.asarray(fq).reshape(-1, 8), wq))


# ---------------------------------------------------------------------------
# Hartree potential: Q1 Poisson solve with monopole Dirichlet data
# ---------------------------------------------------------------------------


def _all_node_index(mesh: P.Mesh):
    """(n_cells, 8) index of each cell node among all (nx+1)(ny+1)(nz+1) nodes, x fastest."""
    nx, ny, nz = mesh.n
    cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    idx = np.zeros((cx.size, 8), dtype=np.int64)
    for az in range(2):
        for ay in range(2):
            for ax in range(2):
                idx[:, ax + 2 * ay + 4 * az] = ((cz + az) * (ny + 1) + (cy + ay)) * (nx + 1) + (cx + ax)
    return idx


def monopole(mesh: P.Mesh, rho_q: np.ndarray):
    """Charge Q = int rho and centre x_c = int rho x / Q of a Gauss-point density."""
    _uniform(mesh)
    _, _, _, wq = P.element_matrices(mesh.h)
    r = np.asarray(rho_q).reshape(-1, 8)
    X = P.gauss_points(mesh).reshape(-1, 8, 3)
    Q = float(np.einsum("cq,q->", r, wq))
    if Q == 0.0:
        return 0.0, np.zeros(3)
    xc = np.einsum("cq,q,cqd->d", r, wq, X) / Q
    return Q, xc


@dataclass
class HartreeResult:
    VH_q: np.ndarray  # at the Gauss points, flat
    VH_nodes: np.ndarray  # at all nodes (nx+1)(ny+1)(nz+1), x fastest
    Q: float
    xc: np.ndarray


def hartree(mesh: P.Mesh, rho_q: np.ndarray) -> HartreeResult:
    """V_H with -Delta V_H = 4 pi rho on the box, V_H = Q / |x - x_c| on its boundary.

    Weak form on Q1: (grad V_H, grad v) = 4 pi (rho, v) for interior test
    functions v, the right-hand side integrated with the Gauss rule at which
    rho is given; the boundary values enter through the interior-boundary
    block of the stiffness matrix.
    """
    _uniform(mesh)
    nx, ny, nz = mesh.n
    Ke, _, Pq, wq = P.element_matrices(mesh.h)
    idx = _all_node_index(mesh)
    n_all = (nx + 1) * (ny + 1) * (nz + 1)
    n_cells = nx * ny * nz
    rows = np.repeat(idx[:, :, None], 8, axis=2).ravel()
    cols = np.repeat(idx[:, None, :], 8, axis=1).ravel()
    K = sp.coo_matrix((np.broadcast_to(Ke, (n_cells, 8, 8)).ravel(), (rows, cols)), shape=(n_all, n_all)).tocsr()
    r = np.asarray(rho_q, dtype=np.float64).reshape(-1, 8)
    be = np.einsum("q,cq,qa->ca", wq, r, Pq)  # (rho, phi_a) per cell
    b = np.zeros(n_all)
    np.add.at(b, idx.ravel(), be.ravel())
    # node coordinates and the boundary mask
    xs = [mesh.lo[d] + mesh.h[d] * np.arange(mesh.n[d] + 1) for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    ii = np.arange(n_all)
    ix, iy, iz = ii % (nx + 1), (ii // (nx + 1)) % (ny + 1), ii // ((nx + 1) * (ny + 1))
    bnd = (ix == 0) | (ix == nx) | (iy == 0) | (iy == ny) | (iz == 0) | (iz == nz)
    Q, xc = monopole(mesh, rho_q)
    g = np.zeros(n_all)
    if Q != 0.0:
        g[bnd] = Q / np.linalg.norm(coords[bnd] - xc, axis=1)
    inner = ~bnd
    Kii = K[inner][:, inner]
    rhs = 4.0 * np.pi * b[inner] - K[inner][:, bnd] @ g[bnd]
    V = g.copy()
    V[inner] = spla.spsolve(Kii.tocsc(), rhs)
    VH_q = np.einsum("qa,ca->cq", Pq, V[idx]).ravel()
    return HartreeResult(VH_q, V, Q, xc)


# ---------------------------------------------------------------------------
# Exchange (LDA, Slater)
# ---------------------------------------------------------------------------


def slater_potential(rho_q: np.ndarray) -> np.ndarray:
    """V_x = -(3 rho / pi)^(1/3) (rho clipped at 0)."""
    r = np.maximum(np.asarray(rho_q, dtype=np.float64), 0.0)
    return -np.cbrt(3.0 * r / np.pi)


def slater_energy(mesh: P.Mesh, rho_q: np.ndarray) -> float:
    """E_x = int -(3/4)(3/pi)^(1/3) rho^(4/3)."""
    r = np.maximum(np.asarray(rho_q, dtype=np.float64), 0.0)
    return integrate(mesh, -0.75 * np.cbrt(3.0 / np.pi) * r ** (4.0 / 3.0))


def effective_potential(mesh: P.Mesh, Vext_q: np.ndarray, rho_q: np.ndarray) -> np.ndarray:
    """V_ext + V_H(rho) + V_x(rho) at the Gauss points."""
    return np.asarray(Vext_q) + hartree(mesh, rho_q).VH_q + slater_potential(rho_q)


def total_energy(mesh: P.Mesh, lam: np.ndarray, occ: np.ndarray, rho_q: np.ndarray) -> float:
    """Kohn-Sham electronic energy in the band-energy form:
        E = sum_i f_i lambda_i - 1/2 int rho V_H[rho] - int rho V_x[rho] + E_x[rho]
    (the eigenvalue sum counts the Hartree energy twice and holds int rho V_x in
    place of E_x).  The nuclei's mutual repulsion is not included."""
    VH = hartree(mesh, rho_q).VH_q
    return float(np.dot(np.asarray(occ, dtype=np.float64), np.asarray(lam, dtype=np.float64))
                 - 0.5 * integrate(mesh, rho_q * VH) - integrate(mesh, rho_q * slater_potential(rho_q))
                 + slater_energy(mesh, rho_q))


def direct_energy(mesh: P.Mesh, Vext_q: np.ndarray, U: np.ndarray, occ: np.ndarray) -> float:
    """The same energy from its definition, for the density of the orbitals U:
        E = sum_i f_i (u_i, (K/2 + M_Vext) u_i) + 1/2 int rho V_H[rho] + E_x[rho]."""
    ops = P.assemble(mesh, Vext_q, 0.0)
    occ = np.asarray(occ, dtype=np.float64)
    rho = density_gauss(mesh, U, occ)
    one = float(np.einsum("i,ni,ni->", occ, U, ops.H @ U))
    return one + 0.5 * integrate(mesh, rho * hartree(mesh, rho).VH_q) + slater_energy(mesh, rho)


# ---------------------------------------------------------------------------
# SCF: Algorithm 3.1 with the Kohn-Sham potential and linear mixing
# ---------------------------------------------------------------------------


def mix_density(rho_in: np.ndarray, rho_out: np.ndarray, mix: float) -> np.ndarray:
    """Linear mixing of the next input density: move rho_in the fraction `mix` of
    the way to the output density (mix = 1: no damping, the plain fixed-point
    step; mix -> 0: the input density stays)."""
    return (1.0 - mix) * rho_in + mix * rho_out


@dataclass
class SCFResult:
    U: np.ndarray
    lam: np.ndarray
    rho_q: np.ndarray
    outer: int
    history: list  # lambda after each outer iteration
    charge: list  # int rho_in after each outer iteration


def scf(mesh: P.Mesh, Vext_q: np.ndarray, U0: np.ndarray, occ: np.ndarray, sigma: float, mix: float = 0.3,
        tol: float = 1e-8, max_outer: int = 200, pcg_tol: float = 1e-12, pcg_maxit: int = 5000,
        fixed_outer: int | None = None, n_check: int | None = None) -> SCFResult:
    """Kohn-Sham ParO.

    Start: one Rayleigh-Ritz on span(U0) with V_ext alone gives orbitals whose
    density is the first rho_in.  Each outer iteration builds V from rho_in,
    solves the N shifted source problems (Step 3) and does Rayleigh-Ritz
    (Step 4) with that potential, then mixes rho_in with the density of the new
    orbitals.  Stops when max |Delta lambda| < tol over the lowest n_check
    orbitals (all by default; Algorithm 3.2 tests the occupied ones and carries
    the others as a buffer), or after fixed_outer.
    """
    ops0 = P.assemble(mesh, Vext_q, sigma)
    rr = P.rayleigh_ritz(ops0, U0)
    U, lam = rr.U, rr.lam
    rho_in = density_gauss(mesh, U, occ)
    history, charge = [], []
    outer = 0
    limit = fixed_outer if fixed_outer is not None else max_outer
    while outer < limit:
        V = effective_potential(mesh, Vext_q, rho_in)
        ops = P.assemble(mesh, V, sigma)
        sol = P.source_problems(ops, U, lam, pcg_tol, pcg_maxit)
        rr = P.rayleigh_ritz(ops, sol.X)
        k = len(lam) if n_check is None else n_check
        dl = np.max(np.abs(rr.lam[:k] - lam[:k]))
        U, lam = rr.U, rr.lam
        rho_out = density_gauss(mesh, U, occ)
        rho_in = mix_density(rho_in, rho_out, mix)
        history.append(lam.copy())
        charge.append(integrate(mesh, rho_in))
        outer += 1
        if fixed_outer is None and dl < tol:
            break
    return SCFResult(U, lam, rho_in, outer, history, charge)
