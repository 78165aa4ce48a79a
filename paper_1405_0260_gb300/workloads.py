"""Seeded synthetic inputs for the ParO hot path.

This module generates problem data only: box, mesh size, the external
potential sampled at the 2x2x2 Gauss points of every cell, the shift sigma and
random Gaussian initial orbitals.  It contains none of the method's
arithmetic (no stencil, solver or projection) and imports neither torch nor
the CUDA library, so both the CUDA path and the CPU oracle consume exactly the
same arrays.

Layouts (shared with the C ABI, see include/paro.h):
  Vq : float64, 8 values per cell, order [cz][cy][cx][qz][qy][qx];
       Gauss abscissae (1 -/+ 1/sqrt(3))/2 in each cell's unit coordinates.
  U0 : float64, (n_interior, N) row-major; interior node (i, j, k), 1-based
       within 1..n-1 per axis, has row ((k-1)(ny-1) + (j-1))(nx-1) + (i-1).

Workloads (paper Section 4 uses molecules on adaptive meshes; these synthetic
stand-ins keep the structure: Coulomb-like wells, N lowest orbitals, Gaussian
initial guesses as suggested for Step 1 of Algorithm 3.1):
  hydrogen       Z=1 at a cell centre, V=-1/r, [-10,10]^3, 32^3 cells, N=5, sigma=2
  harmonic       V=r^2/2, [-8,8]^3, 64^3 cells, N=20, sigma=0
  cluster        softened Coulomb -Z/sqrt(r^2+0.25) from 8 random nuclei (Kohn-Sham SCF)
  batch_systems  64 independent systems, 1-6 nuclei each, meshes 32-96^3, N 4-48
  large_cluster  40 nuclei, [-20,20]^3, 192^3 cells, N=256, standard normal initial block
  random_block   unit-variance orbitals for throughput runs
  graded_hydrogen  the hydrogen-like nucleus on a mesh graded toward it (Section 2.1)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_G = ((1.0 - 1.0 / math.sqrt(3.0)) / 2.0, (1.0 + 1.0 / math.sqrt(3.0)) / 2.0)


@dataclass
class Problem:
    name: str
    n: tuple  # cells per axis (nx, ny, nz)
    lo: tuple
    hi: tuple
    Vq: np.ndarray  # (8*nx*ny*nz,) float64
    sigma: float
    U0: np.ndarray  # (n_interior, N) float64
    tol: float  # stop on max |delta lambda| < tol
    nuclei: np.ndarray | None = None  # (M, 4): x, y, z, Z
    n_occ: int | None = None  # orbitals tested for convergence (Algorithm 3.2 buffer)
    coords: tuple | None = None  # graded mesh: node coordinates per axis (None: uniform)

    @property
    def N(self) -> int:
        return self.U0.shape[1]

    @property
    def n_interior(self) -> int:
        nx, ny, nz = self.n
        return (nx - 1) * (ny - 1) * (nz - 1)

    @property
    def h(self) -> tuple:
        return tuple((self.hi[d] - self.lo[d]) / self.n[d] for d in range(3))


def _axis_nodes(n, lo, hi, coords):
    if coords is not None:
        return [np.asarray(c, dtype=np.float64) for c in coords]
    return [lo[d] + (hi[d] - lo[d]) / n[d] * np.arange(n[d] + 1) for d in range(3)]


def gauss_point_coords(n, lo, hi, coords=None):
    """Coordinates (x, y, z) of the Gauss points, each shaped (nz, ny, nx, 2, 2, 2);
    coords: node coordinates per axis of a graded mesh (None: uniform)."""
    nx, ny, nz = n
    nodes = _axis_nodes(n, lo, hi, coords)
    g = np.array(_G)
    p = [nodes[d][:-1, None] + np.diff(nodes[d])[:, None] * g[None, :] for d in range(3)]  # [cell][q]
    x = p[0][None, None, :, None, None, :]
    y = p[1][None, :, None, None, :, None]
    z = p[2][:, None, None, :, None, None]
    shape = (nz, ny, nx, 2, 2, 2)
    return np.broadcast_to(x, shape), np.broadcast_to(y, shape), np.broadcast_to(z, shape)


def interior_node_coords(n, lo, hi, coords=None):
    """(n_interior, 3) coordinates of the interior nodes in unknown order."""
    nodes = _axis_nodes(n, lo, hi, coords)
    xs = [nodes[d][1:-1] for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def graded_axis(nc, L, beta):
    """nc + 1 node coordinates on [-L, L], finest at 0: x_i = L sinh(beta t_i) / sinh(beta),
    t_i = -1 + 2 i / nc (beta -> 0: uniform; cells grow by about e^(2 beta / nc) outward)."""
    t = -1.0 + 2.0 * np.arange(nc + 1) / nc
    if beta == 0.0:
        return L * t
    x = L * np.sinh(beta * t) / np.sinh(beta)
    x[0], x[-1] = -L, L
    return x


def gaussian_orbitals(n, lo, hi, N, rng, width=(0.5, 3.0), centre=(-1.0, 1.0), coords=None):
    """N seeded Gaussians exp(-|x-c|^2 / (2 w^2)) at the interior nodes.

    Draw order: all N widths w ~ U[width], then the N x 3 centres c ~ U[centre].
    """
    w = rng.uniform(width[0], width[1], size=N)
    c = rng.uniform(centre[0], centre[1], size=(N, 3))
    xyz = interior_node_coords(n, lo, hi, coords)
    d2 = ((xyz[:, None, :] - c[None, :, :]) ** 2).sum(axis=2)
    return np.exp(-d2 / (2.0 * w[None, :] ** 2))


def place_nuclei(rng, M, zmax, box, min_sep, max_tries=100000):
    """M nuclei uniform in [-box, box]^3, pairwise >= min_sep apart (rejection), Z ~ U{1..zmax}."""
    pos = []
    tries = 0
    while len(pos) < M:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place nuclei with the requested separation")
        p = rng.uniform(-box, box, size=3)
        if all(np.linalg.norm(p - q) >= min_sep for q in pos):
            pos.append(p)
    Z = rng.integers(1, zmax + 1, size=M)
    return np.concatenate([np.array(pos), Z[:, None].astype(np.float64)], axis=1)


def softened_coulomb(n, lo, hi, nuclei, soft=0.25):
    """V = -sum_k Z_k / sqrt(|x - R_k|^2 + soft) at the Gauss points (flat, Vq order)."""
    x, y, z = gauss_point_coords(n, lo, hi)
    V = np.zeros(x.shape)
    for R0, R1, R2, Zk in nuclei:
        V -= Zk / np.sqrt((x - R0) ** 2 + (y - R1) ** 2 + (z - R2) ** 2 + soft)
    return np.ascontiguousarray(V.ravel())


def hydrogen(nc=32, L=10.0, N=5, seed=1000, sigma=2.0, Z=1.0, tol=1e-8):
    """Hydrogen-like single nucleus at the centre of the cell whose lower corner is the origin.

    V = -Z/|x - R| at the Gauss points (never singular there: R is a cell centre).
    """
    n = (nc, nc, nc)
    lo, hi = (-L, -L, -L), (L, L, L)
    h = 2.0 * L / nc
    R = np.array([h / 2, h / 2, h / 2])
    x, y, z = gauss_point_coords(n, lo, hi)
    V = -Z / np.sqrt((x - R[0]) ** 2 + (y - R[1]) ** 2 + (z - R[2]) ** 2)
    rng = np.random.default_rng(seed)
    U0 = gaussian_orbitals(n, lo, hi, N, rng)
    nuc = np.array([[R[0], R[1], R[2], Z]])
    return Problem(f"hydrogen-{nc}^3-N{N}", n, lo, hi, np.ascontiguousarray(V.ravel()), sigma, U0, tol, nuc)


def graded_hydrogen(nc=16, L=10.0, beta=2.0, N=5, seed=1100, sigma=2.0, Z=1.0, tol=1e-8):
    """Hydrogen-like nucleus at the origin on a graded mesh (Section 2.1: a mesh
    refined where the orbitals vary fast): every axis graded_axis(nc, L, beta),
    nc even so the nucleus sits on a node, V = -Z/r at the Gauss points (never
    singular there), Gaussian initial orbitals as for the uniform workload."""
    ax = graded_axis(nc, L, beta)
    coords = (ax, ax, ax)
    n = (nc, nc, nc)
    lo, hi = (-L, -L, -L), (L, L, L)
    x, y, z = gauss_point_coords(n, lo, hi, coords)
    V = -Z / np.sqrt(x ** 2 + y ** 2 + z ** 2)
    rng = np.random.default_rng(seed)
    U0 = gaussian_orbitals(n, lo, hi, N, rng, coords=coords)
    nuc = np.array([[0.0, 0.0, 0.0, Z]])
    return Problem(f"graded-hydrogen-{nc}^3-b{beta}-N{N}", n, lo, hi, np.ascontiguousarray(V.ravel()), sigma, U0,
                   tol, nuc, coords=coords)


def harmonic(nc=64, L=8.0, N=20, seed=2000, sigma=0.0, omega=1.0, tol=1e-10):
    """3-D harmonic oscillator V = omega^2 r^2 / 2 at the Gauss points."""
    n = (nc, nc, nc)
    lo, hi = (-L, -L, -L), (L, L, L)
    x, y, z = gauss_point_coords(n, lo, hi)
    V = 0.5 * omega ** 2 * (x ** 2 + y ** 2 + z ** 2)
    rng = np.random.default_rng(seed)
    U0 = gaussian_orbitals(n, lo, hi, N, rng)
    return Problem(f"harmonic-{nc}^3-N{N}", n, lo, hi, np.ascontiguousarray(V.ravel()), sigma, U0, tol)


def free_box(n=(8, 8, 8), L=(1.0, 1.0, 1.0), N=4, seed=7, sigma=0.0, tol=1e-10):
    """V = 0 in [-L, L] (particle in a box); the discrete spectrum has a closed form."""
    lo = tuple(-float(v) for v in L)
    hi = tuple(float(v) for v in L)
    V = np.zeros(8 * n[0] * n[1] * n[2])
    rng = np.random.default_rng(seed)
    U0 = gaussian_orbitals(n, lo, hi, N, rng, width=(0.3 * min(L), 0.8 * min(L)),
                           centre=(-0.2 * min(L), 0.2 * min(L)))
    return Problem(f"box-{n}-N{N}", tuple(n), lo, hi, V, sigma, U0, tol)


def cluster(nc=128, L=12.0, n_nuclei=8, zmax=4, box=6.0, min_sep=2.0, seed=3000,
            extra=8, sigma=None, tol=1e-7):
    """Synthetic softened-Coulomb cluster; N = ceil(sum Z / 2) + extra orbitals.

    sigma None: left to the caller (the shift must make H + sigma M SPD).
    """
    rng = np.random.default_rng(seed)
    nuc = place_nuclei(rng, n_nuclei, zmax, box, min_sep)
    n = (nc, nc, nc)
    lo, hi = (-L, -L, -L), (L, L, L)
    V = softened_coulomb(n, lo, hi, nuc)
    n_occ = int(math.ceil(nuc[:, 3].sum() / 2.0))
    N = n_occ + extra
    U0 = gaussian_orbitals(n, lo, hi, N, rng, centre=(-box, box))
    return Problem(f"cluster-{nc}^3-{n_nuclei}nuc-N{N}", n, lo, hi, V,
                   float(sigma) if sigma is not None else 0.0, U0, tol, nuc, n_occ)


def random_block(n, N, seed):
    """Unit-variance random orbitals for throughput runs (no physics)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    return rng.standard_normal(((nx - 1) * (ny - 1) * (nz - 1), N))


def batch_systems(count=64, seed=4000, L=10.0, meshes=(32, 48, 64, 96), n_range=(4, 48), n_nuclei=(1, 6),
                  zmax=3, box=4.0, min_sep=1.5, tol=1e-7):
    """Independent fixed-potential systems for batched runs.

    Each system: 1-6 softened-Coulomb nuclei (Z ~ U{1..zmax}) uniform in
    [-box, box]^3, pairwise >= min_sep apart, on [-L, L]^3 with nc drawn from
    meshes and N ~ U{n_range}; Gaussian initial orbitals.  sigma is left to the
    caller (it must make H + sigma M SPD).
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nc = int(rng.choice(meshes))
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        M = int(rng.integers(n_nuclei[0], n_nuclei[1] + 1))
        nuc = place_nuclei(rng, M, zmax, box, min_sep)
        n = (nc, nc, nc)
        lo, hi = (-L, -L, -L), (L, L, L)
        V = softened_coulomb(n, lo, hi, nuc)
        U0 = gaussian_orbitals(n, lo, hi, N, rng)
        out.append(Problem(f"batch{k}-{nc}^3-{M}nuc-N{N}", n, lo, hi, V, 0.0, U0, tol, nuc))
    return out


def large_cluster(nc=192, L=20.0, n_nuclei=40, zmax=4, box=14.0, min_sep=1.8, N=256, seed=5000, tol=1e-7):
    """The large fixed-potential workload: 40 softened-Coulomb nuclei (Z ~ U{1..4})
    uniform in [-14, 14]^3 at least 1.8 bohr apart, cube [-20, 20]^3, nc^3 cells,
    N orbitals.  Initial block: seeded standard normal values (N seeded Gaussians
    on this mesh would be numerically dependent); sigma is left to the caller."""
    rng = np.random.default_rng(seed)
    nuc = place_nuclei(rng, n_nuclei, zmax, box, min_sep)
    n = (nc, nc, nc)
    lo, hi = (-L, -L, -L), (L, L, L)
    V = softened_coulomb(n, lo, hi, nuc)
    U0 = rng.standard_normal(((nc - 1) ** 3, N))
    return Problem(f"large-{nc}^3-{n_nuclei}nuc-N{N}", n, lo, hi, V, 0.0, U0, tol, nuc)

