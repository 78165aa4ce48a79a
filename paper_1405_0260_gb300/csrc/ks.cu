// Kohn-Sham pieces of the SCF workload (Section 2.2): the electron density at
// the Gauss points, the Hartree potential by a Poisson solve through the same
// stencil and CG (-Delta V_H = 4 pi rho with the monopole of rho as Dirichlet
// data), Slater exchange, and linear density mixing.  All fields live at the
// 2x2x2 Gauss points of every cell, [cz][cy][cx][qz][qy][qx], the points at
// which the operator takes its potential.
#include <cmath>

#include "common.cuh"
#include "q1.cuh"

namespace paro {

namespace {

inline unsigned nblk(long long work, int threads) { return (unsigned)((work + threads - 1) / threads); }

// sum_q r[q] phi_a(x_q) for one corner a of the cell, axis by axis
__device__ __forceinline__ double project1(const double* r, int a) {
  const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
  double s = 0.0;
#pragma unroll
  for (int qz = 0; qz < 2; ++qz) {
    double t = 0.0;
#pragma unroll
    for (int qy = 0; qy < 2; ++qy) {
      const double* rr = r + 4 * qz + 2 * qy;
      t += gq(ay, qy) * (gq(ax, 0) * rr[0] + gq(ax, 1) * rr[1]);
    }
    s += gq(az, qz) * t;
  }
  return s;
}

// rho_q = sum_i f_i (sum_a phi_a(x_q) u_i(a))^2, one thread per cell (its 8 Gauss
// points), orbitals two at a time (16-byte loads of the 8 corner rows).
// U in the padded layout [node][Np] (boundary rows zero, Np even).
__global__ void __launch_bounds__(128) k_density(Grid g, int N, int Np, const double* __restrict__ U,
                                                 const double* __restrict__ occ, double* __restrict__ rho) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ncell = (long long)g.nx * g.ny * g.nz;
  if (c >= ncell) return;
  const int cx = (int)(c % g.nx), cy = (int)((c / g.nx) % g.ny), cz = (int)(c / ((long long)g.nx * g.ny));
  long long node[8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
    node[a] = ((long long)(cz + ((a >> 2) & 1)) * g.Py + (cy + ((a >> 1) & 1))) * g.Px + (cx + (a & 1));
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < N; i += 2) {
    double c0[8], c1[8], v[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const double2 u = __ldg(reinterpret_cast<const double2*>(U + node[a] * Np + i));
      c0[a] = u.x;
      c1[a] = u.y;
    }
    const double f0 = occ[i];
    interp8(c0, v);
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] += f0 * v[q] * v[q];
    if (i + 1 < N) {
      const double f1 = occ[i + 1];
      interp8(c1, v);
#pragma unroll
      for (int q = 0; q < 8; ++q) s[q] += f1 * v[q] * v[q];
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) rho[c * 8 + q] = s[q];
}

// Per-block partial sums of (w rho, w rho x, w rho y, w rho z) over the Gauss points.
__global__ void k_moments(Grid g, double lox, double loy, double loz, const double* __restrict__ rho,
                          double* __restrict__ part) {
  __shared__ double sm[4][256];
  const long long ncell = (long long)g.nx * g.ny * g.nz;
  const double w = g.hx * g.hy * g.hz / 8.0;
  const double gp[2] = {0.5 - 0.5 / 1.7320508075688772935, 0.5 + 0.5 / 1.7320508075688772935};
  double a[4] = {0, 0, 0, 0};
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < ncell * 8;
       t += (long long)gridDim.x * blockDim.x) {
    const long long c = t / 8;
    const int q = (int)(t % 8);
    const int cx = (int)(c % g.nx), cy = (int)((c / g.nx) % g.ny), cz = (int)(c / ((long long)g.nx * g.ny));
    const double r = w * rho[t];
    a[0] += r;
    a[1] += r * (lox + g.hx * (cx + gp[q & 1]));
    a[2] += r * (loy + g.hy * (cy + gp[(q >> 1) & 1]));
    a[3] += r * (loz + g.hz * (cz + gp[(q >> 2) & 1]));
  }
  for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 4) part[blockIdx.x * 4 + threadIdx.x] = sm[threadIdx.x][0];
}

// Fixed-order sum of the block partials: out[0] = Q, out[1..3] = centre.
__global__ void k_moments_final(int nblocks, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a[4] = {0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b)
    for (int k = 0; k < 4; ++k) a[k] += part[b * 4 + k];
  out[0] = a[0];
  for (int k = 1; k < 4; ++k) out[k] = a[0] != 0.0 ? a[k] / a[0] : 0.0;
}

__device__ __forceinline__ double monopole_at(const double* mom, double x, double y, double z) {
  const double Q = mom[0];
  if (Q == 0.0) return 0.0;
  const double dx = x - mom[1], dy = y - mom[2], dz = z - mom[3];
  return Q / sqrt(dx * dx + dy * dy + dz * dz);
}

// Right-hand side of (K/2) w = 2 pi (rho, phi_i) - (K/2)_{i,boundary} g at the
// interior nodes, padded layout with Np = 4 (column 0); kcoef = the 27 weights
// of K/2 (a handle with V = 0, sigma = 0).
__global__ void k_hartree_rhs(Grid g, double lox, double loy, double loz, const double* __restrict__ rho,
                              const double* __restrict__ kcoef, const double* __restrict__ mom,
                              double* __restrict__ rhs) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nI) return;
  const int ix = (int)(n % (g.nx - 1)) + 1, iy = (int)((n / (g.nx - 1)) % (g.ny - 1)) + 1,
            iz = (int)(n / ((long long)(g.nx - 1) * (g.ny - 1))) + 1;
  const long long gp = ((long long)iz * g.Py + iy) * g.Px + ix;
  const double w = g.hx * g.hy * g.hz / 8.0;
  double b = 0.0;
  // the 8 cells around the node: cell (ix - 1 + ex, ...), the node is local corner a = (1-ex, 1-ey, 1-ez)
  for (int ez = 0; ez < 2; ++ez)
    for (int ey = 0; ey < 2; ++ey)
      for (int ex = 0; ex < 2; ++ex) {
        const long long c = ((long long)(iz - 1 + ez) * g.ny + (iy - 1 + ey)) * g.nx + (ix - 1 + ex);
        const int a = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
        b += w * project1(rho + c * 8, a);
      }
  double bnd = 0.0;
  for (int o = 0; o < 27; ++o) {
    const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
    const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
    if (jx == 0 || jx == g.nx || jy == 0 || jy == g.ny || jz == 0 || jz == g.nz)
      bnd += kcoef[(long long)o * g.G + gp] *
             monopole_at(mom, lox + jx * g.hx, loy + jy * g.hy, loz + jz * g.hz);
  }
  rhs[gp * 4] = 2.0 * M_PI * b - bnd;
}

// V_q = V_ext + V_H + V_x at the Gauss points: V_H interpolated from the nodal
// solution (interior: w, padded layout with Np = 4; boundary: the monopole).
__global__ void __launch_bounds__(128) k_ks_potential(Grid g, double lox, double loy, double loz,
                                                      const double* __restrict__ w, const double* __restrict__ mom,
                                                      const double* __restrict__ rho,
                                                      const double* __restrict__ vext, double* __restrict__ vout,
                                                      double* __restrict__ vh_out) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ncell = (long long)g.nx * g.ny * g.nz;
  if (c >= ncell) return;
  const int cx = (int)(c % g.nx), cy = (int)((c / g.nx) % g.ny), cz = (int)(c / ((long long)g.nx * g.ny));
  double cv[8], vh[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int jx = cx + (a & 1), jy = cy + ((a >> 1) & 1), jz = cz + ((a >> 2) & 1);
    if (jx == 0 || jx == g.nx || jy == 0 || jy == g.ny || jz == 0 || jz == g.nz)
      cv[a] = monopole_at(mom, lox + jx * g.hx, loy + jy * g.hy, loz + jz * g.hz);
    else
      cv[a] = w[(((long long)jz * g.Py + jy) * g.Px + jx) * 4];
  }
  interp8(cv, vh);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const long long t = c * 8 + q;
    const double r = rho[t] > 0.0 ? rho[t] : 0.0;
    const double vx = -cbrt(3.0 * r / M_PI);  // Slater exchange
    if (vh_out) vh_out[t] = vh[q];
    if (vout) vout[t] = vext[t] + vh[q] + vx;
  }
}

// Per-block partial sums over the Gauss points (weight w = hx hy hz / 8) of
// w rho V_H, w rho V_x and w e_x(rho), Slater: V_x = -(3 rho / pi)^(1/3),
// e_x = 3/4 rho V_x.
__global__ void k_energy_terms(Grid g, const double* __restrict__ rho, const double* __restrict__ vh,
                               double* __restrict__ part) {
  __shared__ double sm[3][256];
  const long long n = (long long)g.nx * g.ny * g.nz * 8;
  const double w = g.hx * g.hy * g.hz / 8.0;
  double a[3] = {0, 0, 0};
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double r = rho[t] > 0.0 ? rho[t] : 0.0;
    const double vx = -cbrt(3.0 * r / M_PI);
    a[0] += w * r * vh[t];
    a[1] += w * r * vx;
    a[2] += w * 0.75 * r * vx;
  }
  for (int k = 0; k < 3; ++k) sm[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 3; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 3) part[blockIdx.x * 3 + threadIdx.x] = sm[threadIdx.x][0];
}

// Fixed-order sum of the block partials: out[0..2].
__global__ void k_energy_final(int nblocks, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a[3] = {0, 0, 0};
  for (int b = 0; b < nblocks; ++b)
    for (int k = 0; k < 3; ++k) a[k] += part[b * 3 + k];
  for (int k = 0; k < 3; ++k) out[k] = a[k];
}

// rho_in <- (1 - beta) rho_in + beta rho_out
__global__ void k_mix(long long n, double beta, double* __restrict__ rho_in, const double* __restrict__ rho_out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) rho_in[t] = (1.0 - beta) * rho_in[t] + beta * rho_out[t];
}

}  // namespace

cudaError_t launch_density(const Grid& g, int N, int Np, const double* U, const double* occ, double* rho,
                           cudaStream_t st) {
  k_density<<<nblk((long long)g.nx * g.ny * g.nz, 128), 128, 0, st>>>(g, N, Np, U, occ, rho);
  return cudaGetLastError();
}

int moments_blocks() { return 152 * 2; }

cudaError_t launch_moments(const Grid& g, const double lo[3], const double* rho, double* part, double* mom,
                           cudaStream_t st) {
  const int nb = moments_blocks();
  k_moments<<<nb, 256, 0, st>>>(g, lo[0], lo[1], lo[2], rho, part);
  k_moments_final<<<1, 32, 0, st>>>(nb, part, mom);
  return cudaGetLastError();
}

cudaError_t launch_hartree_rhs(const Grid& g, const double lo[3], const double* rho, const double* kcoef,
                               const double* mom, double* rhs, cudaStream_t st) {
  k_hartree_rhs<<<nblk(g.nI, 128), 128, 0, st>>>(g, lo[0], lo[1], lo[2], rho, kcoef, mom, rhs);
  return cudaGetLastError();
}

cudaError_t launch_ks_potential(const Grid& g, const double lo[3], const double* w, const double* mom,
                                const double* rho, const double* vext, double* vout, double* vh_out,
                                cudaStream_t st) {
  k_ks_potential<<<nblk((long long)g.nx * g.ny * g.nz, 128), 128, 0, st>>>(g, lo[0], lo[1], lo[2], w, mom, rho,
                                                                           vext, vout, vh_out);
  return cudaGetLastError();
}

cudaError_t launch_energy_terms(const Grid& g, const double* rho, const double* vh, double* part, double* out,
                                cudaStream_t st) {
  const int nb = moments_blocks();
  k_energy_terms<<<nb, 256, 0, st>>>(g, rho, vh, part);
  k_energy_final<<<1, 32, 0, st>>>(nb, part, out);
  return cudaGetLastError();
}

cudaError_t launch_mix(long long n, double beta, double* rho_in, const double* rho_out, cudaStream_t st) {
  k_mix<<<nblk(n, 256), 256, 0, st>>>(n, beta, rho_in, rho_out);
  return cudaGetLastError();
}

}  // namespace paro
