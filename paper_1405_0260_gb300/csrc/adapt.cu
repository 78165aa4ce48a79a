// The adaptive loop of Section 2.1 (Solve -> Estimate -> Mark -> Refine) on
// tensor-product meshes.
//
// Estimate: an error indicator per element.  The paper names a-posteriori
// indicators eta_k(., tau) without a formula; here the residual indicator of
// -1/2 Lap u + V u = lambda u with Q1 elements, summed over the orbitals:
//   eta_tau^2 = sum_i [ h_tau^2 ||(lambda_i - V) u_i||^2_tau
//                       + 1/2 sum_{interior F of tau} h_F ||1/2 [d_n u_i]||^2_F ]
// (Lap u = 0 inside a trilinear element; V at the cell's 2x2x2 Gauss points;
// the normal-derivative jump is bilinear on a face and its square is integrated
// exactly with the bilinear face mass matrix; h_tau, h_F: cell and face
// diameters; Dirichlet boundary faces carry no jump).  One thread per cell.
//
// Mark: Doerfler's strategy, eq. (2.2) (least cardinality, largest indicators
// first) or the maximum strategy, eq. (2.3), on the host.
//
// Refine: every marked element refined at least once: on a tensor-product mesh
// every axis interval that holds a marked cell is bisected (host).
//
// Transfer: the coarse Q1 space lies in the refined one (old nodes are kept), so
// the orbitals move to the new mesh by trilinear interpolation of their nodal
// values (one thread per new interior node and orbital block of four).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "../../include/paro.h"
#include "common.cuh"

namespace paro {

namespace {

__device__ __forceinline__ double axis_h(const Grid& g, int d, int c) {
  if (g.graded) return cell_h(g, d, c);
  return d == 0 ? g.hx : (d == 1 ? g.hy : g.hz);
}

// Bilinear mass matrix of the unit square on corner values c (order (0,0),
// (1,0), (0,1), (1,1)): c^T B c, B = [4 2 2 1; 2 4 1 2; 2 1 4 2; 1 2 2 4] / 36.
__device__ __forceinline__ double face_quad(const double c[4]) {
  const double d = 4.0 * (c[0] * c[0] + c[1] * c[1] + c[2] * c[2] + c[3] * c[3]) +
                   4.0 * (c[0] * c[1] + c[0] * c[2] + c[1] * c[3] + c[2] * c[3]) + 2.0 * (c[0] * c[3] + c[1] * c[2]);
  return d / 36.0;
}

__global__ void k_estimate(Grid g, int N, int Np, const double* __restrict__ u, const double* __restrict__ lam,
                           const double* __restrict__ Vq, double* __restrict__ eta2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ncell = (long long)g.nx * g.ny * g.nz;
  if (t >= ncell) return;
  const int cx = (int)(t % g.nx);
  const int cy = (int)((t / g.nx) % g.ny);
  const int cz = (int)(t / ((long long)g.nx * g.ny));
  const double hx = axis_h(g, 0, cx), hy = axis_h(g, 1, cy), hz = axis_h(g, 2, cz);
  // padded node index of (i, j, k)
  auto node = [&](int i, int j, int k) { return ((long long)k * g.Py + j) * g.Px + i; };
  // the two Gauss points of [0, 1] and the linear Lagrange values there
  const double gp0 = 0.5 - 0.5 / sqrt(3.0), gp1 = 0.5 + 0.5 / sqrt(3.0);
  const double l[2][2] = {{1.0 - gp0, 1.0 - gp1}, {gp0, gp1}};  // l[a][q]
  const double vol = hx * hy * hz, diam2 = hx * hx + hy * hy + hz * hz;
  const double* V = Vq + t * 8;  // [qz][qy][qx] of this cell
  double acc = 0.0;
  for (int o = 0; o < N; ++o) {
    const double lo = lam[o];
    double w[2][2][2];  // [az][ay][ax]
    for (int az = 0; az < 2; ++az)
      for (int ay = 0; ay < 2; ++ay)
        for (int ax = 0; ax < 2; ++ax) w[az][ay][ax] = u[node(cx + ax, cy + ay, cz + az) * Np + o];
    // element residual (lambda - V) u at the Gauss points
    for (int qz = 0; qz < 2; ++qz)
      for (int qy = 0; qy < 2; ++qy)
        for (int qx = 0; qx < 2; ++qx) {
          double uq = 0.0;
          for (int az = 0; az < 2; ++az)
            for (int ay = 0; ay < 2; ++ay)
              for (int ax = 0; ax < 2; ++ax) uq += l[ax][qx] * l[ay][qy] * l[az][qz] * w[az][ay][ax];
          const double r = (lo - V[(qz * 2 + qy) * 2 + qx]) * uq;
          acc += diam2 * (0.125 * vol) * r * r;
        }
    // faces: the jump of d/dx across the x-planes cx (left face) and cx + 1 (right
    // face), and likewise in y and z, at the face's four corner node lines
    for (int dir = 0; dir < 3; ++dir) {
      const int n_d = dir == 0 ? g.nx : (dir == 1 ? g.ny : g.nz);
      const int c_d = dir == 0 ? cx : (dir == 1 ? cy : cz);
      // the other two axes of the face: sizes and the corner offsets
      const double ha = dir == 0 ? hy : hx, hb = dir == 2 ? hy : hz;
      for (int side = 0; side < 2; ++side) {
        const int plane = c_d + side;  // node plane of the face
        if (plane < 1 || plane > n_d - 1) continue;  // boundary face: no jump term
        const double hl = axis_h(g, dir, plane - 1), hr = axis_h(g, dir, plane);
        double cj[4];
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a) {
            // corner (a, b) of the face in its two tangential axes
            int i0, j0, k0;
            if (dir == 0) {
              i0 = plane; j0 = cy + a; k0 = cz + b;
            } else if (dir == 1) {
              i0 = cx + a; j0 = plane; k0 = cz + b;
            } else {
              i0 = cx + a; j0 = cy + b; k0 = plane;
            }
            const int di = dir == 0, dj = dir == 1, dk = dir == 2;
            const double um = u[node(i0 - di, j0 - dj, k0 - dk) * Np + o];
            const double u0 = u[node(i0, j0, k0) * Np + o];
            const double up = u[node(i0 + di, j0 + dj, k0 + dk) * Np + o];
            cj[b * 2 + a] = (up - u0) / hr - (u0 - um) / hl;
          }
        const double hF = sqrt(ha * ha + hb * hb);
        acc += 0.5 * hF * 0.25 * ha * hb * face_quad(cj);
      }
    }
  }
  eta2[t] = acc;
}

// U_to[n][o] for the interior nodes n of the fine mesh: trilinear interpolation of
// U_from (interior rows of the coarse mesh, zero on its boundary) in the coarse
// cell (kx, ky, kz) with local coordinates (tx, ty, tz) of each fine node axis.
__global__ void k_transfer(Grid gc, Grid gf, int N, const double* __restrict__ Uc, const int* __restrict__ kmap,
                           const double* __restrict__ tmap, double* __restrict__ Uf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)gf.nI * N) return;
  const int o = (int)(t % N);
  const long long n = t / N;
  const int fx = gf.nx - 1, fy = gf.ny - 1;
  const int i = (int)(n % fx), j = (int)((n / fx) % fy), k = (int)(n / ((long long)fx * fy));
  // per-axis maps: x entries [0, fx), y [fx, fx + fy), z after
  const int kx = kmap[i], ky = kmap[fx + j], kz = kmap[fx + fy + k];
  const double tx = tmap[i], ty = tmap[fx + j], tz = tmap[fx + fy + k];
  const int cx = gc.nx - 1, cy = gc.ny - 1;
  double v = 0.0;
  for (int az = 0; az < 2; ++az)
    for (int ay = 0; ay < 2; ++ay)
      for (int ax = 0; ax < 2; ++ax) {
        const int a = kx + ax, b = ky + ay, c = kz + az;  // coarse node
        if (a < 1 || a > gc.nx - 1 || b < 1 || b > gc.ny - 1 || c < 1 || c > gc.nz - 1) continue;  // boundary: 0
        const double w = (ax ? tx : 1.0 - tx) * (ay ? ty : 1.0 - ty) * (az ? tz : 1.0 - tz);
        const long long cn = ((long long)(c - 1) * cy + (b - 1)) * cx + (a - 1);
        v += w * Uc[cn * N + o];
      }
  Uf[t] = v;
}

}  // namespace

cudaError_t launch_estimate(const Grid& g, int N, int Np, const double* u, const double* lam, const double* Vq,
                            double* eta2, cudaStream_t st) {
  const long long ncell = (long long)g.nx * g.ny * g.nz;
  k_estimate<<<(unsigned)((ncell + 127) / 128), 128, 0, st>>>(g, N, Np, u, lam, Vq, eta2);
  return cudaGetLastError();
}

cudaError_t launch_transfer(const Grid& gc, const Grid& gf, int N, const double* Uc, const int* kmap,
                            const double* tmap, double* Uf, cudaStream_t st) {
  const long long work = (long long)gf.nI * N;
  k_transfer<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(gc, gf, N, Uc, kmap, tmap, Uf);
  return cudaGetLastError();
}

}  // namespace paro

extern "C" {

int paro_mark(long long ncells, const double* eta2, int strategy, double theta, unsigned char* marked) {
  if (ncells < 1 || !eta2 || !marked || !(theta > 0.0 && theta < 1.0)) return PARO_ERR_ARG;
  if (strategy != PARO_MARK_DORFLER && strategy != PARO_MARK_MAXIMUM) return PARO_ERR_ARG;
  double total = 0.0, mx = 0.0;
  for (long long c = 0; c < ncells; ++c) {
    if (!(eta2[c] >= 0.0) || !std::isfinite(eta2[c])) return PARO_ERR_NONFINITE;
    total += eta2[c];
    mx = std::max(mx, eta2[c]);
  }
  std::fill(marked, marked + ncells, (unsigned char)0);
  long long count = 0;
  if (strategy == PARO_MARK_MAXIMUM) {
    // eq. (2.3): eta >= theta max eta, i.e. eta^2 >= theta^2 max eta^2
    for (long long c = 0; c < ncells; ++c)
      if (eta2[c] >= theta * theta * mx) {
        marked[c] = 1;
        ++count;
      }
    return (int)std::min<long long>(count, 0x7fffffff);
  }
  // eq. (2.2): largest indicators first (ties by cell index) until theta of the total
  std::vector<long long> order((size_t)ncells);
  std::iota(order.begin(), order.end(), 0LL);
  std::stable_sort(order.begin(), order.end(), [&](long long a, long long b) { return eta2[a] > eta2[b]; });
  double acc = 0.0;
  for (long long k : order) {
    if (acc >= theta * total) break;
    marked[k] = 1;
    acc += eta2[k];
    ++count;
  }
  return (int)std::min<long long>(count, 0x7fffffff);
}

int paro_refine_coords(const int n[3], const double* coords, const unsigned char* marked, int n_out[3],
                       double* coords_out) {
  if (!n || !coords || !marked || !n_out || !coords_out) return PARO_ERR_ARG;
  const int nx = n[0], ny = n[1], nz = n[2];
  if (nx < 2 || ny < 2 || nz < 2) return PARO_ERR_ARG;
  std::vector<char> hit[3] = {std::vector<char>(nx, 0), std::vector<char>(ny, 0), std::vector<char>(nz, 0)};
  for (int cz = 0; cz < nz; ++cz)
    for (int cy = 0; cy < ny; ++cy)
      for (int cx = 0; cx < nx; ++cx)
        if (marked[((long long)cz * ny + cy) * nx + cx]) {
          hit[0][cx] = 1;
          hit[1][cy] = 1;
          hit[2][cz] = 1;
        }
  const double* in = coords;
  double* out = coords_out;
  for (int d = 0; d < 3; ++d) {
    const int nd = n[d];
    for (int k = 0; k < nd; ++k)
      if (!(in[k + 1] > in[k])) return PARO_ERR_ARG;
    int m = 0;
    out[m++] = in[0];
    for (int k = 0; k < nd; ++k) {
      if (hit[d][k]) out[m++] = 0.5 * (in[k] + in[k + 1]);
      out[m++] = in[k + 1];
    }
    n_out[d] = m - 1;
    in += nd + 1;
    out += m;
  }
  return PARO_OK;
}

}  // extern "C"
