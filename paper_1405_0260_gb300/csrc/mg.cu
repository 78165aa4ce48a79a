// Geometric multigrid V-cycle and the MG-preconditioned CG kernels (see mg.cuh).
//
// All level kernels map one thread to one (interior node, group of 4 orbitals)
// pair, x fastest, so a warp reads the orbital-minor vectors of consecutive
// nodes with 16-byte accesses and the 27 operator weights of a node once per
// node (the same address in every group).
#include <cmath>

#include "cgutil.cuh"
#include "mg.cuh"

namespace paro {

namespace {

constexpr int kMGThreads = 256;

__device__ __forceinline__ void interior_ijk(const Grid& g, long long n, int& i, int& j, int& k) {
  const int ix = g.nx - 1, iy = g.ny - 1;
  i = (int)(n % ix) + 1;
  const long long t = n / ix;
  j = (int)(t % iy) + 1;
  k = (int)(t / iy) + 1;
}

__device__ __forceinline__ long long padded(const Grid& g, int i, int j, int k) {
  return ((long long)k * g.Py + j) * g.Px + i;
}

__device__ __forceinline__ bool group_active(const int* act, int q) {
  return act == nullptr || (act[4 * q] | act[4 * q + 1] | act[4 * q + 2] | act[4 * q + 3]) != 0;
}

// (y += w x) on 4 orbitals
__device__ __forceinline__ void axpy4(float w, const Vec4<float>& x, Vec4<float>& y) {
#pragma unroll
  for (int c = 0; c < 4; ++c) y.v[c] = fmaf(w, x.v[c], y.v[c]);
}

// A x at padded node gp for orbital group q (27 weights, SoA [27][G])
__device__ __forceinline__ Vec4<float> stencil(const Grid& g, int Np, const float* __restrict__ coef,
                                               const float* __restrict__ x, long long gp, int q) {
  const long long plane = (long long)g.Px * g.Py;
  Vec4<float> acc{};
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const float w = __ldg(coef + (long long)o * g.G + gp);
    const long long nb = gp + dz * plane + (long long)dy * g.Px + dx;
    axpy4(w, lds4(x + nb * Np + 4 * q), acc);
  }
  return acc;
}

// MODE 0: out = b - A x.  MODE 1: out = x + omega D^-1 (b - A x).  MODE 2: out = omega D^-1 b.
template <int MODE>
__global__ void __launch_bounds__(kMGThreads) k_mg_level(Grid g, int Np, const float* __restrict__ coef,
                                                         const float* __restrict__ dinv, float omega,
                                                         const float* __restrict__ b, const float* __restrict__ x,
                                                         float* __restrict__ out, const int* __restrict__ act) {
  const int G4 = Np >> 2;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = idx / G4;
  const int q = (int)(idx - n * G4);
  if (n >= g.nI || !group_active(act, q)) return;
  int i, j, k;
  interior_ijk(g, n, i, j, k);
  const long long gp = padded(g, i, j, k);
  const long long e = gp * Np + 4 * q;
  const Vec4<float> bv = lds4(b + e);
  Vec4<float> r;
  if (MODE == 2) {
    const float d = omega * dinv[gp];
#pragma unroll
    for (int c = 0; c < 4; ++c) r.v[c] = d * bv.v[c];
  } else {
    const Vec4<float> ax = stencil(g, Np, coef, x, gp, q);
    if (MODE == 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) r.v[c] = bv.v[c] - ax.v[c];
    } else {
      const Vec4<float> xv = lds4(x + e);
      const float d = omega * dinv[gp];
#pragma unroll
      for (int c = 0; c < 4; ++c) r.v[c] = fmaf(d, bv.v[c] - ax.v[c], xv.v[c]);
    }
  }
  sts4(out + e, r);
}

// 1-D weight of fine offset e in {-1, 0, 1} from the coinciding coarse node
__device__ __forceinline__ float pw(int e) { return e == 0 ? 1.f : 0.5f; }

// b_c = P^T t_f: coarse node I gathers the 27 fine nodes 2I + e
__global__ void __launch_bounds__(kMGThreads) k_mg_restrict(Grid gf, Grid gc, int Np, const float* __restrict__ tf,
                                                            float* __restrict__ bc, const int* __restrict__ act) {
  const int G4 = Np >> 2;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = idx / G4;
  const int q = (int)(idx - n * G4);
  if (n >= gc.nI || !group_active(act, q)) return;
  int I, J, K;
  interior_ijk(gc, n, I, J, K);
  Vec4<float> acc{};
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int ex = o % 3 - 1, ey = (o / 3) % 3 - 1, ez = o / 9 - 1;
    const float w = pw(ex) * pw(ey) * pw(ez);
    const long long f = padded(gf, 2 * I + ex, 2 * J + ey, 2 * K + ez);
    axpy4(w, lds4(tf + f * Np + 4 * q), acc);
  }
  sts4(bc + padded(gc, I, J, K) * Np + 4 * q, acc);
}

// y_f += P x_c: fine node i takes coarse node i/2 (i even) or the two nodes
// (i -/+ 1)/2 with weight 1/2 (i odd), per axis; coarse boundary values are zero
__global__ void __launch_bounds__(kMGThreads) k_mg_prolong(Grid gf, Grid gc, int Np, const float* __restrict__ xc,
                                                           float* __restrict__ yf, const int* __restrict__ act) {
  const int G4 = Np >> 2;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = idx / G4;
  const int q = (int)(idx - n * G4);
  if (n >= gf.nI || !group_active(act, q)) return;
  int i, j, k;
  interior_ijk(gf, n, i, j, k);
  const int ax0 = i >> 1, ax1 = (i + 1) >> 1, ay0 = j >> 1, ay1 = (j + 1) >> 1, az0 = k >> 1, az1 = (k + 1) >> 1;
  const float wx = (i & 1) ? 0.5f : 1.f, wy = (j & 1) ? 0.5f : 1.f, wz = (k & 1) ? 0.5f : 1.f;
  const long long e = padded(gf, i, j, k) * Np + 4 * q;
  Vec4<float> acc = lds4(yf + e);
  // an even axis has ax0 == ax1 and takes one node (weight 1); an odd axis two (1/2 each)
  for (int cz = 0; cz < ((k & 1) ? 2 : 1); ++cz)
    for (int cy = 0; cy < ((j & 1) ? 2 : 1); ++cy)
      for (int cx = 0; cx < ((i & 1) ? 2 : 1); ++cx) {
        const long long c = padded(gc, cx ? ax1 : ax0, cy ? ay1 : ay0, cz ? az1 : az0);
        axpy4(wx * wy * wz, lds4(xc + c * Np + 4 * q), acc);
      }
  sts4(yf + e, acc);
}

// Galerkin coarse operator, one thread per coarse interior node I:
//   A_c[I, I + d] = sum_{k = 2I + e} P[k, I] sum_o A_f[k, k + o] P[k + o, I + d]
// (the coarse nodes J with P[l, J] != 0 are l/2 for even l and (l -/+ 1)/2 for odd l,
// per axis; coarse boundary nodes carry no unknown and are left out).
__global__ void __launch_bounds__(128) k_mg_galerkin(Grid gf, Grid gc, const double* __restrict__ cf,
                                                     double* __restrict__ cc64, float* __restrict__ cc32,
                                                     float* __restrict__ dc32) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= gc.nI) return;
  int I[3];
  interior_ijk(gc, n, I[0], I[1], I[2]);
  const int nc[3] = {gc.nx, gc.ny, gc.nz};
  double w[27];
#pragma unroll
  for (int o = 0; o < 27; ++o) w[o] = 0.0;
  for (int e = 0; e < 27; ++e) {
    const int ek[3] = {e % 3 - 1, (e / 3) % 3 - 1, e / 9 - 1};
    const double pk = (ek[0] ? 0.5 : 1.0) * (ek[1] ? 0.5 : 1.0) * (ek[2] ? 0.5 : 1.0);
    const int kf[3] = {2 * I[0] + ek[0], 2 * I[1] + ek[1], 2 * I[2] + ek[2]};
    const long long gk = padded(gf, kf[0], kf[1], kf[2]);
    for (int o = 0; o < 27; ++o) {
      const double a = cf[(long long)o * gf.G + gk];
      if (a == 0.0) continue;
      const int l[3] = {kf[0] + o % 3 - 1, kf[1] + (o / 3) % 3 - 1, kf[2] + o / 9 - 1};
      int J0[3], J1[3], cnt[3];
      for (int d = 0; d < 3; ++d) {
        J0[d] = l[d] >> 1;
        J1[d] = (l[d] + 1) >> 1;
        cnt[d] = (l[d] & 1) ? 2 : 1;
      }
      const double pl = ((l[0] & 1) ? 0.5 : 1.0) * ((l[1] & 1) ? 0.5 : 1.0) * ((l[2] & 1) ? 0.5 : 1.0);
      for (int cz = 0; cz < cnt[2]; ++cz)
        for (int cy = 0; cy < cnt[1]; ++cy)
          for (int cx = 0; cx < cnt[0]; ++cx) {
            const int J[3] = {cx ? J1[0] : J0[0], cy ? J1[1] : J0[1], cz ? J1[2] : J0[2]};
            bool inner = true;
            for (int d = 0; d < 3; ++d) inner = inner && J[d] >= 1 && J[d] <= nc[d] - 1;
            if (!inner) continue;
            const int od = (J[2] - I[2] + 1) * 9 + (J[1] - I[1] + 1) * 3 + (J[0] - I[0] + 1);
            w[od] += pk * a * pl;
          }
    }
  }
  const long long gp = padded(gc, I[0], I[1], I[2]);
  for (int o = 0; o < 27; ++o) {
    cc64[(long long)o * gc.G + gp] = w[o];
    cc32[(long long)o * gc.G + gp] = (float)w[o];
  }
  dc32[gp] = 1.0f / (float)w[13];
}

// Gershgorin: out = max over interior rows of sum_j |A_ij| / A_ii (interior j only),
// as the bit pattern of a positive double (ordered like the value)
__global__ void __launch_bounds__(256) k_mg_rho(Grid g, const double* __restrict__ coef, unsigned long long* out) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double ratio = 0.0;
  if (n < g.nI) {
    int i, j, k;
    interior_ijk(g, n, i, j, k);
    const long long gp = padded(g, i, j, k);
    double s = 0.0;
    for (int o = 0; o < 27; ++o) {
      const int x = i + o % 3 - 1, y = j + (o / 3) % 3 - 1, z = k + o / 9 - 1;
      if (x < 1 || x > g.nx - 1 || y < 1 || y > g.ny - 1 || z < 1 || z > g.nz - 1) continue;
      s += fabs(coef[(long long)o * g.G + gp]);
    }
    ratio = s / coef[13LL * g.G + gp];
  }
  // block max, then one atomic per block
  __shared__ double red[256];
  red[threadIdx.x] = ratio;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0 && red[0] > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(red[0]));
}

// w = A u on the fine grid; partial sums (r, u), (w, u), (r, r) per orbital; the
// last CTA forms alpha, beta and the masks (the recurrences of the CG kernel).
__global__ void __launch_bounds__(256) k_mg_wdots(CGArgs<float> a, const float* __restrict__ coef) {
  extern __shared__ double dsm[];
  const int Np = a.Np, G4 = Np / 4;
  const int nt = blockDim.x;  // a multiple of G4
  const int q = threadIdx.x % G4;
  const float* u = a.r2;
  float acc[3][4] = {};
  const bool gact = group_active(a.st->active, q);
  if (gact) {
    const long long rowlen = (long long)(a.g.nx - 1) * G4;
    const long long total = rowlen * (long long)(a.g.ny - 1) * (a.g.nz - 1);
    for (long long t = (long long)blockIdx.x * nt + threadIdx.x; t < total; t += (long long)gridDim.x * nt) {
      const long long row = t / rowlen;
      const long long off = t - row * rowlen;
      const int y = (int)(row % (a.g.ny - 1)) + 1, z = (int)(row / (a.g.ny - 1)) + 1;
      const long long gp = ((long long)z * a.g.Py + y) * a.g.Px + 1 + off / G4;
      const long long e = gp * Np + 4 * q;
      const Vec4<float> w = stencil(a.g, Np, coef, u, gp, q);
      const Vec4<float> uv = lds4(u + e), rv = lds4(a.r + e);
      sts4(a.q + e, w);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        acc[0][c] = fmaf(rv.v[c], uv.v[c], acc[0][c]);
        acc[1][c] = fmaf(w.v[c], uv.v[c], acc[1][c]);
        acc[2][c] = fmaf(rv.v[c], rv.v[c], acc[2][c]);
      }
    }
  }
  double* red = dsm;
  const int NTs = nt / G4;
  const int j = threadIdx.x / G4;
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 4; ++c) red[j * 3 * Np + k * Np + 4 * q + c] = (double)acc[k][c];
  __syncthreads();
  double* ctmp = red + (size_t)NTs * 3 * Np;
  block_colsum(red, NTs, 3 * Np, ctmp);
  for (int t = threadIdx.x; t < 3 * Np; t += nt) {
    const int k = t / Np, o = t % Np;
    a.part[((long long)k * gridDim.x + blockIdx.x) * Np + o] = ctmp[t];
  }
  if (!last_cta(&a.st->ticket)) return;
  double* tot = dsm + (nt > 3 * Np ? nt : 3 * Np);
  reduce_over_ctas<3>(a.part, gridDim.x, Np, dsm, tot);
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const double tol = a.st->tol;
  const int maxit = a.st->maxit;
  for (int o = threadIdx.x; o < Np; o += nt) {
    double alpha = 0.0, beta = 0.0;
    bool act = a.st->active[o] != 0;
    if (act) {
      const double gam = tot[o], del = tot[Np + o], rr = tot[2 * Np + o];
      const int it = a.st->iters[o];
      a.st->rr[o] = rr;
      if (!(isfinite(gam) && isfinite(del) && isfinite(rr))) {
        atomicOr(&a.st->status, kStatNonFinite);
        act = false;
      } else if (rr <= tol * tol * a.st->bb[o]) {
        act = false;
      } else if (it >= maxit) {
        atomicOr(&a.st->status, kStatNotConverged);
        act = false;
      } else {
        beta = it > 0 ? gam / a.st->rz[o] : 0.0;
        const double den = it > 0 ? del - beta * gam / a.st->alpha[o] : del;  // = (p, A p)
        if (!(gam > 0.0) || !(den > 0.0)) {
          atomicOr(&a.st->status, kStatNotSPD);
          act = false;
          beta = 0.0;
        } else {
          alpha = gam / den;
          a.st->rz[o] = gam;
          a.st->iters[o] = it + 1;  // x is updated with this alpha
        }
      }
    }
    a.st->alpha[o] = act ? alpha : 0.0;
    a.st->beta[o] = act ? beta : 0.0;
    a.st->active[o] = act ? 1 : 0;
    if (act) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a.st->n_active = cnt;
    a.st->ticket = 0u;
  }
}

// p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s (active groups)
__global__ void __launch_bounds__(kMGThreads) k_mg_update(CGArgs<float> a) {
  __shared__ float sal[kMaxN], sbe[kMaxN];
  const int Np = a.Np, G4 = Np / 4;
  for (int o = threadIdx.x; o < Np; o += blockDim.x) {
    sal[o] = (float)a.st->alpha[o];
    sbe[o] = (float)a.st->beta[o];
  }
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = idx / G4;
  const int q = (int)(idx - n * G4);
  if (n >= a.g.nI || !group_active(a.st->active, q)) return;
  int i, j, k;
  interior_ijk(a.g, n, i, j, k);
  const long long e = padded(a.g, i, j, k) * Np + 4 * q;
  Vec4<float> u = lds4(a.r2 + e), w = lds4(a.q + e), p = lds4(a.p + e), s = lds4(a.s + e);
  Vec4<float> x = lds4(a.x + e), r = lds4(a.r + e);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float al = sal[4 * q + c], be = sbe[4 * q + c];
    p.v[c] = fmaf(be, p.v[c], u.v[c]);
    s.v[c] = fmaf(be, s.v[c], w.v[c]);
    x.v[c] = fmaf(al, p.v[c], x.v[c]);
    r.v[c] = fmaf(-al, s.v[c], r.v[c]);
  }
  sts4(a.p + e, p);
  sts4(a.s + e, s);
  sts4(a.x + e, x);
  sts4(a.r + e, r);
}

unsigned blocks_for(long long threads, int per) { return (unsigned)((threads + per - 1) / per); }

}  // namespace

int mg_plan_levels(const Grid& g0, Grid* out, int max_levels) {
  int n = 0;
  Grid g = g0;
  while (n + 1 < max_levels && g.nx % 2 == 0 && g.ny % 2 == 0 && g.nz % 2 == 0 && g.nx >= 4 && g.ny >= 4 &&
         g.nz >= 4) {
    Grid c{};
    c.nx = g.nx / 2, c.ny = g.ny / 2, c.nz = g.nz / 2;
    c.Px = c.nx + 1, c.Py = c.ny + 1, c.Pz = c.nz + 1;
    c.G = (long long)c.Px * c.Py * c.Pz;
    c.nI = (c.nx - 1) * (c.ny - 1) * (c.nz - 1);
    c.hx = 2 * g.hx, c.hy = 2 * g.hy, c.hz = 2 * g.hz;
    out[n++] = c;
    g = c;
  }
  return n;
}

cudaError_t launch_mg_galerkin(const Grid& gf, const Grid& gc, const double* cf, double* cc64, float* cc32,
                               float* dc32, cudaStream_t st) {
  k_mg_galerkin<<<blocks_for(gc.nI, 128), 128, 0, st>>>(gf, gc, cf, cc64, cc32, dc32);
  return cudaGetLastError();
}

cudaError_t launch_mg_rho(const Grid& g, const double* coef, unsigned long long* out, cudaStream_t st) {
  k_mg_rho<<<blocks_for(g.nI, 256), 256, 0, st>>>(g, coef, out);
  return cudaGetLastError();
}

cudaError_t mg_vcycle(const MGHier& h, int Np, const float* r, float* out, float* y0, float* t0, const int* active,
                      int nu, int nu_c, cudaStream_t st, long long* launches) {
  const int G4 = Np / 4;
  cudaError_t e = cudaSuccess;
  auto level = [&](int mode, const MGLevel& L, const float* b, const float* x, float* o) {
    const unsigned nb = blocks_for((long long)L.g.nI * G4, kMGThreads);
    if (mode == 0)
      k_mg_level<0><<<nb, kMGThreads, 0, st>>>(L.g, Np, L.coef32, L.dinv32, L.omega, b, x, o, active);
    else if (mode == 1)
      k_mg_level<1><<<nb, kMGThreads, 0, st>>>(L.g, Np, L.coef32, L.dinv32, L.omega, b, x, o, active);
    else
      k_mg_level<2><<<nb, kMGThreads, 0, st>>>(L.g, Np, L.coef32, L.dinv32, L.omega, b, x, o, active);
    ++*launches;
    if (e == cudaSuccess) e = cudaGetLastError();
  };
  // nu sweeps from x = 0 into the pair (X, Y), ending in X after the post-sweeps
  // (see the buffer rule below); returns the buffer that holds the iterate
  for (int l = 0; l < h.nlev; ++l) {
    const MGLevel& L = h.lev[l];
    const float* b = l == 0 ? r : L.b;
    float* X = l == 0 ? out : L.x;
    float* Y = l == 0 ? y0 : L.y;
    float* T = l == 0 ? t0 : L.t;
    const bool coarsest = l == h.nlev - 1;
    const int sweeps = coarsest ? nu_c : nu;
    // pre-sweeps alternate Y, X, Y, ...: the first goes to Y, except on the
    // coarsest level with an odd count, which must end in X
    float* cur = (coarsest && (sweeps & 1)) ? X : Y;
    level(2, L, b, nullptr, cur);
    for (int s = 1; s < sweeps; ++s) {
      float* nxt = cur == X ? Y : X;
      level(1, L, b, cur, nxt);
      cur = nxt;
    }
    if (coarsest) break;
    level(0, L, b, cur, T);
    const MGLevel& C = h.lev[l + 1];
    k_mg_restrict<<<blocks_for((long long)C.g.nI * G4, kMGThreads), kMGThreads, 0, st>>>(L.g, C.g, Np, T, C.b,
                                                                                          active);
    ++*launches;
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  // upward: prolongate the coarse correction into the level's iterate, post-sweeps
  for (int l = h.nlev - 2; l >= 0; --l) {
    const MGLevel& L = h.lev[l];
    const MGLevel& C = h.lev[l + 1];
    const float* b = l == 0 ? r : L.b;
    float* X = l == 0 ? out : L.x;
    float* Y = l == 0 ? y0 : L.y;
    // the pre-sweeps ended in Y (nu odd) or X (nu even); nu post-sweeps then end in X
    float* cur = (nu & 1) ? Y : X;
    k_mg_prolong<<<blocks_for((long long)L.g.nI * G4, kMGThreads), kMGThreads, 0, st>>>(L.g, C.g, Np, C.x, cur,
                                                                                         active);
    ++*launches;
    if (e == cudaSuccess) e = cudaGetLastError();
    for (int s = 0; s < nu; ++s) {
      float* nxt = cur == X ? Y : X;
      level(1, L, b, cur, nxt);
      cur = nxt;
    }
  }
  return e;
}

cudaError_t mg_launch_wdots(CGPlan<float>* P, const float* coef32, cudaStream_t st) {
  k_mg_wdots<<<P->grid_stream, P->nt_stream, P->smem_init, st>>>(P->args, coef32);
  return cudaGetLastError();
}

cudaError_t mg_launch_update(CGPlan<float>* P, cudaStream_t st) {
  const int G4 = P->args.Np / 4;
  k_mg_update<<<blocks_for((long long)P->args.g.nI * G4, kMGThreads), kMGThreads, 0, st>>>(P->args);
  return cudaGetLastError();
}

}  // namespace paro
