// Float64 iterative refinement around the float32 CG of the mixed mode
// (cg.cu): the residual r = b - A x of the source problems (Step 3, eq. 3.2)
// in float64, its float32 rounding as the correction right-hand side, and the
// update x += d.  The residual kernel reduces ||r||^2 and ||b||^2 per orbital
// (block partials, then the last block sums them in a fixed order) and flags
// converged orbitals so the next correction solve skips them.
#include <cmath>

#include "cg.cuh"
#include "common.cuh"
#include "ff.cuh"

namespace paro {

namespace {

// Block-level deterministic reduction of K per-orbital sums held as acc[k][4]
// by each thread (thread owns orbitals 4*grp .. 4*grp+3), then last-block
// detection.  Returns true in the last block, with tot[k*Np + o] filled (shared;
// tot may alias sred: K*Np <= K*kRedThreads*4 and sred is consumed first).
template <int K>
__device__ bool reduce_partials(const double (&acc)[K][4], int Np, int grp, int nl, bool live, double* partial,
                                unsigned int* ticket, double* sred, double* tot) {
  NodeMap nm = node_map(Np);
  for (int k = 0; k < K; ++k)
    if (live)
      for (int c = 0; c < 4; ++c) sred[k * kRedThreads * 4 + nl * Np + 4 * grp + c] = acc[k][c];
  __syncthreads();
  for (int t = threadIdx.x; t < K * Np; t += blockDim.x) {
    int k = t / Np, o = t % Np;
    double s = 0.0;
    for (int b = 0; b < nm.npb; ++b) s += sred[k * kRedThreads * 4 + b * Np + o];
    partial[((long long)k * kMaxRedBlocks + blockIdx.x) * Np + o] = s;
  }
  __threadfence();
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(ticket, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // Fixed-order sum over blocks: one warp per (k, o), lanes stride the blocks,
  // then a butterfly of fixed shape.
  int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nwarps = blockDim.x / 32;
  for (int t = warp; t < K * Np; t += nwarps) {
    int k = t / Np, o = t % Np;
    const double* src = partial + (long long)k * kMaxRedBlocks * Np + o;
    double s = 0.0;
    // eight loads in flight a lane before the additions (one L2 round trip per 256 blocks)
    for (int b0 = lane; b0 < (int)gridDim.x; b0 += 32 * 8) {
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int b = b0 + 32 * q;
        v[q] = b < (int)gridDim.x ? __ldcg(src + (long long)b * Np) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) s += v[q];
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) tot[t] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

template <typename T>
__device__ __forceinline__ V4<T> ld4v(const T* base, long long node, int Np, int grp) {
  return ld4(base + node * Np + 4 * grp);
}

// Mixed refinement residual in float64: r = b - A x; its float32 rounding is the
// right-hand side of the correction solve.  Orbitals with ||r|| <= tol ||b||
// (or padding) are flagged in skip[] and excluded from the correction solve.
__global__ void __launch_bounds__(kRedThreads) k_refine_residual(Grid g, int N, int Np, const double* __restrict__ coef,
                                                                 const double* __restrict__ x,
                                                                 const double* __restrict__ b, float* __restrict__ rhs,
                                                                 CGState s, double tol) {
  __shared__ double sred[2 * kRedThreads * 4];
  double* tot = sred;
  __shared__ int cnt;
  NodeMap nm = node_map(Np);
  int grp = threadIdx.x % nm.groups;
  int nl = threadIdx.x / nm.groups;
  bool live = nl < nm.npb;
  double acc[2][4] = {};
  if (live) {
    for (int n = blockIdx.x * nm.npb + nl; n < g.nI; n += gridDim.x * nm.npb) {
      long long gp = interior_to_padded(g, n);
      double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
      for (int o = 0; o < 27; ++o) {
        const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
        long long nb = gp + ((long long)dz * g.Py + dy) * g.Px + dx;
        double w = coef[(long long)o * g.G + gp];
        V4<double> xv = ld4v(x, nb, Np, grp);
        a0 += w * xv.a;
        a1 += w * xv.b;
        a2 += w * xv.c;
        a3 += w * xv.d;
      }
      V4<double> bv = ld4v(b, gp, Np, grp);
      double r[4] = {bv.a - a0, bv.b - a1, bv.c - a2, bv.d - a3};
      if (rhs != nullptr) st4(rhs + gp * Np + 4 * grp, V4<float>{(float)r[0], (float)r[1], (float)r[2], (float)r[3]});
      acc[0][0] += r[0] * r[0]; acc[0][1] += r[1] * r[1]; acc[0][2] += r[2] * r[2]; acc[0][3] += r[3] * r[3];
      acc[1][0] += bv.a * bv.a; acc[1][1] += bv.b * bv.b; acc[1][2] += bv.c * bv.c; acc[1][3] += bv.d * bv.d;
    }
  }
  if (!reduce_partials<2>(acc, Np, grp, nl, live, s.partial, s.ticket, sred, tot)) return;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int o = threadIdx.x; o < Np; o += blockDim.x) {
    double rr = tot[o], bb = tot[Np + o];
    s.rr[o] = rr;
    s.bb[o] = bb;
    bool done = (o >= N) || rr <= tol * tol * bb;
    if (o < N && !(isfinite(rr) && isfinite(bb))) {
      atomicOr(s.status, kStatNonFinite);
      done = true;
    }
    s.skip[o] = done ? 1 : 0;
    if (!done) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *s.n_active = cnt;
}

// The same residual in float-float arithmetic (ff.cuh): x and b as hi/lo arrays,
// the packed per-node float-float weights of A.
__global__ void __launch_bounds__(kRedThreads, 2) k_refine_residual_ff(Grid g, int N, int Np, const float* __restrict__ whi,
                                                                    const float* __restrict__ wlo,
                                                                    const float* __restrict__ xhi,
                                                                    const float* __restrict__ xlo,
                                                                    const float* __restrict__ bhi,
                                                                    const float* __restrict__ blo,
                                                                    float* __restrict__ rhs, CGState s, double tol,
                                                                    int gm) {
  __shared__ double sred[2 * kRedThreads * 4];
  double* tot = sred;
  __shared__ int cnt;
  NodeMap nm = node_map(Np);
  int grp = threadIdx.x % nm.groups;
  int nl = threadIdx.x / nm.groups;
  bool live = nl < nm.npb;
  double acc[2][4] = {};
  if (live) {
    float arr[4] = {0, 0, 0, 0}, abb[4] = {0, 0, 0, 0};
    for (int n = blockIdx.x * nm.npb + nl; n < g.nI; n += gridDim.x * nm.npb) {
      long long gp = interior_to_padded(g, n);
      float wh[28], wl[28];
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        const float4 a = reinterpret_cast<const float4*>(whi + gp * kPackedW)[q];
        const float4 c = reinterpret_cast<const float4*>(wlo + gp * kPackedW)[q];
        wh[4 * q] = a.x, wh[4 * q + 1] = a.y, wh[4 * q + 2] = a.z, wh[4 * q + 3] = a.w;
        wl[4 * q] = c.x, wl[4 * q + 1] = c.y, wl[4 * q + 2] = c.z, wl[4 * q + 3] = c.w;
      }
      FF ax[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
#pragma unroll
      for (int o = 0; o < 27; ++o) {
        const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
        const long long nb = gp + ((long long)dz * g.Py + dy) * g.Px + dx;
        const FF w{wh[o], wl[o]};
        const float4 h = *reinterpret_cast<const float4*>(xhi + nb * Np + 4 * grp);
        const float4 l = *reinterpret_cast<const float4*>(xlo + nb * Np + 4 * grp);
        ff_mac(ax[0], FF{h.x, l.x}, w);
        ff_mac(ax[1], FF{h.y, l.y}, w);
        ff_mac(ax[2], FF{h.z, l.z}, w);
        ff_mac(ax[3], FF{h.w, l.w}, w);
      }
      const float4 bh4 = *reinterpret_cast<const float4*>(bhi + gp * Np + 4 * grp);
      const float4 bl4 = *reinterpret_cast<const float4*>(blo + gp * Np + 4 * grp);
      const float bh[4] = {bh4.x, bh4.y, bh4.z, bh4.w}, bl[4] = {bl4.x, bl4.y, bl4.z, bl4.w};
      float r[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        FF rc{bh[c], bl[c]};
        ff_add(rc, ff_neg(ax[c]));
        rc = ff_norm(rc);
        r[c] = rc.hi;
        arr[c] = fmaf(rc.hi, rc.hi, arr[c]);
        abb[c] = fmaf(bh[c], bh[c], abb[c]);
      }
      if (rhs != nullptr) {
        // node-major [G][Np], or group-major [Np/4][G][4] for the single-pass CG
        const long long e = gm ? ((long long)grp * g.G + gp) * 4 : gp * Np + 4 * grp;
        st4(rhs + e, V4<float>{r[0], r[1], r[2], r[3]});
      }
    }
    for (int c = 0; c < 4; ++c) {
      acc[0][c] = arr[c];
      acc[1][c] = abb[c];
    }
  }
  if (!reduce_partials<2>(acc, Np, grp, nl, live, s.partial, s.ticket, sred, tot)) return;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int o = threadIdx.x; o < Np; o += blockDim.x) {
    double rr = tot[o], bb = tot[Np + o];
    s.rr[o] = rr;
    s.bb[o] = bb;
    bool done = (o >= N) || rr <= tol * tol * bb;
    if (o < N && !(isfinite(rr) && isfinite(bb))) {
      atomicOr(s.status, kStatNonFinite);
      done = true;
    }
    s.skip[o] = done ? 1 : 0;
    if (!done) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *s.n_active = cnt;
}

// The refinement's closing check when a Rayleigh-Ritz step follows on the same x:
// y = H x (27 points, float-float, the packed H weights), r = b - y - sigma M x
// with M x given (mhi, mlo), the norms and skip flags as in k_refine_residual_ff
// (A = H + sigma M), and y written over b (each thread reads b at its own node
// before writing y there), so the Rayleigh-Ritz step finds H x and M x formed.
__global__ void __launch_bounds__(kRedThreads, 2) k_refine_check_hff(Grid g, int N, int Np, const float* __restrict__ whi,
                                                                  const float* __restrict__ wlo,
                                                                  const float* __restrict__ xhi,
                                                                  const float* __restrict__ xlo,
                                                                  const float* __restrict__ mhi,
                                                                  const float* __restrict__ mlo, FF sig, float* bhy,
                                                                  float* bly, CGState s, double tol) {
  __shared__ double sred[2 * kRedThreads * 4];
  double* tot = sred;
  __shared__ int cnt;
  NodeMap nm = node_map(Np);
  int grp = threadIdx.x % nm.groups;
  int nl = threadIdx.x / nm.groups;
  bool live = nl < nm.npb;
  double acc[2][4] = {};
  if (live) {
    float arr[4] = {0, 0, 0, 0}, abb[4] = {0, 0, 0, 0};
    for (int n = blockIdx.x * nm.npb + nl; n < g.nI; n += gridDim.x * nm.npb) {
      long long gp = interior_to_padded(g, n);
      float wh[28], wl[28];
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        const float4 a = reinterpret_cast<const float4*>(whi + gp * kPackedW)[q];
        const float4 c = reinterpret_cast<const float4*>(wlo + gp * kPackedW)[q];
        wh[4 * q] = a.x, wh[4 * q + 1] = a.y, wh[4 * q + 2] = a.z, wh[4 * q + 3] = a.w;
        wl[4 * q] = c.x, wl[4 * q + 1] = c.y, wl[4 * q + 2] = c.z, wl[4 * q + 3] = c.w;
      }
      FF hx[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
#pragma unroll
      for (int o = 0; o < 27; ++o) {
        const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
        const long long nb = gp + ((long long)dz * g.Py + dy) * g.Px + dx;
        const FF w{wh[o], wl[o]};
        const float4 h = *reinterpret_cast<const float4*>(xhi + nb * Np + 4 * grp);
        const float4 l = *reinterpret_cast<const float4*>(xlo + nb * Np + 4 * grp);
        ff_mac(hx[0], FF{h.x, l.x}, w);
        ff_mac(hx[1], FF{h.y, l.y}, w);
        ff_mac(hx[2], FF{h.z, l.z}, w);
        ff_mac(hx[3], FF{h.w, l.w}, w);
      }
      const long long e = gp * Np + 4 * grp;
      const float4 bh4 = *reinterpret_cast<const float4*>(bhy + e);
      const float4 bl4 = *reinterpret_cast<const float4*>(bly + e);
      const float4 mh4 = *reinterpret_cast<const float4*>(mhi + e);
      const float4 ml4 = *reinterpret_cast<const float4*>(mlo + e);
      const float bh[4] = {bh4.x, bh4.y, bh4.z, bh4.w}, bl[4] = {bl4.x, bl4.y, bl4.z, bl4.w};
      const float mh[4] = {mh4.x, mh4.y, mh4.z, mh4.w}, ml[4] = {ml4.x, ml4.y, ml4.z, ml4.w};
      float yh[4], yl[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const FF y = ff_norm(hx[c]);
        yh[c] = y.hi;
        yl[c] = y.lo;
        FF t = y;  // H x + sigma M x = A x
        ff_mac(t, FF{mh[c], ml[c]}, sig);
        FF rc{bh[c], bl[c]};
        ff_add(rc, ff_neg(ff_norm(t)));
        rc = ff_norm(rc);
        arr[c] = fmaf(rc.hi, rc.hi, arr[c]);
        abb[c] = fmaf(bh[c], bh[c], abb[c]);
      }
      *reinterpret_cast<float4*>(bhy + e) = make_float4(yh[0], yh[1], yh[2], yh[3]);
      *reinterpret_cast<float4*>(bly + e) = make_float4(yl[0], yl[1], yl[2], yl[3]);
    }
    for (int c = 0; c < 4; ++c) {
      acc[0][c] = arr[c];
      acc[1][c] = abb[c];
    }
  }
  if (!reduce_partials<2>(acc, Np, grp, nl, live, s.partial, s.ticket, sred, tot)) return;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int o = threadIdx.x; o < Np; o += blockDim.x) {
    double rr = tot[o], bb = tot[Np + o];
    s.rr[o] = rr;
    s.bb[o] = bb;
    bool done = (o >= N) || rr <= tol * tol * bb;
    if (o < N && !(isfinite(rr) && isfinite(bb))) {
      atomicOr(s.status, kStatNonFinite);
      done = true;
    }
    s.skip[o] = done ? 1 : 0;
    if (!done) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *s.n_active = cnt;
}

// x += d for the orbitals the correction solve ran for (d group-major), and the
// float-float split of the new x for the next residual; skipped orbitals keep x
// (and, the split being a function of x, the same split).  Vector loads and
// stores of a thread's four orbitals; one float64 addition an element.
// x = x_in + d for the orbitals not skipped, x = x_in for the others, and the
// float-float split of the new x.  x_in == x: in place (groups whose four
// orbitals are all skipped are left alone); x_in != x (the first sweep, x_in
// the orbitals u the solve starts from): every group is written.
__global__ void k_refine_update_split(Grid g, int Np, const double* x_in, double* x, const float* __restrict__ d,
                                      const int* __restrict__ skip, float* __restrict__ xh, float* __restrict__ xl) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int groups = Np / 4;
  if (t >= (long long)g.nI * groups) return;
  const int n = (int)(t / groups), grp = (int)(t % groups);
  const int4 sk = *reinterpret_cast<const int4*>(skip + 4 * grp);
  if (x_in == x && sk.x && sk.y && sk.z && sk.w) return;
  const long long gp = interior_to_padded(g, n);
  const float4 dv = *reinterpret_cast<const float4*>(d + ((long long)grp * g.G + gp) * 4);
  const long long e = gp * Np + 4 * grp;
  const double2* xq = reinterpret_cast<const double2*>(x_in + e);
  double2* xp = reinterpret_cast<double2*>(x + e);
  const double2 a = xq[0], b = xq[1];
  const double v0 = sk.x ? a.x : a.x + f2d_exact(dv.x);
  const double v1 = sk.y ? a.y : a.y + f2d_exact(dv.y);
  const double v2 = sk.z ? b.x : b.x + f2d_exact(dv.z);
  const double v3 = sk.w ? b.y : b.y + f2d_exact(dv.w);
  xp[0] = make_double2(v0, v1);
  xp[1] = make_double2(v2, v3);
  const FF f0 = ff_split(v0), f1 = ff_split(v1), f2 = ff_split(v2), f3 = ff_split(v3);
  *reinterpret_cast<float4*>(xh + e) = make_float4(f0.hi, f1.hi, f2.hi, f3.hi);
  *reinterpret_cast<float4*>(xl + e) = make_float4(f0.lo, f1.lo, f2.lo, f3.lo);
}

__global__ void k_refine_update(Grid g, int Np, double* __restrict__ x, const float* __restrict__ d,
                                const int* __restrict__ skip) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.nI * Np) return;
  int n = (int)(t / Np), o = (int)(t % Np);
  if (skip[o]) return;
  long long gp = interior_to_padded(g, n);
  x[gp * Np + o] += (double)d[gp * Np + o];
}

}  // namespace

int red_blocks(const Grid& g, int Np) {
  NodeMap nm = node_map(Np);
  long long need = (g.nI + nm.npb - 1) / nm.npb;
  long long cap = kMaxRedBlocks;
  return (int)(need < cap ? need : cap);
}

cudaError_t launch_refine_residual(const Grid& g, int N, int Np, const double* coef64, const double* x64,
                                   const double* b64, float* rhs32, const CGState& s, double tol, cudaStream_t st) {
  k_refine_residual<<<red_blocks(g, Np), kRedThreads, 0, st>>>(g, N, Np, coef64, x64, b64, rhs32, s, tol);
  return cudaGetLastError();
}

cudaError_t launch_refine_residual_ff(const Grid& g, int N, int Np, const float* whi, const float* wlo,
                                      const float* xhi, const float* xlo, const float* bhi, const float* blo,
                                      float* rhs32, const CGState& s, double tol, cudaStream_t st, int gm) {
  // two 256-thread blocks resident a SM (up to 128 registers a thread), two waves
  const int grid = red_blocks(g, Np) < 152 * 4 ? red_blocks(g, Np) : 152 * 4;
  k_refine_residual_ff<<<grid, kRedThreads, 0, st>>>(g, N, Np, whi, wlo, xhi, xlo, bhi, blo, rhs32, s, tol, gm);
  return cudaGetLastError();
}

cudaError_t launch_refine_check_hff(const Grid& g, int N, int Np, const float* whi, const float* wlo,
                                    const float* xhi, const float* xlo, const float* mhi, const float* mlo,
                                    double sigma, float* bhy, float* bly, const CGState& s, double tol,
                                    cudaStream_t st) {
  const int grid = red_blocks(g, Np) < 152 * 4 ? red_blocks(g, Np) : 152 * 4;
  k_refine_check_hff<<<grid, kRedThreads, 0, st>>>(g, N, Np, whi, wlo, xhi, xlo, mhi, mlo, ff_split_host(sigma), bhy,
                                                   bly, s, tol);
  return cudaGetLastError();
}

cudaError_t launch_refine_update(const Grid& g, int Np, double* x64, const float* d32, const int* skip,
                                 cudaStream_t st) {
  long long work = (long long)g.nI * Np;
  k_refine_update<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(g, Np, x64, d32, skip);
  return cudaGetLastError();
}

cudaError_t launch_refine_update_split(const Grid& g, int Np, const double* x_in, double* x64, const float* d32gm,
                                       const int* skip, float* xh, float* xl, cudaStream_t st) {
  const long long work = (long long)g.nI * (Np / 4);
  k_refine_update_split<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(g, Np, x_in, x64, d32gm, skip, xh, xl);
  return cudaGetLastError();
}

}  // namespace paro
