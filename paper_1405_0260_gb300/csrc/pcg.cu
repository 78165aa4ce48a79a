// Batched Jacobi-preconditioned CG: one independent CG per orbital (Step 3 of
// Algorithms 3.1 / A.1, eq. alg-bvp, shifted to the SPD form A x = b), with a
// per-orbital convergence mask.  Two kernels per iteration:
//   cg_q      p <- D^-1 r + beta p   (computed on the fly, also at the 26
//             neighbours, so p never needs its own pass), q = A p, (p, q)
//   cg_update x += alpha p, r -= alpha q, z = D^-1 r, (r, z), (r, r)
// Each kernel reduces its dot products per orbital: block partials, then the
// last block to finish (atomic ticket) sums them in a fixed order and updates
// the per-orbital scalars, so results are deterministic and no extra launch or
// host round trip is needed.  p ping-pongs between two buffers because cg_q
// reads the old p at neighbours that another block may already be updating.
#include <cmath>

#include "common.cuh"

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
    double s = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(&partial[((long long)k * kMaxRedBlocks + b) * Np + o]);
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

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_cg_init(Grid g, int N, int Np, CGVectors<T> v, CGState s, bool x_zero,
                                                         double tol, int maxit) {
  __shared__ double sred[3 * kRedThreads * 4];
  double* tot = sred;  // reused once the block partials are written
  __shared__ int cnt;
  NodeMap nm = node_map(Np);
  int grp = threadIdx.x % nm.groups;
  int nl = threadIdx.x / nm.groups;
  bool live = nl < nm.npb;
  double acc[3][4] = {};
  if (live) {
    T arz[4] = {}, arr[4] = {}, abb[4] = {};
    for (int n = blockIdx.x * nm.npb + nl; n < g.nI; n += gridDim.x * nm.npb) {
      long long gp = interior_to_padded(g, n);
      V4<T> b = ld4v(v.b, gp, Np, grp);
      V4<T> r;
      if (x_zero) {
        r = b;
        st4(v.x + gp * Np + 4 * grp, V4<T>{0, 0, 0, 0});
      } else {
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
        for (int o = 0; o < 27; ++o) {
          const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
          long long nb = gp + ((long long)dz * g.Py + dy) * g.Px + dx;
          T w = v.coef[(long long)o * g.G + gp];
          V4<T> xv = ld4v(v.x, nb, Np, grp);
          a0 += w * xv.a;
          a1 += w * xv.b;
          a2 += w * xv.c;
          a3 += w * xv.d;
        }
        r = {b.a - a0, b.b - a1, b.c - a2, b.d - a3};
      }
      T di = v.dinv[gp];
      V4<T> z = {di * r.a, di * r.b, di * r.c, di * r.d};
      st4(v.r + gp * Np + 4 * grp, r);
      st4(v.p[0] + gp * Np + 4 * grp, z);
      arz[0] += r.a * z.a; arz[1] += r.b * z.b; arz[2] += r.c * z.c; arz[3] += r.d * z.d;
      arr[0] += r.a * r.a; arr[1] += r.b * r.b; arr[2] += r.c * r.c; arr[3] += r.d * r.d;
      abb[0] += b.a * b.a; abb[1] += b.b * b.b; abb[2] += b.c * b.c; abb[3] += b.d * b.d;
    }
    for (int c = 0; c < 4; ++c) {
      acc[0][c] = arz[c];
      acc[1][c] = arr[c];
      acc[2][c] = abb[c];
    }
  }
  if (!reduce_partials<3>(acc, Np, grp, nl, live, s.partial, s.ticket, sred, tot)) return;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int o = threadIdx.x; o < Np; o += blockDim.x) {
    double rz = tot[o], rr = tot[Np + o], bb = tot[2 * Np + o];
    s.rz[o] = rz;
    s.rr[o] = rr;
    s.bb[o] = bb;
    s.iters[o] = 0;
    s.alpha[o] = 0.0;
    s.beta[o] = 0.0;
    bool skip = (o >= N) || (s.skip != nullptr && s.skip[o] != 0);
    bool act = !skip && maxit > 0 && rr > tol * tol * bb;
    if (!skip && !(isfinite(rr) && isfinite(bb) && isfinite(rz))) {
      atomicOr(s.status, kStatNonFinite);
      act = false;
    } else if (act && !(rz > 0.0)) {  // (r, D^-1 r) <= 0 with r != 0: D, hence A, is not SPD
      atomicOr(s.status, kStatNotSPD);
      act = false;
    }
    s.active[o] = act ? 1 : 0;
    if (act) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *s.n_active = cnt;
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_cg_q(Grid g, int Np, CGVectors<T> v, CGState s, int parity) {
  __shared__ double sred[1 * kRedThreads * 4];
  double* tot = sred;
  NodeMap nm = node_map(Np);
  int grp = threadIdx.x % nm.groups;
  int nl = threadIdx.x / nm.groups;
  bool live = nl < nm.npb;
  double acc[1][4] = {};
  const T* pold = v.p[parity];
  T* pnew = v.p[parity ^ 1];
  if (live) {
    int act = s.active[4 * grp] | s.active[4 * grp + 1] | s.active[4 * grp + 2] | s.active[4 * grp + 3];
    if (act) {
      T be[4] = {(T)s.beta[4 * grp], (T)s.beta[4 * grp + 1], (T)s.beta[4 * grp + 2], (T)s.beta[4 * grp + 3]};
      T apq[4] = {};
      for (int n = blockIdx.x * nm.npb + nl; n < g.nI; n += gridDim.x * nm.npb) {
        long long gp = interior_to_padded(g, n);
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        V4<T> pc;
#pragma unroll
        for (int o = 0; o < 27; ++o) {
          const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
          long long nb = gp + ((long long)dz * g.Py + dy) * g.Px + dx;
          T w = v.coef[(long long)o * g.G + gp];
          T di = v.dinv[nb];
          V4<T> rv = ld4v(v.r, nb, Np, grp);
          V4<T> pv = ld4v(pold, nb, Np, grp);
          V4<T> pn = {di * rv.a + be[0] * pv.a, di * rv.b + be[1] * pv.b, di * rv.c + be[2] * pv.c,
                      di * rv.d + be[3] * pv.d};
          if (o == 13) pc = pn;
          a0 += w * pn.a;
          a1 += w * pn.b;
          a2 += w * pn.c;
          a3 += w * pn.d;
        }
        st4(pnew + gp * Np + 4 * grp, pc);
        st4(v.q + gp * Np + 4 * grp, V4<T>{a0, a1, a2, a3});
        apq[0] += pc.a * a0;
        apq[1] += pc.b * a1;
        apq[2] += pc.c * a2;
        apq[3] += pc.d * a3;
      }
      for (int c = 0; c < 4; ++c) acc[0][c] = apq[c];
    }
  }
  if (!reduce_partials<1>(acc, Np, grp, nl, live, s.partial, s.ticket, sred, tot)) return;
  if (threadIdx.x == 0 && s.work != nullptr) {
    unsigned long long w = 0;
    for (int q = 0; q < Np / 4; ++q)
      if (s.active[4 * q] | s.active[4 * q + 1] | s.active[4 * q + 2] | s.active[4 * q + 3]) w += 4ull * g.nI;
    *s.work += w;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < Np; o += blockDim.x) {
    double pq = tot[o];
    s.pq[o] = pq;
    double alpha = 0.0;
    if (s.active[o]) {
      if (!isfinite(pq)) {
        atomicOr(s.status, kStatNonFinite);
        s.active[o] = 0;
      } else if (!(pq > 0.0)) {
        atomicOr(s.status, kStatNotSPD);
        s.active[o] = 0;
      } else {
        alpha = s.rz[o] / pq;
      }
    }
    s.alpha[o] = alpha;
  }
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_cg_update(Grid g, int Np, CGVectors<T> v, CGState s, int parity,
                                                           double tol, int maxit) {
  __shared__ double sred[2 * kRedThreads * 4];
  double* tot = sred;
  __shared__ int cnt;
  NodeMap nm = node_map(Np);
  int grp = threadIdx.x % nm.groups;
  int nl = threadIdx.x / nm.groups;
  bool live = nl < nm.npb;
  double acc[2][4] = {};
  const T* p = v.p[parity ^ 1];
  if (live) {
    int act = s.active[4 * grp] | s.active[4 * grp + 1] | s.active[4 * grp + 2] | s.active[4 * grp + 3];
    if (act) {
      T al[4] = {(T)s.alpha[4 * grp], (T)s.alpha[4 * grp + 1], (T)s.alpha[4 * grp + 2], (T)s.alpha[4 * grp + 3]};
      T arz[4] = {}, arr[4] = {};
      for (int n = blockIdx.x * nm.npb + nl; n < g.nI; n += gridDim.x * nm.npb) {
        long long gp = interior_to_padded(g, n);
        V4<T> x = ld4v(v.x, gp, Np, grp), r = ld4v(v.r, gp, Np, grp);
        V4<T> pv = ld4v(p, gp, Np, grp), q = ld4v(v.q, gp, Np, grp);
        x = {x.a + al[0] * pv.a, x.b + al[1] * pv.b, x.c + al[2] * pv.c, x.d + al[3] * pv.d};
        r = {r.a - al[0] * q.a, r.b - al[1] * q.b, r.c - al[2] * q.c, r.d - al[3] * q.d};
        st4(v.x + gp * Np + 4 * grp, x);
        st4(v.r + gp * Np + 4 * grp, r);
        T di = v.dinv[gp];
        arz[0] += r.a * r.a * di; arz[1] += r.b * r.b * di; arz[2] += r.c * r.c * di; arz[3] += r.d * r.d * di;
        arr[0] += r.a * r.a; arr[1] += r.b * r.b; arr[2] += r.c * r.c; arr[3] += r.d * r.d;
      }
      for (int c = 0; c < 4; ++c) {
        acc[0][c] = arz[c];
        acc[1][c] = arr[c];
      }
    }
  }
  if (!reduce_partials<2>(acc, Np, grp, nl, live, s.partial, s.ticket, sred, tot)) return;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int o = threadIdx.x; o < Np; o += blockDim.x) {
    double beta = 0.0;
    if (s.active[o]) {
      double rz = tot[o], rr = tot[Np + o];
      int it = s.iters[o] + 1;
      s.iters[o] = it;
      s.rr[o] = rr;
      bool act = true;
      if (!(isfinite(rz) && isfinite(rr))) {
        atomicOr(s.status, kStatNonFinite);
        act = false;
      } else if (rr <= tol * tol * s.bb[o]) {
        act = false;
      } else if (!(rz > 0.0)) {
        atomicOr(s.status, kStatNotSPD);
        act = false;
      } else if (it >= maxit) {
        atomicOr(s.status, kStatNotConverged);
        act = false;
      }
      if (act) {
        beta = rz / s.rz[o];
        atomicAdd(&cnt, 1);
      }
      s.rz[o] = rz;
      s.active[o] = act ? 1 : 0;
    }
    s.beta[o] = beta;
  }
  __syncthreads();
  if (threadIdx.x == 0) *s.n_active = cnt;
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

template <typename T>
cudaError_t launch_cg_init(const Grid& g, int N, int Np, const CGVectors<T>& v, const CGState& s, bool x_zero,
                           double tol, int maxit, cudaStream_t st) {
  k_cg_init<T><<<red_blocks(g, Np), kRedThreads, 0, st>>>(g, N, Np, v, s, x_zero, tol, maxit);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_q(const Grid& g, int Np, const CGVectors<T>& v, const CGState& s, int parity, cudaStream_t st) {
  k_cg_q<T><<<red_blocks(g, Np), kRedThreads, 0, st>>>(g, Np, v, s, parity);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_update(const Grid& g, int Np, const CGVectors<T>& v, const CGState& s, int parity, double tol,
                             int maxit, cudaStream_t st) {
  k_cg_update<T><<<red_blocks(g, Np), kRedThreads, 0, st>>>(g, Np, v, s, parity, tol, maxit);
  return cudaGetLastError();
}

template cudaError_t launch_cg_init<float>(const Grid&, int, int, const CGVectors<float>&, const CGState&, bool,
                                           double, int, cudaStream_t);
template cudaError_t launch_cg_init<double>(const Grid&, int, int, const CGVectors<double>&, const CGState&, bool,
                                            double, int, cudaStream_t);
template cudaError_t launch_cg_q<float>(const Grid&, int, const CGVectors<float>&, const CGState&, int, cudaStream_t);
template cudaError_t launch_cg_q<double>(const Grid&, int, const CGVectors<double>&, const CGState&, int,
                                         cudaStream_t);
template cudaError_t launch_cg_update<float>(const Grid&, int, const CGVectors<float>&, const CGState&, int, double,
                                             int, cudaStream_t);
template cudaError_t launch_cg_update<double>(const Grid&, int, const CGVectors<double>&, const CGState&, int, double,
                                              int, cudaStream_t);

cudaError_t launch_refine_residual(const Grid& g, int N, int Np, const double* coef64, const double* x64,
                                   const double* b64, float* rhs32, const CGState& s, double tol, cudaStream_t st) {
  k_refine_residual<<<red_blocks(g, Np), kRedThreads, 0, st>>>(g, N, Np, coef64, x64, b64, rhs32, s, tol);
  return cudaGetLastError();
}

cudaError_t launch_refine_update(const Grid& g, int Np, double* x64, const float* d32, const int* skip,
                                 cudaStream_t st) {
  long long work = (long long)g.nI * Np;
  k_refine_update<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(g, Np, x64, d32, skip);
  return cudaGetLastError();
}

}  // namespace paro
