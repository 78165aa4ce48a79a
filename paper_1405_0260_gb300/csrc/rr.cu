// Rayleigh-Ritz on span(X) (Step 4 of Algorithms 3.1 / A.1, eq. alg-evp):
//   G_A = X^T H X, G_B = X^T M X                    (gram2: tall-skinny, float64)
//   G_B = L L^T, L^-1 G_A L^-T = Q Theta Q^T         (small_eig: one CTA, float64)
//   C = L^-T Q (columns sorted by ascending theta), U = X C   (rotate)
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "../../include/paro.h"

#include "common.cuh"
#include "ff.cuh"

namespace paro {

namespace {

constexpr int kTile = 32;      // Gram output tile (rows a, columns b)
constexpr int kGramRows = 32;  // nodes staged per step

// Partial Grams over a chunk of padded nodes.  Block (16 x 16) computes a 32 x 32
// tile of both G1 = X^T Y1 and G2 = X^T Y2, each thread 2 x 2 entries of each.
__global__ void __launch_bounds__(256) k_gram2(long long G, int Np, const double* __restrict__ X,
                                               const double* __restrict__ Y1, const double* __restrict__ Y2,
                                               double* __restrict__ part, int nch, long long chunk) {
  __shared__ double xs[kGramRows][kTile + 1];
  __shared__ double y1s[kGramRows][kTile + 1];
  __shared__ double y2s[kGramRows][kTile + 1];
  int ntile = (Np + kTile - 1) / kTile;
  int tile = blockIdx.x % (ntile * ntile);
  int ch = blockIdx.x / (ntile * ntile);
  int a0 = (tile / ntile) * kTile, b0 = (tile % ntile) * kTile;
  int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double g1[2][2] = {}, g2[2][2] = {};
  long long beg = ch * chunk, end = beg + chunk;
  if (end > G) end = G;
  for (long long n0 = beg; n0 < end; n0 += kGramRows) {
    for (int t = threadIdx.x; t < kGramRows * kTile; t += 256) {
      int r = t / kTile, c = t % kTile;
      long long n = n0 + r;
      bool ok = n < end;
      xs[r][c] = (ok && a0 + c < Np) ? X[n * Np + a0 + c] : 0.0;
      y1s[r][c] = (ok && b0 + c < Np) ? Y1[n * Np + b0 + c] : 0.0;
      y2s[r][c] = (ok && b0 + c < Np) ? Y2[n * Np + b0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kGramRows; ++r) {
      double xa0 = xs[r][2 * ty], xa1 = xs[r][2 * ty + 1];
      double yb0 = y1s[r][2 * tx], yb1 = y1s[r][2 * tx + 1];
      double zb0 = y2s[r][2 * tx], zb1 = y2s[r][2 * tx + 1];
      g1[0][0] += xa0 * yb0; g1[0][1] += xa0 * yb1; g1[1][0] += xa1 * yb0; g1[1][1] += xa1 * yb1;
      g2[0][0] += xa0 * zb0; g2[0][1] += xa0 * zb1; g2[1][0] += xa1 * zb0; g2[1][1] += xa1 * zb1;
    }
    __syncthreads();
  }
  long long NN = (long long)Np * Np;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      int a = a0 + 2 * ty + i, b = b0 + 2 * tx + j;
      if (a < Np && b < Np) {
        part[(2LL * ch) * NN + (long long)a * Np + b] = g1[i][j];
        part[(2LL * ch + 1) * NN + (long long)a * Np + b] = g2[i][j];
      }
    }
  (void)nch;
}

// One warp per Gram entry: lanes stride the chunks, then a butterfly of fixed
// shape (deterministic).
__global__ void k_gram_reduce(int Np, int nch, const double* __restrict__ part, double* __restrict__ G1,
                              double* __restrict__ G2) {
  const long long NN = (long long)Np * Np;
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (t >= 2 * NN) return;
  const int w = (int)(t / NN);
  const long long e = t % NN;
  double s = 0.0;
  for (int c = lane; c < nch; c += 32) s += part[(2LL * c + w) * NN + e];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) (w == 0 ? G1 : G2)[e] = s;
}

// Round-robin ("circle") pairing of m = even indices: round r, slot k.
__device__ __forceinline__ void rr_pair(int m, int r, int k, int* p, int* q) {
  int a = (k == 0) ? 0 : ((k - 1 + r) % (m - 1)) + 1;
  int b = ((m - 2 - k + r) % (m - 1)) + 1;
  *p = a < b ? a : b;
  *q = a < b ? b : a;
}

// One CTA: Cholesky of G_B, two triangular solves, parallel cyclic Jacobi on
// S = L^-1 G_A L^-T, sort, back-substitution C = L^-T Q.  All matrices N x N
// row-major (ld N), in dynamic shared memory when the launch provides 4 N^2
// doubles of it (smem != 0), else in `work`; inputs G_A, G_B and output C have
// ld Np, C zero-padded to Np x Np.
constexpr int kJacobiSweeps = 40;  // cyclic Jacobi sweep limit of the one-CTA eigensolve

__global__ void __launch_bounds__(1024) k_small_eig(int N, int Np, const double* __restrict__ GA,
                                                    const double* __restrict__ GB, double* __restrict__ work,
                                                    double* __restrict__ C, double* __restrict__ theta,
                                                    int* __restrict__ status, int smem,
                                                    const int* __restrict__ clus) {
  extern __shared__ double esm[];
  if (smem) work = esm;
  __shared__ int fail;
  __shared__ double red[1024 / 32][2];
  __shared__ double cs[kMaxN / 2 + 1][2];
  __shared__ int pr[kMaxN / 2 + 1][2];
  __shared__ double rdiag[kMaxN];
  const int tid = threadIdx.x, nt = blockDim.x;
  double* L = work;
  double* S = work + (long long)N * N;
  double* V = work + 2LL * N * N;
  double* W = work + 3LL * N * N;
  if (tid == 0) fail = 0;
  for (int t = tid; t < N * N; t += nt) {
    int i = t / N, j = t % N;
    L[t] = 0.5 * (GB[(long long)i * Np + j] + GB[(long long)j * Np + i]);
    S[t] = 0.5 * (GA[(long long)i * Np + j] + GA[(long long)j * Np + i]);
    V[t] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // Cholesky, right-looking, lower triangle of L.
  for (int k = 0; k < N; ++k) {
    if (tid == 0) {
      double d = L[k * N + k];
      if (!(d > 0.0) || !isfinite(d)) fail = 1;
      else L[k * N + k] = sqrt(d);
    }
    __syncthreads();
    if (fail) break;
    const double rk = 1.0 / L[k * N + k];
    for (int i = k + 1 + tid; i < N; i += nt) L[i * N + k] *= rk;
    __syncthreads();
    int m = N - k - 1;
    for (int t = tid; t < m * m; t += nt) {
      int i = k + 1 + t / m, j = k + 1 + t % m;
      if (j <= i) L[i * N + j] -= L[i * N + k] * L[j * N + k];
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) atomicOr(status, kStatNotSPD);
    return;
  }
  for (int t = tid; t < N * N; t += nt) {
    int i = t / N, j = t % N;
    if (j > i) L[t] = 0.0;
  }
  // reciprocals of the diagonal of L (float64 division is slow on this GPU)
  for (int i = tid; i < N; i += nt) rdiag[i] = 1.0 / L[i * N + i];
  __syncthreads();
  // W = L^-1 S  (column j by thread j)
  for (int j = tid; j < N; j += nt)
    for (int i = 0; i < N; ++i) {
      double s = S[i * N + j];
      for (int k = 0; k < i; ++k) s -= L[i * N + k] * W[k * N + j];
      W[i * N + j] = s * rdiag[i];
    }
  __syncthreads();
  // S = L^-1 W^T = L^-1 S L^-T
  for (int j = tid; j < N; j += nt)
    for (int i = 0; i < N; ++i) {
      double s = W[j * N + i];
      for (int k = 0; k < i; ++k) s -= L[i * N + k] * S[k * N + j];
      S[i * N + j] = s * rdiag[i];
    }
  __syncthreads();
  for (int t = tid; t < N * N; t += nt) {
    int i = t / N, j = t % N;
    if (j > i) {
      double a = 0.5 * (S[i * N + j] + S[j * N + i]);
      if (clus != nullptr && clus[i] != clus[j]) a = 0.0;  // cluster-separated: diagonal blocks only
      S[i * N + j] = a;
      S[j * N + i] = a;
    }
  }
  __syncthreads();
  // Parallel cyclic Jacobi.
  const int m = (N % 2 == 0) ? N : N + 1;
  const int half = m / 2;
  bool converged = N <= 1;
  for (int sweep = 0; sweep < kJacobiSweeps && N > 1; ++sweep) {
    double off = 0.0, all = 0.0;
    for (int t = tid; t < N * N; t += nt) {
      double v = S[t];
      all += v * v;
      if (t / N != t % N) off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    if (tid % 32 == 0) {
      red[tid / 32][0] = off;
      red[tid / 32][1] = all;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < nt / 32; ++w) {
        a += red[w][0];
        b += red[w][1];
      }
      red[0][0] = a;
      red[0][1] = b;
    }
    __syncthreads();
    off = red[0][0];
    all = red[0][1];
    __syncthreads();
    // stop at the float64 rounding floor of the rotations: off-norm <= ~3e-15 N norm(S)
    if (!(off > 1e-29 * (double)N * N * all)) {
      converged = true;
      break;
    }
    // entries below 1e-16 of norm(S) are left alone: rotating them changes nothing
    // at float64 precision, and skipping them removes most of the float64 work of
    // the later sweeps (inside the ParO loop the matrix starts nearly diagonal)
    const double skip2 = 1e-32 * all;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = tid; k < half; k += nt) {
        int p, q;
        rr_pair(m, r, k, &p, &q);
        double c = 1.0, s = 0.0;
        if (q < N) {
          // The rotation angle in float32 (float64 division and square root are
          // long sequences on this GPU's float64 pipe), then (c, s) renormalised to
          // c^2 + s^2 = 1 in float64 by two Newton steps for 1/sqrt(c^2 + s^2):
          // the rotation is orthogonal to float64 precision and annihilates
          // a_pq up to a float32-relative residue, which later sweeps remove.
          const double apq = S[p * N + q];
          const float fa = (float)apq;
          if (fa != 0.0f && apq * apq > skip2) {
            const float tau = (float)(S[q * N + q] - S[p * N + p]) / (2.0f * fa);
            const float rt = sqrtf(1.0f + tau * tau);
            const float t = (tau >= 0.0f) ? 1.0f / (tau + rt) : -1.0f / (-tau + rt);
            const float cf = rsqrtf(1.0f + t * t);
            const double cd = cf, sd = (double)(t * cf);
            const double nn = cd * cd + sd * sd;
            double y = 1.5 - 0.5 * nn;
            y = y * (1.5 - 0.5 * nn * y * y);
            c = cd * y;
            s = sd * y;
          }
        }
        cs[k][0] = c;
        cs[k][1] = s;
        pr[k][0] = p;
        pr[k][1] = q;
      }
      __syncthreads();
      // rows p, q of S <- J^T S (cluster-separated: S and V stay block diagonal, so
      // only pairs within a cluster rotate, and only that cluster's entries:
      // O(sum q_k^3) work a sweep instead of O(N^3))
      for (int t = tid; t < half * N; t += nt) {
        int k = t / N, col = t % N;
        int p = pr[k][0], q = pr[k][1];
        if (q >= N || cs[k][1] == 0.0) continue;
        if (clus != nullptr && (clus[p] != clus[q] || clus[col] != clus[p])) continue;
        double c = cs[k][0], s = cs[k][1];
        double sp = S[p * N + col], sq = S[q * N + col];
        S[p * N + col] = c * sp - s * sq;
        S[q * N + col] = s * sp + c * sq;
      }
      __syncthreads();
      // columns p, q of S <- S J ; V <- V J
      for (int t = tid; t < half * N; t += nt) {
        int k = t / N, row = t % N;
        int p = pr[k][0], q = pr[k][1];
        if (q >= N || cs[k][1] == 0.0) continue;
        if (clus != nullptr && (clus[p] != clus[q] || clus[row] != clus[p])) continue;
        double c = cs[k][0], s = cs[k][1];
        double sp = S[row * N + p], sq = S[row * N + q];
        S[row * N + p] = c * sp - s * sq;
        S[row * N + q] = s * sp + c * sq;
        double vp = V[row * N + p], vq = V[row * N + q];
        V[row * N + p] = c * vp - s * vq;
        V[row * N + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // the sweep limit ran out with off-diagonal mass above the rounding floor
  if (!converged && tid == 0) atomicOr(status, kStatNotConverged);
  // Sort by ascending Ritz value (ties by index) and back-substitute C = L^-T V.
  for (int j = tid; j < N; j += nt) {
    double tj = S[j * N + j];
    int rank = 0;
    for (int i = 0; i < N; ++i) {
      double ti = S[i * N + i];
      if (clus != nullptr && clus[i] != clus[j]) {
        if (clus[i] < clus[j]) ++rank;  // every orbital of an earlier cluster comes first
      } else if (ti < tj || (ti == tj && i < j)) {
        ++rank;
      }
    }
    theta[rank] = tj;
    for (int i = N - 1; i >= 0; --i) {
      double s = V[i * N + j];
      for (int k = i + 1; k < N; ++k) s -= L[k * N + i] * C[(long long)k * Np + rank];
      C[(long long)i * Np + rank] = s * rdiag[i];
    }
  }
  for (int t = tid; t < Np * Np; t += nt) {
    int i = t / Np, j = t % Np;
    if (i >= N || j >= N) C[t] = 0.0;
  }
}

// U[g, b] = sum_a X[g, a] C[a, b], interior nodes, 4 columns per thread.
__global__ void __launch_bounds__(kRedThreads) k_rotate(Grid g, int N, int Np, const double* __restrict__ X,
                                                        const double* __restrict__ C, double* __restrict__ U) {
  NodeMap nm = node_map(Np);
  int grp = threadIdx.x % nm.groups;
  int nl = threadIdx.x / nm.groups;
  if (nl >= nm.npb) return;
  for (int n = blockIdx.x * nm.npb + nl; n < g.nI; n += gridDim.x * nm.npb) {
    long long gp = interior_to_padded(g, n);
    const double* xr = X + gp * Np;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int a = 0; a < N; ++a) {
      double xa = xr[a];
      V4<double> c = ld4(C + (long long)a * Np + 4 * grp);
      a0 += xa * c.a;
      a1 += xa * c.b;
      a2 += xa * c.c;
      a3 += xa * c.d;
    }
    st4(U + gp * Np + 4 * grp, V4<double>{a0, a1, a2, a3});
  }
}

}  // namespace

static void gram_shape(const Grid& g, int Np, int* nch, long long* chunk) {
  int ntile = (Np + kTile - 1) / kTile;
  long long want = (1216 + ntile * ntile - 1) / (ntile * ntile);
  long long maxch = (g.G + kGramRows - 1) / kGramRows;
  if (want > maxch) want = maxch;
  if (want < 1) want = 1;
  long long ch = (g.G + want - 1) / want;
  ch = (ch + kGramRows - 1) / kGramRows * kGramRows;
  *chunk = ch;
  *nch = (int)((g.G + ch - 1) / ch);
}

size_t gram_partial_doubles(const Grid& g, int Np) {
  int nch;
  long long chunk;
  gram_shape(g, Np, &nch, &chunk);
  return (size_t)nch * 2 * Np * Np;
}

cudaError_t launch_gram2(const Grid& g, int N, int Np, const double* X, const double* Y1, const double* Y2,
                         double* part, int* n_chunks, double* G1, double* G2, cudaStream_t st) {
  (void)N;
  int nch;
  long long chunk;
  gram_shape(g, Np, &nch, &chunk);
  int ntile = (Np + kTile - 1) / kTile;
  k_gram2<<<ntile * ntile * nch, 256, 0, st>>>(g.G, Np, X, Y1, Y2, part, nch, chunk);
  long long work = 2LL * Np * Np * 32;
  k_gram_reduce<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(Np, nch, part, G1, G2);
  if (n_chunks) *n_chunks = nch;
  return cudaGetLastError();
}

cudaError_t launch_gram_reduce(int Np, int nch, const double* part, double* G1, double* G2, cudaStream_t st) {
  long long work = 2LL * Np * Np * 32;
  k_gram_reduce<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(Np, nch, part, G1, G2);
  return cudaGetLastError();
}

// One Gram from per-chunk partials part[nch][Np][Np]: one warp per entry.
__global__ void k_gram_reduce1(int Np, int nch, const double* __restrict__ part, double* __restrict__ Gm) {
  const long long NN = (long long)Np * Np;
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (t >= NN) return;
  double s = 0.0;
  for (int c = lane; c < nch; c += 32) s += part[(long long)c * NN + t];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) Gm[t] = s;
}

cudaError_t launch_gram_reduce1(int Np, int nch, const double* part, double* Gm, cudaStream_t st) {
  long long work = (long long)Np * Np * 32;
  k_gram_reduce1<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(Np, nch, part, Gm);
  return cudaGetLastError();
}

namespace {

// Grid-wide barrier of the multi-CTA eigensolve: CTAs add 1 to a counter the
// host zeroes before the launch; barrier k completes at k * gridDim.x.  Bounded:
// false after kEigSpinLimit polls.
constexpr unsigned kEigSpinLimit = 1u << 24;
// cluster-separated eigensolves: clusters up to this size are diagonalised one per CTA
constexpr int kEigClusterCtaMaxQ = 128;
__device__ bool eig_barrier(unsigned* count, unsigned target) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    int ok = 0;
    for (unsigned i = 0; i < kEigSpinLimit; ++i) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if (v >= target) {
        ok = 1;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The small generalized eigensolve of k_small_eig for larger N on the whole GPU
// (cooperative launch): the same steps and the same cyclic Jacobi ordering, but
// every Jacobi round's rotations are spread over all CTAs with three grid
// barriers a round (angles, rows, columns).  Cholesky in CTA 0; the triangular
// solves and the back-substitution one warp per column.  work: L, S, V, W
// (N x N each, ld N); C (Np x Np) doubles as scratch until its final write:
// [0, 2 half) rotation (c, s), [2 half, 2 half + 2 grid) the sweep's partial
// norms, then a failure flag.
__global__ void __launch_bounds__(256) k_small_eig_grid(int N, int Np, const double* __restrict__ GA,
                                                        const double* __restrict__ GB, double* __restrict__ work,
                                                        double* __restrict__ C, double* __restrict__ theta,
                                                        int* __restrict__ status, unsigned* __restrict__ bar,
                                                        const int* __restrict__ clus) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long gt = (long long)blockIdx.x * nt + tid, gs = (long long)gridDim.x * nt;
  const int lane = tid % 32;
  const int gw = (int)(gt / 32), nw = (int)(gs / 32);
  const long long NN = (long long)N * N;
  double* L = work;
  double* S = work + NN;
  double* V = work + 2 * NN;
  double* W = work + 3 * NN;
  const int m = (N % 2 == 0) ? N : N + 1;
  const int half = m / 2;
  double* cs = C;                   // [half][2]
  double* part = C + 2 * half;      // [grid][2]
  double* flag = part + 2 * gridDim.x;
  double* rdiag = W;                // after the triangular solves: W holds 1 / L[i][i] in its first row
  __shared__ double red[256 / 32][2];
  __shared__ int s_fail;
  unsigned bno = 0;
  auto sync = [&]() -> bool {
    if (!eig_barrier(bar, ++bno * gridDim.x)) {
      if (tid == 0) atomicOr(status, kStatTimeout);
      return false;
    }
    return true;
  };
  // copy and symmetrise
  for (long long t = gt; t < NN; t += gs) {
    const int i = (int)(t / N), j = (int)(t % N);
    L[t] = 0.5 * (GB[(long long)i * Np + j] + GB[(long long)j * Np + i]);
    S[t] = 0.5 * (GA[(long long)i * Np + j] + GA[(long long)j * Np + i]);
    V[t] = (i == j) ? 1.0 : 0.0;
  }
  if (gt == 0) flag[0] = 0.0;
  if (!sync()) return;
  // Cholesky (right-looking, lower triangle) in CTA 0
  if (blockIdx.x == 0) {
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int k = 0; k < N; ++k) {
      if (tid == 0) {
        const double d = L[(long long)k * N + k];
        if (!(d > 0.0) || !isfinite(d)) s_fail = 1;
        else L[(long long)k * N + k] = sqrt(d);
      }
      __syncthreads();
      if (s_fail) break;
      const double rk = 1.0 / L[(long long)k * N + k];
      for (int i = k + 1 + tid; i < N; i += nt) L[(long long)i * N + k] *= rk;
      __syncthreads();
      const int r = N - k - 1;
      for (long long t = tid; t < (long long)r * r; t += nt) {
        const int i = k + 1 + (int)(t / r), j = k + 1 + (int)(t % r);
        if (j <= i) L[(long long)i * N + j] -= L[(long long)i * N + k] * L[(long long)j * N + k];
      }
      __syncthreads();
    }
    if (s_fail && tid == 0) {
      flag[0] = 1.0;
      atomicOr(status, kStatNotSPD);
    }
  }
  if (!sync()) return;
  if (flag[0] != 0.0) return;
  for (long long t = gt; t < NN; t += gs) {
    const int i = (int)(t / N), j = (int)(t % N);
    if (j > i) L[t] = 0.0;
  }
  if (!sync()) return;
  // W = L^-1 S, then S = L^-1 W^T: one warp per column, the lanes split each row's dot product
  for (int pass = 0; pass < 2; ++pass) {
    const double* Rin = pass == 0 ? S : W;
    double* Rout = pass == 0 ? W : S;
    for (int j = gw; j < N; j += nw) {
      for (int i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int k = lane; k < i; k += 32) acc += L[(long long)i * N + k] * Rout[(long long)k * N + j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
          const double b = pass == 0 ? Rin[(long long)i * N + j] : Rin[(long long)j * N + i];
          Rout[(long long)i * N + j] = (b - acc) / L[(long long)i * N + i];
        }
        __syncwarp();
      }
    }
    if (!sync()) return;
  }
  // symmetrise S, keep 1 / L[i][i] in W's first row (W is free now)
  for (long long t = gt; t < NN; t += gs) {
    const int i = (int)(t / N), j = (int)(t % N);
    if (j > i) {
      double a = 0.5 * (S[t] + S[(long long)j * N + i]);
      if (clus != nullptr && clus[i] != clus[j]) a = 0.0;  // cluster-separated: diagonal blocks only
      S[t] = a;
      S[(long long)j * N + i] = a;
    }
  }
  for (long long i = gt; i < N; i += gs) rdiag[i] = 1.0 / L[i * N + i];
  if (!sync()) return;
  // parallel cyclic Jacobi
  // clusters are consecutive index ranges with ids 0, 1, ... in order; the largest
  // decides the form of the Jacobi phase (every CTA computes the same)
  int qmax = 0;
  if (clus != nullptr)
    for (int i = 0, run = 0; i < N; ++i) {
      run = (i > 0 && clus[i] == clus[i - 1]) ? run + 1 : 1;
      qmax = run > qmax ? run : qmax;
    }
  if (clus != nullptr && qmax <= kEigClusterCtaMaxQ) {
    // Cluster-separated (Section 3): S is block diagonal, so every cluster is its own
    // eigenproblem.  CTA b diagonalises clusters b, b + grid, ... alone, with CTA
    // barriers only: O(sum q_k^3) work and q_k - 1 rounds a sweep instead of N - 1
    // rounds of three grid barriers.
    __shared__ double s_cs[kEigClusterCtaMaxQ];  // (c, s) of the round's q_k / 2 pairs
    __shared__ double s_red[256 / 32][2];
    const int ncl = clus[N - 1] + 1;
    for (int kc = blockIdx.x; kc < ncl; kc += gridDim.x) {
      int c0 = 0;
      while (c0 < N && clus[c0] != kc) ++c0;
      int c1 = c0;
      while (c1 < N && clus[c1] == kc) ++c1;
      const int q = c1 - c0;
      if (q < 2) continue;
      const int mq = (q % 2 == 0) ? q : q + 1, hq = mq / 2;
      for (int sweep = 0; sweep < 40; ++sweep) {
        double off = 0.0, all = 0.0;
        for (int t = tid; t < q * q; t += nt) {
          const int i = c0 + t / q, j = c0 + t % q;
          const double v = S[(long long)i * N + j];
          all += v * v;
          if (i != j) off += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
          off += __shfl_xor_sync(0xffffffffu, off, o);
          all += __shfl_xor_sync(0xffffffffu, all, o);
        }
        if (lane == 0) {
          s_red[tid / 32][0] = off;
          s_red[tid / 32][1] = all;
        }
        __syncthreads();
        off = 0.0;
        all = 0.0;
        for (int w = 0; w < nt / 32; ++w) {
          off += s_red[w][0];
          all += s_red[w][1];
        }
        __syncthreads();
        if (!(off > 1e-29 * (double)q * q * all)) break;
        for (int r = 0; r < mq - 1; ++r) {
          for (int k = tid; k < hq; k += nt) {
            int p, pq;
            rr_pair(mq, r, k, &p, &pq);
            double c = 1.0, sn = 0.0;
            if (pq < q) {
              // angle in float32, (c, s) renormalised in float64 (as k_small_eig)
              const float fa = (float)S[(long long)(c0 + p) * N + c0 + pq];
              if (fa != 0.0f) {
                const float tau =
                    (float)(S[(long long)(c0 + pq) * N + c0 + pq] - S[(long long)(c0 + p) * N + c0 + p]) / (2.0f * fa);
                const float rt = sqrtf(1.0f + tau * tau);
                const float tt = (tau >= 0.0f) ? 1.0f / (tau + rt) : -1.0f / (-tau + rt);
                const float cf = rsqrtf(1.0f + tt * tt);
                const double cd = cf, sd = (double)(tt * cf);
                const double nn = cd * cd + sd * sd;
                double y = 1.5 - 0.5 * nn;
                y = y * (1.5 - 0.5 * nn * y * y);
                c = cd * y;
                sn = sd * y;
              }
            }
            s_cs[2 * k] = c;
            s_cs[2 * k + 1] = sn;
          }
          __syncthreads();
          // rows p, q of the block <- J^T S
          for (int t = tid; t < hq * q; t += nt) {
            const int k = t / q, col = c0 + t % q;
            int p, pq;
            rr_pair(mq, r, k, &p, &pq);
            if (pq >= q) continue;
            const double c = s_cs[2 * k], sn = s_cs[2 * k + 1];
            const long long ep = (long long)(c0 + p) * N + col, eq = (long long)(c0 + pq) * N + col;
            const double sp = S[ep], sq = S[eq];
            S[ep] = c * sp - sn * sq;
            S[eq] = sn * sp + c * sq;
          }
          __syncthreads();
          // columns p, q of the block <- S J; V <- V J (V is block diagonal too)
          for (int t = tid; t < hq * q; t += nt) {
            const int k = t / q, row = c0 + t % q;
            int p, pq;
            rr_pair(mq, r, k, &p, &pq);
            if (pq >= q) continue;
            const double c = s_cs[2 * k], sn = s_cs[2 * k + 1];
            const long long ep = (long long)row * N + c0 + p, eq = (long long)row * N + c0 + pq;
            const double sp = S[ep], sq = S[eq];
            S[ep] = c * sp - sn * sq;
            S[eq] = sn * sp + c * sq;
            const double vp = V[ep], vq = V[eq];
            V[ep] = c * vp - sn * vq;
            V[eq] = sn * vp + c * vq;
          }
          __syncthreads();
        }
      }
    }
  } else {
    for (int sweep = 0; sweep < 40 && N > 1; ++sweep) {
      double off = 0.0, all = 0.0;
      for (long long t = gt; t < NN; t += gs) {
        const double v = S[t];
        all += v * v;
        if (t / N != t % N) off += v * v;
      }
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        all += __shfl_xor_sync(0xffffffffu, all, o);
      }
      if (lane == 0) {
        red[tid / 32][0] = off;
        red[tid / 32][1] = all;
      }
      __syncthreads();
      if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < nt / 32; ++w) {
          a += red[w][0];
          b += red[w][1];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
      }
      if (!sync()) return;
      // every CTA sums the partials in the same order: the same decision everywhere
      off = 0.0;
      all = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) {
        off += part[2 * b];
        all += part[2 * b + 1];
      }
      if (!(off > 1e-29 * (double)N * N * all)) break;
      for (int r = 0; r < m - 1; ++r) {
        for (long long k = gt; k < half; k += gs) {
          int p, q;
          rr_pair(m, r, (int)k, &p, &q);
          double c = 1.0, s = 0.0;
          if (q < N) {
            // angle in float32, (c, s) renormalised in float64 (as k_small_eig)
            const float fa = (float)S[(long long)p * N + q];
            if (fa != 0.0f) {
              const float tau = (float)(S[(long long)q * N + q] - S[(long long)p * N + p]) / (2.0f * fa);
              const float rt = sqrtf(1.0f + tau * tau);
              const float t = (tau >= 0.0f) ? 1.0f / (tau + rt) : -1.0f / (-tau + rt);
              const float cf = rsqrtf(1.0f + t * t);
              const double cd = cf, sd = (double)(t * cf);
              const double nn = cd * cd + sd * sd;
              double y = 1.5 - 0.5 * nn;
              y = y * (1.5 - 0.5 * nn * y * y);
              c = cd * y;
              s = sd * y;
            }
          }
          cs[2 * k] = c;
          cs[2 * k + 1] = s;
        }
        if (!sync()) return;
        // rows p, q of S <- J^T S (cluster-separated: within-cluster entries only, as k_small_eig)
        for (long long t = gt; t < (long long)half * N; t += gs) {
          const int k = (int)(t / N), col = (int)(t % N);
          int p, q;
          rr_pair(m, r, k, &p, &q);
          if (q >= N) continue;
          if (clus != nullptr && (clus[p] != clus[q] || clus[col] != clus[p])) continue;
          const double c = cs[2 * k], s = cs[2 * k + 1];
          const double sp = S[(long long)p * N + col], sq = S[(long long)q * N + col];
          S[(long long)p * N + col] = c * sp - s * sq;
          S[(long long)q * N + col] = s * sp + c * sq;
        }
        if (!sync()) return;
        // columns p, q of S <- S J; V <- V J
        for (long long t = gt; t < (long long)half * N; t += gs) {
          const int k = (int)(t / N), row = (int)(t % N);
          int p, q;
          rr_pair(m, r, k, &p, &q);
          if (q >= N) continue;
          if (clus != nullptr && (clus[p] != clus[q] || clus[row] != clus[p])) continue;
          const double c = cs[2 * k], s = cs[2 * k + 1];
          const double sp = S[(long long)row * N + p], sq = S[(long long)row * N + q];
          S[(long long)row * N + p] = c * sp - s * sq;
          S[(long long)row * N + q] = s * sp + c * sq;
          const double vp = V[(long long)row * N + p], vq = V[(long long)row * N + q];
          V[(long long)row * N + p] = c * vp - s * vq;
          V[(long long)row * N + q] = s * vp + c * vq;
        }
        if (!sync()) return;
      }
    }
  }
  // every CTA has read the sweep's partial norms (C's scratch) before C is written
  if (!sync()) return;
  // sort by ascending Ritz value (ties by index); back-substitution C = L^-T V, one
  // warp per column
  for (int j = gw; j < N; j += nw) {
    const double tj = S[(long long)j * N + j];
    int rank = 0;
    for (int i = lane; i < N; i += 32) {
      const double ti = S[(long long)i * N + i];
      if (clus != nullptr && clus[i] != clus[j]) {
        if (clus[i] < clus[j]) ++rank;  // every orbital of an earlier cluster comes first
      } else if (ti < tj || (ti == tj && i < j)) {
        ++rank;
      }
    }
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    if (lane == 0) theta[rank] = tj;
    for (int i = N - 1; i >= 0; --i) {
      double acc = 0.0;
      for (int k = i + 1 + lane; k < N; k += 32) acc += L[(long long)k * N + i] * C[(long long)k * Np + rank];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) C[(long long)i * Np + rank] = (V[(long long)i * N + j] - acc) * rdiag[i];
      __syncwarp();
    }
  }
  for (long long t = gt; t < (long long)Np * Np; t += gs) {
    const int i = (int)(t / Np), j = (int)(t % Np);
    if (i >= N || j >= N) C[t] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// The small generalized eigensolve of Step 4 in float-float arithmetic (mixed
// precision handles, N <= kEigFFMaxN, no clusters).  On this GPU a float64
// instruction costs ~60x a float32 one, and the one-CTA float64 solve above
// spent ~220 us at N = 20 (Cholesky 21, two triangular solves 20, 44 a Jacobi
// sweep) on a handful of float64 operations a thread between CTA barriers.  Here
// every step runs on hi + lo float pairs (~48 bits, ff.cuh):
//   G_B = Lt D Lt^T           LDL^T elimination, one barrier a column (Lt unit lower)
//   T = Lt^-1 G_A Lt^-T       two unit-triangular solves, one barrier a column
//   S = D^-1/2 T D^-1/2       (= L^-1 G_A L^-T with L = Lt D^1/2)
//   S = Q Theta Q^T           parallel cyclic Jacobi: the pairs of a round are
//                             disjoint, so each thread updates whole 2 x 2 blocks
//                             R_k S_kk' R_k'^T: two barriers a round
//   C = Lt^-T D^-1/2 Q        one barrier a row, columns sorted by ascending theta
// Rotation angles are taken in float32 and (c, s) renormalised so that
// c^2 + s^2 = 1 to float-float precision: every rotation is orthogonal to ~2^-48
// and annihilates its pair to a float32-relative residue that the next sweep
// removes.  A pair rotates while |S_pq| > 2^-44 max(|S_pp|, |S_qq|) + 2^-47 ||S||_F:
// the rotations' own rounding leaves ~2^-48 of the entries they combine, so a
// threshold at that level (tried first) never let a sweep end without rotations.
constexpr int kEigFFMaxN = 64;
constexpr int kJacobiSweepsFF = 40;

__device__ __forceinline__ FF ffe_fast(float a, float b) {
  const float s = __fadd_rn(a, b);
  return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ffe_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ffe_fast(p, e);
}
__device__ __forceinline__ FF ffe_add(FF a, FF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ffe_fast(s, e);
}
__device__ __forceinline__ FF ffe_sub(FF a, FF b) { return ffe_add(a, FF{-b.hi, -b.lo}); }
// 1/d and 1/sqrt(d) by two Newton steps from the float32 estimate
__device__ __forceinline__ FF ffe_recip(FF d) {
  FF x{__frcp_rn(d.hi), 0.f};
  for (int it = 0; it < 2; ++it) x = ffe_add(x, ffe_mul(x, ffe_sub(FF{1.f, 0.f}, ffe_mul(d, x))));
  return x;
}
__device__ __forceinline__ FF ffe_rsqrt(FF d) {
  FF y{rsqrtf(d.hi), 0.f};
  for (int it = 0; it < 2; ++it) {
    const FF r = ffe_sub(FF{1.f, 0.f}, ffe_mul(d, ffe_mul(y, y)));
    y = ffe_add(y, ffe_mul(y, FF{0.5f * r.hi, 0.5f * r.lo}));
  }
  return y;
}

__global__ void __launch_bounds__(512) k_small_eig_ff(int N, int Np, const double* __restrict__ GA,
                                                      const double* __restrict__ GB, double* __restrict__ C,
                                                      double* __restrict__ theta, int* __restrict__ status) {
  extern __shared__ float fsm[];
  const int LD = N | 1;  // odd row pitch: column walks hit distinct banks
  const int NN = N * LD;
  float* Bh = fsm;  // G_B, then Lt (strict lower) and D (diagonal)
  float* Bl = Bh + NN;
  float* Sh = Bl + NN;  // G_A, then W, then S
  float* Sl = Sh + NN;
  float* Vh = Sl + NN;  // the second solve's right-hand side, then Q, then X
  float* Vl = Vh + NN;
  float* yv = Vl + NN;  // [2N] D^-1/2 (hi, lo)
  float* csv = yv + 2 * N;  // [4 * half] rotation of each pair of a round
  __shared__ int pr[kEigFFMaxN / 2][2];
  __shared__ int s_fail, s_big, s_nan;
  __shared__ unsigned s_norm;
  const int tid = threadIdx.x, nt = blockDim.x;
  auto ld = [&](const float* h, const float* l, int i, int j) { return FF{h[i * LD + j], l[i * LD + j]}; };
  auto st = [&](float* h, float* l, int i, int j, FF v) {
    h[i * LD + j] = v.hi;
    l[i * LD + j] = v.lo;
  };
  if (tid == 0) {
    s_fail = 0;
    s_big = 0;
    s_nan = 0;
    s_norm = 0u;
  }
  for (int t = tid; t < N * N; t += nt) {
    const int i = t / N, j = t % N;
    st(Bh, Bl, i, j, ff_split(0.5 * (GB[(long long)i * Np + j] + GB[(long long)j * Np + i])));
    st(Sh, Sl, i, j, ff_split(0.5 * (GA[(long long)i * Np + j] + GA[(long long)j * Np + i])));
  }
  __syncthreads();
  // LDL^T: step k removes column k from the trailing lower triangle
  for (int k = 0; k < N - 1; ++k) {
    const FF rd = ffe_recip(ld(Bh, Bl, k, k));
    const int m = N - 1 - k;
    for (int t = tid; t < m * m; t += nt) {
      const int i = k + 1 + t / m, j = k + 1 + t % m;
      if (j > i) continue;
      const FF bik = ld(Bh, Bl, i, k), bjk = ld(Bh, Bl, j, k);
      st(Bh, Bl, i, j, ffe_sub(ld(Bh, Bl, i, j), ffe_mul(bik, ffe_mul(bjk, rd))));
    }
    __syncthreads();
  }
  // D > 0 (G_B positive definite), Lt = B / d_k below the diagonal, D^-1/2
  for (int k = tid; k < N; k += nt) {
    const FF d = ld(Bh, Bl, k, k);
    if (!(d.hi > 0.f) || !isfinite(d.hi)) atomicOr(&s_fail, 1);
    const FF y = ffe_rsqrt(d);
    yv[2 * k] = y.hi;
    yv[2 * k + 1] = y.lo;
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) atomicOr(status, kStatNotSPD);
    return;
  }
  for (int t = tid; t < N * N; t += nt) {
    const int i = t / N, k = t % N;
    if (k < i) {
      const FF y = FF{yv[2 * k], yv[2 * k + 1]};
      st(Bh, Bl, i, k, ffe_mul(ld(Bh, Bl, i, k), ffe_mul(y, y)));
    }
  }
  __syncthreads();
  // W = Lt^-1 G_A (in S), then V = W^T, V = Lt^-1 V
  for (int pass = 0; pass < 2; ++pass) {
    float* Xh = pass == 0 ? Sh : Vh;
    float* Xl = pass == 0 ? Sl : Vl;
    if (pass == 1) {
      for (int t = tid; t < N * N; t += nt) {
        const int i = t / N, j = t % N;
        st(Vh, Vl, i, j, ld(Sh, Sl, j, i));
      }
      __syncthreads();
    }
    for (int k = 0; k < N - 1; ++k) {
      const int m = N - 1 - k;
      for (int t = tid; t < m * N; t += nt) {
        const int i = k + 1 + t / N, j = t % N;
        st(Xh, Xl, i, j, ffe_sub(ld(Xh, Xl, i, j), ffe_mul(ld(Bh, Bl, i, k), ld(Xh, Xl, k, j))));
      }
      __syncthreads();
    }
  }
  // S = D^-1/2 T D^-1/2, symmetrised; V = I; ||S||_F^2 (rotation-invariant)
  float nrm = 0.f;
  for (int t = tid; t < N * N; t += nt) {
    const int i = t / N, j = t % N;
    const FF yi{yv[2 * i], yv[2 * i + 1]}, yj{yv[2 * j], yv[2 * j + 1]};
    const FF a = ld(Vh, Vl, i, j), b = ld(Vh, Vl, j, i);
    const FF s = ffe_mul(ffe_mul(ffe_add(a, b), FF{0.5f, 0.f}), ffe_mul(yi, yj));
    st(Sh, Sl, i, j, s);
    nrm = fmaf(s.hi, s.hi, nrm);
  }
  __syncthreads();
  for (int t = tid; t < N * N; t += nt) {
    const int i = t / N, j = t % N;
    st(Vh, Vl, i, j, FF{i == j ? 1.f : 0.f, 0.f});
  }
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if ((tid & 31) == 0) atomicAdd(reinterpret_cast<float*>(&s_norm), nrm);
  __syncthreads();
  const float tg = 0x1p-47f * sqrtf(__uint_as_float(s_norm));
  auto thr = [&](int p, int q) { return fmaf(0x1p-44f, fmaxf(fabsf(Sh[p * LD + p]), fabsf(Sh[q * LD + q])), tg); };
  const int m = (N % 2 == 0) ? N : N + 1;
  const int half = m / 2;
  bool converged = N <= 1;
  for (int sweep = 0; sweep < kJacobiSweepsFF && N > 1; ++sweep) {
    // another sweep while some pair is above its threshold (or a value is NaN)
    for (int t = tid; t < N * N; t += nt) {
      const int p = t / N, q = t % N;
      const float a = Sh[p * LD + q];
      if (isnan(a)) s_nan = 1;
      else if (p != q && fabsf(a) > thr(p, q)) s_big = 1;
    }
    __syncthreads();
    if (s_nan || !s_big) {
      converged = !s_nan;
      break;
    }
    for (int r = 0; r < m - 1; ++r) {
      // the rotation of each pair (identity for a pair with the padding index, or
      // whose |a_pq| is at the rounding level)
      for (int k = tid; k < half; k += nt) {
        int p, q;
        rr_pair(m, r, k, &p, &q);
        FF c{1.f, 0.f}, s{0.f, 0.f};
        if (q < N) {
          const FF apq = ld(Sh, Sl, p, q), app = ld(Sh, Sl, p, p), aqq = ld(Sh, Sl, q, q);
          if (fabsf(apq.hi) > thr(p, q)) {
            const float a = __fadd_rn(apq.hi, apq.lo);
            const float dd = __fadd_rn(__fsub_rn(aqq.hi, app.hi), __fsub_rn(aqq.lo, app.lo));
            const float tau = dd / (2.f * a);
            const float rt = sqrtf(fmaf(tau, tau, 1.f));
            const float t = isfinite(rt) ? ((tau >= 0.f) ? 1.f / (tau + rt) : -1.f / (-tau + rt)) : 0.f;
            const float cf = rsqrtf(fmaf(t, t, 1.f)), sf = t * cf;
            // (c, s) = (cf, sf) (cf^2 + sf^2)^-1/2 to float-float precision
            float p1, e1, p2, e2;
            p1 = __fmul_rn(cf, cf);
            e1 = __fmaf_rn(cf, cf, -p1);
            p2 = __fmul_rn(sf, sf);
            e2 = __fmaf_rn(sf, sf, -p2);
            const FF dl = ffe_sub(ffe_add(FF{p1, e1}, FF{p2, e2}), FF{1.f, 0.f});
            FF y = ffe_sub(FF{1.f, 0.f}, FF{0.5f * dl.hi, 0.5f * dl.lo});
            y = ffe_add(y, FF{0.375f * dl.hi * dl.hi, 0.f});
            c = ffe_mul(FF{cf, 0.f}, y);
            s = ffe_mul(FF{sf, 0.f}, y);
          }
        }
        csv[4 * k] = c.hi;
        csv[4 * k + 1] = c.lo;
        csv[4 * k + 2] = s.hi;
        csv[4 * k + 3] = s.lo;
        pr[k][0] = p;
        pr[k][1] = q;
      }
      __syncthreads();
      // S_kk' <- R_k S_kk' R_k'^T for every pair of pairs (disjoint 2 x 2 blocks),
      // V <- V R^T, R = [[c, -s], [s, c]]
      const int nblk = half * half;
      for (int t = tid; t < nblk + N * half; t += nt) {
        if (t < nblk) {
          const int k = t / half, kk = t % half;
          const int p = pr[k][0], q = pr[k][1], p2 = pr[kk][0], q2 = pr[kk][1];
          const FF c{csv[4 * k], csv[4 * k + 1]}, s{csv[4 * k + 2], csv[4 * k + 3]};
          const FF c2{csv[4 * kk], csv[4 * kk + 1]}, s2{csv[4 * kk + 2], csv[4 * kk + 3]};
          const bool qv = q < N, q2v = q2 < N;
          const FF z{0.f, 0.f};
          const FF b00 = ld(Sh, Sl, p, p2), b01 = q2v ? ld(Sh, Sl, p, q2) : z;
          const FF b10 = qv ? ld(Sh, Sl, q, p2) : z, b11 = (qv && q2v) ? ld(Sh, Sl, q, q2) : z;
          // rows: R_k B
          const FF t00 = ffe_sub(ffe_mul(c, b00), ffe_mul(s, b10)), t01 = ffe_sub(ffe_mul(c, b01), ffe_mul(s, b11));
          const FF t10 = ffe_add(ffe_mul(s, b00), ffe_mul(c, b10)), t11 = ffe_add(ffe_mul(s, b01), ffe_mul(c, b11));
          // columns: (R_k B) R_k'^T
          st(Sh, Sl, p, p2, ffe_sub(ffe_mul(c2, t00), ffe_mul(s2, t01)));
          if (q2v) st(Sh, Sl, p, q2, ffe_add(ffe_mul(s2, t00), ffe_mul(c2, t01)));
          if (qv) st(Sh, Sl, q, p2, ffe_sub(ffe_mul(c2, t10), ffe_mul(s2, t11)));
          if (qv && q2v) st(Sh, Sl, q, q2, ffe_add(ffe_mul(s2, t10), ffe_mul(c2, t11)));
        } else {
          const int u = t - nblk, row = u / half, kk = u % half;
          const int p2 = pr[kk][0], q2 = pr[kk][1];
          if (q2 >= N) continue;
          const FF c2{csv[4 * kk], csv[4 * kk + 1]}, s2{csv[4 * kk + 2], csv[4 * kk + 3]};
          const FF vp = ld(Vh, Vl, row, p2), vq = ld(Vh, Vl, row, q2);
          st(Vh, Vl, row, p2, ffe_sub(ffe_mul(c2, vp), ffe_mul(s2, vq)));
          st(Vh, Vl, row, q2, ffe_add(ffe_mul(s2, vp), ffe_mul(c2, vq)));
        }
      }
      __syncthreads();
    }
    if (tid == 0) s_big = 0;
    __syncthreads();
  }
  if (!converged && tid == 0) atomicOr(status, kStatNotConverged);
  // X = D^-1/2 Q, then X = Lt^-T X (unit upper), row k final at step k
  for (int t = tid; t < N * N; t += nt) {
    const int i = t / N, j = t % N;
    st(Vh, Vl, i, j, ffe_mul(ld(Vh, Vl, i, j), FF{yv[2 * i], yv[2 * i + 1]}));
  }
  __syncthreads();
  for (int k = N - 1; k > 0; --k) {
    for (int t = tid; t < k * N; t += nt) {
      const int i = t / N, j = t % N;
      st(Vh, Vl, i, j, ffe_sub(ld(Vh, Vl, i, j), ffe_mul(ld(Bh, Bl, k, i), ld(Vh, Vl, k, j))));
    }
    __syncthreads();
  }
  // columns by ascending Ritz value (ties by index)
  for (int j = tid; j < N; j += nt) {
    const FF tj = ld(Sh, Sl, j, j);
    int rank = 0;
    for (int i = 0; i < N; ++i) {
      const FF ti = ld(Sh, Sl, i, i);
      if (ti.hi < tj.hi || (ti.hi == tj.hi && (ti.lo < tj.lo || (ti.lo == tj.lo && i < j)))) ++rank;
    }
    theta[rank] = ff_to_double(tj);
    for (int i = 0; i < N; ++i) C[(long long)i * Np + rank] = ff_to_double(ld(Vh, Vl, i, j));
  }
  for (int t = tid; t < Np * Np; t += nt) {
    const int i = t / Np, j = t % Np;
    if (i >= N || j >= N) C[t] = 0.0;
  }
}

}  // namespace

cudaError_t launch_small_eig(int N, const double* GA, const double* GB, double* work, double* C, double* theta,
                             int* status, cudaStream_t st, unsigned* bar, const int* clus, bool ff) {
  int Np = (N + 3) / 4 * 4;
  if (ff && clus == nullptr && N <= kEigFFMaxN) {
    const int LD = N | 1;
    const size_t smem = ((size_t)6 * N * LD + 2 * N + 4 * ((N + 1) / 2)) * sizeof(float);
    cudaError_t e = allow_max_dyn_smem((const void*)k_small_eig_ff);
    if (e != cudaSuccess) return e;
    // one thread per 2 x 2 block and per V row segment of a round, and per entry of
    // an elimination or solve step, where possible: no more warps than that (their
    // barriers are the kernel's latency), 64 to 512 threads
    const int half = (N + 1) / 2;
    int need = half * half + N * half;
    if (N * (N - 1) > need) need = N * (N - 1);
    int nt = (need + 31) / 32 * 32;
    nt = nt < 64 ? 64 : (nt > 512 ? 512 : nt);
    k_small_eig_ff<<<1, nt, smem, st>>>(N, Np, GA, GB, C, theta, status);
    return cudaGetLastError();
  }
  if (bar != nullptr && N > kEigGridMinN) {
    // the whole GPU: a cooperative grid of up to 128 CTAs (co-resident by construction)
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int half = (N + 1) / 2;
    int grid = half < nsm ? half : nsm;
    if (grid > 128) grid = 128;
    if ((e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    int n = N, np = Np;
    void* args[] = {&n, &np, (void*)&GA, (void*)&GB, &work, &C, &theta, &status, &bar, (void*)&clus};
    return cudaLaunchCooperativeKernel((const void*)k_small_eig_grid, dim3(grid), dim3(256), args, 0, st);
  }
  // threads: about one per rotation-pair row element, a multiple of 32
  int nt = (N * N / 2 + 31) / 32 * 32;
  if (nt < 64) nt = 64;
  if (nt > 1024) nt = 1024;
  const size_t smem = (size_t)4 * N * N * sizeof(double);
  if (smem <= 160 * 1024) {
    cudaError_t e = allow_max_dyn_smem((const void*)k_small_eig);
    if (e != cudaSuccess) return e;
    k_small_eig<<<1, nt, smem, st>>>(N, Np, GA, GB, work, C, theta, status, 1, clus);
  } else {
    k_small_eig<<<1, nt, 0, st>>>(N, Np, GA, GB, work, C, theta, status, 0, clus);
  }
  return cudaGetLastError();
}

cudaError_t launch_rotate(const Grid& g, int N, int Np, const double* X, const double* C, double* U,
                          cudaStream_t st) {
  NodeMap nm = node_map(Np);
  long long need = (g.nI + nm.npb - 1) / nm.npb;
  int nb = (int)(need < 152 * 16 ? need : 152 * 16);
  k_rotate<<<nb, kRedThreads, 0, st>>>(g, N, Np, X, C, U);
  return cudaGetLastError();
}

}  // namespace paro

// ---------------------------------------------------------------------------
// paro_small_eig_static: the small generalized eigensolve of k_small_eig with
// its scratch in a fixed, statically sized device array instead of memory the
// library allocates.
// ---------------------------------------------------------------------------

namespace {

constexpr int kStaticEigMaxN = PARO_STATIC_EIG_MAX_N;
// Work matrices L, S, V, W (4 N^2 doubles at N <= kStaticEigMaxN), then the
// status word.  Every GPU that loads this library holds the array until the
// process exits; all calls share it.
constexpr size_t kStaticEigDoubles = 4ull * kStaticEigMaxN * kStaticEigMaxN + 32;
__device__ __align__(256) double g_static_eig_scratch[kStaticEigDoubles];

// Device addresses of the array, one per CUDA context: the array lives in the
// module loaded into a context, so its address belongs to that context, not to
// a device ordinal (a context destroyed by cudaDeviceReset, or a caller's own
// driver-API context on the same device, has its own copy).  Contexts are told
// apart by their unique id (cuCtxGetId), which is never reused in a process.
constexpr int kMaxContexts = 64;
std::mutex g_static_eig_mu;
unsigned long long g_static_eig_ctx[kMaxContexts] = {};
void* g_static_eig_ptr[kMaxContexts] = {};
int g_static_eig_used = 0;

}  // namespace

extern "C" int paro_small_eig_static(int N, const double* GA, const double* GB, double* C, double* theta,
                                     void* cuda_stream) {
  if (N < 1 || N > kStaticEigMaxN) return PARO_ERR_ARG;
  if (!GA || !GB || !C || !theta) return PARO_ERR_ARG;
  // the calling thread's current context; with none yet, the current device's
  // primary context (what the runtime would bind on the launch)
  // (driver entry points through the runtime: the library does not link libcuda)
  typedef CUresult (*PFN_ctxGetCurrent)(CUcontext*);
  typedef CUresult (*PFN_ctxGetId)(CUcontext, unsigned long long*);
  static PFN_ctxGetCurrent get_current = nullptr;
  static PFN_ctxGetId get_id = nullptr;
  std::unique_lock<std::mutex> entry_lock(g_static_eig_mu);
  if (!get_current || !get_id) {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
      return PARO_ERR_CUDA;
    get_current = reinterpret_cast<PFN_ctxGetCurrent>(a);
    get_id = reinterpret_cast<PFN_ctxGetId>(b);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return PARO_ERR_CUDA;
  if (ctx == nullptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) return PARO_ERR_CUDA;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return PARO_ERR_CUDA;
  }
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return PARO_ERR_CUDA;
  entry_lock.unlock();
  double* scratch = nullptr;
  {
    // Once per context, with it current: the device address of the array (in
    // host code its name is only a host-side stand-in).
    std::lock_guard<std::mutex> lock(g_static_eig_mu);
    for (int i = 0; i < g_static_eig_used; ++i)
      if (g_static_eig_ctx[i] == id) scratch = static_cast<double*>(g_static_eig_ptr[i]);
    if (scratch == nullptr) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_static_eig_scratch) != cudaSuccess || ptr == nullptr) return PARO_ERR_CUDA;
      scratch = static_cast<double*>(ptr);
      if (g_static_eig_used < kMaxContexts) {  // beyond that, looked up on every call
        g_static_eig_ctx[g_static_eig_used] = id;
        g_static_eig_ptr[g_static_eig_used] = ptr;
        ++g_static_eig_used;
      }
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int* status = reinterpret_cast<int*>(scratch + 4ull * kStaticEigMaxN * kStaticEigMaxN);
  // The status word keeps the previous call's value: clear it.  The work
  // matrices are fully written by the kernel before they are read.
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return PARO_ERR_CUDA;
  paro::k_small_eig<<<1, 1024, 0, st>>>(N, N, GA, GB, scratch, C, theta, status, 0, nullptr);
  if (cudaGetLastError() != cudaSuccess) return PARO_ERR_CUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return PARO_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PARO_ERR_CUDA;
  if (h & paro::kStatNotSPD) return PARO_ERR_NOT_SPD;
  if (h & paro::kStatNotConverged) return PARO_ERR_NOT_CONVERGED;
  return PARO_OK;
}

