// Float64-accurate kernels of the mixed-precision path in float-float
// arithmetic (ff.cuh): the operator applies of Step 3's right-hand sides and of
// the Rayleigh-Ritz step (Step 4), the Gram matrices G_A = X^T H X and
// G_B = X^T M X, and the rotation U = X C.  Inputs in float64 are first split
// into hi/lo float arrays (one streaming pass), so the stencil and Gram inner
// loops read pairs of floats and use only float32 instructions.
#include <cmath>

#include "cg.cuh"
#include "common.cuh"
#include "ff.cuh"

namespace paro {

namespace {

inline unsigned nblk(long long work, int threads) { return (unsigned)((work + threads - 1) / threads); }

// hi/lo split of a float64 vector (every padded node, so boundary rows stay zero).
__global__ void k_split(long long n, const double* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo) {
  long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (i + 1 < n) {
    const double2 v = reinterpret_cast<const double2*>(x)[i / 2];
    const FF a = ff_split(v.x), b = ff_split(v.y);
    reinterpret_cast<float2*>(hi)[i / 2] = make_float2(a.hi, b.hi);
    reinterpret_cast<float2*>(lo)[i / 2] = make_float2(a.lo, b.lo);
  } else if (i < n) {
    const FF a = ff_split(x[i]);
    hi[i] = a.hi;
    lo[i] = a.lo;
  }
}

// Packed float-float operator weights per padded node: w[g][o], o < 27 the
// weights of row g of A (mode 0) or of H = A - sigma M (mode 1); o = 27 pads.
__global__ void k_build_wff(Grid g, const double* __restrict__ coef, Weights27 mw, double sigma, float* __restrict__ ahi,
                            float* __restrict__ alo, float* __restrict__ hhi, float* __restrict__ hlo,
                            const double* __restrict__ mcoef) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.G * kPackedW) return;
  const long long node = t / kPackedW;
  const int o = (int)(t % kPackedW);
  double a = 0.0, h = 0.0;
  const int x = (int)(node % g.Px), y = (int)((node / g.Px) % g.Py), z = (int)(node / ((long long)g.Px * g.Py));
  if (o < 27 && x > 0 && x < g.Px - 1 && y > 0 && y < g.Py - 1 && z > 0 && z < g.Pz - 1) {
    a = coef[(long long)o * g.G + node];
    h = a - sigma * (mcoef != nullptr ? mcoef[(long long)o * g.G + node] : mw.w[o]);
  }
  const FF fa = ff_split(a), fh = ff_split(h);
  ahi[t] = fa.hi;
  alo[t] = fa.lo;
  hhi[t] = fh.hi;
  hlo[t] = fh.lo;
}

struct FFConst27 {
  float hi[27], lo[27];
};

// y = scale_o * (W x) at the interior nodes, W the packed per-node weights
// (CONSTW false) or the 27 constant weights cw (CONSTW true).  x as hi/lo
// arrays [G][Np]; y as float64 (y64) and/or hi/lo arrays (yhi, ylo).
template <bool CONSTW>
__global__ void __launch_bounds__(kRedThreads, 2) k_ff_apply(Grid g, int Np, const float* __restrict__ whi,
                                                          const float* __restrict__ wlo, FFConst27 cw,
                                                          const float* __restrict__ xhi,
                                                          const float* __restrict__ xlo,
                                                          const double* __restrict__ scale, double* __restrict__ y64,
                                                          float* __restrict__ yhi, float* __restrict__ ylo) {
  const NodeMap nm = node_map(Np);
  const int grp = threadIdx.x % nm.groups;
  const int nl = threadIdx.x / nm.groups;
  if (nl >= nm.npb) return;
  FF s[4] = {{1.0f, 0.0f}, {1.0f, 0.0f}, {1.0f, 0.0f}, {1.0f, 0.0f}};
  if (scale != nullptr)
    for (int c = 0; c < 4; ++c) s[c] = ff_split(scale[4 * grp + c]);
  for (int n = blockIdx.x * nm.npb + nl; n < g.nI; n += gridDim.x * nm.npb) {
    const long long gp = interior_to_padded(g, n);
    float wh[28], wl[28];
    if (!CONSTW) {
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        const float4 a = reinterpret_cast<const float4*>(whi + gp * kPackedW)[q];
        const float4 b = reinterpret_cast<const float4*>(wlo + gp * kPackedW)[q];
        wh[4 * q] = a.x, wh[4 * q + 1] = a.y, wh[4 * q + 2] = a.z, wh[4 * q + 3] = a.w;
        wl[4 * q] = b.x, wl[4 * q + 1] = b.y, wl[4 * q + 2] = b.z, wl[4 * q + 3] = b.w;
      }
    }
    FF acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
#pragma unroll
    for (int o = 0; o < 27; ++o) {
      const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
      const long long nb = gp + ((long long)dz * g.Py + dy) * g.Px + dx;
      const FF w = CONSTW ? FF{cw.hi[o], cw.lo[o]} : FF{wh[o], wl[o]};
      const float4 h = *reinterpret_cast<const float4*>(xhi + nb * Np + 4 * grp);
      const float4 l = *reinterpret_cast<const float4*>(xlo + nb * Np + 4 * grp);
      ff_mac(acc[0], FF{h.x, l.x}, w);
      ff_mac(acc[1], FF{h.y, l.y}, w);
      ff_mac(acc[2], FF{h.z, l.z}, w);
      ff_mac(acc[3], FF{h.w, l.w}, w);
    }
    FF r[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      FF t = {0.0f, 0.0f};
      ff_mac(t, ff_norm(acc[c]), s[c]);
      r[c] = ff_norm(t);
    }
    const long long e = gp * Np + 4 * grp;
    if (y64 != nullptr)
      st4(y64 + e, V4<double>{ff_to_double(r[0]), ff_to_double(r[1]), ff_to_double(r[2]), ff_to_double(r[3])});
    if (yhi != nullptr) {
      *reinterpret_cast<float4*>(yhi + e) = make_float4(r[0].hi, r[1].hi, r[2].hi, r[3].hi);
      *reinterpret_cast<float4*>(ylo + e) = make_float4(r[0].lo, r[1].lo, r[2].lo, r[3].lo);
    }
  }
}

// Gram matrices of Rayleigh-Ritz in float-float, for Np <= 32:
//   G1[a][b] = sum_n X[n][a] Y1[n][b],  G2[a][b] = sum_n X[n][a] Y2[n][b]
// over the padded nodes of one chunk per CTA (boundary rows are zero).  Thread
// (pair block q, slice sl) owns the 2 x 2 entries (2qa.., 2qb..) of both Grams
// and the chunk's staged nodes sl, sl + S, ...; slices are summed in order.
constexpr int kGramNodes = 64;  // nodes staged per step
__global__ void __launch_bounds__(256) k_gram2_ff(long long G, int Np, const float* __restrict__ xh,
                                                  const float* __restrict__ xl, const float* __restrict__ ah,
                                                  const float* __restrict__ al, const float* __restrict__ bh,
                                                  const float* __restrict__ bl, double* __restrict__ part,
                                                  long long chunk) {
  extern __shared__ float gsm[];  // 6 arrays [kGramNodes][Np]
  const int NS = kGramNodes * Np;
  float* sxh = gsm;
  float* sxl = gsm + NS;
  float* sah = gsm + 2 * NS;
  float* sal = gsm + 3 * NS;
  float* sbh = gsm + 4 * NS;
  float* sbl = gsm + 5 * NS;
  const int h2 = Np / 2;
  const int nq = h2 * h2;
  int S = blockDim.x / nq;
  if (S < 1) S = 1;
  const int q = threadIdx.x % nq, sl = threadIdx.x / nq;
  const bool live = threadIdx.x < nq * S;
  const int a0 = 2 * (q / h2), b0 = 2 * (q % h2);
  FF g1[2][2] = {}, g2[2][2] = {};
  const long long beg = (long long)blockIdx.x * chunk;
  long long end = beg + chunk;
  if (end > G) end = G;
  for (long long n0 = beg; n0 < end; n0 += kGramNodes) {
    const int rows = (int)((end - n0) < kGramNodes ? (end - n0) : kGramNodes);
    for (int t = threadIdx.x; t < kGramNodes * Np; t += blockDim.x) {
      const int r = t / Np;
      const long long e = n0 * Np + t;
      const bool ok = r < rows;
      sxh[t] = ok ? xh[e] : 0.0f;
      sxl[t] = ok ? xl[e] : 0.0f;
      sah[t] = ok ? ah[e] : 0.0f;
      sal[t] = ok ? al[e] : 0.0f;
      sbh[t] = ok ? bh[e] : 0.0f;
      sbl[t] = ok ? bl[e] : 0.0f;
    }
    __syncthreads();
    if (live) {
      for (int r = sl; r < rows; r += S) {
        const int base = r * Np;
        const FF x0{sxh[base + a0], sxl[base + a0]}, x1{sxh[base + a0 + 1], sxl[base + a0 + 1]};
        const FF y0{sah[base + b0], sal[base + b0]}, y1{sah[base + b0 + 1], sal[base + b0 + 1]};
        const FF z0{sbh[base + b0], sbl[base + b0]}, z1{sbh[base + b0 + 1], sbl[base + b0 + 1]};
        ff_mac(g1[0][0], x0, y0);
        ff_mac(g1[0][1], x0, y1);
        ff_mac(g1[1][0], x1, y0);
        ff_mac(g1[1][1], x1, y1);
        ff_mac(g2[0][0], x0, z0);
        ff_mac(g2[0][1], x0, z1);
        ff_mac(g2[1][0], x1, z0);
        ff_mac(g2[1][1], x1, z1);
      }
    }
    __syncthreads();
  }
  // slices in order: reuse the staging area as [S][nq][8] doubles
  double* red = reinterpret_cast<double*>(gsm);
  if (live) {
    double* dst = red + ((long long)sl * nq + q) * 8;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        dst[i * 2 + j] = ff_to_double(ff_norm(g1[i][j]));
        dst[4 + i * 2 + j] = ff_to_double(ff_norm(g2[i][j]));
      }
  }
  __syncthreads();
  const long long NN = (long long)Np * Np;
  for (int t = threadIdx.x; t < nq * 8; t += blockDim.x) {
    const int qq = t / 8, k = t % 8;
    double v = 0.0;
    for (int s2 = 0; s2 < S; ++s2) v += red[((long long)s2 * nq + qq) * 8 + k];
    const int w = k / 4, i = (k / 2) % 2, j = k % 2;
    const int a = 2 * (qq / h2) + i, b = 2 * (qq % h2) + j;
    part[(2LL * blockIdx.x + w) * NN + (long long)a * Np + b] = v;
  }
}

// U[g, b] = sum_a X[g, a] C[a, b] at the interior nodes in float-float; C (Np x Np,
// float64) is split into shared memory once per CTA.
__global__ void __launch_bounds__(kRedThreads) k_rotate_ff(Grid g, int N, int Np, const float* __restrict__ xh,
                                                           const float* __restrict__ xl, const double* __restrict__ C,
                                                           double* __restrict__ U) {
  extern __shared__ float csm[];  // hi [Np][Np], lo [Np][Np]
  float* ch = csm;
  float* cl = csm + Np * Np;
  for (int t = threadIdx.x; t < Np * Np; t += blockDim.x) {
    const FF c = ff_split(C[t]);
    ch[t] = c.hi;
    cl[t] = c.lo;
  }
  __syncthreads();
  const NodeMap nm = node_map(Np);
  const int grp = threadIdx.x % nm.groups;
  const int nl = threadIdx.x / nm.groups;
  if (nl >= nm.npb) return;
  for (int n = blockIdx.x * nm.npb + nl; n < g.nI; n += gridDim.x * nm.npb) {
    const long long gp = interior_to_padded(g, n);
    FF acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int a = 0; a < N; ++a) {
      const FF xa{xh[gp * Np + a], xl[gp * Np + a]};
      const float4 h = *reinterpret_cast<const float4*>(ch + a * Np + 4 * grp);
      const float4 l = *reinterpret_cast<const float4*>(cl + a * Np + 4 * grp);
      ff_mac(acc[0], xa, FF{h.x, l.x});
      ff_mac(acc[1], xa, FF{h.y, l.y});
      ff_mac(acc[2], xa, FF{h.z, l.z});
      ff_mac(acc[3], xa, FF{h.w, l.w});
    }
    st4(U + gp * Np + 4 * grp, V4<double>{ff_to_double(ff_norm(acc[0])), ff_to_double(ff_norm(acc[1])),
                                          ff_to_double(ff_norm(acc[2])), ff_to_double(ff_norm(acc[3]))});
  }
}

// U = X C for any Np (float-float): CTA y takes output columns [64 y, 64 y + 64);
// C's rows pass through shared memory 64 at a time as hi/lo [64][64]; a thread
// owns 4 output columns of one node (16 threads a node, 16 nodes a pass).
constexpr int kRotCB = 64, kRotKC = 64;
__global__ void __launch_bounds__(256) k_rotate_ff_cols(Grid g, int N, int Np, const float* __restrict__ xh,
                                                         const float* __restrict__ xl, const double* __restrict__ C,
                                                         double* __restrict__ U) {
  __shared__ float ch[kRotKC][kRotCB], cl[kRotKC][kRotCB];
  const int b0 = blockIdx.y * kRotCB;
  const int grp = threadIdx.x % (kRotCB / 4);  // 4 columns each
  const int nl = threadIdx.x / (kRotCB / 4);   // 16 nodes a pass
  const int npb = blockDim.x / (kRotCB / 4);
  const int b = b0 + 4 * grp;
  for (int n0 = blockIdx.x * npb; n0 < g.nI; n0 += gridDim.x * npb) {
    const int n = n0 + nl;
    const long long gp = n < g.nI ? interior_to_padded(g, n) : 0;
    FF acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int a0 = 0; a0 < N; a0 += kRotKC) {
      __syncthreads();  // the previous chunk's C is no longer read
      for (int t = threadIdx.x; t < kRotKC * kRotCB; t += blockDim.x) {
        const int r = t / kRotCB, c = t % kRotCB;
        const int a = a0 + r, bb = b0 + c;
        const FF f = (a < N && bb < Np) ? ff_split(C[(long long)a * Np + bb]) : FF{0.f, 0.f};
        ch[r][c] = f.hi;
        cl[r][c] = f.lo;
      }
      __syncthreads();
      const int na = N - a0 < kRotKC ? N - a0 : kRotKC;
      if (n < g.nI && b < Np)
        for (int r = 0; r < na; ++r) {
          const long long e = gp * Np + a0 + r;
          const FF xa{xh[e], xl[e]};
          const float4 h = *reinterpret_cast<const float4*>(&ch[r][4 * grp]);
          const float4 l = *reinterpret_cast<const float4*>(&cl[r][4 * grp]);
          ff_mac(acc[0], xa, FF{h.x, l.x});
          ff_mac(acc[1], xa, FF{h.y, l.y});
          ff_mac(acc[2], xa, FF{h.z, l.z});
          ff_mac(acc[3], xa, FF{h.w, l.w});
        }
    }
    if (n < g.nI && b < Np)
      st4(U + gp * Np + b, V4<double>{ff_to_double(ff_norm(acc[0])), ff_to_double(ff_norm(acc[1])),
                                      ff_to_double(ff_norm(acc[2])), ff_to_double(ff_norm(acc[3]))});
  }
}

int apply_grid(const Grid& g, int Np) {
  const NodeMap nm = node_map(Np);
  const long long need = (g.nI + nm.npb - 1) / nm.npb;
  // two 256-thread blocks resident a SM (up to 128 registers a thread: the 27 neighbours'
  // loads stay in flight; 6-8% faster than four blocks at 64 registers), two waves
  const long long cap = 152LL * 4;
  return (int)(need < cap ? need : cap);
}

}  // namespace

cudaError_t launch_split_ff(long long n, const double* x, float* hi, float* lo, cudaStream_t st) {
  k_split<<<nblk((n + 1) / 2, 256), 256, 0, st>>>(n, x, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_build_wff(const Grid& g, const double* coef64, const Weights27& mw, double sigma, float* ahi,
                             float* alo, float* hhi, float* hlo, cudaStream_t st, const double* mcoef) {
  k_build_wff<<<nblk(g.G * kPackedW, 256), 256, 0, st>>>(g, coef64, mw, sigma, ahi, alo, hhi, hlo, mcoef);
  return cudaGetLastError();
}

cudaError_t launch_ff_apply(const Grid& g, int Np, const float* whi, const float* wlo, const Weights27* cw,
                            const float* xhi, const float* xlo, const double* scale, double* y64, float* yhi,
                            float* ylo, cudaStream_t st) {
  FFConst27 c{};
  if (cw != nullptr) {
    for (int o = 0; o < 27; ++o) {
      const FF f = ff_split_host(cw->w[o]);
      c.hi[o] = f.hi;
      c.lo[o] = f.lo;
    }
    k_ff_apply<true><<<apply_grid(g, Np), kRedThreads, 0, st>>>(g, Np, nullptr, nullptr, c, xhi, xlo, scale, y64, yhi,
                                                                ylo);
  } else {
    k_ff_apply<false><<<apply_grid(g, Np), kRedThreads, 0, st>>>(g, Np, whi, wlo, c, xhi, xlo, scale, y64, yhi, ylo);
  }
  return cudaGetLastError();
}

static void gram_ff_shape(const Grid& g, long long* chunk, int* nch) {
  const long long want = 152 * 2;
  long long ch = (g.G + want - 1) / want;
  ch = (ch + kGramNodes - 1) / kGramNodes * kGramNodes;
  *chunk = ch;
  *nch = (int)((g.G + ch - 1) / ch);
}

size_t gram_ff_partial_doubles(const Grid& g, int Np) {
  long long chunk;
  int nch;
  gram_ff_shape(g, &chunk, &nch);
  return (size_t)nch * 2 * Np * Np;
}

cudaError_t launch_gram2_ff(const Grid& g, int Np, const float* xh, const float* xl, const float* ah, const float* al,
                            const float* bh, const float* bl, double* part, int* n_chunks, cudaStream_t st) {
  if (Np > 32) return cudaErrorInvalidValue;
  long long chunk;
  int nch;
  gram_ff_shape(g, &chunk, &nch);
  // staging (6 arrays of kGramNodes x Np floats), reused for the slice sums (<= 256 x 8 doubles)
  size_t smem = (size_t)6 * kGramNodes * Np * sizeof(float);
  if (smem < (size_t)256 * 8 * sizeof(double)) smem = (size_t)256 * 8 * sizeof(double);
  k_gram2_ff<<<nch, 256, smem, st>>>(g.G, Np, xh, xl, ah, al, bh, bl, part, chunk);
  *n_chunks = nch;
  return cudaGetLastError();
}

cudaError_t launch_rotate_ff(const Grid& g, int N, int Np, const float* xh, const float* xl, const double* C,
                             double* U, cudaStream_t st) {
  if (Np > kRotateFFMaxNp) {
    // column blocks of 64 outputs, C through shared memory 64 rows at a time
    const int ncb = (Np + kRotCB - 1) / kRotCB;
    long long nb = ((long long)g.nI + 15) / 16;
    const long long cap = 152LL * 8 / ncb + 1;
    dim3 grid((unsigned)(nb < cap ? nb : cap), (unsigned)ncb);
    k_rotate_ff_cols<<<grid, 256, 0, st>>>(g, N, Np, xh, xl, C, U);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)2 * Np * Np * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_dyn_smem((const void*)k_rotate_ff);
    if (e != cudaSuccess) return e;
  }
  k_rotate_ff<<<apply_grid(g, Np), kRedThreads, smem, st>>>(g, N, Np, xh, xl, C, U);
  return cudaGetLastError();
}

}  // namespace paro
