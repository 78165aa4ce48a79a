// Operator set-up and the 27-point Q1 stencil apply.
//
// Discrete form (eq. 2.7, linear part, with the shift of the source problems):
//   A = K/2 + M_{V+sigma}
// K/2 is built from its Kronecker closed form: with the 1-D Q1 matrices
//   k(0) = 2/h, k(+-1) = -1/h,   m(0) = 4h/6, m(+-1) = h/6,
// K = k_x m_y m_z + m_x k_y m_z + m_x m_y k_z  (weight of offset (dx,dy,dz)).
// M_{V+sigma} is integrated cell by cell with the 2x2x2 Gauss rule at which V is
// given; the rule is exact for sigma * mass, so sigma folds into V.
// The weights of a node are the 27 entries of its row of A.
#include "cg.cuh"
#include <mutex>
#include <set>
#include "common.cuh"
#include "q1.cuh"

namespace paro {

namespace {

__host__ __device__ inline double k1(int d, double h) { return d == 0 ? 2.0 / h : -1.0 / h; }
__host__ __device__ inline double m1(int d, double h) { return d == 0 ? 4.0 * h / 6.0 : h / 6.0; }

__global__ void k_build_coef(Grid g, const double* __restrict__ Vq, double sigma, double* __restrict__ coef64,
                             float* __restrict__ coef32, double* __restrict__ dinv64, float* __restrict__ dinv32) {
  // phi_a(x_q) on the reference cell, [a][q] with a = ax + 2 ay + 4 az, q likewise
  __shared__ double sa[64];
  for (int t = threadIdx.x; t < 64; t += blockDim.x) {
    const int a = t >> 3, q = t & 7;
    sa[t] = gq(a & 1, q & 1) * gq((a >> 1) & 1, (q >> 1) & 1) * gq((a >> 2) & 1, (q >> 2) & 1);
  }
  __syncthreads();
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nI) return;
  int ix = g.nx - 1, iy = g.ny - 1;
  int i = n % ix + 1;
  int t = n / ix;
  int j = t % iy + 1;
  int k = t / iy + 1;
  long long gp = ((long long)k * g.Py + j) * g.Px + i;
  double w[27];
  // 1-D stiffness and mass rows at the node, from the sizes of its two cells
  // along each axis (uniform: k = (-1, 2, -1)/h, m = (1, 4, 1) h/6)
  double kr[3][3], mr[3][3];
  const int ijk[3] = {i, j, k};
  const double hu[3] = {g.hx, g.hy, g.hz};
  for (int d = 0; d < 3; ++d) {
    const double hl = g.graded ? cell_h(g, d, ijk[d] - 1) : hu[d];
    const double hr = g.graded ? cell_h(g, d, ijk[d]) : hu[d];
    kr[d][0] = -1.0 / hl, kr[d][1] = 1.0 / hl + 1.0 / hr, kr[d][2] = -1.0 / hr;
    mr[d][0] = hl / 6.0, mr[d][1] = (hl + hr) / 3.0, mr[d][2] = hr / 6.0;
  }
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        double kk = kr[0][dx + 1] * mr[1][dy + 1] * mr[2][dz + 1] + mr[0][dx + 1] * kr[1][dy + 1] * mr[2][dz + 1] +
                    mr[0][dx + 1] * mr[1][dy + 1] * kr[2][dz + 1];
        w[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = 0.5 * kk;
      }
  // The 8 cells around the node; (cx, cy, cz) selects the cell, the node sits at
  // local corner a = (1-cx, 1-cy, 1-cz) of it.
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        int ex = i - 1 + cx, ey = j - 1 + cy, ez = k - 1 + cz;
        long long cell = ((long long)ez * g.ny + ey) * g.nx + ex;
        // Gauss weight of the cell: its volume / 8
        const double wq = g.graded ? cell_h(g, 0, ex) * cell_h(g, 1, ey) * cell_h(g, 2, ez) / 8.0
                                   : g.hx * g.hy * g.hz / 8.0;
        // row a of the cell's potential matrix: sum_q (V_q + sigma) phi_a(x_q) phi_b(x_q)
        // for the 8 corners b, i.e. the values (V + sigma) phi_a at the Gauss points
        // projected on the corners (the transpose of interp8, which has the same form)
        const int ax = 1 - cx, ay = 1 - cy, az = 1 - cz;
        const double* s_a = sa + (ax + 2 * ay + 4 * az) * 8;
        double ua[8], row[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) ua[q] = (Vq[cell * 8 + q] + sigma) * s_a[q];
        interp8(ua, row);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
          w[(bz - az + 1) * 9 + (by - ay + 1) * 3 + (bx - ax + 1)] += wq * row[b];
        }
      }
  for (int o = 0; o < 27; ++o) {
    coef64[(long long)o * g.G + gp] = w[o];
    coef32[(long long)o * g.G + gp] = (float)w[o];
  }
  dinv64[gp] = 1.0 / w[13];
  dinv32[gp] = 1.0f / (float)w[13];
}

// Graded meshes: the mass weights of every interior node, m_x (x) m_y (x) m_z with
// the 1-D mass rows of the node's two cells per axis; zero on boundary nodes.
__global__ void k_build_mass(Grid g, double* __restrict__ coefM) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nI) return;
  const int ix = g.nx - 1, iy = g.ny - 1;
  const int i = n % ix + 1, t = n / ix;
  const int j = t % iy + 1, k = t / iy + 1;
  const long long gp = ((long long)k * g.Py + j) * g.Px + i;
  const int ijk[3] = {i, j, k};
  double mr[3][3];
  for (int d = 0; d < 3; ++d) {
    const double hl = cell_h(g, d, ijk[d] - 1), hr = cell_h(g, d, ijk[d]);
    mr[d][0] = hl / 6.0, mr[d][1] = (hl + hr) / 3.0, mr[d][2] = hr / 6.0;
  }
  for (int o = 0; o < 27; ++o)
    coefM[(long long)o * g.G + gp] = mr[0][o % 3] * mr[1][(o / 3) % 3] * mr[2][o / 9];
}

__global__ void k_sub_scaled(long long n, const double* __restrict__ a, double s, const double* __restrict__ b,
                             double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = a[t] - s * b[t];
}

// MODE 0: y = coef x.  MODE 1: y = (coef - csub * cw) x.  MODE 2: y = cw x.
// Optional per-orbital scale of the result.
template <typename T, int MODE>
__global__ void __launch_bounds__(kRedThreads) k_apply(Grid g, int Np, const T* __restrict__ coef, Weights27 cw,
                                                       double csub, const T* __restrict__ x, T* __restrict__ y,
                                                       const double* __restrict__ scale) {
  NodeMap nm = node_map(Np);
  int grp = threadIdx.x % nm.groups;
  int nl = threadIdx.x / nm.groups;
  if (nl >= nm.npb) return;
  V4<double> s = {1.0, 1.0, 1.0, 1.0};
  if (scale != nullptr) s = {scale[4 * grp], scale[4 * grp + 1], scale[4 * grp + 2], scale[4 * grp + 3]};
  for (int n = blockIdx.x * nm.npb + nl; n < g.nI; n += gridDim.x * nm.npb) {
    long long gp = interior_to_padded(g, n);
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
    for (int o = 0; o < 27; ++o) {
      const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
      long long nb = gp + ((long long)dz * g.Py + dy) * g.Px + dx;
      T w;
      if (MODE == 0) w = coef[(long long)o * g.G + gp];
      else if (MODE == 1) w = (T)(coef[(long long)o * g.G + gp] - csub * cw.w[o]);
      else w = (T)cw.w[o];
      V4<T> v = ld4(x + nb * Np + 4 * grp);
      a0 += w * v.a;
      a1 += w * v.b;
      a2 += w * v.c;
      a3 += w * v.d;
    }
    V4<T> out = {(T)(a0 * s.a), (T)(a1 * s.b), (T)(a2 * s.c), (T)(a3 * s.d)};
    st4(y + gp * Np + 4 * grp, out);
  }
}

int apply_blocks(const Grid& g, int Np) {
  NodeMap nm = node_map(Np);
  long long need = (g.nI + nm.npb - 1) / nm.npb;
  long long cap = 152LL * 16;
  return (int)(need < cap ? need : cap);
}

__global__ void k_pack(Grid g, int N, int Np, const double* __restrict__ src, double* __restrict__ dst) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.nI * Np) return;
  int n = (int)(t / Np), o = (int)(t % Np);
  long long gp = interior_to_padded(g, n);
  dst[gp * Np + o] = o < N ? src[(long long)n * N + o] : 0.0;
}

__global__ void k_unpack(Grid g, int N, int Np, const double* __restrict__ src, double* __restrict__ dst) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.nI * N) return;
  int n = (int)(t / N), o = (int)(t % N);
  long long gp = interior_to_padded(g, n);
  dst[t] = src[gp * Np + o];
}

__global__ void k_pack_f32(Grid g, int N, int Np, const float* __restrict__ src, float* __restrict__ dst) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.nI * Np) return;
  int n = (int)(t / Np), o = (int)(t % Np);
  long long gp = interior_to_padded(g, n);
  dst[gp * Np + o] = o < N ? src[(long long)n * N + o] : 0.0f;
}

__global__ void k_unpack_f32(Grid g, int N, int Np, const float* __restrict__ src, float* __restrict__ dst) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.nI * N) return;
  int n = (int)(t / N), o = (int)(t % N);
  long long gp = interior_to_padded(g, n);
  dst[t] = src[gp * Np + o];
}

inline unsigned nblk(long long work, int threads) { return (unsigned)((work + threads - 1) / threads); }

// Operator weights keyed by input plane, for the z-marching tiled kernel, packed
// per output node:  W[s][yi][xi][o] = weight (dx, dy, dz) of the row of node
// (x, y, t), t = s - dz, x = xi + 1, y = yi + 1, o = (dz+1)*9 + (dy+1)*3 + (dx+1):
// the weight that multiplies the value at (x+dx, y+dy, s) in output row (x, y, t).
// Zero where t is not an interior plane; entry o = 27 pads the node to kPackedW.
template <typename T>
__global__ void k_build_w(Grid g, const T* __restrict__ coef, T* __restrict__ W) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)packed_weights_count(g);
  if (n >= total) return;
  const int o = (int)(n % kPackedW);
  long long r = n / kPackedW;
  const int xi = (int)(r % (g.nx - 1));
  r /= (g.nx - 1);
  const int yi = (int)(r % (g.ny - 1));
  const int s = (int)(r / (g.ny - 1));
  T w = 0;
  if (o < 27) {
    const int t = s - (o / 9 - 1), x = xi + 1, y = yi + 1;
    if (t >= 1 && t <= g.nz - 1) w = coef[(long long)o * g.G + ((long long)t * g.Py + y) * g.Px + x];
  }
  W[n] = w;
}

// D^-1 on the padded grid with row pitch dpitch (a multiple of 4): zero outside the interior.
template <typename T>
__global__ void k_build_dinv_tma(Grid g, const T* __restrict__ dinv, T* __restrict__ D, int dpitch) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)g.Pz * g.Py * dpitch;
  if (n >= total) return;
  int x = (int)(n % dpitch);
  long long r = n / dpitch;
  D[n] = (x < g.Px) ? dinv[r * g.Px + x] : (T)0;
}

}  // namespace

template <typename T>
cudaError_t launch_build_tma_operator(const Grid& g, const T* coef, const T* dinv, T* wcoef, T* dinv_tma, int dpitch,
                                      cudaStream_t st) {
  long long nw = (long long)packed_weights_count(g);
  k_build_w<T><<<nblk(nw, 256), 256, 0, st>>>(g, coef, wcoef);
  long long nd = (long long)g.Pz * g.Py * dpitch;
  k_build_dinv_tma<T><<<nblk(nd, 256), 256, 0, st>>>(g, dinv, dinv_tma, dpitch);
  return cudaGetLastError();
}
template cudaError_t launch_build_tma_operator<float>(const Grid&, const float*, const float*, float*, float*, int,
                                                      cudaStream_t);
template cudaError_t launch_build_tma_operator<double>(const Grid&, const double*, const double*, double*, double*, int,
                                                       cudaStream_t);

template <typename T>
cudaError_t graph_add_apply(cudaGraph_t gr, cudaGraphNode_t* node, const Grid& g, int Np, const T* coef, const T* x,
                            T* y) {
  Weights27 w{};
  double csub = 0.0;
  const double* scale = nullptr;
  Grid gg = g;
  int np = Np;
  void* args[] = {&gg, &np, (void*)&coef, &w, &csub, (void*)&x, (void*)&y, (void*)&scale};
  cudaKernelNodeParams p{};
  p.func = (void*)k_apply<T, 0>;
  p.gridDim = dim3(apply_blocks(g, Np));
  p.blockDim = dim3(kRedThreads);
  p.sharedMemBytes = 0;
  p.kernelParams = args;
  return cudaGraphAddKernelNode(node, gr, nullptr, 0, &p);
}
template cudaError_t graph_add_apply<float>(cudaGraph_t, cudaGraphNode_t*, const Grid&, int, const float*,
                                            const float*, float*);
template cudaError_t graph_add_apply<double>(cudaGraph_t, cudaGraphNode_t*, const Grid&, int, const double*,
                                             const double*, double*);

void mass_weights(const Grid& g, Weights27* mw) {
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx)
        mw->w[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = m1(dx, g.hx) * m1(dy, g.hy) * m1(dz, g.hz);
}

cudaError_t launch_build_coef(const Grid& g, const double* Vq, double sigma, double* coef64, float* coef32,
                              double* dinv64, float* dinv32, cudaStream_t st) {
  k_build_coef<<<nblk(g.nI, 128), 128, 0, st>>>(g, Vq, sigma, coef64, coef32, dinv64, dinv32);
  return cudaGetLastError();
}

cudaError_t launch_build_mass(const Grid& g, double* coefM, cudaStream_t st) {
  k_build_mass<<<nblk(g.nI, 128), 128, 0, st>>>(g, coefM);
  return cudaGetLastError();
}

cudaError_t launch_sub_scaled(long long n, const double* a, double s, const double* b, double* out, cudaStream_t st) {
  k_sub_scaled<<<nblk(n, 256), 256, 0, st>>>(n, a, s, b, out);
  return cudaGetLastError();
}

cudaError_t launch_apply_f64(const Grid& g, int Np, const double* coef, const Weights27* cw, double csub,
                             const double* x, double* y, const double* scale, cudaStream_t st) {
  Weights27 w{};
  if (cw) w = *cw;
  int nb = apply_blocks(g, Np);
  if (coef == nullptr)
    k_apply<double, 2><<<nb, kRedThreads, 0, st>>>(g, Np, coef, w, csub, x, y, scale);
  else if (cw != nullptr)
    k_apply<double, 1><<<nb, kRedThreads, 0, st>>>(g, Np, coef, w, csub, x, y, scale);
  else
    k_apply<double, 0><<<nb, kRedThreads, 0, st>>>(g, Np, coef, w, csub, x, y, scale);
  return cudaGetLastError();
}

cudaError_t launch_apply_f32(const Grid& g, int Np, const float* coef, const float* x, float* y, cudaStream_t st) {
  Weights27 w{};
  k_apply<float, 0><<<apply_blocks(g, Np), kRedThreads, 0, st>>>(g, Np, coef, w, 0.0, x, y, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_pack(const Grid& g, int N, int Np, const double* src, double* dst, cudaStream_t st) {
  k_pack<<<nblk((long long)g.nI * Np, 256), 256, 0, st>>>(g, N, Np, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_unpack(const Grid& g, int N, int Np, const double* src, double* dst, cudaStream_t st) {
  k_unpack<<<nblk((long long)g.nI * N, 256), 256, 0, st>>>(g, N, Np, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_pack_f32(const Grid& g, int N, int Np, const float* src, float* dst, cudaStream_t st) {
  k_pack_f32<<<nblk((long long)g.nI * Np, 256), 256, 0, st>>>(g, N, Np, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_unpack_f32(const Grid& g, int N, int Np, const float* src, float* dst, cudaStream_t st) {
  k_unpack_f32<<<nblk((long long)g.nI * N, 256), 256, 0, st>>>(g, N, Np, src, dst);
  return cudaGetLastError();
}

cudaError_t allow_max_dyn_smem(const void* f) {
  static std::mutex mu;
  static std::set<const void*> done;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(f)) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.insert(f);
  return e;
}

}  // namespace paro
