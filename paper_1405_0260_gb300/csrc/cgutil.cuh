// Device helpers shared by the CG kernels (cg.cu) and the multigrid kernels
// (mg.cu): 4-wide vector loads and stores, and the deterministic (fixed-order)
// reductions of per-orbital partial sums within a CTA and across CTAs.
#pragma once
#include <cuda_runtime.h>

namespace paro {
namespace {

template <typename T>
struct Vec4 {
  T v[4];
};

template <typename T>
__device__ __forceinline__ Vec4<T> lds4(const T* p) {
  Vec4<T> r;
  if constexpr (sizeof(T) == 4) {
    float4 a = *reinterpret_cast<const float4*>(p);
    r.v[0] = a.x, r.v[1] = a.y, r.v[2] = a.z, r.v[3] = a.w;
  } else {
    double2 a = reinterpret_cast<const double2*>(p)[0];
    double2 b = reinterpret_cast<const double2*>(p)[1];
    r.v[0] = a.x, r.v[1] = a.y, r.v[2] = b.x, r.v[3] = b.y;
  }
  return r;
}

// 16-byte (float) or 32-byte (double) vector load through L2 only (data other
// CTAs of the same launch wrote)
template <typename T>
__device__ __forceinline__ Vec4<T> ldcg4(const T* p) {
  Vec4<T> r;
  if constexpr (sizeof(T) == 4) {
    const float4 a = __ldcg(reinterpret_cast<const float4*>(p));
    r.v[0] = a.x, r.v[1] = a.y, r.v[2] = a.z, r.v[3] = a.w;
  } else {
    const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
    r.v[0] = a.x, r.v[1] = a.y, r.v[2] = b.x, r.v[3] = b.y;
  }
  return r;
}

template <typename T>
__device__ __forceinline__ void sts4(T* p, const Vec4<T>& r) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(r.v[0], r.v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(r.v[2], r.v[3]);
  }
}

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// p_new = D^-1 r + beta p_old (the same expression in K1 and K2).
template <typename T>
__device__ __forceinline__ T pnew(T di, T r, T beta, T pold) {
  return fmaT(beta, pold, di * r);
}

// Deterministic reduction of K per-orbital partial vectors over the CTAs of a
// kernel, run by the last CTA: tot[k*Np + o] = sum_b part[(k*G + b)*Np + o].
// Threads take (item, slice) pairs; slices are summed in order.
template <int K>
__device__ void reduce_over_ctas(const double* part, int G, int Np, double* sm, double* tot) {
  const int items = K * Np;
  const int nt = blockDim.x;
  int S = nt / items;
  if (S < 1) S = 1;
  if (S > 32) S = 32;
  for (int t = threadIdx.x; t < items * S; t += nt) {
    int item = t % items, sl = t / items;
    int k = item / Np, o = item % Np;
    const double* base = part + (long long)k * G * Np + o;
    // the 16 loads of a batch are issued before any addition (one L2 round trip
    // per batch instead of one per addition), then summed pairwise; the order is
    // fixed, so every CTA obtains the same totals
    double acc = 0.0;
    for (int b0 = sl; b0 < G; b0 += 16 * S) {
      double v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int b = b0 + q * S;
        v[q] = b < G ? __ldcg(base + (long long)b * Np) : 0.0;
      }
#pragma unroll
      for (int w = 8; w > 0; w >>= 1)
#pragma unroll
        for (int q = 0; q < w; ++q) v[q] += v[q + w];
      acc += v[0];
    }
    sm[sl * items + item] = acc;
  }
  __syncthreads();
  for (int item = threadIdx.x; item < items; item += nt) {
    double s = 0.0;
    for (int sl = 0; sl < S; ++sl) s += sm[sl * items + item];
    tot[item] = s;
  }
  __syncthreads();
}

// Fixed-order column sums of a [rows][cols] block of doubles in shared memory by
// every thread of the CTA: thread t sums rows sl, sl+S, ... of column c (t = sl*cols + c),
// then one thread per column adds the S slices in order.  tmp holds S*cols <= blockDim.x
// values.  Returns with the sums in tmp[0 .. cols) (after a barrier).
__device__ void block_colsum(const double* in, int rows, int cols, double* tmp) {
  const int nt = blockDim.x;
  int S = nt / cols;
  if (S < 1) S = 1;
  if (S > rows) S = rows;
  for (int t = threadIdx.x; t < S * cols; t += nt) {
    const int c = t % cols, sl = t / cols;
    double a0 = 0, a1 = 0;
    int r = sl;
    for (; r + S < rows; r += 2 * S) {
      a0 += in[r * cols + c];
      a1 += in[(r + S) * cols + c];
    }
    if (r < rows) a0 += in[r * cols + c];
    tmp[t] = a0 + a1;
  }
  __syncthreads();
  double v = 0.0;
  if (threadIdx.x < cols)
    for (int sl = 0; sl < S; ++sl) v += tmp[sl * cols + threadIdx.x];
  __syncthreads();
  if (threadIdx.x < cols) tmp[threadIdx.x] = v;
  __syncthreads();
}

// Writes this CTA's partials, takes a ticket; true in the last CTA.
__device__ bool last_cta(unsigned int* ticket) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(ticket, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

}  // namespace
}  // namespace paro
