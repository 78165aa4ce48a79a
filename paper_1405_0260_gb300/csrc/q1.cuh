// Reference-cell Q1 tables shared by the set-up and Kohn-Sham kernels: the 1-D
// linear functions at the two Gauss points of [0, 1] and the trilinear
// interpolation of 8 corner values to the 8 Gauss points of a cell.
#pragma once
#include <cuda_runtime.h>

namespace paro {
namespace {

// The 1-D Q1 functions at the two Gauss points of [0, 1]: gq(a, q) = g0 when the
// node a is the one nearer to point q, g1 otherwise.
__device__ __forceinline__ double gq(int a, int q) {
  const double g0 = 0.5 + 0.5 / 1.7320508075688772935;
  const double g1 = 0.5 - 0.5 / 1.7320508075688772935;
  return a == q ? g0 : g1;
}

// Values at the 8 Gauss points of a cell of the trilinear function with corner
// values c[a] (a = ax + 2 ay + 4 az), axis by axis (sum factorisation):
// v[q] = sum_a phi_a(x_q) c[a], q = qx + 2 qy + 4 qz.
__device__ __forceinline__ void interp8(const double (&c)[8], double (&v)[8]) {
  double X[8], Y[8];
#pragma unroll
  for (int yz = 0; yz < 4; ++yz)
#pragma unroll
    for (int qx = 0; qx < 2; ++qx) X[2 * yz + qx] = gq(0, qx) * c[2 * yz] + gq(1, qx) * c[2 * yz + 1];
#pragma unroll
  for (int az = 0; az < 2; ++az)
#pragma unroll
    for (int qy = 0; qy < 2; ++qy)
#pragma unroll
      for (int qx = 0; qx < 2; ++qx)
        Y[4 * az + 2 * qy + qx] = gq(0, qy) * X[4 * az + qx] + gq(1, qy) * X[4 * az + 2 + qx];
#pragma unroll
  for (int qz = 0; qz < 2; ++qz)
#pragma unroll
    for (int r = 0; r < 4; ++r) v[4 * qz + r] = gq(0, qz) * Y[r] + gq(1, qz) * Y[4 + r];
}

}  // namespace
}  // namespace paro
