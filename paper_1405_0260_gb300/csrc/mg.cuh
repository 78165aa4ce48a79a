// Geometric multigrid preconditioner for the float32 correction solves (mg.cu).
//
// Section 3 (two-level parallelisation): the N source problems run in parallel
// (the orbital blocks of every kernel) and each one is solved by a parallel
// multigrid method.  Hierarchy: the cell counts are halved while all three are
// even and >= 4, the coarse Q1 space being a subspace of the fine one;
// prolongation P = trilinear interpolation (the coarse basis in the fine one);
// Galerkin coarse operators A_c = P^T A P (built in float64, stored as 27
// weights per node like the fine operator); damped Jacobi smoothing with
// w = min(1, 4 / (3 rho)), rho the Gershgorin bound max_i sum_j |A_ij| / A_ii of
// D^-1 A; a symmetric V(nu, nu) cycle with nu_c sweeps on the coarsest level.
// Every level stores its vectors orbital-minor [node][Np] on its padded grid
// (zero on the boundary nodes, which no kernel writes).
#pragma once
#include <cuda_runtime.h>

#include "cg.cuh"
#include "common.cuh"

namespace paro {

constexpr int kMaxMGLevels = 12;

struct MGLevel {
  Grid g{};
  double* coef64 = nullptr;  // [27][G] (level 0: the handle's operator)
  float* coef32 = nullptr;   // [27][G]
  float* dinv32 = nullptr;   // [G]
  float omega = 1.f;         // Jacobi weight
  double rho = 0.0;          // Gershgorin bound of D^-1 A
  // levels >= 1: right-hand side, residual, and the two iterates of the sweeps
  float *b = nullptr, *t = nullptr, *x = nullptr, *y = nullptr;  // [G][Np]
};

struct MGHier {
  int nlev = 0;
  int Np = 0;          // width the level vectors were allocated for
  bool built = false;  // coefficients match the current operator
  MGLevel lev[kMaxMGLevels];
  unsigned long long* rho_bits = nullptr;  // device [kMaxMGLevels]
};

// Grids of the hierarchy below the fine grid g0 (host only); returns the level count.
int mg_plan_levels(const Grid& g0, Grid* out, int max_levels);

// Galerkin operator of level l+1 from level l (float64 coefficients), its float32
// copy and inverse diagonal; Gershgorin bounds of every level into rho_bits.
cudaError_t launch_mg_galerkin(const Grid& gf, const Grid& gc, const double* cf, double* cc64, float* cc32,
                               float* dc32, cudaStream_t st);
cudaError_t launch_mg_rho(const Grid& g, const double* coef, unsigned long long* out, cudaStream_t st);

// One V(nu, nu) cycle on all Np columns (groups of 4 orbitals with no active
// orbital are skipped when active != nullptr): out = B r on the fine grid h.lev[0].
// y0, t0: fine-grid scratch [G][Np].  *launches += kernels launched.
cudaError_t mg_vcycle(const MGHier& h, int Np, const float* r, float* out, float* y0, float* t0, const int* active,
                      int nu, int nu_c, cudaStream_t st, long long* launches);

// MG-preconditioned CG (float32, the single-reduction recurrences of the CG kernel
// with u = B r): after the V-cycle left u in args.r2, w = A u with the partial sums
// (r, u), (w, u), (r, r); the last CTA updates alpha, beta, masks and counts.
cudaError_t mg_launch_wdots(CGPlan<float>* P, const float* coef32, cudaStream_t st);
// p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s.
cudaError_t mg_launch_update(CGPlan<float>* P, cudaStream_t st);

}  // namespace paro
