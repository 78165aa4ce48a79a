// Internal definitions shared by the CUDA translation units of libparo.
//
// Storage (all device, library-owned unless noted):
//   node grid   padded with the Dirichlet boundary layer: Px = nx+1, Py = ny+1,
//               Pz = nz+1 nodes per axis, node g = (k*Py + j)*Px + i.  Boundary
//               rows of every vector are zero and are never written by a kernel,
//               which makes the 27-point stencil branch-free.
//   vectors     T[G][Np]: node-major, orbital-minor, Np = N rounded up to 4, so a
//               thread owns 4 consecutive orbitals of one node (16 B float /
//               32 B double vector access, coalesced across a warp).
//   operator    27 weights per node, SoA: coef[o][g], o = (dz+1)*9 + (dy+1)*3 + (dx+1),
//               plus the inverse diagonal dinv[g], in float64 and float32.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace paro {

constexpr int kMaxN = 1024;        // orbitals per block handled by one handle
constexpr int kRedThreads = 256;   // threads per block of the node-wise kernels
constexpr int kMaxRedBlocks = 1216;  // 152 SMs x 8: grid cap of the reducing kernels

// Device-side status bits (OR-ed into Grid::status).
constexpr int kStatNotSPD = 1;
constexpr int kStatNonFinite = 2;
constexpr int kStatNotConverged = 4;
constexpr int kStatTimeout = 8;

struct Grid {
  int nx, ny, nz;      // cells
  int Px, Py, Pz;      // padded nodes per axis
  long long G;         // padded node count
  int nI;              // interior node count
  double hx, hy, hz;   // cell sizes (graded meshes: their means)
  int graded;          // 1: the cell sizes vary along the axes (tensor-product grading)
  const double* hc;    // graded: device cell sizes, nx of x, then ny of y, then nz of z
};

// Graded meshes: the size of cell c along axis d (0 x, 1 y, 2 z).
__device__ __forceinline__ double cell_h(const Grid& g, int d, int c) {
  return g.hc[(d >= 1 ? g.nx : 0) + (d >= 2 ? g.ny : 0) + c];
}

template <typename T>
struct V4 {
  T a, b, c, d;
};

__device__ __forceinline__ V4<float> ld4(const float* p) {
  float4 v = *reinterpret_cast<const float4*>(p);
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  double2 u = reinterpret_cast<const double2*>(p)[0];
  double2 v = reinterpret_cast<const double2*>(p)[1];
  return {u.x, u.y, v.x, v.y};
}
__device__ __forceinline__ void st4(float* p, V4<float> v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.a, v.b, v.c, v.d);
}
__device__ __forceinline__ void st4(double* p, V4<double> v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v.a, v.b);
  reinterpret_cast<double2*>(p)[1] = make_double2(v.c, v.d);
}

// Mapping of a thread of a node-wise kernel: `groups` threads per node (4 orbitals
// each), `npb` nodes per block; threads tid >= groups*npb idle.
struct NodeMap {
  int groups;  // Np / 4
  int npb;     // nodes per block pass
};

__host__ __device__ inline NodeMap node_map(int Np) {
  NodeMap m;
  m.groups = Np / 4;
  m.npb = kRedThreads / m.groups;
  if (m.npb < 1) m.npb = 1;
  return m;
}

// Interior linear index n -> padded node index.
__device__ __forceinline__ long long interior_to_padded(const Grid& g, int n) {
  int ix = g.nx - 1, iy = g.ny - 1;
  int i = n % ix + 1;
  int t = n / ix;
  int j = t % iy + 1;
  int k = t / iy + 1;
  return ((long long)k * g.Py + j) * g.Px + i;
}

// Allows a kernel the device's largest dynamic shared memory (its opt-in maximum
// less the kernel's static shared memory), once per kernel and never lowered.
// Handles used from several host threads at once would otherwise race: a launch
// size set by one thread could lower the limit under another thread's launch.
// The limit is only a cap; occupancy follows the size a launch requests.
cudaError_t allow_max_dyn_smem(const void* f);

// ---------------------------------------------------------------------------
// Host-side launch wrappers (defined in stencil.cu, pcg.cu, rr.cu)
// ---------------------------------------------------------------------------

// Operator weights (constant part) for op selection in apply kernels.
struct Weights27 {
  double w[27];
};

// stencil.cu
cudaError_t launch_build_coef(const Grid& g, const double* Vq, double sigma, double* coef64, float* coef32,
                              double* dinv64, float* dinv32, cudaStream_t st);
// graded meshes: the 27 mass weights of every node (coefM, SoA like coef), and
// out = a - s b over n values (the H weights A - sigma M)
cudaError_t launch_build_mass(const Grid& g, double* coefM, cudaStream_t st);
cudaError_t launch_sub_scaled(long long n, const double* a, double s, const double* b, double* out, cudaStream_t st);
void mass_weights(const Grid& g, Weights27* mw);  // constant mass stencil M
// y = scale_o * (op x), op = coef (+ cw * wsub) ; T = float or double.  scale may be null.
cudaError_t launch_apply_f64(const Grid& g, int Np, const double* coef, const Weights27* cw, double csub,
                             const double* x, double* y, const double* scale, cudaStream_t st);
cudaError_t launch_apply_f32(const Grid& g, int Np, const float* coef, const float* x, float* y, cudaStream_t st);
cudaError_t launch_pack(const Grid& g, int N, int Np, const double* src, double* dst, cudaStream_t st);
cudaError_t launch_unpack(const Grid& g, int N, int Np, const double* src, double* dst, cudaStream_t st);
cudaError_t launch_pack_f32(const Grid& g, int N, int Np, const float* src, float* dst, cudaStream_t st);
cudaError_t launch_unpack_f32(const Grid& g, int N, int Np, const float* src, float* dst, cudaStream_t st);

// pcg.cu: per-orbital CG state, in device memory.
struct CGState {
  double* rz;      // (r, z)
  double* pq;      // (p, A p)
  double* alpha;
  double* beta;
  double* bb;      // ||b||^2
  double* rr;      // ||r||^2
  int* active;
  int* iters;
  int* skip;       // orbitals excluded from this solve (mixed: already converged)
  int* n_active;   // orbitals still iterating
  int* status;     // OR of kStat* bits
  double* partial; // [3][kMaxRedBlocks][Np]
  unsigned int* ticket;
  unsigned long long* work;  // cg_q adds (interior nodes) x (orbitals it processed) per launch
};

// Mixed refinement: r64 = b64 - A64 x64 -> rhs32 (float); convergence flags in s.skip.
cudaError_t launch_refine_residual(const Grid& g, int N, int Np, const double* coef64, const double* x64,
                                   const double* b64, float* rhs32, const CGState& s, double tol, cudaStream_t st);
cudaError_t launch_refine_update(const Grid& g, int Np, double* x64, const float* d32, const int* skip,
                                 cudaStream_t st);
// The same residual in float-float arithmetic (x and b as hi/lo arrays, packed weights of A).
// pcg.cu: the refinement's closing check before a Rayleigh-Ritz step on the same x:
// H x written over b (hi/lo), r = b - H x - sigma M x (M x given), norms and skip flags
cudaError_t launch_refine_check_hff(const Grid& g, int N, int Np, const float* whi, const float* wlo,
                                    const float* xhi, const float* xlo, const float* mhi, const float* mlo,
                                    double sigma, float* bhy, float* bly, const CGState& s, double tol,
                                    cudaStream_t st);
cudaError_t launch_refine_residual_ff(const Grid& g, int N, int Np, const float* whi, const float* wlo,
                                      const float* xhi, const float* xlo, const float* bhi, const float* blo,
                                      float* rhs32, const CGState& s, double tol, cudaStream_t st, int gm = 0);
// x64 = x_in + d (group-major d, orbitals not skipped; x_in for the skipped ones)
// and the float-float split of the new x; x_in may be x64 (in place)
cudaError_t launch_refine_update_split(const Grid& g, int Np, const double* x_in, double* x64, const float* d32gm,
                                       const int* skip, float* xh, float* xl, cudaStream_t st);

// ff.cu: float64-accurate applies, Grams and rotation in float-float arithmetic
cudaError_t launch_split_ff(long long n, const double* x, float* hi, float* lo, cudaStream_t st);
// mcoef (graded meshes, per-node mass weights) replaces the constant mw in H = A - sigma M
cudaError_t launch_build_wff(const Grid& g, const double* coef64, const Weights27& mw, double sigma, float* ahi,
                             float* alo, float* hhi, float* hlo, cudaStream_t st, const double* mcoef = nullptr);
// y = scale_o (W x): W the packed per-node weights (whi/wlo) or the constant weights cw
cudaError_t launch_ff_apply(const Grid& g, int Np, const float* whi, const float* wlo, const Weights27* cw,
                            const float* xhi, const float* xlo, const double* scale, double* y64, float* yhi,
                            float* ylo, cudaStream_t st);
size_t gram_ff_partial_doubles(const Grid& g, int Np);
cudaError_t launch_gram2_ff(const Grid& g, int Np, const float* xh, const float* xl, const float* ah, const float* al,
                            const float* bh, const float* bl, double* part, int* n_chunks, cudaStream_t st);
cudaError_t launch_gram_reduce(int Np, int nch, const double* part, double* G1, double* G2, cudaStream_t st);
cudaError_t launch_gram_reduce1(int Np, int nch, const double* part, double* Gm, cudaStream_t st);
// gram_tc.cu: one Gram X^T Y on the tensor cores (exact BF16 digit products, Np <= kTcMaxNp),
// from the hi parts of the float-float arrays; per-CTA partials
constexpr int kTcMaxNp = 256;
size_t gram_tc_partial_doubles(const Grid& g, int Np);
cudaError_t launch_gram_tc(const Grid& g, int Np, const float* xh, const float* yh, double* part, int* n_chunks,
                           int* status, cudaStream_t st);
// both Grams X^T A and X^T B in one launch (Np <= 32), partials into partA and partB
cudaError_t launch_gram_tc_pair(const Grid& g, int Np, const float* xh, const float* ah, const float* bh,
                                double* partA, double* partB, int* n_chunks, int* status, cudaStream_t st);
// gram_tc.cu: the rotation U = X C on the tensor cores (Np <= kRotTcMaxNp, X as float32 hi parts;
// above 128 in blocks of 128 K rows and columns, later K blocks added in float64)
constexpr int kRotTcMaxNp = 256;
cudaError_t launch_rotate_tc(const Grid& g, int N, int Np, const float* xh, const double* C, double* U, int* status,
                             cudaStream_t st);
constexpr int kRotateFFMaxNp = 144;  // whole C as float-float in shared memory (8 Np^2 bytes); column blocks above
cudaError_t launch_rotate_ff(const Grid& g, int N, int Np, const float* xh, const float* xl, const double* C,
                             double* U, cudaStream_t st);

// rr.cu
cudaError_t launch_gram2(const Grid& g, int N, int Np, const double* X, const double* Y1, const double* Y2,
                         double* part, int* n_chunks, double* G1, double* G2, cudaStream_t st);
size_t gram_partial_doubles(const Grid& g, int Np);
// N > kEigGridMinN with a barrier counter (bar, device): the whole-GPU form;
// else one CTA.  C (Np x Np) needs room for N + 2 x 128 + 1 doubles of scratch.
constexpr int kEigGridMinN = 64;
// clus (device, N cluster ids ascending, optional): cluster-separated form, the
// eigenproblem of each cluster's diagonal block alone, sorted within clusters.
// ff: float-float arithmetic on the float32 pipes (one CTA, N <= 64, no clusters).
cudaError_t launch_small_eig(int N, const double* GA, const double* GB, double* work, double* C, double* theta,
                             int* status, cudaStream_t st, unsigned* bar = nullptr, const int* clus = nullptr,
                             bool ff = false);
cudaError_t launch_rotate(const Grid& g, int N, int Np, const double* X, const double* C, double* U,
                          cudaStream_t st);

// adapt.cu: the adaptive loop on tensor-product meshes (Section 2.1)
// eta2[cell] = residual indicator of the orbitals u (padded [G][Np]), lam device[N],
// Vq the potential at the Gauss points ([cz][cy][cx][qz][qy][qx])
cudaError_t launch_estimate(const Grid& g, int N, int Np, const double* u, const double* lam, const double* Vq,
                            double* eta2, cudaStream_t st);
// Uf (fine interior rows x N) = trilinear interpolation of Uc (coarse interior rows x N);
// kmap/tmap: coarse interval and local coordinate of the fine interior nodes, x then y then z
cudaError_t launch_transfer(const Grid& gc, const Grid& gf, int N, const double* Uc, const int* kmap,
                            const double* tmap, double* Uf, cudaStream_t st);

// ks.cu: Kohn-Sham pieces (fields at the Gauss points)
cudaError_t launch_density(const Grid& g, int N, int Np, const double* U, const double* occ, double* rho,
                           cudaStream_t st);
int moments_blocks();
cudaError_t launch_moments(const Grid& g, const double lo[3], const double* rho, double* part, double* mom,
                           cudaStream_t st);
cudaError_t launch_hartree_rhs(const Grid& g, const double lo[3], const double* rho, const double* kcoef,
                               const double* mom, double* rhs, cudaStream_t st);
cudaError_t launch_ks_potential(const Grid& g, const double lo[3], const double* w, const double* mom,
                                const double* rho, const double* vext, double* vout, double* vh_out,
                                cudaStream_t st);
// out[0..2] = int rho V_H, int rho V_x, E_x (Slater) over the Gauss points; part: moments_blocks() x 3
cudaError_t launch_energy_terms(const Grid& g, const double* rho, const double* vh, double* part, double* out,
                                cudaStream_t st);
cudaError_t launch_mix(long long n, double beta, double* rho_in, const double* rho_out, cudaStream_t st);

}  // namespace paro
