/*
 * paro.h -- C ABI of the GB300 (sm_103a) parallel orbital-updating library.
 *
 * The method (Dai, Gong, Zhou, Zhu, "A parallel orbital-updating approach for
 * electronic structure calculations"): given orbitals u_i and eigenvalue
 * estimates lambda_i, Step 3 of Algorithms 1.1, 3.1 and A.1 solves N independent
 * source problems a(u_i^(n+1/2), v) = lambda_i (u_i, v) (eq. alg-bvp), Step 4
 * projects onto span{u_i^(n+1/2)} (Rayleigh-Ritz, eq. alg-evp), Step 5 loops.
 *
 * Discretisation: Q1 finite elements on a uniform nx x ny x nz hexahedral mesh
 * of the box [lo, hi], homogeneous Dirichlet data on the whole boundary (the
 * truncated domain of Section 2.2).  The bilinear form is the linear part of
 * eq. (2.7):  a(w, v) = 1/2 (grad w, grad v) + (V w, v), with V given at the
 * 2x2x2 Gauss points of every cell.  Discrete operators on interior nodes:
 *     H = K/2 + M_V,   M = mass,   A = H + sigma M   (SPD for a suitable sigma).
 * The source problem is solved in its shifted form
 *     A x_i = (lambda_i + sigma) M u_i,
 * whose solution spans the same space as the paper's (sigma = 0 is the paper's
 * form; the shift keeps every system SPD when lambda_1 < 0).
 *
 * Conventions shared by every entry point
 *  - All array arguments marked "device" are caller-owned device pointers; the
 *    library never frees them.  Host arrays are caller-owned host memory.
 *  - Orbital blocks U, X are float64, row-major (n_interior x N): the row of
 *    interior node (i, j, k) (1 <= i <= nx-1, ...) is ((k-1)(ny-1) + (j-1))(nx-1)
 *    + (i-1), i.e. x varies fastest, and the N orbital values of a node are
 *    contiguous.
 *  - Vq (potential) is float64, 8 values per cell, order [cz][cy][cx][qz][qy][qx],
 *    Gauss abscissae (1 -/+ 1/sqrt 3)/2 in the cell's unit coordinates (q = 0 is
 *    the smaller one).
 *  - Every call is ordered on the handle's CUDA stream and returns a paro_status;
 *    calls that return host values (eigenvalues, statistics) synchronise that
 *    stream.  No exception crosses the ABI; paro_last_error() gives a message.
 *  - The library owns the handle and its workspace (device memory sized for the
 *    largest N seen, allocated on first use and released by paro_mesh_destroy).
 *  - A handle must not be used from two host threads at once.
 */
#ifndef PARO_H
#define PARO_H

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
  PARO_OK = 0,
  PARO_ERR_ARG = -1,           /* invalid argument (null pointer, size out of range) */
  PARO_ERR_CUDA = -2,          /* a CUDA runtime call failed (message has the CUDA error) */
  PARO_ERR_NOT_SPD = -3,       /* p^T A p <= 0 in CG, or a non-positive Cholesky pivot */
  PARO_ERR_NOT_CONVERGED = -4, /* an iteration limit was reached before its tolerance */
  PARO_ERR_NONFINITE = -5,     /* NaN/Inf met in a reduction */
  PARO_ERR_TIMEOUT = -6,       /* a bounded device-side wait (grid barrier, mbarrier) ran out */
  PARO_ERR_OOM = -7,           /* device allocation failed */
  PARO_ERR_STATE = -8          /* call out of order (e.g. no potential set) */
} paro_status;

/* Precision modes of a mesh handle. */
#define PARO_FP64 0  /* every operator apply, CG and projection in float64 */
#define PARO_MIXED 1 /* float32 CG inside float64-residual iterative refinement */

/* Operators for paro_apply. */
#define PARO_OP_A 0 /* A = K/2 + M_V + sigma M */
#define PARO_OP_H 1 /* H = K/2 + M_V            */
#define PARO_OP_M 2 /* M                       */

/* Arithmetic type for paro_apply. */
#define PARO_F64 0
#define PARO_F32 1
#define PARO_FF 2 /* float64 X, Y; float-float arithmetic (the mixed path's float64-accurate applies) */

/* Preconditioner of the float32 correction solves (paro_params.precond). */
#define PARO_PRECOND_JACOBI 0 /* Jacobi (D^-1), fused into the single-reduction CG kernel */
#define PARO_PRECOND_MG 1     /* one geometric-multigrid V-cycle (see paro_mg_vcycle); PARO_MIXED handles */
#define PARO_PRECOND_AUTO -1  /* hartree_precond only: multigrid on PARO_MIXED handles whose mesh coarsens at
                                 least twice, else Jacobi */

typedef struct paro_mesh_s* paro_mesh;

/* Solver controls.  paro_default_params fills the defaults noted here. */
typedef struct {
  double tol;         /* paro_iterate: stop when max_i |lambda_i^(n+1) - lambda_i^(n)| < tol (1e-10) */
  int max_outer;      /* paro_iterate: outer-iteration limit (500) */
  int n_check;        /* paro_iterate: test only the lowest n_check values; 0 = all N (0) */
  double solve_tol;   /* source problem: stop orbital i when ||b_i - A x_i||_2 <= solve_tol ||b_i||_2 (1e-12) */
  int pcg_maxit;      /* CG iteration limit per solve (FP64 mode) or per correction solve (mixed) (5000) */
  double inner_tol;   /* mixed: relative tolerance of each float32 correction solve; <= 0: sqrt(solve_tol)
                         clamped to [1e-6, 1e-3], so that two refinement sweeps reach solve_tol (0) */
  int max_refine;     /* mixed: refinement sweeps per source problem (20) */
  int check_every;    /* CG iterations between host convergence checks (16) */
  int fixed_outer;    /* paro_iterate: if > 0, run exactly this many outer iterations (0) */
  int profile;        /* 1: time every launch of the CG kernel (the persistent CG loop, one launch per
                         solve) with CUDA events on the handle's stream and report it in paro_stats.prof_*;
                         2: the same for a host-driven loop that launches the operator pass and the
                         update as separate kernels (timing the operator pass); 0: off (0) */
  int n_clusters;     /* paro_iterate: > 0 separates the Rayleigh-Ritz step of the outer iterations by
                         eigenvalue clusters (Section 3): orbitals come in n_clusters consecutive groups
                         of cluster_size[k] (ascending; the sizes add up to N); each group is made
                         M-orthogonal to the groups before it and gets its own small eigenproblem, and
                         the Ritz values are sorted within each group.  0: one problem of size N (0) */
  const int* cluster_size; /* host[n_clusters], read during the call (NULL) */
  int precond;        /* PARO_PRECOND_JACOBI or PARO_PRECOND_MG: the preconditioner of the float32
                         correction solves of the N source problems on a PARO_MIXED handle
                         (Section 3: each source problem solved by a parallel multigrid method).
                         PARO_PRECOND_MG on a PARO_FP64 handle: PARO_ERR_ARG (PARO_PRECOND_JACOBI) */
  int mg_nu;          /* multigrid: damped-Jacobi sweeps before and after the coarse correction, 1..8 (1) */
  int mg_coarse_sweeps; /* multigrid: sweeps on the coarsest level, 1..64 (4) */
  int hartree_precond; /* preconditioner of the Hartree (Poisson) solves of the Kohn-Sham calls:
                          PARO_PRECOND_AUTO, PARO_PRECOND_JACOBI or PARO_PRECOND_MG (PARO_PRECOND_AUTO) */
  int wait_polls;     /* mixed handles, Jacobi correction solves: polls of every bounded device-side wait
                         (TMA completion, the cross-CTA reduction) before the CG kernel gives up, records
                         PARO_ERR_TIMEOUT and returns; the handle stays usable.  <= 0: the built-in limit,
                         about a second of polling (0) */
} paro_params;

/* Statistics of a call.  Counters and times (cg_iters*, ms_*, stencil_applies,
 * kernel_launches, prof_*) are ADDED to what the struct holds, so zero it first;
 * the other fields are overwritten.  Counts are summed over orbitals. */
typedef struct {
  int outer_iters;             /* outer iterations done by paro_iterate */
  int refine_sweeps;           /* mixed mode: refinement sweeps in the last source solve */
  long long cg_iters;          /* CG updates, summed over orbitals and solves */
  long long cg_iters_f32;      /* of which in float32 */
  int cg_iters_max;            /* largest per-orbital CG count in the last source solve */
  double max_relres;           /* largest final ||b - A x|| / ||b|| of the last source solve (float64 residual) */
  double max_dlambda;          /* last max |delta lambda| */
  double ms_solve;             /* device time in source problems (CUDA events) */
  double ms_rr;                /* device time in Rayleigh-Ritz */
  long long stencil_applies;   /* orbital-operator applies (one orbital, one apply = 1) */
  long long kernel_launches;   /* CUDA kernels this library launched during the call */
  long long prof_launches;     /* profile != 0: timed launches (see paro_params.profile) */
  double prof_ms;              /* profile != 0: their summed device time (ms) */
  long long prof_dof_orb;      /* profile != 0: sum over their operator passes of n_interior x orbitals processed */
  long long prof_node_passes;  /* profile != 0: sum over their operator passes of n_interior x orbital blocks */
  int rr_tc_steps;             /* Rayleigh-Ritz steps whose Gram matrices ran on the tensor cores (mixed handles) */
  long long poisson_cg_iters;  /* CG iterations of the Hartree (Poisson) solves of a Kohn-Sham call */
  long long prof_dof_orb_active; /* profile != 0: sum over their operator passes of n_interior x orbitals still
                                    iterating (prof_dof_orb counts every orbital of a streamed group) */
} paro_stats;

void paro_default_params(paro_params* p);

/* Create a handle for the uniform Q1 mesh of [lo, hi] with nx x ny x nz cells
 * (each >= 2, at most 1024), Dirichlet on all faces.
 * precision: PARO_FP64 or PARO_MIXED.  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream) on which every later call is ordered.  Allocates the operator
 * storage (27 stencil weights per node in float64 and float32). */
int paro_mesh_create(paro_mesh* out, int nx, int ny, int nz, const double lo[3], const double hi[3],
                     int precision, void* cuda_stream);

/* A graded tensor-product mesh (Section 2.1: finite element spaces on meshes
 * refined where the orbitals vary fast; here the refinement runs along each
 * axis): x, y, z are host arrays of nx + 1, ny + 1 and nz + 1 node coordinates,
 * finite and strictly increasing (the box is [x[0], x[nx]] x ...; Dirichlet on
 * all faces).  The potential of paro_set_potential is then given at the 2x2x2
 * Gauss points of these cells (same order).  Every call works as on a uniform
 * mesh (the Q1 weights follow the cell sizes; the mass matrix is stored per
 * node), except the Kohn-Sham calls and PARO_PRECOND_MG, which return
 * PARO_ERR_ARG on a graded handle.  Other arguments and errors as
 * paro_mesh_create. */
int paro_mesh_create_graded(paro_mesh* out, int nx, int ny, int nz, const double* x, const double* y,
                            const double* z, int precision, void* cuda_stream);

/* Release the handle and all library-owned device memory.  Synchronises the stream. */
int paro_mesh_destroy(paro_mesh m);

/* Set the potential and shift: builds A = K/2 + M_{V+sigma} as 27 weights per
 * interior node (M_{V+sigma} by 2x2x2 Gauss quadrature, exact for sigma M) and
 * its Jacobi diagonal.  Vq: device, 8*nx*ny*nz float64 in the layout above.
 * eq. (2.7) with V = V_ext (+ V_H + V_xc for Kohn-Sham, supplied by the caller). */
int paro_set_potential(paro_mesh m, const double* Vq, double sigma);

/* Step 3 (eq. alg-bvp), all N orbitals at once:  A x_i = (lambda_i + sigma) M u_i,
 * warm start x_i = u_i, Jacobi-preconditioned CG per orbital with its own
 * convergence mask.  FP64 mode: float64 CG to solve_tol.  Mixed mode: float64
 * residual, float32 CG correction to inner_tol, x += d, repeated until solve_tol
 * or max_refine.  lambda: host[N].  U, X: device (n_interior x N) float64; X may
 * not alias U.  Returns PARO_ERR_NOT_CONVERGED (X still written) if a limit was hit. */
int paro_orbital_solve(paro_mesh m, int N, const double* lambda, const double* U, double* X,
                       const paro_params* p, paro_stats* s);

/* Step 4 (eq. alg-evp): Rayleigh-Ritz on span(X).  G_A = X^T H X, G_B = X^T M X,
 * Cholesky G_B = L L^T, symmetric eigen of L^-1 G_A L^-T (ascending), C = L^-T Q,
 * U_out = X C (M-orthonormal), lambda_out = Ritz values.  X, U_out: device
 * (n_interior x N) float64, may alias (the rotation goes through workspace).
 * lambda_out: host[N].  PARO_ERR_NOT_SPD if G_B is not positive definite
 * (X rank-deficient). */
int paro_rayleigh_ritz(paro_mesh m, int N, const double* X, double* U_out, double* lambda_out,
                       paro_stats* s);

/* Steps 3-5 repeated (Algorithm A.1 with a fixed potential; Algorithm 3.2 when
 * n_check < N).  U: device (n_interior x N) float64, in: initial orbitals, out:
 * final M-orthonormal Ritz vectors.  lambda: host[N], in: estimates, or NaN in
 * lambda[0] to start with one Rayleigh-Ritz step on span(U); out: Ritz values.
 * Stops on max |delta lambda| < tol (or after fixed_outer iterations). */
int paro_iterate(paro_mesh m, int N, double* U, double* lambda, const paro_params* p, paro_stats* s);

/* Z = B R: one V(mg_nu, mg_nu) cycle of the geometric multigrid preconditioner of
 * A = K/2 + M_{V+sigma} (the handle's current operator), float32, all N columns at
 * once (Section 3, two-level parallelisation).  Hierarchy: the cell counts are halved
 * while all three are even and >= 4; prolongation P = trilinear interpolation (the
 * coarse Q1 basis in the fine one); coarse operators A_c = P^T A P (Galerkin, built
 * in float64); damped Jacobi x <- x + w D^-1 (b - A x), w = min(1, 4/(3 rho)) with
 * rho = max_i sum_j |A_ij| / A_ii; mg_coarse_sweeps sweeps on the coarsest level; the
 * first sweep of every level starts from x = 0.  B is symmetric positive definite.
 * R, Z: device (n_interior x N) float32, must not alias.  PARO_MIXED handles only.
 * p: mg_nu and mg_coarse_sweeps are read (NULL: defaults). */
int paro_mg_vcycle(paro_mesh m, int N, const float* R, float* Z, const paro_params* p);

/* Y = op X for a block of N orbitals (op: PARO_OP_A/H/M), in float64 (dtype
 * PARO_F64: X, Y double) or float32 (PARO_F32: X, Y float, float32 weights).
 * X, Y: device (n_interior x N), must not alias.  The kernel the CG iterations use. */
int paro_apply(paro_mesh m, int N, int op, int dtype, const void* X, void* Y);

/* ---------------------------------------------------------------------------
 * Kohn-Sham (Section 2.2): fields at the 2x2x2 Gauss points of every cell,
 * device float64 arrays of 8*nx*ny*nz values in the order of paro_set_potential.
 * ------------------------------------------------------------------------- */

/* Electron density rho(x_q) = sum_i occ_i u_i(x_q)^2 (eq. (2.6)'s rho with
 * occupations).  U: device (n_interior x N) float64; occ: host[N]; rho_q: device,
 * written.  Needs a potential set on the handle (its workspace). */
int paro_density(paro_mesh m, int N, const double* U, const double* occ, double* rho_q);

/* v_q = vext_q + V_H(rho) + V_x(rho) and/or vh_q = V_H(rho).  V_H solves
 * -Delta V_H = 4 pi rho (the Poisson form of Section 2.2) with Q1 elements on the
 * box, Dirichlet data Q/|x - x_c| (the monopole of rho: charge Q, centre x_c),
 * by float64 Jacobi-PCG to p->solve_tol through the library's own stencil and CG
 * (an internal handle whose operator is K/2).  V_x = -(3 rho/pi)^(1/3) (Slater
 * exchange, the local-density approximation).  rho_q, vext_q: device in;
 * v_q, vh_q: device out (either may be NULL, not both).  p may be NULL (defaults). */
int paro_ks_potential(paro_mesh m, const double* rho_q, const double* vext_q, double* v_q, double* vh_q,
                      const paro_params* p);

/* Kohn-Sham ParO (Algorithm 3.1 with the Kohn-Sham potential): one
 * Rayleigh-Ritz on span(U) with vext_q gives the first density rho_in; each
 * outer iteration sets the potential vext + V_H(rho_in) + V_x(rho_in) with the
 * handle's sigma (from the last paro_set_potential), solves the N source
 * problems and does Rayleigh-Ritz with it, then mixes
 * rho_in <- (1 - mix) rho_in + mix rho_out (rho_out: density of the new
 * orbitals).  Stops when max |Delta lambda_i| over the lowest p->n_check
 * orbitals (0: all; Algorithm 3.2 tests the occupied ones and carries the rest
 * as a buffer) is below p->tol, or after p->fixed_outer.
 * The Hartree solve is warm-started from the previous one; PARO_FP64 handles
 * solve it to p->solve_tol, PARO_MIXED handles to max(p->solve_tol,
 * min(1e-4, 1e-2 x the previous iteration's max |Delta lambda|)).
 * occ: host[N] occupations; vext_q: device; U: device (n_interior x N) in/out;
 * lambda: host[N] out.  The handle's potential is the last effective potential
 * on return.  Errors as paro_iterate. */
int paro_scf_iterate(paro_mesh m, int N, const double* occ, const double* vext_q, double mix, double* U,
                     double* lambda, const paro_params* p, paro_stats* s);

/* Kohn-Sham electronic energy of the orbitals U (device, n_interior x N) with
 * occupations occ and eigenvalues lambda (host[N] each), in the band-energy form
 *     E = sum_i f_i lambda_i - 1/2 int rho V_H - int rho V_x + E_x,
 * rho = sum_i f_i u_i^2, V_H by a Hartree solve (p->solve_tol), Slater exchange;
 * at self-consistency this is the Kohn-Sham energy functional (the nuclei's
 * mutual repulsion not included).  *energy: host out.  Leaves the handle's SCF
 * density (rho_in) untouched. */
int paro_ks_energy(paro_mesh m, int N, const double* occ, const double* lambda, const double* U,
                   const paro_params* p, double* energy);

/* Copy the mixed density rho_in of the last paro_scf_iterate to rho_q (device). */
int paro_ks_density_in(paro_mesh m, double* rho_q);

/* Largest N accepted by paro_small_eig_static. */
#define PARO_STATIC_EIG_MAX_N 128

/* The small generalized eigenproblem of the Rayleigh-Ritz step, for callers
 * that must not allocate device memory.  The paper has no counterpart: this is
 * a library convenience.  Some callers cannot call cudaMalloc: applications
 * that hand all device memory to their own pool up front and forbid other
 * allocations, and latency-critical loops where a cudaMalloc (which may
 * synchronise the device) would stall other streams.  This entry point
 * allocates nothing: its work matrices live in one file-scope, statically sized
 * device array of 4*128*128 + 32 doubles (about 512 KiB), which every GPU that
 * loads the library holds until the process exits.
 *
 * Computes, in float64, the same thing as the small solve inside
 * paro_rayleigh_ritz: G_B = L L^T (Cholesky), L^-1 G_A L^-T = Q Theta Q^T
 * (cyclic Jacobi, ascending), C = L^-T Q.
 *   N      : 1 <= N <= PARO_STATIC_EIG_MAX_N, else PARO_ERR_ARG (nothing launched).
 *   GA, GB : device, N x N float64 row-major (symmetrised as (G + G^T)/2); GB SPD.
 *   C      : device, N x N float64 row-major out: column j is the eigenvector of theta[j],
 *            G_B-orthonormal (C^T G_B C = I, C^T G_A C = diag(theta)).
 *   theta  : device, N float64 out, ascending.
 *   cuda_stream : cudaStream_t the work is ordered on (NULL = legacy default stream).
 * Returns PARO_OK, PARO_ERR_ARG, PARO_ERR_NOT_SPD (non-positive Cholesky pivot:
 * C and theta are then not written), PARO_ERR_NOT_CONVERGED (the cyclic Jacobi
 * sweep limit ran out before the off-diagonal part reached the float64 rounding
 * floor: C and theta are written but C^T G_A C is only close to diagonal) or
 * PARO_ERR_CUDA.  Every call waits for the stream to finish: it reads the
 * status word back to the host.
 * The caller owns GA, GB, C and theta; the library allocates nothing, neither
 * cudaMalloc nor any allocating library routine.  The array's device address
 * belongs to the CUDA context the call runs in (the thread's current context,
 * else the current device's primary context): the first call in each context
 * looks it up once with that context current (a one-time set-up; make that
 * first call before any stream capture), later calls in the same context reuse
 * it, and a new context (for instance after cudaDeviceReset) gets its own
 * look-up.  All calls share the one array and it keeps the last call's
 * contents, so calls whose work overlaps on the GPU (different streams,
 * threads) race: order them. */
int paro_small_eig_static(int N, const double* GA, const double* GB, double* C, double* theta,
                          void* cuda_stream);

/* Measurement aid (the paper has no counterpart): the float32 (dtype PARO_F32)
 * or float64 (PARO_F64) fused multiply-add rate of the GPU's SIMT pipes, the
 * roofline denominator of the library's float-float and float64 kernels.  Runs
 * 8 x SMs blocks of 256 threads, each thread 8 independent FMA chains for
 * 16 x iters steps, twice, and times the second run with CUDA events on
 * cuda_stream.  out: device scratch of at least 8 x SMs x 256 elements of the
 * dtype (caller-owned, overwritten).  *tflops: host out, 10^12 flop/s (an FMA
 * counts 2).  Returns PARO_OK, PARO_ERR_ARG or PARO_ERR_CUDA; synchronises the
 * stream. */
int paro_peak_fma(int dtype, int iters, void* out, double* tflops, void* cuda_stream);

/* Message describing the last error on this handle ("" if none).  NULL handle:
 * the last paro_mesh_create failure on the calling host thread.  The string
 * lives until the next call. */
const char* paro_last_error(paro_mesh m);

/* Interior node count (nx-1)(ny-1)(nz-1) of a handle (PARO_ERR_ARG on NULL). */
long long paro_interior_nodes(paro_mesh m);

/* The adaptive loop of Section 2.1 (Solve -> Estimate -> Mark -> Refine) on
 * tensor-product meshes: solve on a handle (paro_iterate), estimate the error
 * per cell, mark cells, refine the axis coordinates, create the handle of the
 * refined mesh (paro_mesh_create_graded), move the orbitals to it
 * (paro_transfer) and solve again. */
#define PARO_MARK_DORFLER 0 /* eq. (2.2): least-cardinality set with sum eta^2 >= theta sum eta^2 */
#define PARO_MARK_MAXIMUM 1 /* eq. (2.3): eta >= theta max eta */

/* Estimate (Section 2.1: an a-posteriori indicator eta(., tau) per element; the
 * paper gives no formula, this is the residual indicator of -1/2 Lap u + V u =
 * lambda u for Q1 elements, summed over the N orbitals):
 *   eta_tau^2 = sum_i [ h_tau^2 ||(lambda_i - V) u_i||^2_tau
 *                       + 1/2 sum_{interior faces F of tau} h_F ||1/2 [d_n u_i]||^2_F ]
 * (Lap u = 0 inside trilinear elements; V at the cell's 2x2x2 Gauss points; the
 * normal-derivative jump is integrated exactly on each face; h_tau, h_F cell and
 * face diameters; Dirichlet boundary faces carry no jump).  U: device
 * (n_interior x N) float64 orbitals of this handle's mesh; lambda: host[N];
 * Vq: device potential at the Gauss points (layout of paro_set_potential);
 * eta2: device out, nx*ny*nz float64 in [cz][cy][cx] order.  Uses the handle's
 * workspace (not thread-safe with other calls on the handle); synchronises its
 * stream.  Errors: PARO_ERR_ARG (null pointer, N out of range), PARO_ERR_STATE
 * (no potential set), PARO_ERR_CUDA. */
int paro_estimate(paro_mesh m, int N, const double* U, const double* lambda, const double* Vq, double* eta2);

/* Mark (Section 2.1, eqs. (2.2)-(2.3)), on the host: marked[c] = 1 for the chosen
 * cells, 0 for the others.  PARO_MARK_DORFLER takes the largest indicators first
 * (ties by cell index) until their sum reaches theta of the total;
 * PARO_MARK_MAXIMUM marks eta >= theta max eta.  eta2: host[ncells] (>= 0,
 * finite); theta in (0, 1).  Returns the number of marked cells, or
 * PARO_ERR_ARG / PARO_ERR_NONFINITE. */
int paro_mark(long long ncells, const double* eta2, int strategy, double theta, unsigned char* marked);

/* Refine (Section 2.1: every marked element refined at least once), on the host:
 * on a tensor-product mesh every axis interval that holds a marked cell is
 * bisected (the cells sharing it are bisected too, so the mesh stays a tensor
 * product).  n: cells per axis; coords: host, the nx+1 x, then ny+1 y, then
 * nz+1 z node coordinates (strictly increasing); marked: host[nx*ny*nz] in
 * [cz][cy][cx] order; n_out: the new cell counts; coords_out: host, room for
 * (2nx+1) + (2ny+1) + (2nz+1) values, filled like coords.  PARO_ERR_ARG on null
 * pointers, fewer than 2 cells an axis or coordinates not increasing. */
int paro_refine_coords(const int n[3], const double* coords, const unsigned char* marked, int n_out[3],
                       double* coords_out);

/* Move N orbitals from one mesh to another covering the same box: the trilinear
 * interpolant of U_from's nodal values (zero on the boundary) at the interior
 * nodes of `to`.  Exact when `to` refines `from` (nested Q1 spaces).  U_from:
 * device (n_interior(from) x N), read after from's stream has synchronised;
 * U_to: device (n_interior(to) x N) out, must not alias U_from.  Runs on to's
 * stream and synchronises it.  PARO_ERR_ARG for different boxes, N out of range
 * or null / aliased pointers. */
int paro_transfer(paro_mesh from, paro_mesh to, int N, const double* U_from, double* U_to);

/* Batches of independent systems (meshes, orbital counts and potentials of
 * their own), Step 3 of Algorithm 3.1 solved for many systems at once.
 * paro_batch_iterate runs paro_iterate on every system.  Batched mode (the
 * default, paro_batch_set_fused(b, 1)): one host thread per system, and the
 * float32 correction solves of every PARO_MIXED, Jacobi-preconditioned system
 * (at least two, at most 256; profile = 0) run as ONE cooperative launch per
 * refinement sweep over all of them: work items (system, orbital block, tile
 * column, z-chunk) are taken from a counter in global memory, so converged
 * systems drop out and the rest spread over every SM.  The systems advance in
 * lockstep, one correction solve at a time; everything between two solves runs
 * on each system's own stream.  Float64 and multigrid systems iterate alone in
 * their threads.  The first call plans and autotunes the batched kernel over
 * the systems' buffers (PARO_AUTOTUNE=0: untuned).  Pool mode
 * (paro_batch_set_fused(b, 0)): a pool of n_workers host threads runs
 * paro_iterate per system, largest (interior nodes x N) first.
 * Give every handle its own CUDA stream (paro_mesh_create's cuda_stream): the
 * kernels of different systems then overlap on the GPU and the host-side waits
 * of one system hide behind the others' work; handles that share a stream stay
 * correct, only serialised.  A handle may appear in one entry of a batch. */
typedef struct paro_batch_s* paro_batch;
int paro_batch_create(paro_batch* out, int n_workers); /* 1 <= n_workers <= 256 */
/* Registers system (m, N, U, lambda, p) and returns its index (>= 0), or an
 * error status.  U: device (n_interior x N) in/out; lambda: host[N] in/out (NaN
 * in lambda[0]: initial Rayleigh-Ritz, as paro_iterate); p is copied (NULL:
 * defaults).  U and lambda must stay valid until paro_batch_iterate returns. */
int paro_batch_add(paro_batch b, paro_mesh m, int N, double* U, double* lambda, const paro_params* p);
int paro_batch_size(paro_batch b);
/* Iterates every system to its tolerance (paro_iterate).  rc: host[size] out,
 * every system's status; stats: host[size] out or NULL.  Returns PARO_OK if all
 * converged, else the status of the first failing system in index order. */
int paro_batch_iterate(paro_batch b, int* rc, paro_stats* stats);
/* on = 1: batched correction solves (default); 0: the pool of host workers.
 * PARO_ERR_ARG for other values or a NULL batch. */
int paro_batch_set_fused(paro_batch b, int on);
/* Batched launches of the last paro_batch_iterate (0: no batch was formed, e.g.
 * fewer than two qualifying systems, or pool mode). */
long long paro_batch_fused_launches(paro_batch b);
/* Message of the last batch-level failure (planning the batched kernel); the
 * systems' own failures are in paro_last_error of their handles. */
const char* paro_batch_last_error(paro_batch b);
int paro_batch_destroy(paro_batch b); /* the handles are not destroyed */

#ifdef __cplusplus
}
#endif
#endif /* PARO_H */
