// Device state, arguments and host plan of the batched CG (cg.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <vector>

#include "common.cuh"

namespace paro {

// Per-orbital CG scalars and controls, in device memory (one per handle).
struct CGDevState {
  double rz[kMaxN];     // (r, D^-1 r) of the current residual
  double pq[kMaxN];     // (p, A p)
  double alpha[kMaxN];  // step of the current iteration (set by K1)
  double beta[kMaxN];   // direction update for the next K1 (set by K2)
  double bb[kMaxN];     // ||b||^2
  double rr[kMaxN];     // ||r||^2
  int active[kMaxN];
  int iters[kMaxN];
  int skip[kMaxN];      // orbitals excluded from this solve
  int n_active;
  int status;           // OR of kStat* bits
  double tol;           // stop orbital i when ||r_i|| <= tol ||b_i||
  int maxit;
  unsigned int ticket;  // last-CTA detection; every last CTA resets it
  unsigned long long work;  // sum over operator passes of interior nodes x orbitals processed
  unsigned int bar_count;   // grid barrier counter of the persistent CG kernel (zeroed per launch)
  unsigned long long work_nodes;  // sum over operator passes of interior nodes x orbital blocks processed
  unsigned long long work_act;    // sum over operator passes of interior nodes x orbitals still iterating
  long long it_sum;               // single-pass CG: iterations of every orbital, summed over solves
  int it_max;                     // single-pass CG: largest per-orbital iteration count since the last reset
};

template <typename T>
struct CGArgs {
  Grid g;
  int N, Np;
  T *x, *b, *r, *p, *q;  // padded-grid vectors [node][Np]
  T* s;                  // single-reduction CG: s = A p (null in the two-reduction form); q holds w = A u
  T *r2, *q2, *s2;       // single-reduction CG: the second buffer set of r, w, s
  const T* dinv;         // inverse diagonal, padded grid (pitch Px)
  double* part;          // per-CTA partial sums
  CGDevState* st;
  int in_graph;          // kernels set the graph's while condition only inside a graph
};

// Geometry of the tiled operator kernel K1.
constexpr int kMaxGrid1 = 512;  // CTAs of the single-reduction CG kernel (split table size)

struct K1Geom {
  int TX, TY, DX;     // tile (x, y) of a z-marching column, staged row pitch of D^-1
  int ncx, ncy, nob;  // columns per axis, orbital blocks of width 4*G4
  int grid, G4;       // CTAs (each takes an equal share of the column-planes), float4 groups per block
  int npt, nthr;      // tile nodes per thread; node slots per CTA (TX * TY = nthr * npt)
  int slots;          // single-pass CG: depth of the TMA ring (planes in flight)
  int off_p, off_s, off_d, off_w, slot_bytes;  // byte offsets inside one ring slot
  uint32_t tx_bytes;                    // TMA bytes per slot
  size_t smem;                          // dynamic shared memory per CTA
  // single-reduction kernel: CTA c takes the column-planes [split[c], split[c+1])
  int split[kMaxGrid1 + 1];
};

template <typename T>
struct CGPlan {
  CGArgs<T> args{};
  K1Geom geo{};
  int nsm = 152;
  int dpitch = 0;  // row pitch of dinv_tma (elements)
  const T* dinv_tma = nullptr;
  const T* wcoef = nullptr;
  CUtensorMap mr;  // CUtensorMap carries its own 64-byte alignment
  CUtensorMap mp;
  CUtensorMap md;
  CUtensorMap mw;
  int grid_stream = 0, nt_stream = 0;  // init kernel
  int grid_upd = 0, nt_upd = 0;        // update kernel
  size_t smem_init = 0, smem_upd = 0;
  cudaGraphExec_t exec_zero = nullptr, exec_warm = nullptr;
  int graph_N = -1;  // N the graphs were built for
  bool coop_ok = false;  // the persistent CG kernel's grid can be co-resident
  // single-reduction CG (float32): geometry, tensor maps of r, w (= q), s, D^-1, weights
  K1Geom geo1{};
  bool cg1_ok = false;
  CUtensorMap m1r[2];
  CUtensorMap m1q[2];
  CUtensorMap m1s[2];
  CUtensorMap m1d;
  CUtensorMap m1w;
  // adds q = A x (the warm-start apply) as a graph node
  std::function<cudaError_t(cudaGraph_t, cudaGraphNode_t*)> add_apply;
};

template <typename T>
cudaError_t cg_plan_geometry(const Grid& g, int Np, int nsm, K1Geom* geo, int* bw_out);
// Tensor maps, kernel attributes and launch shapes (after args, pitches and pointers are set).
template <typename T>
cudaError_t cg_prepare(CGPlan<T>* P);
// Encodes the tensor maps, sets kernel attributes and instantiates the graph
// (warm start: with the apply node; else x0 = 0).
template <typename T>
cudaError_t cg_build_graph(CGPlan<T>* P, cudaStream_t st, bool with_apply);
// Host-driven form of the same loop (no graph): init, then K1/K2 pairs with
// CUDA events around every K1 launch.  *iters_done: K1 launches issued.
template <typename T>
cudaError_t cg_launch_init(CGPlan<T>* P, cudaStream_t st, bool x_zero);
template <typename T>
cudaError_t cg_launch_k1(CGPlan<T>* P, cudaStream_t st);
template <typename T>
cudaError_t cg_launch_k2(CGPlan<T>* P, cudaStream_t st);
// The whole CG loop as one cooperative launch (after cg_launch_init); returns an
// error (and launches nothing) if the grid cannot be co-resident.
template <typename T>
cudaError_t cg_launch_loop(CGPlan<T>* P, cudaStream_t st);
// Single-reduction CG (float32): plan (after the tensor maps' pointers are set) and launch.
// The feasible geometries for (mesh, Np), widest orbital blocks first; the first
// is the untuned default.
void cg1_candidates(const Grid& g, int Np, int nsm, std::vector<K1Geom>* out);
cudaError_t cg1_prepare(CGPlan<float>* P);                           // the default geometry
cudaError_t cg1_prepare_geo(CGPlan<float>* P, const K1Geom& geo);     // a given geometry
cudaError_t cg_launch_cg1(CGPlan<float>* P, cudaStream_t st);
// Autotuner: times `passes` CG passes of every candidate on the plan's own
// operator and workspace (b = 1, x = 0, tol = 0; overwrites b, x and the CG
// state) and prepares the fastest; *chosen: its index in cg1_candidates (-1 if
// none ran), *best_us: its time per pass, *tried: candidates timed.
cudaError_t cg1_autotune(CGPlan<float>* P, cudaStream_t st, int passes, int* chosen, float* best_us, int* tried);

// Single-pass Jacobi PCG of the float32 correction solves (cg2.cu).  Vectors are
// group-major: element (orbital 4 g + c, padded node n) at (g G + n) 4 + c, so a
// group of four orbitals is one contiguous [Pz][Py][Px][4] array and a converged
// group is neither loaded nor stored.  r[0] holds the right-hand side on entry
// (x0 = 0) and is overwritten; x receives the solution.
struct CG2Args {
  Grid g;
  int N, Np;
  float* x;
  float *r[2], *q[2], *p[2];  // the two buffer sets (read by pass parity, written by the other)
  double* part;               // per-CTA partial sums [2][Np][5][grid] (two buffers by pass parity)
  double* pub;                // per-orbital step of a pass, [2][Np][4]: alpha, beta, still iterating
  CGDevState* st;
  unsigned spin;              // poll limit of every bounded wait
  int inner;                  // 1: reaching maxit is not an error (refinement carries on)
};

struct CG2Plan {
  CG2Args args{};
  K1Geom geo{};
  int nsm = 152;
  int dpitch = 0;
  const float* dinv_tma = nullptr;
  const float* wcoef = nullptr;
  bool ok = false;
  CUtensorMap mr[2];
  CUtensorMap mq[2];
  CUtensorMap mp[2];
  CUtensorMap md;
  CUtensorMap mw;
};

// Geometries (tile shape, orbital block width) for (mesh, Np), widest blocks first.
void cg2_candidates(const Grid& g, int Np, int nsm, std::vector<K1Geom>* out);
cudaError_t cg2_prepare_geo(CG2Plan* P, const K1Geom& geo);
// One solve: zeroes the barrier words, then one cooperative launch.
cudaError_t cg2_launch(CG2Plan* P, cudaStream_t st);
// Times `passes` passes of every candidate (b = 1, tol = 0; overwrites the
// vectors and the CG state) and prepares the fastest.
cudaError_t cg2_autotune(CG2Plan* P, cudaStream_t st, int passes, int* chosen, float* best_us, int* tried);
void balanced_split(long long F, int nzo, int grid, int* out);

// Batched single-pass CG (cg2b.cu): the float32 correction solves of several
// independent systems (meshes, orbital counts, potentials) in one cooperative
// launch.  Work items are (system, orbital block, tile column, z-chunk); each
// pass the CTAs take items from a counter in global memory (dynamic balance as
// systems converge), and every system's vectors keep the group-major layout
// of the single-system kernel.
struct CG2BSys {
  Grid g;
  int Np, N;      // orbitals allocated (a multiple of 4) and solved
  int ncx, ncy;   // tile columns of the batch geometry
  int o0;         // first orbital of the system in the batch's numbering
  int job0;       // first orbital block (job) of the system
  float* x;
  float *r[2], *q[2], *p[2];
  CGDevState* st;
};
struct CG2BJob {
  int sys, ob, ng;  // system, orbital block, groups of four orbitals in the block
  int it0, nit;     // the block's work items [it0, it0 + nit)
  int pad[3];
};
constexpr int kMaxBatchSys = 256;
struct CG2BArgs {
  const CG2BSys* sys;
  const CG2BJob* jobs;
  const int4* items;      // (job, tile x, tile y, z-chunk)
  const CUtensorMap* maps;  // [system][8]: r0 q0 p0 r1 q1 p1 D^-1 weights
  const int* osys;        // system of each batch orbital
  int nsys, njobs, nitems, norb;
  int zlen;               // planes of a z-chunk
  int wpg;                // consumer warps per group slot (per-warp partial sums)
  unsigned long long part_mask[kMaxBatchSys / 64];  // systems taking part in the launch
  double* part;           // [item][warp of the group slot][5][block width]
  double* obb;            // [norb] ||b||^2
  int* oit;               // [norb] iterations
  int* oact;              // [norb] still iterating
  float *oal, *obe;       // [norb] alpha, beta of the next pass
  unsigned* jmask;        // [2][njobs] active groups of each block, by pass parity
  unsigned* bar;          // grid barrier counter (zeroed per launch)
  unsigned long long* ictr;  // work-item counter (zeroed per launch)
  unsigned spin;
  int inner;              // 1: reaching maxit is not an error (refinement carries on)
};
// One system of a batch plan: its float32 CG buffers and operator (the
// single-system plan's group-major vectors, D^-1 and packed weights).
struct CG2BSysDesc {
  Grid g;
  int Np, N;
  float* x;
  float *r[2], *q[2], *p[2];
  CGDevState* st;
  const float* dinv_tma;
  int dpitch;
  const float* wcoef;
};
struct CG2BPlan {
  CG2BArgs args{};
  K1Geom geo{};
  int nsm = 152;
  bool ok = false;
  std::vector<CG2BSysDesc> desc;
  std::vector<CG2BSys> hsys;
  // device buffers owned by the plan
  CG2BSys* dsys = nullptr;
  CG2BJob* djobs = nullptr;
  int4* ditems = nullptr;
  CUtensorMap* dmaps = nullptr;
  int* dosys = nullptr;
  double* dpart = nullptr;
  size_t part_cap = 0;
  size_t jobs_cap = 0, items_cap = 0;
  double* dobb = nullptr;
  int *doit = nullptr, *doact = nullptr;
  float *doal = nullptr, *dobe = nullptr;
  unsigned* djmask = nullptr;
  unsigned* dbar = nullptr;  // [0]: barrier; then the item counter (8-byte aligned)
};
// A plan over the given systems (device buffers allocated here; every call
// returns a CUDA status).  The geometry is the first candidate until
// cg2b_autotune or cg2b_prepare_geo picks another.
cudaError_t cg2b_create(CG2BPlan* P, const std::vector<CG2BSysDesc>& sys, int nsm);
void cg2b_destroy(CG2BPlan* P);
void cg2b_candidates(const CG2BPlan* P, std::vector<K1Geom>* out);
// Host only: the orbital blocks (jobs) and work items of a geometry (G.TX, G.TY,
// G.G4, G.grid), and the z-chunk length.
void cg2b_tables(const std::vector<CG2BSysDesc>& desc, const K1Geom& G, std::vector<CG2BJob>* jobs,
                 std::vector<int4>* items, int* zlen);
cudaError_t cg2b_prepare_geo(CG2BPlan* P, const K1Geom& geo);
// One batched solve of the systems whose bit is set in mask (their CG state:
// tol, maxit, skip, and r[0] = b, as for the single-system kernel).
cudaError_t cg2b_launch(CG2BPlan* P, const unsigned long long* mask, unsigned spin, cudaStream_t st);
// Times `passes` passes of every candidate over all systems (b = 1, tol = 0;
// overwrites their vectors and CG state) and prepares the fastest.
cudaError_t cg2b_autotune(CG2BPlan* P, cudaStream_t st, int passes, int* chosen, float* best_us, int* tried);

// Packed operator weights per input plane, [Pz][ny-1][nx-1][kPackedW], for the tiled kernel.
constexpr int kPackedW = 28;
__host__ __device__ inline size_t packed_weights_count(const Grid& g) { return (size_t)kPackedW * g.Pz * (g.ny - 1) * (g.nx - 1); }
// Build the tiled-kernel operator arrays from the 27-weight SoA coefficients.
template <typename T>
cudaError_t launch_build_tma_operator(const Grid& g, const T* coef, const T* dinv, T* wcoef, T* dinv_tma, int dpitch,
                                      cudaStream_t st);
template <typename T>
cudaError_t graph_add_apply(cudaGraph_t gr, cudaGraphNode_t* node, const Grid& g, int Np, const T* coef, const T* x,
                            T* y);

}  // namespace paro
