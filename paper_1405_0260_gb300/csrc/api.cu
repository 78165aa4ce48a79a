// C ABI of libparo (declared in include/paro.h): handle, workspace and the host
// orchestration of Steps 3-5 of the parallel orbital-updating method.  Every
// arithmetic step runs in the kernels of stencil.cu, pcg.cu and rr.cu; this file
// only sequences launches on the handle's stream and reads back the per-orbital
// convergence counters and the Ritz values.
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/paro.h"
#include "cg.cuh"
#include "mg.cuh"
#include "common.cuh"
#include "tma.cuh"

using namespace paro;

namespace {
struct BatchCG;
}

struct paro_mesh_s {
  Grid g{};
  // a batch whose correction solves this handle joins (one batched launch for
  // every system of the batch), and the handle's index in it
  BatchCG* bcg = nullptr;
  int bcg_index = -1;
  long long rr_tc = 0;  // Rayleigh-Ritz steps with tensor-core Grams (for paro_stats)
  int* clus = nullptr;  // cluster ids of the cluster-separated Rayleigh-Ritz (device, kMaxN)
  const char* tune_source = "default";  // how the float32 CG geometry was chosen
  long long ks_pois_iters = 0;  // CG iterations of the Hartree solves (for paro_stats)
  int precision = PARO_FP64;
  cudaStream_t st = nullptr;
  std::string err;
  double sigma = 0.0;
  bool have_pot = false;
  double* coef64 = nullptr;
  float* coef32 = nullptr;
  // graded meshes: cell sizes (device), per-node mass weights, the weights of
  // H = A - sigma M, and the packed float-float mass weights (mixed handles)
  double* hcell = nullptr;
  double* coefM64 = nullptr;
  double* coefH64 = nullptr;
  float *wMh = nullptr, *wMl = nullptr;
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  Weights27 mw{};
  // workspace sized for Np_alloc orbitals
  int Np_alloc = 0;
  double *u = nullptr, *x = nullptr, *b = nullptr, *r = nullptr, *p0 = nullptr, *q = nullptr;
  float *b32 = nullptr, *x32 = nullptr, *r32 = nullptr, *p32a = nullptr, *q32 = nullptr, *s32 = nullptr;
  float *r32b = nullptr, *q32b = nullptr, *s32b = nullptr;  // second buffer set of the single-reduction CG
  // mixed mode: float-float (hi/lo) copies of a float64 input vector and of two
  // operator images, [G][Np] each; float-float weights of A and H, [G][28] each
  float *fxh = nullptr, *fxl = nullptr, *fah = nullptr, *fal = nullptr, *fbh = nullptr, *fbl = nullptr;
  double* gpart_ff = nullptr;
  double* gpart_tc = nullptr;  // tensor-core Gram partials (32 < Np <= kTcMaxNp)
  float *wAh = nullptr, *wAl = nullptr, *wHh = nullptr, *wHl = nullptr;
  double *gpart = nullptr, *GA = nullptr, *GB = nullptr, *C = nullptr, *theta = nullptr, *eigwork = nullptr;
  double* dscal = nullptr;  // per-orbital double scalars
  int* dint = nullptr;      // per-orbital int scalars
  double* partial = nullptr;
  unsigned int* ticket = nullptr;
  double* h_dbl = nullptr;  // pinned host staging
  int* h_int = nullptr;
  // pinned staging of the CG controls only: h_dbl may still be the source of a
  // queued copy (the per-orbital right-hand-side scales) when a solve starts
  double* h_ctl = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // phase timings of the statistics: event pairs recorded on the stream and read
  // once at the end of the call (no synchronisation per phase)
  std::vector<cudaEvent_t> tev;
  int tev_used = 0;
  std::vector<std::pair<double*, int>> tev_pending;
  std::vector<void*> allocs;
  // launch accounting and optional per-launch timing of the CG operator kernel
  long long launches = 0;
  int profile = 0;
  std::vector<cudaEvent_t> pev;       // kProfPairs start/stop pairs
  int pev_used = 0;
  long long prof_launches = 0;
  double prof_ms = 0.0;
  // batched CG: device state, partial sums, TMA-layout operator, plans (graphs)
  int nsm = 152;
  CGDevState* cgst = nullptr;
  double* cgpart = nullptr;
  int dpitch = 0;
  float *w32 = nullptr, *dt32 = nullptr;
  double *w64 = nullptr, *dt64 = nullptr;
  CGPlan<float>* plan32 = nullptr;
  CGPlan<double>* plan64 = nullptr;
  // single-pass float32 CG (group-major vectors over the same float32 buffers)
  CG2Plan* plan2 = nullptr;
  double* cg2part = nullptr;
  const char* tune2_source = "default";
  // layout of the float32 CG buffers: 0 node-major (two-reduction and single-reduction
  // CG, multigrid, paro_apply), 1 group-major (single-pass CG).  A change zeroes them,
  // since each layout relies on zero Dirichlet rows at its own positions.
  int f32_layout = 0;
  // fxh/fxl hold the float-float split of x (set where x = u was just split)
  bool x_split_fresh = false;
  // x holds the start of a mixed solve only logically: x = u, not yet copied (the
  // first refinement update reads u and writes x)
  bool x_pending_u = false;
  // fxh/fxl = split(x) when a single-pass refinement has just ended (the
  // Rayleigh-Ritz step that follows in the ParO loop reuses it)
  bool x_split_valid = false;
  bool hm_ready = false;  // fah/fal = H x and fbh/fbl = M x of the current x (the refinement's closing check)
  // h_dbl holds the last refinement's ||r_i||^2 and ||b_i||^2 (read with its final check)
  bool relres_staged = false;
  // Kohn-Sham: box origin, the float64 handle of the Poisson operator K/2 (V = 0,
  // sigma = 0) that solves for the Hartree potential, and Gauss-point fields
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  // node coordinates per axis on the host (uniform or graded), for the transfer
  // of orbitals between meshes; per-axis maps of a transfer on the device
  std::vector<double> nodes[3];
  int* xmap_k = nullptr;
  double* xmap_t = nullptr;
  int xmap_cap = 0;
  paro_mesh pois = nullptr;
  double* ks_mom = nullptr;   // [Q, x_c, y_c, z_c]
  double* ks_part = nullptr;  // block partials of the moments
  double* ks_rho = nullptr;   // rho_in
  double* ks_rho2 = nullptr;  // rho_out
  double* ks_v = nullptr;     // the effective potential
  double* ks_occ = nullptr;   // occupations [Np]
  double* ks_vh = nullptr;    // V_H of the energy evaluation (Gauss points)
  double* ks_energy = nullptr;  // [int rho V_H, int rho V_x, E_x]
  // multigrid preconditioner of the float32 correction solves (built on first use,
  // coefficients rebuilt after every new potential)
  MGHier mg;
};

// Message of the last paro_mesh_create failure, one per host thread (creations on
// different threads do not race on it).
static thread_local std::string g_create_err;

namespace {

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      m->err = std::string(#call) + ": " + cudaGetErrorString(e_);                    \
      (void)cudaGetLastError(); /* a non-sticky error must not surface in a later call */ \
      return e_ == cudaErrorMemoryAllocation ? PARO_ERR_OOM : PARO_ERR_CUDA;          \
    }                                                                                 \
  } while (0)

#define TRY(expr)                  \
  do {                             \
    int rc_ = (expr);              \
    if (rc_ != PARO_OK) return rc_; \
  } while (0)

// A library kernel launch (nk kernels): checked and counted.
#define LAUNCH(nk, call)     \
  do {                       \
    CK(call);                \
    m->launches += (nk);     \
  } while (0)

constexpr int kProfPairs = 256;

// The mass and Hamiltonian applies: constant 27-point weights on uniform meshes,
// per-node weights on graded ones.
cudaError_t apply_M_f64(paro_mesh m, int Np, const double* x, double* y, const double* scale) {
  if (m->g.graded) return launch_apply_f64(m->g, Np, m->coefM64, nullptr, 0.0, x, y, scale, m->st);
  return launch_apply_f64(m->g, Np, nullptr, &m->mw, 0.0, x, y, scale, m->st);
}
cudaError_t apply_H_f64(paro_mesh m, int Np, const double* x, double* y) {
  if (m->g.graded) return launch_apply_f64(m->g, Np, m->coefH64, nullptr, 0.0, x, y, nullptr, m->st);
  return launch_apply_f64(m->g, Np, m->coef64, &m->mw, m->sigma, x, y, nullptr, m->st);
}
cudaError_t apply_M_ff(paro_mesh m, int Np, const float* xh, const float* xl, const double* scale, double* y64,
                       float* yh, float* yl) {
  if (m->g.graded) return launch_ff_apply(m->g, Np, m->wMh, m->wMl, nullptr, xh, xl, scale, y64, yh, yl, m->st);
  return launch_ff_apply(m->g, Np, nullptr, nullptr, &m->mw, xh, xl, scale, y64, yh, yl, m->st);
}

int set_f32_layout(paro_mesh m, int want);

int fail(paro_mesh m, int code, const std::string& msg) {
  m->err = msg;
  return code;
}

template <typename T>
int dalloc(paro_mesh m, T** p, size_t count, bool zero = true) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
  if (e != cudaSuccess) {
    m->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PARO_ERR_OOM : PARO_ERR_CUDA;
  }
  m->allocs.push_back(v);
  if (zero) {
    e = cudaMemsetAsync(v, 0, count * sizeof(T), m->st);
    if (e != cudaSuccess) return fail(m, PARO_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  }
  *p = static_cast<T*>(v);
  return PARO_OK;
}

void dfree(paro_mesh m, void* p) {
  if (!p) return;
  for (auto& a : m->allocs)
    if (a == p) {
      cudaFree(a);
      a = nullptr;
    }
}

// Per-orbital scalar slots in dscal (doubles) and dint (ints), each kMaxN long.
enum { S_RZ, S_PQ, S_ALPHA, S_BETA, S_BB, S_RR, S_RBB, S_RRR, S_SCALE, S_COUNT };
enum { I_ACTIVE, I_ITERS, I_SKIP, I_COUNT };
// then single ints after 3*kMaxN: n_active, status

CGState cg_state(paro_mesh m, bool refine) {
  CGState s;
  s.rz = m->dscal + S_RZ * kMaxN;
  s.pq = m->dscal + S_PQ * kMaxN;
  s.alpha = m->dscal + S_ALPHA * kMaxN;
  s.beta = m->dscal + S_BETA * kMaxN;
  s.bb = m->dscal + (refine ? S_RBB : S_BB) * kMaxN;
  s.rr = m->dscal + (refine ? S_RRR : S_RR) * kMaxN;
  s.active = m->dint + I_ACTIVE * kMaxN;
  s.iters = m->dint + I_ITERS * kMaxN;
  s.skip = m->cgst->skip;
  s.n_active = &m->cgst->n_active;
  s.status = &m->cgst->status;
  s.partial = m->partial;
  s.ticket = m->ticket;
  s.work = nullptr;
  return s;
}

void free_plans(paro_mesh m) {
  delete m->plan2;
  m->plan2 = nullptr;
  if (m->plan32) {
    if (m->plan32->exec_zero) cudaGraphExecDestroy(m->plan32->exec_zero);
    if (m->plan32->exec_warm) cudaGraphExecDestroy(m->plan32->exec_warm);
    delete m->plan32;
    m->plan32 = nullptr;
  }
  if (m->plan64) {
    if (m->plan64->exec_zero) cudaGraphExecDestroy(m->plan64->exec_zero);
    if (m->plan64->exec_warm) cudaGraphExecDestroy(m->plan64->exec_warm);
    delete m->plan64;
    m->plan64 = nullptr;
  }
}

// Autotuner of the single-reduction CG geometry (tile shape, orbital block width).
// PARO_AUTOTUNE=0 keeps the untuned default.  PARO_AUTOTUNE_CACHE=<file>: a JSON
// object mapping "<device>|<nx>x<ny>x<nz>|Np<Np>" to [TX, TY, block width, us per
// pass], read before and rewritten after a tuning run.
struct TuneEntry {
  int TX = 0, TY = 0, bw = 0;
  double us = 0.0;
};

std::map<std::string, TuneEntry> tune_cache_read(const char* path) {
  std::map<std::string, TuneEntry> out;
  FILE* f = std::fopen(path, "r");
  if (!f) return out;
  std::string txt;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, n);
  std::fclose(f);
  size_t pos = 0;
  while ((pos = txt.find('"', pos)) != std::string::npos) {
    const size_t end = txt.find('"', pos + 1);
    if (end == std::string::npos) break;
    const size_t lb = txt.find('[', end), rb = lb == std::string::npos ? lb : txt.find(']', lb);
    if (rb == std::string::npos) break;
    TuneEntry e;
    if (std::sscanf(txt.c_str() + lb + 1, " %d , %d , %d , %lf", &e.TX, &e.TY, &e.bw, &e.us) == 4)
      out[txt.substr(pos + 1, end - pos - 1)] = e;
    pos = rb + 1;
  }
  return out;
}

void tune_cache_write(const char* path, const std::map<std::string, TuneEntry>& c) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : c)
    std::fprintf(f, "  \"%s\": [%d, %d, %d, %.2f]%s\n", kv.first.c_str(), kv.second.TX, kv.second.TY, kv.second.bw,
                 kv.second.us, ++i < c.size() ? "," : "");
  std::fprintf(f, "}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path);
}

// Chooses the geometry of a float32 plan's single-reduction kernel: from the
// cache, else by timing the candidates (cg1_autotune).
int autotune_cg1(paro_mesh m, CGPlan<float>* P) {
  const char* off = std::getenv("PARO_AUTOTUNE");
  if ((off && off[0] == '0') || !P->cg1_ok) return PARO_OK;
  std::vector<K1Geom> cand;
  cg1_candidates(m->g, P->args.Np, m->nsm, &cand);
  if (cand.size() < 2) return PARO_OK;
  int dev = 0;
  cudaDeviceProp prop{};
  CK(cudaGetDevice(&dev));
  CK(cudaGetDeviceProperties(&prop, dev));
  const std::string key = std::string(prop.name) + "|" + std::to_string(m->g.nx) + "x" + std::to_string(m->g.ny) +
                          "x" + std::to_string(m->g.nz) + "|Np" + std::to_string(P->args.Np);
  const char* path = std::getenv("PARO_AUTOTUNE_CACHE");
  std::map<std::string, TuneEntry> cache;
  if (path) {
    cache = tune_cache_read(path);
    auto it = cache.find(key);
    if (it != cache.end())
      for (const K1Geom& G : cand)
        if (G.TX == it->second.TX && G.TY == it->second.TY && G.G4 * 4 == it->second.bw) {
          CK(cg1_prepare_geo(P, G));
          m->tune_source = "cache";
          return PARO_OK;
        }
  }
  int chosen = -1, tried = 0;
  float us = 0.f;
  CK(cg1_autotune(P, m->st, 8, &chosen, &us, &tried));
  m->tune_source = "timed";
  if (chosen >= 0 && path) {
    TuneEntry e;
    e.TX = cand[chosen].TX;
    e.TY = cand[chosen].TY;
    e.bw = cand[chosen].G4 * 4;
    e.us = us;
    cache[key] = e;
    tune_cache_write(path, cache);
  }
  return PARO_OK;
}

template <typename T>
int make_plan(paro_mesh m, int Np, CGPlan<T>** out, T* x, T* b, T* r, T* p, T* q, const T* dinv, const T* dinv_tma,
              const T* wcoef, const T* coef, T* s = nullptr, T* r2 = nullptr, T* q2 = nullptr, T* s2 = nullptr) {
  CGPlan<T>* P = new CGPlan<T>();
  P->nsm = m->nsm;
  P->args.g = m->g;
  P->args.N = Np;  // set per solve
  P->args.Np = Np;
  P->args.x = x;
  P->args.b = b;
  P->args.r = r;
  P->args.p = p;
  P->args.q = q;
  P->args.s = s;
  P->args.r2 = r2;
  P->args.q2 = q2;
  P->args.s2 = s2;
  P->args.dinv = dinv;
  P->args.part = m->cgpart;
  P->args.st = m->cgst;
  P->args.in_graph = 0;
  P->dpitch = m->dpitch;
  P->dinv_tma = dinv_tma;
  P->wcoef = wcoef;
  int bw = 0;
  cudaError_t e = cg_plan_geometry<T>(m->g, Np, m->nsm, &P->geo, &bw);
  if (e == cudaSuccess) e = cg_prepare<T>(P);
  if constexpr (sizeof(T) == 4) {
    if (e == cudaSuccess) e = cg1_prepare(P);
  }
  if (e != cudaSuccess) {
    delete P;
    return fail(m, PARO_ERR_CUDA, std::string("CG plan: ") + cudaGetErrorString(e));
  }
  if constexpr (sizeof(T) == 4) m->tune_source = "default";  // tuned in make_plans when it is the solver used
  if (std::getenv("PARO_PRINT_PLAN"))
    std::fprintf(stderr, "paro CG plan (%s): tile %dx%d, %d node(s)/thread, block %d orbitals x %d, %d threads, grid %d, "
                 "smem %zu B, persistent %d\n", sizeof(T) == 4 ? "float32" : "float64", P->geo.TX, P->geo.TY,
                 P->geo.npt, P->geo.G4 * 4, P->geo.nob, P->geo.nthr * P->geo.G4, P->geo.grid, P->geo.smem,
                 (int)P->coop_ok);
  if constexpr (sizeof(T) == 4) {
    if (std::getenv("PARO_PRINT_PLAN"))
      std::fprintf(stderr, "paro single-reduction CG plan: tile %dx%d, block %d orbitals x %d, %d threads, grid %d, "
                   "smem %zu B, usable %d, geometry %s\n", P->geo1.TX, P->geo1.TY, P->geo1.G4 * 4, P->geo1.nob,
                   P->geo1.nthr * P->geo1.G4, P->geo1.grid, P->geo1.smem, (int)P->cg1_ok, m->tune_source);
  }
  Grid g = m->g;
  P->add_apply = [g, Np, coef, x, q](cudaGraph_t gr, cudaGraphNode_t* node) {
    return graph_add_apply<T>(gr, node, g, Np, coef, x, q);
  };
  *out = P;
  return PARO_OK;
}

// Geometry of the single-pass CG: from the cache (key suffix "|cg2"), else timed.
int autotune_cg2(paro_mesh m, CG2Plan* P) {
  std::vector<K1Geom> cand;
  cg2_candidates(m->g, P->args.Np, m->nsm, &cand);
  if (cand.empty()) return PARO_OK;
  // PARO_CG2_GEOMETRY=<i>: candidate i, untimed (the tests run every geometry this way)
  if (const char* f = std::getenv("PARO_CG2_GEOMETRY")) {
    const int i = std::atoi(f);
    if (i >= 0 && i < (int)cand.size()) {
      CK(cg2_prepare_geo(P, cand[i]));
      m->tune2_source = "forced";
      return PARO_OK;
    }
  }
  const char* off = std::getenv("PARO_AUTOTUNE");
  CK(cg2_prepare_geo(P, cand[0]));
  m->tune2_source = "default";
  if ((off && off[0] == '0') || cand.size() < 2) return PARO_OK;
  int dev = 0;
  cudaDeviceProp prop{};
  CK(cudaGetDevice(&dev));
  CK(cudaGetDeviceProperties(&prop, dev));
  const std::string key = std::string(prop.name) + "|" + std::to_string(m->g.nx) + "x" + std::to_string(m->g.ny) +
                          "x" + std::to_string(m->g.nz) + "|Np" + std::to_string(P->args.Np) + "|cg2";
  const char* path = std::getenv("PARO_AUTOTUNE_CACHE");
  std::map<std::string, TuneEntry> cache;
  if (path) {
    cache = tune_cache_read(path);
    auto it = cache.find(key);
    if (it != cache.end())
      for (const K1Geom& G : cand)
        if (G.TX == it->second.TX && G.TY == it->second.TY && G.G4 * 4 == it->second.bw) {
          CK(cg2_prepare_geo(P, G));
          m->tune2_source = "cache";
          return PARO_OK;
        }
  }
  int chosen = -1, tried = 0;
  float us = 0.f;
  CK(cg2_autotune(P, m->st, 8, &chosen, &us, &tried));
  m->tune2_source = "timed";
  if (chosen >= 0 && path) {
    TuneEntry e;
    e.TX = cand[chosen].TX;
    e.TY = cand[chosen].TY;
    e.bw = cand[chosen].G4 * 4;
    e.us = us;
    cache[key] = e;
    tune_cache_write(path, cache);
  }
  return PARO_OK;
}

int make_plans(paro_mesh m, int Np) {
  free_plans(m);
  TRY(make_plan<double>(m, Np, &m->plan64, m->x, m->b, m->r, m->p0, m->q, m->dinv64, m->dt64, m->w64, m->coef64));
  if (m->precision == PARO_MIXED) {
    m->f32_layout = 0;
    TRY(make_plan<float>(m, Np, &m->plan32, m->x32, m->b32, m->r32, m->p32a, m->q32, m->dinv32, m->dt32, m->w32,
                         m->coef32, m->s32, m->r32b, m->q32b, m->s32b));
    CG2Plan* P = new CG2Plan();
    m->plan2 = P;
    P->nsm = m->nsm;
    P->dpitch = m->dpitch;
    P->dinv_tma = m->dt32;
    P->wcoef = m->w32;
    CG2Args& a = P->args;
    a.g = m->g;
    a.N = Np;
    a.Np = Np;
    a.x = m->x32;
    a.r[0] = m->b32;
    a.r[1] = m->r32;
    a.q[0] = m->q32;
    a.q[1] = m->q32b;
    a.p[0] = m->p32a;
    a.p[1] = m->s32;
    a.part = m->cg2part;
    a.pub = m->cg2part + (size_t)2 * 5 * kMaxGrid1 * Np;
    a.st = m->cgst;
    a.spin = kSpinLimit;
    a.inner = 1;
    TRY(set_f32_layout(m, 1));
    TRY(autotune_cg2(m, P));
    // the single-reduction kernel solves the float32 correction problems only where
    // the single-pass plan cannot run: its geometry is timed only then
    if (!P->ok) TRY(autotune_cg1(m, m->plan32));
    if (std::getenv("PARO_PRINT_PLAN"))
      std::fprintf(stderr, "paro single-pass CG plan: tile %dx%d, %d nodes a thread, block %d orbitals x %d, %d threads, "
                   "grid %d, smem %zu B, usable %d, geometry %s\n", P->geo.TX, P->geo.TY, P->geo.npt, P->geo.G4 * 4,
                   P->geo.nob,
                   P->geo.nthr * P->geo.G4, P->geo.grid, P->geo.smem, (int)P->ok, m->tune2_source);
  }
  return PARO_OK;
}

int ensure_workspace(paro_mesh m, int Np) {
  if (Np == m->Np_alloc) return PARO_OK;
  free_plans(m);
  // release the previous vector workspace
  void* olds[] = {m->u,    m->x,   m->b,   m->r,   m->p0,  m->q,     m->b32,    m->x32, m->r32,
                  m->p32a, m->q32, m->s32, m->r32b, m->q32b, m->s32b, m->fxh, m->fxl, m->fah, m->fal,   m->fbh,    m->fbl, m->gpart_ff, m->gpart_tc,
                  m->gpart, m->GA, m->GB,  m->C,   m->theta, m->eigwork, m->cgpart, m->cg2part};
  CK(cudaStreamSynchronize(m->st));
  for (void* p : olds) dfree(m, p);
  // the Gram workspaces below are allocated only for some Np: no stale pointers
  m->gpart_ff = nullptr;
  m->gpart_tc = nullptr;
  size_t n = (size_t)m->g.G * Np;
  TRY(dalloc(m, &m->u, n));
  TRY(dalloc(m, &m->x, n));
  TRY(dalloc(m, &m->b, n));
  TRY(dalloc(m, &m->r, n));
  TRY(dalloc(m, &m->p0, n));
  TRY(dalloc(m, &m->q, n));
  if (m->precision == PARO_MIXED) {
    TRY(dalloc(m, &m->b32, n));
    TRY(dalloc(m, &m->x32, n));
    TRY(dalloc(m, &m->r32, n));
    TRY(dalloc(m, &m->p32a, n));
    TRY(dalloc(m, &m->q32, n));
    TRY(dalloc(m, &m->s32, n));
    TRY(dalloc(m, &m->r32b, n));
    TRY(dalloc(m, &m->q32b, n));
    TRY(dalloc(m, &m->s32b, n));
    TRY(dalloc(m, &m->fxh, n));
    TRY(dalloc(m, &m->fxl, n));
    TRY(dalloc(m, &m->fah, n));
    TRY(dalloc(m, &m->fal, n));
    TRY(dalloc(m, &m->fbh, n));
    TRY(dalloc(m, &m->fbl, n));
    if (Np <= kTcMaxNp) TRY(dalloc(m, &m->gpart_tc, gram_tc_partial_doubles(m->g, Np)));
    if (Np <= 32) TRY(dalloc(m, &m->gpart_ff, gram_ff_partial_doubles(m->g, Np)));
  }
  TRY(dalloc(m, &m->gpart, gram_partial_doubles(m->g, Np)));
  TRY(dalloc(m, &m->GA, (size_t)Np * Np));
  TRY(dalloc(m, &m->GB, (size_t)Np * Np));
  TRY(dalloc(m, &m->C, (size_t)Np * Np));
  TRY(dalloc(m, &m->theta, (size_t)Np));
  TRY(dalloc(m, &m->eigwork, (size_t)4 * Np * Np));
  // per-CTA partials: up to 4 CTAs per SM, 3 values per orbital, two buffers
  TRY(dalloc(m, &m->cgpart, (size_t)2 * 3 * 4 * m->nsm * Np));
  // single-pass CG: 5 partial sums per orbital and CTA, two buffers
  TRY(dalloc(m, &m->cg2part, (size_t)2 * 5 * kMaxGrid1 * Np + (size_t)2 * 4 * Np));  // partials, then steps
  m->Np_alloc = Np;
  TRY(make_plans(m, Np));
  return PARO_OK;
}

int check_status(paro_mesh m, const char* where) {
  int* st = &m->cgst->status;
  CK(cudaMemcpyAsync(m->h_int, st, sizeof(int), cudaMemcpyDeviceToHost, m->st));
  CK(cudaStreamSynchronize(m->st));
  int bits = m->h_int[0];
  if (bits == 0) return PARO_OK;
  CK(cudaMemsetAsync(st, 0, sizeof(int), m->st));
  if (bits & kStatNonFinite) return fail(m, PARO_ERR_NONFINITE, std::string(where) + ": non-finite value in a reduction");
  if (bits & kStatNotSPD)
    return fail(m, PARO_ERR_NOT_SPD, std::string(where) + ": operator or Gram matrix not positive definite");
  if (bits & kStatTimeout)
    return fail(m, PARO_ERR_TIMEOUT, std::string(where) + ": a bounded device-side wait ran out");
  if (bits & kStatNotConverged)
    return fail(m, PARO_ERR_NOT_CONVERGED, std::string(where) + ": iteration limit reached");
  return PARO_OK;
}

int set_f32_layout(paro_mesh m, int want) {
  if (m->precision != PARO_MIXED || m->f32_layout == want) return PARO_OK;
  const size_t n = sizeof(float) * (size_t)m->g.G * m->Np_alloc;
  float* bufs[] = {m->b32, m->x32, m->r32, m->p32a, m->q32, m->s32, m->r32b, m->q32b, m->s32b};
  for (float* b : bufs)
    if (b) CK(cudaMemsetAsync(b, 0, n, m->st));
  m->f32_layout = want;
  return PARO_OK;
}

int read_n_active(paro_mesh m, int* out) {
  CK(cudaMemcpyAsync(m->h_int, &m->cgst->n_active, sizeof(int), cudaMemcpyDeviceToHost, m->st));
  CK(cudaStreamSynchronize(m->st));
  *out = m->h_int[0];
  return PARO_OK;
}

// Sum and max of the per-orbital CG counts of the last solve.
// PARO_TRACE=1 in the environment: one line per CG solve on stderr with the
// iteration count of every orbital (how unevenly the masked orbitals finish).
bool trace_on() {
  static const bool on = [] {
    const char* t = std::getenv("PARO_TRACE");
    return t != nullptr && t[0] == '1';
  }();
  return on;
}

int read_iters(paro_mesh m, int N, long long* sum, int* mx) {
  CK(cudaMemcpyAsync(m->h_int, m->cgst->iters, sizeof(int) * N, cudaMemcpyDeviceToHost, m->st));
  CK(cudaStreamSynchronize(m->st));
  long long s = 0;
  int x = 0;
  for (int i = 0; i < N; ++i) {
    s += m->h_int[i];
    if (m->h_int[i] > x) x = m->h_int[i];
  }
  *sum = s;
  *mx = x;
  if (trace_on()) {
    std::fprintf(stderr, "paro-trace cg N=%d iters:", N);
    for (int i = 0; i < N; ++i) std::fprintf(stderr, " %d", m->h_int[i]);
    std::fprintf(stderr, "\n");
  }
  return PARO_OK;
}

// Sum the recorded start/stop pairs (the stream has been synchronised).
int drain_profile(paro_mesh m) {
  for (int i = 0; i < m->pev_used; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, m->pev[2 * i], m->pev[2 * i + 1]));
    m->prof_ms += ms;
    m->prof_launches += 1;
  }
  m->pev_used = 0;
  return PARO_OK;
}

cudaError_t launch_apply_T(paro_mesh m, CGPlan<double>* P) {
  return launch_apply_f64(m->g, P->args.Np, m->coef64, nullptr, 0.0, P->args.x, P->args.q, nullptr, m->st);
}
cudaError_t launch_apply_T(paro_mesh m, CGPlan<float>* P) {
  return launch_apply_f32(m->g, P->args.Np, m->coef32, P->args.x, P->args.q, m->st);
}

// One batched CG solve with the plan P: A x = b from x (warm) or from x = 0.
// Graph mode: one graph launch (init + device-side while loop).  Profile
// mode: the same kernels launched from the host with CUDA events around every
// operator (K1) launch; the host tests the active count every check_every.
template <typename T>
int run_cg(paro_mesh m, CGPlan<T>* P, int N, bool warm, double tol, int maxit, int check_every, long long* it_sum,
           int* it_max) {
  P->args.N = N;
  // controls
  // the previous solve's copies from h_ctl completed: every run_cg ends with a stream synchronisation
  m->h_ctl[0] = tol;
  int* ctl_int = reinterpret_cast<int*>(m->h_ctl + 1);
  ctl_int[0] = maxit;
  CK(cudaMemcpyAsync(&m->cgst->tol, m->h_ctl, sizeof(double), cudaMemcpyHostToDevice, m->st));
  CK(cudaMemcpyAsync(&m->cgst->maxit, ctl_int, sizeof(int), cudaMemcpyHostToDevice, m->st));
  // float32: the whole loop in one cooperative launch (profile 1: CUDA events
  // around it).  float64 keeps the graph (or host-driven) loop of two kernels per
  // iteration, which runs its longer float64 passes with less synchronisation.
  if constexpr (sizeof(T) == 4) {
    // float32: the single-reduction CG, one cooperative launch per correction solve
    if (P->cg1_ok && m->profile != 2) {
      if (warm) LAUNCH(1, launch_apply_T(m, P));
      LAUNCH(1, cg_launch_init<T>(P, m->st, !warm));
      if (m->profile) CK(cudaEventRecord(m->pev[2 * m->pev_used], m->st));
      LAUNCH(1, cg_launch_cg1(P, m->st));
      if (m->profile) {
        CK(cudaEventRecord(m->pev[2 * m->pev_used + 1], m->st));
        m->pev_used++;
      }
      TRY(read_iters(m, N, it_sum, it_max));  // synchronises the stream
      if (m->profile) TRY(drain_profile(m));
      return PARO_OK;
    }
  }
  if (P->coop_ok && m->profile != 2 && sizeof(T) == 4) {
    if (warm) LAUNCH(1, launch_apply_T(m, P));
    LAUNCH(1, cg_launch_init<T>(P, m->st, !warm));
    if (m->profile) CK(cudaEventRecord(m->pev[2 * m->pev_used], m->st));
    LAUNCH(1, cg_launch_loop<T>(P, m->st));
    if (m->profile) {
      CK(cudaEventRecord(m->pev[2 * m->pev_used + 1], m->st));
      m->pev_used++;
    }
    TRY(read_iters(m, N, it_sum, it_max));  // synchronises the stream
    if (m->profile) TRY(drain_profile(m));
    return PARO_OK;
  }
  if (!m->profile) {
    // N is baked into the graph arguments: rebuild when it changes
    cudaGraphExec_t* ex = warm ? &P->exec_warm : &P->exec_zero;
    if (P->graph_N != N) {
      if (P->exec_warm) cudaGraphExecDestroy(P->exec_warm);
      if (P->exec_zero) cudaGraphExecDestroy(P->exec_zero);
      P->exec_warm = P->exec_zero = nullptr;
      P->graph_N = N;
    }
    if (!*ex) {
      cudaError_t e = cg_build_graph<T>(P, m->st, warm);
      if (e != cudaSuccess) return fail(m, PARO_ERR_CUDA, std::string("CG graph: ") + cudaGetErrorString(e));
    }
    CK(cudaGraphLaunch(*ex, m->st));
    TRY(read_iters(m, N, it_sum, it_max));
    m->launches += (warm ? 1 : 0) + 1 + 2LL * (*it_max);
    return PARO_OK;
  }
  if (warm) LAUNCH(1, launch_apply_T(m, P));
  LAUNCH(1, cg_launch_init<T>(P, m->st, !warm));
  int nact = 0;
  TRY(read_n_active(m, &nact));
  int done = 0;
  if (check_every > kProfPairs) check_every = kProfPairs;
  while (nact > 0 && done < maxit) {
    int k = check_every;
    if (k > maxit - done) k = maxit - done;
    for (int i = 0; i < k; ++i) {
      CK(cudaEventRecord(m->pev[2 * m->pev_used], m->st));
      LAUNCH(1, cg_launch_k1<T>(P, m->st));
      CK(cudaEventRecord(m->pev[2 * m->pev_used + 1], m->st));
      m->pev_used++;
      LAUNCH(1, cg_launch_k2<T>(P, m->st));
    }
    done += k;
    TRY(read_n_active(m, &nact));
    TRY(drain_profile(m));
  }
  TRY(read_iters(m, N, it_sum, it_max));
  return PARO_OK;
}

// Multigrid hierarchy for Np-wide level vectors: grids and storage on first use
// (again when Np changes), Galerkin coefficients and Jacobi weights whenever the
// operator changed since the last build.
int ensure_mg(paro_mesh m, int Np) {
  MGHier& h = m->mg;
  if (h.nlev == 0 || h.Np != Np) {
    CK(cudaStreamSynchronize(m->st));
    for (int l = 1; l < h.nlev; ++l) {
      MGLevel& L = h.lev[l];
      void* olds[] = {L.coef64, L.coef32, L.dinv32, L.b, L.t, L.x, L.y};
      for (void* o : olds) dfree(m, o);
      L = MGLevel{};
    }
    Grid gs[kMaxMGLevels];
    const int nc = mg_plan_levels(m->g, gs, kMaxMGLevels);
    h.lev[0] = MGLevel{};
    h.lev[0].g = m->g;
    for (int l = 1; l <= nc; ++l) {
      MGLevel& L = h.lev[l];
      L.g = gs[l - 1];
      const size_t G = (size_t)L.g.G;
      TRY(dalloc(m, &L.coef64, 27 * G));
      TRY(dalloc(m, &L.coef32, 27 * G));
      TRY(dalloc(m, &L.dinv32, G));
      TRY(dalloc(m, &L.b, G * Np));
      TRY(dalloc(m, &L.t, G * Np));
      TRY(dalloc(m, &L.x, G * Np));
      TRY(dalloc(m, &L.y, G * Np));
    }
    if (!h.rho_bits) TRY(dalloc(m, &h.rho_bits, kMaxMGLevels));
    h.nlev = nc + 1;
    h.Np = Np;
    h.built = false;
  }
  MGLevel& F = h.lev[0];
  F.coef64 = m->coef64;
  F.coef32 = m->coef32;
  F.dinv32 = m->dinv32;
  if (h.built) return PARO_OK;
  CK(cudaMemsetAsync(h.rho_bits, 0, sizeof(unsigned long long) * kMaxMGLevels, m->st));
  for (int l = 0; l < h.nlev; ++l) {
    if (l > 0)
      LAUNCH(1, launch_mg_galerkin(h.lev[l - 1].g, h.lev[l].g, h.lev[l - 1].coef64, h.lev[l].coef64,
                                   h.lev[l].coef32, h.lev[l].dinv32, m->st));
    LAUNCH(1, launch_mg_rho(h.lev[l].g, h.lev[l].coef64, h.rho_bits + l, m->st));
  }
  static_assert(kMaxMGLevels * sizeof(unsigned long long) <= kMaxN * sizeof(double), "h_dbl staging");
  CK(cudaMemcpyAsync(m->h_dbl, h.rho_bits, sizeof(unsigned long long) * h.nlev, cudaMemcpyDeviceToHost, m->st));
  CK(cudaStreamSynchronize(m->st));
  for (int l = 0; l < h.nlev; ++l) {
    const double rho = m->h_dbl[l];  // the bit pattern of the bound, a positive double
    if (!(rho > 0.0) || !std::isfinite(rho)) return fail(m, PARO_ERR_NOT_SPD, "multigrid: non-positive diagonal");
    h.lev[l].rho = rho;
    h.lev[l].omega = (float)std::fmin(1.0, 4.0 / (3.0 * rho));
  }
  h.built = true;
  return PARO_OK;
}

// One MG-preconditioned float32 CG solve A x = b from x = 0 on the plan P (x, b,
// r, p, s, w = q; u = r2; V-cycle scratch s2, q2), per-orbital masks as in the
// Jacobi CG; the host tests the active count every check_every iterations.
int run_mg(paro_mesh m, CGPlan<float>* P, int N, double tol, int maxit, int check_every, int nu, int nu_c,
           long long* it_sum, int* it_max) {
  P->args.N = N;
  TRY(ensure_mg(m, P->args.Np));
  m->h_ctl[0] = tol;
  int* ctl_int = reinterpret_cast<int*>(m->h_ctl + 1);
  ctl_int[0] = maxit;
  CK(cudaMemcpyAsync(&m->cgst->tol, m->h_ctl, sizeof(double), cudaMemcpyHostToDevice, m->st));
  CK(cudaMemcpyAsync(&m->cgst->maxit, ctl_int, sizeof(int), cudaMemcpyHostToDevice, m->st));
  LAUNCH(1, cg_launch_init<float>(P, m->st, true));
  int nact = 0;
  TRY(read_n_active(m, &nact));
  int done = 0;
  while (nact > 0 && done < maxit) {
    int k = check_every;
    if (k > maxit - done) k = maxit - done;
    for (int i = 0; i < k; ++i) {
      long long nl = 0;
      CK(mg_vcycle(m->mg, P->args.Np, P->args.r, P->args.r2, P->args.s2, P->args.q2, m->cgst->active, nu, nu_c,
                   m->st, &nl));
      m->launches += nl;
      LAUNCH(1, mg_launch_wdots(P, m->coef32, m->st));
      LAUNCH(1, mg_launch_update(P, m->st));
    }
    done += k;
    TRY(read_n_active(m, &nact));
  }
  TRY(read_iters(m, N, it_sum, it_max));
  return PARO_OK;
}

int check_precond(paro_mesh m, const paro_params& p) {
  if (p.precond != PARO_PRECOND_JACOBI && p.precond != PARO_PRECOND_MG)
    return fail(m, PARO_ERR_ARG, "unknown preconditioner");
  if (p.precond == PARO_PRECOND_MG) {
    if (m->g.graded) return fail(m, PARO_ERR_ARG, "the multigrid preconditioner needs a uniform mesh");
    if (m->precision != PARO_MIXED)
      return fail(m, PARO_ERR_ARG, "the multigrid preconditioner runs in the float32 solves of a PARO_MIXED handle");
    if (p.mg_nu < 1 || p.mg_nu > 8 || p.mg_coarse_sweeps < 1 || p.mg_coarse_sweeps > 64)
      return fail(m, PARO_ERR_ARG, "mg_nu must be in [1, 8] and mg_coarse_sweeps in [1, 64]");
  }
  return PARO_OK;
}

// ---------------------------------------------------------------------------
// Batches: the correction solves of every system in one launch.
// Each system of a batch runs its own ParO loop (paro_iterate) in a host thread
// of its own.  When a system reaches a float32 correction solve it records an
// event on its stream and waits here; once every system still iterating has
// arrived, the last one makes the batch stream wait on all their events,
// launches the batched single-pass CG over them (the systems' bits in the
// launch mask), records `done`, and every system's stream waits on it.  A
// system that finishes its loop leaves, and a launch is issued for the others
// if they are all waiting.  Systems therefore advance in lockstep at the
// granularity of a correction solve, while everything between two solves
// (right-hand sides, refinement residuals, Rayleigh-Ritz) runs on each system's
// own stream, overlapping the others.
// ---------------------------------------------------------------------------
struct BatchCG {
  std::mutex mu;
  std::condition_variable cv;
  CG2BPlan plan;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<cudaEvent_t> ready;
  std::vector<paro_mesh> ms;
  std::vector<char> waiting_flag;
  std::vector<unsigned> spin;
  int live = 0, waiting = 0;
  unsigned long long gen = 0;
  cudaError_t launch_err = cudaSuccess;
  long long launches = 0;
  int chosen = -1, tried = 0;
  float best_us = 0.f;
  std::vector<CG2BSysDesc> desc;  // what the plan was built over (reuse check)
};

void bcg_launch_locked(BatchCG* B) {
  unsigned long long mask[kMaxBatchSys / 64] = {0, 0, 0, 0};
  unsigned spin = kSpinLimit;
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < B->ms.size(); ++i) {
    if (!B->waiting_flag[i]) continue;
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->st, B->ready[i], 0);
    mask[i >> 6] |= 1ull << (i & 63);
    if (B->spin[i] < spin) spin = B->spin[i];
    B->waiting_flag[i] = 0;
  }
  if (e == cudaSuccess) e = cg2b_launch(&B->plan, mask, spin, B->st);
  if (e == cudaSuccess) e = cudaEventRecord(B->done, B->st);
  B->launch_err = e;
  ++B->launches;
  B->waiting = 0;
  ++B->gen;
  B->cv.notify_all();
}

// Replaces the single-system launch in the refinement sweeps of a batch member.
int batch_cg_solve(paro_mesh m, unsigned spin) {
  BatchCG* B = m->bcg;
  std::unique_lock<std::mutex> lk(B->mu);
  const int i = m->bcg_index;
  CK(cudaEventRecord(B->ready[i], m->st));
  B->waiting_flag[i] = 1;
  B->spin[i] = spin;
  ++B->waiting;
  const unsigned long long g0 = B->gen;
  if (B->waiting == B->live) bcg_launch_locked(B);
  else B->cv.wait(lk, [&] { return B->gen != g0; });
  // the next launch needs this system to arrive again: B->done and launch_err
  // still describe the launch that ran its solve
  if (B->launch_err != cudaSuccess)
    return fail(m, PARO_ERR_CUDA, std::string("batched CG launch: ") + cudaGetErrorString(B->launch_err));
  CK(cudaStreamWaitEvent(m->st, B->done, 0));
  return PARO_OK;
}

// Step 3 on the packed buffers: u (current orbitals) -> x (source solutions).
// Mixed-precision solve of A x = b for N columns: x (float64, padded) holds the
// initial guess, b is given as a float-float pair in fah/fal.  Each sweep forms
// r = b - A x in float-float arithmetic (float64-accurate), stops the columns with
// |r| <= solve_tol |b|, solves A d = r to inner_tol with the float32 CG and adds d.
// The same refinement around the single-pass CG (group-major correction
// vectors).  Sweeps run without host synchronisation: residual (its float32
// rounding goes straight into the CG's right-hand side, converged orbitals are
// flagged skip), correction solve (a launch with no active orbital returns at
// once), x += d with the float-float split of the new x; two sweeps, then a
// residual whose active count the host reads, and one sweep more at a time
// while orbitals remain open.  fxh/fxl hold the split of x on entry.
// x = u when no refinement update wrote x (no sweep ran, or an early return):
// every return of the single-pass refinement leaves x materialised.
struct MaterialiseX {
  paro_mesh m;
  ~MaterialiseX() {
    if (!m->x_pending_u) return;
    if (cudaMemcpyAsync(m->x, m->u, sizeof(double) * m->g.G * m->Np_alloc, cudaMemcpyDeviceToDevice, m->st) !=
        cudaSuccess)
      (void)cudaGetLastError();
    m->x_pending_u = false;
  }
};

int refine_solve_cg2(paro_mesh m, int N, const paro_params& p, paro_stats* st, double itol, bool rr_next) {
  MaterialiseX mx{m};
  const int Np = m->Np_alloc;
  Grid& g = m->g;
  CG2Plan* P = m->plan2;
  CGState rs = cg_state(m, true);
  if (p.pcg_maxit < 1) return fail(m, PARO_ERR_ARG, "pcg_maxit must be at least 1");
  TRY(set_f32_layout(m, 1));
  P->args.N = N;
  P->args.spin = p.wait_polls > 0 ? (unsigned)p.wait_polls : kSpinLimit;
  m->h_ctl[0] = itol;
  int* ctl_int = reinterpret_cast<int*>(m->h_ctl + 1);
  ctl_int[0] = p.pcg_maxit;
  CK(cudaMemcpyAsync(&m->cgst->tol, m->h_ctl, sizeof(double), cudaMemcpyHostToDevice, m->st));
  CK(cudaMemcpyAsync(&m->cgst->maxit, ctl_int, sizeof(int), cudaMemcpyHostToDevice, m->st));
  CK(cudaMemsetAsync(&m->cgst->it_sum, 0, sizeof(long long), m->st));
  CK(cudaMemsetAsync(&m->cgst->it_max, 0, sizeof(int), m->st));
  if (!m->x_split_fresh) LAUNCH(1, launch_split_ff((long long)g.G * Np, m->x, m->fxh, m->fxl, m->st));
  m->x_split_fresh = false;
  int sweep = 0;
  for (;;) {
    int batch = sweep == 0 ? 2 : 1;
    if (batch > p.max_refine - sweep) batch = p.max_refine - sweep;
    for (int b = 0; b < batch; ++b) {
      LAUNCH(1, launch_refine_residual_ff(g, N, Np, m->wAh, m->wAl, m->fxh, m->fxl, m->fah, m->fal, m->b32, rs,
                                          p.solve_tol, m->st, 1));
      if (st) st->stencil_applies += N;
      if (m->profile) CK(cudaEventRecord(m->pev[2 * m->pev_used], m->st));
      if (m->bcg) {
        TRY(batch_cg_solve(m, P->args.spin));
        m->launches += 1;
      } else {
        LAUNCH(1, cg2_launch(P, m->st));
      }
      if (m->profile) {
        CK(cudaEventRecord(m->pev[2 * m->pev_used + 1], m->st));
        m->pev_used++;
      }
      if (trace_on()) {
        long long s0 = 0;
        int mx = 0;
        TRY(read_iters(m, N, &s0, &mx));
      }
      LAUNCH(1, launch_refine_update_split(g, Np, m->x_pending_u ? m->u : m->x, m->x, m->x32, m->cgst->skip, m->fxh,
                                           m->fxl, m->st));
      m->x_pending_u = false;
      ++sweep;
    }
    if (rr_next) {
      // a Rayleigh-Ritz step on this x follows: M x, then H x with the check
      // r = b - H x - sigma M x, H x written over b (both applies of that step)
      LAUNCH(1, apply_M_ff(m, Np, m->fxh, m->fxl, nullptr, nullptr, m->fbh, m->fbl));
      LAUNCH(1, launch_refine_check_hff(g, N, Np, m->wHh, m->wHl, m->fxh, m->fxl, m->fbh, m->fbl, m->sigma, m->fah,
                                        m->fal, rs, p.solve_tol, m->st));
    } else {
      LAUNCH(1, launch_refine_residual_ff(g, N, Np, m->wAh, m->wAl, m->fxh, m->fxl, m->fah, m->fal, nullptr, rs,
                                          p.solve_tol, m->st, 1));
    }
    if (st) st->stencil_applies += N;
    // the open count and the status word in one round trip (with the statistics'
    // iteration counts and residual norms when they are asked for); a failed
    // correction solve (timeout, non-finite value, indefinite operator) ends the
    // refinement
    CK(cudaMemcpyAsync(m->h_int, &m->cgst->n_active, sizeof(int), cudaMemcpyDeviceToHost, m->st));
    CK(cudaMemcpyAsync(m->h_int + 1, &m->cgst->status, sizeof(int), cudaMemcpyDeviceToHost, m->st));
    if (st) {
      CK(cudaMemcpyAsync(m->h_int + 2, &m->cgst->it_sum, sizeof(long long), cudaMemcpyDeviceToHost, m->st));
      CK(cudaMemcpyAsync(m->h_int + 4, &m->cgst->it_max, sizeof(int), cudaMemcpyDeviceToHost, m->st));
      CK(cudaMemcpyAsync(m->h_dbl, m->dscal + S_RRR * kMaxN, sizeof(double) * N, cudaMemcpyDeviceToHost, m->st));
      CK(cudaMemcpyAsync(m->h_dbl + kMaxN, m->dscal + S_RBB * kMaxN, sizeof(double) * N, cudaMemcpyDeviceToHost,
                         m->st));
    }
    CK(cudaStreamSynchronize(m->st));
    const int open = m->h_int[0];
    if (m->h_int[1] != 0) TRY(check_status(m, "orbital_solve (float32 correction)"));
    if (m->profile) TRY(drain_profile(m));
    if (open == 0) {
      m->hm_ready = rr_next;
      break;
    }
    if (rr_next) {
      // b was overwritten by H x: b = (lambda + sigma) M u again, u's split staged in fbh/fbl
      LAUNCH(1, launch_split_ff((long long)g.G * Np, m->u, m->fbh, m->fbl, m->st));
      LAUNCH(1, apply_M_ff(m, Np, m->fbh, m->fbl, m->dscal + S_SCALE * kMaxN, nullptr, m->fah, m->fal));
    }
    if (sweep >= p.max_refine) {
      if (st) st->refine_sweeps = sweep;
      TRY(check_status(m, "orbital_solve"));
      m->err = "mixed refinement: max_refine sweeps reached";
      return PARO_ERR_NOT_CONVERGED;
    }
  }
  TRY(check_status(m, "orbital_solve (float32 correction)"));
  m->x_split_valid = true;  // every sweep ended with x and its split updated together
  if (st) {
    long long its = 0;
    std::memcpy(&its, m->h_int + 2, sizeof(its));
    const int imax = m->h_int[4];
    m->relres_staged = true;  // h_dbl holds the final ||r||^2 and ||b||^2
    st->cg_iters += its;
    st->cg_iters_f32 += its;
    st->cg_iters_max = imax;
    st->refine_sweeps = sweep;
    st->stencil_applies += its;
  }
  return PARO_OK;
}

int refine_solve(paro_mesh m, int N, const paro_params& p, paro_stats* st, bool rr_next = false) {
  TRY(check_precond(m, p));
  // inner tolerance: given, or sqrt(solve_tol) so that two sweeps reach solve_tol
  // (clamped to what float32 CG reliably attains and to a useful minimum)
  const double itol = p.inner_tol > 0.0 ? p.inner_tol : std::fmin(1e-3, std::fmax(1e-6, std::sqrt(p.solve_tol)));
  if (p.precond == PARO_PRECOND_JACOBI && m->plan2 && m->plan2->ok && m->profile != 2)
    return refine_solve_cg2(m, N, p, st, itol, rr_next);
  if (m->x_pending_u) {
    CK(cudaMemcpyAsync(m->x, m->u, sizeof(double) * m->g.G * m->Np_alloc, cudaMemcpyDeviceToDevice, m->st));
    m->x_pending_u = false;
  }
  m->x_split_fresh = false;
  TRY(set_f32_layout(m, 0));
  const int Np = m->Np_alloc;
  Grid& g = m->g;
  CGState rs = cg_state(m, true);
  int sweep = 0;
  long long its32 = 0;
  int maxit_seen = 0;
  for (;;) {
    // r = b - A x, float64-accurate (float-float arithmetic); its float32 rounding
    // is the correction right-hand side
    LAUNCH(1, launch_split_ff((long long)g.G * Np, m->x, m->fxh, m->fxl, m->st));
    LAUNCH(1, launch_refine_residual_ff(g, N, Np, m->wAh, m->wAl, m->fxh, m->fxl, m->fah, m->fal, m->b32, rs,
                                        p.solve_tol, m->st));
    if (st) st->stencil_applies += N;
    int open = 0;
    TRY(read_n_active(m, &open));
    if (open == 0) break;
    if (sweep >= p.max_refine) {
      if (st) st->refine_sweeps = sweep;
      TRY(check_status(m, "orbital_solve"));
      m->err = "mixed refinement: max_refine sweeps reached";
      return PARO_ERR_NOT_CONVERGED;
    }
    long long i1 = 0;
    int imx = 0;
    if (p.precond == PARO_PRECOND_MG)
      TRY(run_mg(m, m->plan32, N, itol, p.pcg_maxit, p.check_every, p.mg_nu, p.mg_coarse_sweeps, &i1, &imx));
    else
      TRY(run_cg<float>(m, m->plan32, N, false, itol, p.pcg_maxit, p.check_every, &i1, &imx));
    // an inner limit is not fatal: refinement carries on from the partial correction
    int* stw = &m->cgst->status;
    CK(cudaMemcpyAsync(m->h_int, stw, sizeof(int), cudaMemcpyDeviceToHost, m->st));
    CK(cudaStreamSynchronize(m->st));
    if (m->h_int[0] & kStatNotConverged) {
      m->h_int[0] &= ~kStatNotConverged;
      CK(cudaMemcpyAsync(stw, m->h_int, sizeof(int), cudaMemcpyHostToDevice, m->st));
    }
    TRY(check_status(m, "orbital_solve (float32 correction)"));
    LAUNCH(1, launch_refine_update(g, Np, m->x, m->x32, m->cgst->skip, m->st));
    its32 += i1;
    if (imx > maxit_seen) maxit_seen = imx;
    ++sweep;
  }
  if (st) {
    st->cg_iters += its32;
    st->cg_iters_f32 += its32;
    st->cg_iters_max = maxit_seen;
    st->refine_sweeps = sweep;
    st->stencil_applies += its32;
  }
  return PARO_OK;
}

int solve_packed(paro_mesh m, int N, const double* lam, const paro_params& p, paro_stats* st, bool rr_next = false) {
  const int Np = m->Np_alloc;
  Grid& g = m->g;
  m->x_split_valid = false;
  m->hm_ready = false;
  m->relres_staged = false;
  // b = (lambda + sigma) M u
  for (int i = 0; i < Np; ++i) m->h_dbl[i] = i < N ? lam[i] + m->sigma : 0.0;
  double* scale = m->dscal + S_SCALE * kMaxN;
  CK(cudaMemcpyAsync(scale, m->h_dbl, sizeof(double) * Np, cudaMemcpyHostToDevice, m->st));
  if (m->precision == PARO_MIXED) {
    // float-float mass apply (float64 accuracy on the float32 pipes); b stays as a
    // hi/lo pair in fah/fal for the solve (the Rayleigh-Ritz step reuses them after)
    LAUNCH(1, launch_split_ff((long long)g.G * Np, m->u, m->fxh, m->fxl, m->st));
    LAUNCH(1, apply_M_ff(m, Np, m->fxh, m->fxl, scale, nullptr, m->fah, m->fal));
  } else {
    LAUNCH(1, apply_M_f64(m, Np, m->u, m->b, scale));
  }
  if (m->precision == PARO_MIXED) {
    m->x_pending_u = true;  // x = u: the refinement materialises it
  } else {
    CK(cudaMemcpyAsync(m->x, m->u, sizeof(double) * g.G * Np, cudaMemcpyDeviceToDevice, m->st));
  }
  m->x_split_fresh = m->precision == PARO_MIXED;  // fxh/fxl = split(u) = split(x)
  long long its = 0;
  int itmax = 0;
  TRY(check_precond(m, p));
  if (m->precision == PARO_FP64) {
    CK(cudaMemsetAsync(m->cgst->skip, 0, sizeof(int) * kMaxN, m->st));
    TRY(run_cg<double>(m, m->plan64, N, true, p.solve_tol, p.pcg_maxit, p.check_every, &its, &itmax));
    if (st) {
      st->cg_iters += its;
      st->cg_iters_max = itmax;
      st->refine_sweeps = 0;
      st->stencil_applies += its + N;
    }
    // float64 true residual for the statistics
    CGState rs = cg_state(m, true);
    LAUNCH(1, launch_refine_residual(g, N, Np, m->coef64, m->x, m->b, nullptr, rs, p.solve_tol, m->st));
  } else {
    TRY(refine_solve(m, N, p, st, rr_next));
  }
  if (st) {
    if (!m->relres_staged) {
      double* rr = m->dscal + S_RRR * kMaxN;
      double* bb = m->dscal + S_RBB * kMaxN;
      CK(cudaMemcpyAsync(m->h_dbl, rr, sizeof(double) * N, cudaMemcpyDeviceToHost, m->st));
      CK(cudaMemcpyAsync(m->h_dbl + kMaxN, bb, sizeof(double) * N, cudaMemcpyDeviceToHost, m->st));
      CK(cudaStreamSynchronize(m->st));
    }
    m->relres_staged = false;
    double worst = 0.0;
    for (int i = 0; i < N; ++i) {
      double b = m->h_dbl[kMaxN + i];
      double rel = b > 0 ? std::sqrt(m->h_dbl[i] / b) : std::sqrt(m->h_dbl[i]);
      if (rel > worst) worst = rel;
    }
    st->max_relres = worst;
  }
  return check_status(m, "orbital_solve");
}

// Gram precision of one Rayleigh-Ritz step on a mixed handle.
enum RRMode {
  kRRFast,      // tensor-core Grams (~1e-9 of |x| |y|; float64 Grams where Np > kTcMaxNp)
  kRRAccurate,  // float-float Grams (Np <= 32), float64 Grams otherwise
  kRRFP64,      // float64 Grams and rotation
};

// The ParO loop of a mixed handle takes the fast Grams while the Ritz values
// still move by more than this (relative to max(1, |lambda|_max)); below it the
// tensor-core Grams' rounding would show in |delta lambda|, so the loop switches
// to the accurate Grams for the last iterations.
constexpr double kRRSwitchRel = 1e-6;

RRMode next_rr_mode(paro_mesh m, RRMode cur, double dl, const std::vector<double>& lam) {
  if (m->precision != PARO_MIXED || cur != kRRFast) return cur;
  double scale = 1.0;
  for (double v : lam) scale = std::fmax(scale, std::fabs(v));
  return dl < kRRSwitchRel * scale ? kRRAccurate : kRRFast;
}

// Step 4 on packed buffers: src -> dst (Ritz vectors), lam (host, ascending).
// kRRFP64 is used for the start on user guesses, whose overlap matrix can be
// ill-conditioned far beyond what the mixed path's Grams resolve (their error is
// amplified by cond(X^T M X)); inside the ParO loop X stays near M-orthonormal.
// src_split: fxh/fxl already hold the float-float split of src.
// Host check of an overlap matrix G (N x N, leading dimension ld) before the
// fast Rayleigh-Ritz trusts Grams from 24-bit inputs: with G scaled to unit
// diagonal, its Cholesky factor L exists and trace(G^-1) = ||L^-1||_F^2 stays
// below 4 N (near M-orthonormal X gives ~N).  The Grams' relative error is
// amplified by ||G^-1|| <= trace(G^-1), so raw, nearly dependent guesses fail
// the check.
static bool overlap_well_conditioned(const std::vector<double>& G, int N, int ld) {
  std::vector<double> L((size_t)N * N, 0.0), d(N);
  for (int i = 0; i < N; ++i) {
    const double gii = G[(size_t)i * ld + i];
    if (!(gii > 0.0) || !std::isfinite(gii)) return false;
    d[i] = 1.0 / std::sqrt(gii);
  }
  for (int j = 0; j < N; ++j) {
    double s = G[(size_t)j * ld + j] * d[j] * d[j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * N + k] * L[(size_t)j * N + k];
    if (!(s > 0.0)) return false;
    const double ljj = std::sqrt(s);
    L[(size_t)j * N + j] = ljj;
    for (int i = j + 1; i < N; ++i) {
      double t = 0.5 * (G[(size_t)i * ld + j] + G[(size_t)j * ld + i]) * d[i] * d[j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * N + k] * L[(size_t)j * N + k];
      L[(size_t)i * N + j] = t / ljj;
    }
  }
  // ||L^-1||_F^2, column by column of L^-1 (forward substitution)
  double tr = 0.0;
  std::vector<double> y(N);
  for (int c = 0; c < N; ++c) {
    for (int i = 0; i < N; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) t -= L[(size_t)i * N + k] * y[k];
      y[i] = i < c ? 0.0 : t / L[(size_t)i * N + i];
      tr += y[i] * y[i];
    }
  }
  return std::isfinite(tr) && tr <= 4.0 * N;
}

int rr_packed(paro_mesh m, int N, const double* src, double* dst, double* lam, RRMode mode = kRRFast,
              const int* clus = nullptr, bool src_split = false, bool guard = false) {
  const int Np = m->Np_alloc;
  Grid& g = m->g;
  m->x_split_valid = false;
  // H X and M X already formed by the refinement's closing check on this X
  const bool hm = m->hm_ready && src_split && src == m->x;
  m->hm_ready = false;
  const bool mixed = m->precision == PARO_MIXED;
  const bool tc = mixed && mode == kRRFast && m->gpart_tc != nullptr;
  const bool ff = mixed && mode == kRRAccurate && m->gpart_ff != nullptr;
  if (tc) {
    // float-float X, HX and MX; both Grams on the tensor cores from their hi parts
    // (exact BF16 digit products, float-float across 128-node chunks)
    if (!src_split) LAUNCH(1, launch_split_ff((long long)g.G * Np, src, m->fxh, m->fxl, m->st));
    if (!hm) {
      LAUNCH(1, launch_ff_apply(g, Np, m->wHh, m->wHl, nullptr, m->fxh, m->fxl, nullptr, nullptr, m->fah, m->fal,
                                m->st));
      LAUNCH(1, apply_M_ff(m, Np, m->fxh, m->fxl, nullptr, nullptr, m->fbh, m->fbl));
    }
    int nch = 0;
    if (Np <= 32) {
      // both Grams in one launch (X loaded and converted once)
      double* partB = m->gpart_tc + gram_tc_partial_doubles(g, Np) / 2;
      LAUNCH(1, launch_gram_tc_pair(g, Np, m->fxh, m->fah, m->fbh, m->gpart_tc, partB, &nch, &m->cgst->status,
                                    m->st));
      LAUNCH(1, launch_gram_reduce1(Np, nch, m->gpart_tc, m->GA, m->st));
      LAUNCH(1, launch_gram_reduce1(Np, nch, partB, m->GB, m->st));
    } else {
      LAUNCH(1, launch_gram_tc(g, Np, m->fxh, m->fah, m->gpart_tc, &nch, &m->cgst->status, m->st));
      LAUNCH(1, launch_gram_reduce1(Np, nch, m->gpart_tc, m->GA, m->st));
      LAUNCH(1, launch_gram_tc(g, Np, m->fxh, m->fbh, m->gpart_tc, &nch, &m->cgst->status, m->st));
      LAUNCH(1, launch_gram_reduce1(Np, nch, m->gpart_tc, m->GB, m->st));
    }
    if (guard) {
      // arbitrary X (the public call): an overlap too ill-conditioned for these
      // Grams takes the float64 step instead
      std::vector<double> hG((size_t)Np * Np);
      CK(cudaMemcpyAsync(hG.data(), m->GB, sizeof(double) * Np * Np, cudaMemcpyDeviceToHost, m->st));
      CK(cudaStreamSynchronize(m->st));
      if (!overlap_well_conditioned(hG, N, Np)) {
        if (trace_on()) std::fprintf(stderr, "paro rayleigh_ritz: ill-conditioned overlap, float64 step\n");
        return rr_packed(m, N, src, dst, lam, kRRFP64, clus, false);
      }
    }
    ++m->rr_tc;
  } else if (ff) {
    // float-float: HX and MX as hi/lo arrays, both Grams and the rotation from the split X
    if (!src_split) LAUNCH(1, launch_split_ff((long long)g.G * Np, src, m->fxh, m->fxl, m->st));
    if (!hm) {
      LAUNCH(1, launch_ff_apply(g, Np, m->wHh, m->wHl, nullptr, m->fxh, m->fxl, nullptr, nullptr, m->fah, m->fal,
                                m->st));
      LAUNCH(1, apply_M_ff(m, Np, m->fxh, m->fxl, nullptr, nullptr, m->fbh, m->fbl));
    }
    int nch = 0;
    LAUNCH(1, launch_gram2_ff(g, Np, m->fxh, m->fxl, m->fah, m->fal, m->fbh, m->fbl, m->gpart_ff, &nch, m->st));
    LAUNCH(1, launch_gram_reduce(Np, nch, m->gpart_ff, m->GA, m->GB, m->st));
  } else {
    LAUNCH(1, apply_H_f64(m, Np, src, m->r));           // H = A - sigma M
    LAUNCH(1, apply_M_f64(m, Np, src, m->q, nullptr));  // M
    LAUNCH(2, launch_gram2(g, N, Np, src, m->r, m->q, m->gpart, nullptr, m->GA, m->GB, m->st));
  }
  // mixed handles inside the loop: the eigensolve in float-float on the float32
  // pipes; the start on user guesses (ill-conditioned overlaps) and the public
  // call on arbitrary X (guard) stay float64: the float-float Jacobi reaches its
  // sweep limit on an X that already diagonalises the pencil with degenerate
  // Ritz values (the converged orbitals of a shell)
  LAUNCH(1, launch_small_eig(N, m->GA, m->GB, m->eigwork, m->C, m->theta, &m->cgst->status, m->st,
                             &m->cgst->bar_count, clus, mixed && mode != kRRFP64 && !guard));
  // An input the fast arithmetic cannot resolve (the overlap of raw guesses can
  // be ill-conditioned far beyond the Grams' 24-bit inputs) makes the fast
  // eigensolve report an indefinite overlap or its sweep limit; the step is then
  // redone in float64 (Grams, eigensolve and rotation) from the same X, which the
  // fast step leaves untouched.  Inside the ParO loop the status is read with the
  // Ritz values after the rotation (one round trip a step); elsewhere before it.
  const bool fast = mixed && mode != kRRFP64;
  if (!fast || guard) {
    const int rc = check_status(m, "rayleigh_ritz");
    if ((rc == PARO_ERR_NOT_CONVERGED || rc == PARO_ERR_NOT_SPD) && fast) {
      if (trace_on()) std::fprintf(stderr, "paro rayleigh_ritz: fast eigensolve %s, float64 step\n", m->err.c_str());
      return rr_packed(m, N, src, dst, lam, kRRFP64, clus, false);
    }
    TRY(rc);
  }
  // the rotation: on the tensor cores from the hi parts of X with the tensor-core
  // Grams (the same 24-bit inputs), else in float-float from the split X (C staged
  // in shared memory whole, or in column blocks above kRotateFFMaxNp), or float64
  if (tc && Np <= kRotTcMaxNp)
    LAUNCH(1, launch_rotate_tc(g, N, Np, m->fxh, m->C, dst, &m->cgst->status, m->st));
  else if (ff || tc)
    LAUNCH(1, launch_rotate_ff(g, N, Np, m->fxh, m->fxl, m->C, dst, m->st));
  else
    LAUNCH(1, launch_rotate(g, N, Np, src, m->C, dst, m->st));
  // the Ritz values and the status word (a bounded wait of the rotation) in one round trip
  CK(cudaMemcpyAsync(m->h_dbl, m->theta, sizeof(double) * N, cudaMemcpyDeviceToHost, m->st));
  CK(cudaMemcpyAsync(m->h_int, &m->cgst->status, sizeof(int), cudaMemcpyDeviceToHost, m->st));
  CK(cudaStreamSynchronize(m->st));
  if (m->h_int[0] != 0) {
    const int rc = check_status(m, "rayleigh_ritz");
    if ((rc == PARO_ERR_NOT_CONVERGED || rc == PARO_ERR_NOT_SPD) && fast && !guard) {
      if (trace_on()) std::fprintf(stderr, "paro rayleigh_ritz: fast eigensolve %s, float64 step\n", m->err.c_str());
      return rr_packed(m, N, src, dst, lam, kRRFP64, clus, false);
    }
    TRY(rc);
  }
  for (int i = 0; i < N; ++i) lam[i] = m->h_dbl[i];
  return PARO_OK;
}

int check_common(paro_mesh m, int N) {
  if (!m) return PARO_ERR_ARG;
  if (N < 1 || N > kMaxN) return fail(m, PARO_ERR_ARG, "N out of range [1, 1024]");
  if (!m->have_pot) return fail(m, PARO_ERR_STATE, "paro_set_potential has not been called");
  return PARO_OK;
}

constexpr int kTimerPairs = 64;

// Adds the elapsed time of every stopped phase to its statistic (waits for the
// last of them) and frees the event pairs.
void timers_resolve(paro_mesh m) {
  for (const auto& pk : m->tev_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(m->tev[2 * pk.second + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, m->tev[2 * pk.second], m->tev[2 * pk.second + 1]) == cudaSuccess)
      *pk.first += ms;
  }
  (void)cudaGetLastError();
  m->tev_pending.clear();
  m->tev_used = 0;
}

// One timed phase of a call (statistics only): events around it on the stream,
// read when the call ends (CallScope) or when the pool of pairs is used up.
struct Timer {
  paro_mesh m;
  double* acc;
  int k = -1;
  Timer(paro_mesh mm, double* a) : m(mm), acc(a) {
    if (!acc) return;
    if (m->tev_used >= kTimerPairs) timers_resolve(m);
    k = m->tev_used;
    while ((int)m->tev.size() < 2 * (k + 1)) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        acc = nullptr;
        return;
      }
      m->tev.push_back(e);
    }
    ++m->tev_used;
    cudaEventRecord(m->tev[2 * k], m->st);
  }
  void stop() {
    if (!acc) return;
    cudaEventRecord(m->tev[2 * k + 1], m->st);
    m->tev_pending.push_back({acc, k});
    acc = nullptr;
  }
  ~Timer() { stop(); }
};

// Per-call accounting: kernel launches, and (params.profile) the timed CG
// operator launches with the work they processed.
struct CallScope {
  paro_mesh m;
  paro_stats* s;
  long long l0, tc0, pi0;
  CallScope(paro_mesh mm, paro_stats* ss, int profile)
      : m(mm), s(ss), l0(mm->launches), tc0(mm->rr_tc), pi0(mm->ks_pois_iters) {
    m->profile = 0;
    m->prof_launches = 0;
    m->prof_ms = 0.0;
    m->pev_used = 0;
    if (!profile || !s) return;
    if (m->pev.empty()) {
      m->pev.resize(2 * kProfPairs, nullptr);
      for (auto& e : m->pev)
        if (cudaEventCreate(&e) != cudaSuccess) {
          m->pev.clear();
          return;
        }
    }
    if (cudaMemsetAsync(&m->cgst->work, 0, sizeof(unsigned long long), m->st) != cudaSuccess) return;
    if (cudaMemsetAsync(&m->cgst->work_nodes, 0, sizeof(unsigned long long), m->st) != cudaSuccess) return;
    if (cudaMemsetAsync(&m->cgst->work_act, 0, sizeof(unsigned long long), m->st) != cudaSuccess) return;
    m->profile = profile == 2 ? 2 : 1;
  }
  ~CallScope() {
    timers_resolve(m);
    if (s) {
      s->kernel_launches += m->launches - l0;
      s->rr_tc_steps += (int)(m->rr_tc - tc0);
      s->poisson_cg_iters += m->ks_pois_iters - pi0;
      if (m->profile) {
        unsigned long long w = 0, wn = 0, wa = 0;
        if (cudaMemcpyAsync(m->h_dbl, &m->cgst->work, sizeof(w), cudaMemcpyDeviceToHost, m->st) == cudaSuccess &&
            cudaMemcpyAsync(m->h_dbl + 1, &m->cgst->work_nodes, sizeof(wn), cudaMemcpyDeviceToHost, m->st) ==
                cudaSuccess &&
            cudaMemcpyAsync(m->h_dbl + 2, &m->cgst->work_act, sizeof(wa), cudaMemcpyDeviceToHost, m->st) ==
                cudaSuccess &&
            cudaStreamSynchronize(m->st) == cudaSuccess) {
          std::memcpy(&w, m->h_dbl, sizeof(w));
          std::memcpy(&wn, m->h_dbl + 1, sizeof(wn));
          std::memcpy(&wa, m->h_dbl + 2, sizeof(wa));
        }
        s->prof_launches += m->prof_launches;
        s->prof_ms += m->prof_ms;
        s->prof_dof_orb += (long long)w;
        s->prof_node_passes += (long long)wn;
        s->prof_dof_orb_active += (long long)wa;
      }
    }
    m->profile = 0;
  }
};


// ---------------------------------------------------------------------------
// Kohn-Sham helpers
// ---------------------------------------------------------------------------

long long gauss_count(const Grid& g) { return (long long)g.nx * g.ny * g.nz * 8; }

int ensure_ks(paro_mesh m) {
  if (m->g.graded) return fail(m, PARO_ERR_ARG, "the Kohn-Sham calls need a uniform mesh");
  if (m->ks_rho) return PARO_OK;
  const long long nq = gauss_count(m->g);
  TRY(dalloc(m, &m->ks_mom, 4));
  TRY(dalloc(m, &m->ks_part, (size_t)4 * moments_blocks()));
  TRY(dalloc(m, &m->ks_rho, (size_t)nq));
  TRY(dalloc(m, &m->ks_rho2, (size_t)nq));
  TRY(dalloc(m, &m->ks_v, (size_t)nq));
  TRY(dalloc(m, &m->ks_occ, (size_t)kMaxN));
  TRY(dalloc(m, &m->ks_vh, (size_t)nq));
  TRY(dalloc(m, &m->ks_energy, 3));
  return PARO_OK;
}

// The float64 handle of K/2 on the same mesh (V = 0, sigma = 0), for the Poisson solve.
int ensure_poisson(paro_mesh m) {
  if (m->pois) return PARO_OK;
  paro_mesh c = nullptr;
  // the Poisson problem takes the parent's precision: float32 CG in float-float
  // refinement on mixed handles
  int rc = paro_mesh_create(&c, m->g.nx, m->g.ny, m->g.nz, m->lo, m->hi, m->precision, m->st);
  if (rc != PARO_OK) return fail(m, rc, std::string("Poisson handle: ") + paro_last_error(nullptr));
  m->pois = c;
  double* zeros = nullptr;
  TRY(dalloc(m, &zeros, (size_t)gauss_count(m->g)));  // zeroed on the stream
  rc = paro_set_potential(c, zeros, 0.0);
  if (rc != PARO_OK) return fail(m, rc, std::string("Poisson handle: ") + paro_last_error(c));
  TRY(ensure_workspace(c, 4));  // zeroed: the first solve starts from w = 0
  return PARO_OK;
}

// Hartree potential of rho (Gauss points): monopole, right-hand side, solve of
// (K/2) w = 2 pi (rho, phi) - (K/2)_{I,boundary} g on the Poisson handle, warm-
// started from the previous solution (the density of an SCF loop changes little
// from one iteration to the next); the solution is left in m->pois->x (padded,
// column 0).  Mixed handles: float32 CG in float-float refinement to
// pp.solve_tol; float64 handles: float64 CG.
int hartree_solve(paro_mesh m, const double* rho, const paro_params& p) {
  if (p.hartree_precond < PARO_PRECOND_AUTO || p.hartree_precond > PARO_PRECOND_MG)
    return fail(m, PARO_ERR_ARG, "unknown Hartree preconditioner");
  TRY(ensure_ks(m));
  TRY(ensure_poisson(m));
  paro_mesh c = m->pois;
  // the Poisson problem is where multigrid pays most (Jacobi-PCG iterations grow
  // like 1/h there, without a mass term to bound them)
  paro_params pp = p;
  pp.precond = p.hartree_precond;
  if (pp.precond == PARO_PRECOND_AUTO) {
    Grid gs[kMaxMGLevels];
    pp.precond = (c->precision == PARO_MIXED && mg_plan_levels(c->g, gs, kMaxMGLevels) >= 2) ? PARO_PRECOND_MG
                                                                                                : PARO_PRECOND_JACOBI;
  }
  TRY(check_precond(m, pp));
  LAUNCH(2, launch_moments(m->g, m->lo, rho, m->ks_part, m->ks_mom, m->st));
  CK(cudaMemsetAsync(c->b, 0, sizeof(double) * c->g.G * 4, m->st));
  LAUNCH(1, launch_hartree_rhs(c->g, m->lo, rho, c->coef64, m->ks_mom, c->b, m->st));
  CK(cudaMemsetAsync(c->cgst->skip, 0, sizeof(int) * kMaxN, m->st));
  int rc;
  if (c->precision == PARO_MIXED) {
    rc = launch_split_ff((long long)c->g.G * 4, c->b, c->fah, c->fal, m->st) == cudaSuccess ? PARO_OK : PARO_ERR_CUDA;
    if (rc == PARO_OK) {
      ++m->launches;
      paro_stats ps{};
      rc = refine_solve(c, 1, pp, &ps);
      m->ks_pois_iters += ps.cg_iters;
    }
  } else {
    long long its = 0;
    int itmax = 0;
    rc = run_cg<double>(c, c->plan64, 1, true, pp.solve_tol, pp.pcg_maxit, 16, &its, &itmax);
    m->ks_pois_iters += its;
  }
  if (rc != PARO_OK) return fail(m, rc, std::string("Hartree solve: ") + c->err);
  rc = check_status(c, "Hartree solve");
  if (rc != PARO_OK) return fail(m, rc, c->err);
  m->launches += c->launches;
  c->launches = 0;
  return PARO_OK;
}

// v = V_ext + V_H(rho) + V_x(rho) at the Gauss points (vh: V_H alone, optional).
int ks_potential(paro_mesh m, const double* rho, const double* vext, double* v, double* vh, const paro_params& pp) {
  TRY(hartree_solve(m, rho, pp));
  LAUNCH(1, launch_ks_potential(m->g, m->lo, m->pois->x, m->ks_mom, rho, vext, v, vh, m->st));
  return PARO_OK;
}

int upload_occ(paro_mesh m, int N, const double* occ) {
  TRY(ensure_ks(m));
  for (int i = 0; i < N; ++i) m->h_dbl[i] = occ[i];
  CK(cudaMemcpyAsync(m->ks_occ, m->h_dbl, sizeof(double) * N, cudaMemcpyHostToDevice, m->st));
  CK(cudaStreamSynchronize(m->st));
  return PARO_OK;
}

}  // namespace

namespace paro {

// Joins the mixed-precision, Jacobi-preconditioned systems of a batch (at least
// two, at most kMaxBatchSys) to one coordinator: their workspaces and
// single-pass plans are made, the batched plan is built over their CG buffers
// and autotuned (PARO_AUTOTUNE=0: the first candidate; PARO_CG2B_GEOMETRY=<i>:
// candidate i), and each handle points to the coordinator.  *coord carries the
// coordinator from one paro_batch_iterate to the next: it is kept when the same
// systems come back with the same buffers, else rebuilt.  *coord is null when
// fewer than two systems qualify or the batched kernel cannot run co-resident;
// the systems then solve alone.
static bool same_desc(const CG2BSysDesc& a, const CG2BSysDesc& b) {
  return a.Np == b.Np && a.N == b.N && a.x == b.x && a.r[0] == b.r[0] && a.r[1] == b.r[1] && a.q[0] == b.q[0] &&
         a.q[1] == b.q[1] && a.p[0] == b.p[0] && a.p[1] == b.p[1] && a.st == b.st && a.dinv_tma == b.dinv_tma &&
         a.dpitch == b.dpitch && a.wcoef == b.wcoef && a.g.nx == b.g.nx && a.g.ny == b.g.ny && a.g.nz == b.g.nz;
}

void batch_cg_destroy(void* h) {
  BatchCG* B = static_cast<BatchCG*>(h);
  if (!B) return;
  if (B->st) cudaStreamSynchronize(B->st);
  cg2b_destroy(&B->plan);
  for (auto ev : B->ready)
    if (ev) cudaEventDestroy(ev);
  if (B->done) cudaEventDestroy(B->done);
  if (B->st) cudaStreamDestroy(B->st);
  delete B;
}

int batch_cg_begin(const std::vector<paro_mesh>& ms, const std::vector<int>& Ns, const std::vector<paro_params>& ps,
                   void** coord, std::string* err) {
  std::vector<int> idx;
  for (size_t i = 0; i < ms.size(); ++i) {
    paro_mesh m = ms[i];
    if (m->precision != PARO_MIXED || ps[i].precond != PARO_PRECOND_JACOBI || ps[i].profile) continue;
    const int N = Ns[i];
    if (N < 1 || N > kMaxN || !m->have_pot) continue;
    const int rc = ensure_workspace(m, (N + 3) / 4 * 4);
    if (rc != PARO_OK) {
      *err = m->err;
      return rc;
    }
    if (m->plan2 && m->plan2->ok) idx.push_back((int)i);
  }
  if (idx.size() < 2 || idx.size() > (size_t)kMaxBatchSys) {
    batch_cg_destroy(*coord);
    *coord = nullptr;
    return PARO_OK;
  }
  std::vector<CG2BSysDesc> desc;
  for (int i : idx) {
    paro_mesh m = ms[i];
    const int rc = set_f32_layout(m, 1);
    if (rc != PARO_OK) {
      *err = m->err;
      return rc;
    }
    const CG2Plan* P = m->plan2;
    CG2BSysDesc d{};
    d.g = m->g;
    d.Np = P->args.Np;
    d.N = Ns[i];
    d.x = P->args.x;
    for (int b = 0; b < 2; ++b) {
      d.r[b] = P->args.r[b];
      d.q[b] = P->args.q[b];
      d.p[b] = P->args.p[b];
    }
    d.st = m->cgst;
    d.dinv_tma = P->dinv_tma;
    d.dpitch = P->dpitch;
    d.wcoef = P->wcoef;
    desc.push_back(d);
  }
  BatchCG* B = static_cast<BatchCG*>(*coord);
  bool reuse = B && B->desc.size() == desc.size();
  for (size_t k = 0; reuse && k < desc.size(); ++k) reuse = B->ms[k] == ms[idx[k]] && same_desc(B->desc[k], desc[k]);
  if (!reuse) {
    batch_cg_destroy(B);
    *coord = nullptr;
    B = new BatchCG();
    B->desc = desc;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cg2b_create(&B->plan, desc, ms[idx[0]]->nsm);
    const char* off = std::getenv("PARO_AUTOTUNE");
    const char* force = std::getenv("PARO_CG2B_GEOMETRY");  // candidate i, untimed (tests run several)
    if (e == cudaSuccess && force) {
      std::vector<K1Geom> cand;
      cg2b_candidates(&B->plan, &cand);
      const int i = std::atoi(force);
      if (i >= 0 && i < (int)cand.size()) {
        e = cg2b_prepare_geo(&B->plan, cand[i]);
        B->chosen = i;
      }
    } else if (e == cudaSuccess && !(off && off[0] == '0')) {
      e = cg2b_autotune(&B->plan, B->st, 4, &B->chosen, &B->best_us, &B->tried);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->st);
    B->ready.assign(idx.size(), nullptr);
    for (size_t k = 0; k < idx.size() && e == cudaSuccess; ++k)
      e = cudaEventCreateWithFlags(&B->ready[k], cudaEventDisableTiming);
    if (e != cudaSuccess || !B->plan.ok) {
      const bool cuda_failed = e != cudaSuccess;
      if (cuda_failed) *err = std::string("batched CG plan: ") + cudaGetErrorString(e);
      (void)cudaGetLastError();
      batch_cg_destroy(B);
      return cuda_failed ? PARO_ERR_CUDA : PARO_OK;
    }
    if (std::getenv("PARO_PRINT_PLAN"))
      std::fprintf(stderr, "paro batched CG plan: %zu systems, tile %dx%d, %d nodes a thread, block %d, %d slots, "
                   "z-chunk %d, %d items, %d orbital blocks, candidate %d (%d timed, %.1f us a pass)\n", idx.size(),
                   B->plan.geo.TX, B->plan.geo.TY, B->plan.geo.npt, B->plan.geo.G4 * 4, B->plan.geo.slots,
                   B->plan.args.zlen, B->plan.args.nitems, B->plan.args.njobs, B->chosen, B->tried, B->best_us);
    for (size_t k = 0; k < idx.size(); ++k) B->ms.push_back(ms[idx[k]]);
    *coord = B;
  } else {
    // the systems' streams may still run earlier work on these buffers
    for (int i : idx) {
      paro_mesh m = ms[i];
      CK(cudaStreamSynchronize(m->st));
    }
  }
  for (size_t k = 0; k < idx.size(); ++k) {
    paro_mesh m = ms[idx[k]];
    m->bcg = B;
    m->bcg_index = (int)k;
  }
  B->live = (int)idx.size();
  B->waiting = 0;
  B->launches = 0;
  B->launch_err = cudaSuccess;
  B->waiting_flag.assign(idx.size(), 0);
  B->spin.assign(idx.size(), kSpinLimit);
  return PARO_OK;
}

// The system's loop has ended (converged, limit or error): it no longer takes
// part, and the others are launched if they were all waiting for it.
void batch_cg_leave(paro_mesh m) {
  BatchCG* B = m->bcg;
  if (!B) return;
  std::lock_guard<std::mutex> lk(B->mu);
  m->bcg = nullptr;
  --B->live;
  if (B->live > 0 && B->waiting == B->live) bcg_launch_locked(B);
}

// After every system has left: the batched launches of this paro_batch_iterate.
long long batch_cg_finish(void* h) {
  BatchCG* B = static_cast<BatchCG*>(h);
  if (!B) return 0;
  cudaStreamSynchronize(B->st);
  return B->launches;
}

}  // namespace paro

extern "C" {

void paro_default_params(paro_params* p) {
  if (!p) return;
  p->tol = 1e-10;
  p->max_outer = 500;
  p->n_check = 0;
  p->solve_tol = 1e-12;
  p->pcg_maxit = 5000;
  p->inner_tol = 0.0;
  p->max_refine = 20;
  p->check_every = 16;
  p->fixed_outer = 0;
  p->profile = 0;
  p->n_clusters = 0;
  p->cluster_size = nullptr;
  p->precond = PARO_PRECOND_JACOBI;
  p->mg_nu = 1;
  p->mg_coarse_sweeps = 4;
  p->hartree_precond = PARO_PRECOND_AUTO;
  p->wait_polls = 0;
}

static int mesh_create(paro_mesh* out, int nx, int ny, int nz, const double lo_in[3], const double hi_in[3],
                       const double* const ax[3], int precision, void* cuda_stream);

int paro_mesh_create(paro_mesh* out, int nx, int ny, int nz, const double lo[3], const double hi[3], int precision,
                     void* cuda_stream) {
  const double* const none[3] = {nullptr, nullptr, nullptr};
  return mesh_create(out, nx, ny, nz, lo, hi, none, precision, cuda_stream);
}

int paro_mesh_create_graded(paro_mesh* out, int nx, int ny, int nz, const double* x, const double* y,
                            const double* z, int precision, void* cuda_stream) {
  if (!out || !x || !y || !z) {
    g_create_err = "null argument";
    return PARO_ERR_ARG;
  }
  if (nx < 2 || ny < 2 || nz < 2 || nx > 1024 || ny > 1024 || nz > 1024) {
    g_create_err = "cells per axis must be in [2, 1024]";
    return PARO_ERR_ARG;
  }
  const double* const ax[3] = {x, y, z};
  const int n[3] = {nx, ny, nz};
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    for (int i = 0; i <= n[d]; ++i)
      if (!std::isfinite(ax[d][i]) || (i > 0 && !(ax[d][i] > ax[d][i - 1]))) {
        g_create_err = "node coordinates must be finite and strictly increasing along every axis";
        return PARO_ERR_ARG;
      }
    lo[d] = ax[d][0];
    hi[d] = ax[d][n[d]];
  }
  return mesh_create(out, nx, ny, nz, lo, hi, ax, precision, cuda_stream);
}

static int mesh_create(paro_mesh* out, int nx, int ny, int nz, const double lo_in[3], const double hi_in[3],
                       const double* const ax[3], int precision, void* cuda_stream) {
  const double* lo = lo_in;
  const double* hi = hi_in;
  if (!out || !lo || !hi) {
    g_create_err = "null argument";
    return PARO_ERR_ARG;
  }
  *out = nullptr;
  if (nx < 2 || ny < 2 || nz < 2 || nx > 1024 || ny > 1024 || nz > 1024) {
    g_create_err = "cells per axis must be in [2, 1024]";
    return PARO_ERR_ARG;
  }
  if (precision != PARO_FP64 && precision != PARO_MIXED) {
    g_create_err = "precision must be PARO_FP64 or PARO_MIXED";
    return PARO_ERR_ARG;
  }
  for (int d = 0; d < 3; ++d)
    if (!(hi[d] > lo[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d])) {
      g_create_err = "box must satisfy lo < hi (finite)";
      return PARO_ERR_ARG;
    }
  paro_mesh m = new paro_mesh_s();
  m->precision = precision;
  m->st = static_cast<cudaStream_t>(cuda_stream);
  Grid& g = m->g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.Px = nx + 1;
  g.Py = ny + 1;
  g.Pz = nz + 1;
  g.G = (long long)g.Px * g.Py * g.Pz;
  g.nI = (nx - 1) * (ny - 1) * (nz - 1);
  g.hx = (hi[0] - lo[0]) / nx;
  g.hy = (hi[1] - lo[1]) / ny;
  g.hz = (hi[2] - lo[2]) / nz;
  for (int d = 0; d < 3; ++d) {
    m->lo[d] = lo[d];
    m->hi[d] = hi[d];
    const int nd = d == 0 ? nx : (d == 1 ? ny : nz);
    m->nodes[d].resize(nd + 1);
    for (int i = 0; i <= nd; ++i)
      m->nodes[d][i] = ax[d] ? ax[d][i] : (i == nd ? hi[d] : lo[d] + (hi[d] - lo[d]) * i / nd);
  }
  mass_weights(g, &m->mw);
  m->dpitch = (g.Px + 3) / 4 * 4;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
      m->nsm = nsm;
  }
  int rc = PARO_OK;
  cudaError_t e;
  if ((rc = dalloc(m, &m->coef64, (size_t)27 * g.G)) || (rc = dalloc(m, &m->coef32, (size_t)27 * g.G)) ||
      (rc = dalloc(m, &m->dinv64, (size_t)g.G)) || (rc = dalloc(m, &m->dinv32, (size_t)g.G)) ||
      (rc = dalloc(m, &m->dscal, (size_t)S_COUNT * kMaxN)) ||
      (rc = dalloc(m, &m->dint, (size_t)I_COUNT * kMaxN + 8)) ||
      (rc = dalloc(m, &m->partial, (size_t)3 * kMaxRedBlocks * kMaxN)) || (rc = dalloc(m, &m->ticket, 4)) ||
      (rc = dalloc(m, &m->cgst, 1)) || (rc = dalloc(m, &m->w32, packed_weights_count(g))) ||
      (rc = dalloc(m, &m->w64, packed_weights_count(g))) ||
      (rc = dalloc(m, &m->dt32, (size_t)g.Pz * g.Py * m->dpitch)) ||
      (rc = dalloc(m, &m->dt64, (size_t)g.Pz * g.Py * m->dpitch)) ||
      (precision == PARO_MIXED &&
       ((rc = dalloc(m, &m->wAh, (size_t)g.G * kPackedW)) || (rc = dalloc(m, &m->wAl, (size_t)g.G * kPackedW)) ||
        (rc = dalloc(m, &m->wHh, (size_t)g.G * kPackedW)) || (rc = dalloc(m, &m->wHl, (size_t)g.G * kPackedW))))) {
    g_create_err = m->err;
    paro_mesh_destroy(m);
    return rc;
  }
  if ((e = cudaMallocHost(&m->h_dbl, sizeof(double) * 2 * kMaxN)) != cudaSuccess ||
      (e = cudaMallocHost(&m->h_ctl, sizeof(double) * 2)) != cudaSuccess ||
      (e = cudaMallocHost(&m->h_int, sizeof(int) * kMaxN)) != cudaSuccess ||
      (e = cudaEventCreate(&m->e0)) != cudaSuccess || (e = cudaEventCreate(&m->e1)) != cudaSuccess) {
    g_create_err = std::string("host setup: ") + cudaGetErrorString(e);
    paro_mesh_destroy(m);
    return PARO_ERR_CUDA;
  }
  if (ax[0] != nullptr) {
    // graded: cell sizes on the device, the per-node mass weights (fixed by the
    // mesh) and, on mixed handles, their packed float-float copy
    const int n3[3] = {nx, ny, nz};
    std::vector<double> hc;
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < n3[d]; ++c) hc.push_back(ax[d][c + 1] - ax[d][c]);
    if ((rc = dalloc(m, &m->hcell, hc.size())) || (rc = dalloc(m, &m->coefM64, (size_t)27 * g.G)) ||
        (rc = dalloc(m, &m->coefH64, (size_t)27 * g.G)) ||
        (precision == PARO_MIXED && ((rc = dalloc(m, &m->wMh, (size_t)g.G * kPackedW)) ||
                                     (rc = dalloc(m, &m->wMl, (size_t)g.G * kPackedW))))) {
      g_create_err = m->err;
      paro_mesh_destroy(m);
      return rc;
    }
    g.graded = 1;
    g.hc = m->hcell;
    e = cudaMemcpyAsync(m->hcell, hc.data(), sizeof(double) * hc.size(), cudaMemcpyHostToDevice, m->st);
    if (e == cudaSuccess) e = launch_build_mass(g, m->coefM64, m->st);
    if (e == cudaSuccess && precision == PARO_MIXED) {
      Weights27 zero{};
      e = launch_build_wff(g, m->coefM64, zero, 0.0, m->wMh, m->wMl, m->wMh, m->wMl, m->st);
    }
    if (e != cudaSuccess) {
      g_create_err = std::string("graded mesh set-up: ") + cudaGetErrorString(e);
      paro_mesh_destroy(m);
      return PARO_ERR_CUDA;
    }
  }
  if ((e = cudaStreamSynchronize(m->st)) != cudaSuccess) {
    g_create_err = std::string("stream: ") + cudaGetErrorString(e);
    paro_mesh_destroy(m);
    return PARO_ERR_CUDA;
  }
  *out = m;
  return PARO_OK;
}

int paro_mesh_destroy(paro_mesh m) {
  if (!m) return PARO_ERR_ARG;
  cudaStreamSynchronize(m->st);
  if (m->pois) paro_mesh_destroy(m->pois);
  free_plans(m);
  for (void* p : m->allocs)
    if (p) cudaFree(p);
  if (m->h_dbl) cudaFreeHost(m->h_dbl);
  if (m->h_int) cudaFreeHost(m->h_int);
  if (m->h_ctl) cudaFreeHost(m->h_ctl);
  if (m->e0) cudaEventDestroy(m->e0);
  if (m->e1) cudaEventDestroy(m->e1);
  for (auto e : m->pev)
    if (e) cudaEventDestroy(e);
  for (auto e : m->tev)
    if (e) cudaEventDestroy(e);
  delete m;
  return PARO_OK;
}

int paro_set_potential(paro_mesh m, const double* Vq, double sigma) {
  if (!m) return PARO_ERR_ARG;
  if (!Vq) return fail(m, PARO_ERR_ARG, "Vq is null");
  if (!std::isfinite(sigma)) return fail(m, PARO_ERR_ARG, "sigma must be finite");
  LAUNCH(1, launch_build_coef(m->g, Vq, sigma, m->coef64, m->coef32, m->dinv64, m->dinv32, m->st));
  LAUNCH(2, launch_build_tma_operator<double>(m->g, m->coef64, m->dinv64, m->w64, m->dt64, m->dpitch,
                                               m->st));
  LAUNCH(2, launch_build_tma_operator<float>(m->g, m->coef32, m->dinv32, m->w32, m->dt32, m->dpitch,
                                              m->st));
  if (m->g.graded)  // H = A - sigma M with the per-node mass weights
    LAUNCH(1, launch_sub_scaled((long long)27 * m->g.G, m->coef64, sigma, m->coefM64, m->coefH64, m->st));
  if (m->precision == PARO_MIXED)
    LAUNCH(1, launch_build_wff(m->g, m->coef64, m->mw, sigma, m->wAh, m->wAl, m->wHh, m->wHl, m->st,
                               m->g.graded ? m->coefM64 : nullptr));
  m->sigma = sigma;
  m->have_pot = true;
  m->mg.built = false;
  return PARO_OK;
}

int paro_orbital_solve(paro_mesh m, int N, const double* lambda, const double* U, double* X, const paro_params* p,
                       paro_stats* s) {
  TRY(check_common(m, N));
  if (!lambda || !U || !X) return fail(m, PARO_ERR_ARG, "null pointer");
  if (U == X) return fail(m, PARO_ERR_ARG, "X must not alias U");
  paro_params pp;
  if (p) pp = *p;
  else paro_default_params(&pp);
  if (pp.check_every < 1) pp.check_every = 1;
  const int Np = (N + 3) / 4 * 4;
  TRY(ensure_workspace(m, Np));
  CallScope cs(m, s, pp.profile);
  LAUNCH(1, launch_pack(m->g, N, Np, U, m->u, m->st));
  Timer t(m, s ? &s->ms_solve : nullptr);
  int rc = solve_packed(m, N, lambda, pp, s);
  t.stop();
  if (rc != PARO_OK && rc != PARO_ERR_NOT_CONVERGED) return rc;
  LAUNCH(1, launch_unpack(m->g, N, Np, m->x, X, m->st));
  CK(cudaStreamSynchronize(m->st));
  return rc;
}

int paro_rayleigh_ritz(paro_mesh m, int N, const double* X, double* U_out, double* lambda_out, paro_stats* s) {
  TRY(check_common(m, N));
  if (!X || !U_out || !lambda_out) return fail(m, PARO_ERR_ARG, "null pointer");
  const int Np = (N + 3) / 4 * 4;
  TRY(ensure_workspace(m, Np));
  CallScope cs(m, s, 0);
  LAUNCH(1, launch_pack(m->g, N, Np, X, m->x, m->st));
  Timer t(m, s ? &s->ms_rr : nullptr);
  TRY(rr_packed(m, N, m->x, m->u, lambda_out, kRRFast, nullptr, false, true));
  t.stop();
  LAUNCH(1, launch_unpack(m->g, N, Np, m->u, U_out, m->st));
  CK(cudaStreamSynchronize(m->st));
  return PARO_OK;
}

int paro_iterate(paro_mesh m, int N, double* U, double* lambda, const paro_params* p, paro_stats* s) {
  TRY(check_common(m, N));
  if (!U || !lambda) return fail(m, PARO_ERR_ARG, "null pointer");
  paro_params pp;
  if (p) pp = *p;
  else paro_default_params(&pp);
  if (pp.check_every < 1) pp.check_every = 1;
  const int Np = (N + 3) / 4 * 4;
  TRY(ensure_workspace(m, Np));
  CallScope cs(m, s, pp.profile);
  LAUNCH(1, launch_pack(m->g, N, Np, U, m->u, m->st));
  std::vector<double> lam(lambda, lambda + N), lam_new(N);
  if (std::isnan(lambda[0])) {
    Timer t(m, s ? &s->ms_rr : nullptr);
    TRY(rr_packed(m, N, m->u, m->x, lam.data(), kRRFP64));
    t.stop();
    // copy rather than swap: the CG plans hold the addresses of the workspace vectors
    CK(cudaMemcpyAsync(m->u, m->x, sizeof(double) * m->g.G * Np, cudaMemcpyDeviceToDevice, m->st));
  }
  const int nchk = (pp.n_check > 0 && pp.n_check < N) ? pp.n_check : N;
  RRMode rr_mode = kRRFast;
  const int* clus = nullptr;
  if (pp.n_clusters > 0) {
    if (!pp.cluster_size) return fail(m, PARO_ERR_ARG, "cluster_size is NULL");
    int total = 0;
    for (int k = 0; k < pp.n_clusters; ++k) {
      if (pp.cluster_size[k] < 1) return fail(m, PARO_ERR_ARG, "cluster sizes must be positive");
      total += pp.cluster_size[k];
    }
    if (total != N) return fail(m, PARO_ERR_ARG, "cluster sizes must add up to N");
    if (!m->clus) TRY(dalloc(m, &m->clus, (size_t)kMaxN));
    int* ids = m->h_int;  // pinned host staging
    for (int k = 0, o = 0; k < pp.n_clusters; ++k)
      for (int j = 0; j < pp.cluster_size[k]; ++j) ids[o++] = k;
    CK(cudaMemcpyAsync(m->clus, ids, sizeof(int) * N, cudaMemcpyHostToDevice, m->st));
    CK(cudaStreamSynchronize(m->st));
    clus = m->clus;
  }
  int outer = 0;
  int rc = PARO_ERR_NOT_CONVERGED;
  const int limit = pp.fixed_outer > 0 ? pp.fixed_outer : pp.max_outer;
  double dl = INFINITY;
  while (outer < limit) {
    {
      Timer t(m, s ? &s->ms_solve : nullptr);
      int r1 = solve_packed(m, N, lam.data(), pp, s, true);
      if (r1 != PARO_OK) return r1;
    }
    {
      Timer t(m, s ? &s->ms_rr : nullptr);
      TRY(rr_packed(m, N, m->x, m->u, lam_new.data(), rr_mode, clus, m->x_split_valid));
    }
    dl = 0.0;
    for (int i = 0; i < nchk; ++i) dl = std::fmax(dl, std::fabs(lam_new[i] - lam[i]));
    lam = lam_new;
    rr_mode = next_rr_mode(m, rr_mode, dl, lam);
    ++outer;
    if (pp.fixed_outer <= 0 && dl < pp.tol) {
      rc = PARO_OK;
      break;
    }
  }
  if (pp.fixed_outer > 0) rc = PARO_OK;
  if (s) {
    s->outer_iters = outer;
    s->max_dlambda = dl;
  }
  for (int i = 0; i < N; ++i) lambda[i] = lam[i];
  LAUNCH(1, launch_unpack(m->g, N, Np, m->u, U, m->st));
  CK(cudaStreamSynchronize(m->st));
  if (rc != PARO_OK) m->err = "paro_iterate: max_outer reached before tol";
  return rc;
}

int paro_estimate(paro_mesh m, int N, const double* U, const double* lambda, const double* Vq, double* eta2) {
  TRY(check_common(m, N));
  if (!U || !lambda || !Vq || !eta2) return fail(m, PARO_ERR_ARG, "null pointer");
  const int Np = (N + 3) / 4 * 4;
  TRY(ensure_workspace(m, Np));
  LAUNCH(1, launch_pack(m->g, N, Np, U, m->u, m->st));
  double* lam_d = m->dscal + S_SCALE * kMaxN;
  for (int i = 0; i < N; ++i) m->h_dbl[i] = lambda[i];
  CK(cudaMemcpyAsync(lam_d, m->h_dbl, sizeof(double) * N, cudaMemcpyHostToDevice, m->st));
  LAUNCH(1, launch_estimate(m->g, N, Np, m->u, lam_d, Vq, eta2, m->st));
  CK(cudaStreamSynchronize(m->st));
  return PARO_OK;
}

int paro_transfer(paro_mesh from, paro_mesh to, int N, const double* U_from, double* U_to) {
  if (!from || !to) return PARO_ERR_ARG;
  paro_mesh m = to;
  if (N < 1 || N > kMaxN) return fail(m, PARO_ERR_ARG, "N out of range [1, 1024]");
  if (!U_from || !U_to || (const void*)U_from == (const void*)U_to) return fail(m, PARO_ERR_ARG, "U_from, U_to must be non-null and distinct");
  for (int d = 0; d < 3; ++d) {
    const auto& c = from->nodes[d];
    const auto& f = to->nodes[d];
    if (std::fabs(c.front() - f.front()) > 1e-12 * (1.0 + std::fabs(c.front())) ||
        std::fabs(c.back() - f.back()) > 1e-12 * (1.0 + std::fabs(c.back())))
      return fail(m, PARO_ERR_ARG, "paro_transfer: the two meshes must cover the same box");
  }
  // per-axis maps of the new interior nodes: the old interval and the local coordinate
  const int fx = to->g.nx - 1, fy = to->g.ny - 1, fz = to->g.nz - 1;
  const int total = fx + fy + fz;
  std::vector<int> km(total);
  std::vector<double> tm(total);
  int o = 0;
  for (int d = 0; d < 3; ++d) {
    const auto& c = from->nodes[d];
    const auto& f = to->nodes[d];
    for (size_t i = 1; i + 1 < f.size(); ++i) {
      const double p = f[i];
      long k = (long)(std::upper_bound(c.begin(), c.end(), p) - c.begin()) - 1;
      if (k < 0) k = 0;
      if (k > (long)c.size() - 2) k = (long)c.size() - 2;
      km[o] = (int)k;
      tm[o] = (p - c[k]) / (c[k + 1] - c[k]);
      ++o;
    }
  }
  if (total > m->xmap_cap) {
    if (m->xmap_k) dfree(m, m->xmap_k);
    if (m->xmap_t) dfree(m, m->xmap_t);
    m->xmap_k = nullptr;
    m->xmap_t = nullptr;
    TRY(dalloc(m, &m->xmap_k, (size_t)total, false));
    TRY(dalloc(m, &m->xmap_t, (size_t)total, false));
    m->xmap_cap = total;
  }
  CK(cudaStreamSynchronize(from->st));  // U_from is ordered on the coarse handle's stream
  CK(cudaMemcpyAsync(m->xmap_k, km.data(), sizeof(int) * total, cudaMemcpyHostToDevice, m->st));
  CK(cudaMemcpyAsync(m->xmap_t, tm.data(), sizeof(double) * total, cudaMemcpyHostToDevice, m->st));
  LAUNCH(1, launch_transfer(from->g, to->g, N, U_from, m->xmap_k, m->xmap_t, U_to, m->st));
  CK(cudaStreamSynchronize(m->st));
  return PARO_OK;
}

int paro_apply(paro_mesh m, int N, int op, int dtype, const void* X, void* Y) {
  TRY(check_common(m, N));
  if (!X || !Y || X == Y) return fail(m, PARO_ERR_ARG, "X, Y must be non-null and distinct");
  if (op < PARO_OP_A || op > PARO_OP_M) return fail(m, PARO_ERR_ARG, "unknown op");
  if (dtype != PARO_F64 && dtype != PARO_F32 && dtype != PARO_FF) return fail(m, PARO_ERR_ARG, "unknown dtype");
  if (dtype == PARO_FF && m->precision != PARO_MIXED)
    return fail(m, PARO_ERR_ARG, "float-float apply needs a PARO_MIXED handle");
  if (dtype == PARO_F32 && op != PARO_OP_A) return fail(m, PARO_ERR_ARG, "float32 apply supports PARO_OP_A only");
  if (dtype == PARO_F32 && m->precision != PARO_MIXED)
    return fail(m, PARO_ERR_ARG, "float32 apply needs a PARO_MIXED handle");
  const int Np = (N + 3) / 4 * 4;
  TRY(ensure_workspace(m, Np));
  if (dtype == PARO_F64) {
    LAUNCH(1, launch_pack(m->g, N, Np, static_cast<const double*>(X), m->u, m->st));
    if (op == PARO_OP_A) LAUNCH(1, launch_apply_f64(m->g, Np, m->coef64, nullptr, 0.0, m->u, m->x, nullptr, m->st));
    else if (op == PARO_OP_H) LAUNCH(1, apply_H_f64(m, Np, m->u, m->x));
    else LAUNCH(1, apply_M_f64(m, Np, m->u, m->x, nullptr));
    LAUNCH(1, launch_unpack(m->g, N, Np, m->x, static_cast<double*>(Y), m->st));
  } else if (dtype == PARO_FF) {
    LAUNCH(1, launch_pack(m->g, N, Np, static_cast<const double*>(X), m->u, m->st));
    LAUNCH(1, launch_split_ff((long long)m->g.G * Np, m->u, m->fxh, m->fxl, m->st));
    if (op == PARO_OP_M)
      LAUNCH(1, apply_M_ff(m, Np, m->fxh, m->fxl, nullptr, m->x, nullptr, nullptr));
    else
      LAUNCH(1, launch_ff_apply(m->g, Np, op == PARO_OP_A ? m->wAh : m->wHh, op == PARO_OP_A ? m->wAl : m->wHl,
                                nullptr, m->fxh, m->fxl, nullptr, m->x, nullptr, nullptr, m->st));
    LAUNCH(1, launch_unpack(m->g, N, Np, m->x, static_cast<double*>(Y), m->st));
  } else {
    TRY(set_f32_layout(m, 0));
    LAUNCH(1, launch_pack_f32(m->g, N, Np, static_cast<const float*>(X), m->b32, m->st));
    LAUNCH(1, launch_apply_f32(m->g, Np, m->coef32, m->b32, m->q32, m->st));
    LAUNCH(1, launch_unpack_f32(m->g, N, Np, m->q32, static_cast<float*>(Y), m->st));
  }
  CK(cudaStreamSynchronize(m->st));
  return PARO_OK;
}

int paro_mg_vcycle(paro_mesh m, int N, const float* R, float* Z, const paro_params* p) {
  TRY(check_common(m, N));
  if (!R || !Z || (const void*)R == (const void*)Z) return fail(m, PARO_ERR_ARG, "R, Z must be non-null and distinct");
  paro_params pp;
  if (p) pp = *p;
  else paro_default_params(&pp);
  pp.precond = PARO_PRECOND_MG;
  TRY(check_precond(m, pp));
  const int Np = (N + 3) / 4 * 4;
  TRY(ensure_workspace(m, Np));
  TRY(ensure_mg(m, Np));
  CGArgs<float>& a = m->plan32->args;
  LAUNCH(1, launch_pack_f32(m->g, N, Np, R, a.r, m->st));
  long long nl = 0;
  CK(mg_vcycle(m->mg, Np, a.r, a.r2, a.s2, a.q2, nullptr, pp.mg_nu, pp.mg_coarse_sweeps, m->st, &nl));
  m->launches += nl;
  LAUNCH(1, launch_unpack_f32(m->g, N, Np, a.r2, Z, m->st));
  CK(cudaStreamSynchronize(m->st));
  return PARO_OK;
}

int paro_density(paro_mesh m, int N, const double* U, const double* occ, double* rho_q) {
  TRY(check_common(m, N));
  if (m->g.graded) return fail(m, PARO_ERR_ARG, "the Kohn-Sham calls need a uniform mesh");
  if (!U || !occ || !rho_q) return fail(m, PARO_ERR_ARG, "null pointer");
  const int Np = (N + 3) / 4 * 4;
  TRY(ensure_workspace(m, Np));
  TRY(upload_occ(m, N, occ));
  LAUNCH(1, launch_pack(m->g, N, Np, U, m->u, m->st));
  LAUNCH(1, launch_density(m->g, N, Np, m->u, m->ks_occ, rho_q, m->st));
  CK(cudaStreamSynchronize(m->st));
  return PARO_OK;
}

int paro_ks_potential(paro_mesh m, const double* rho_q, const double* vext_q, double* v_q, double* vh_q,
                      const paro_params* p) {
  if (!m) return PARO_ERR_ARG;
  if (!rho_q || !vext_q || (!v_q && !vh_q)) return fail(m, PARO_ERR_ARG, "null pointer");
  paro_params pp;
  if (p) pp = *p;
  else paro_default_params(&pp);
  TRY(ks_potential(m, rho_q, vext_q, v_q, vh_q, pp));
  CK(cudaStreamSynchronize(m->st));
  return PARO_OK;
}

int paro_scf_iterate(paro_mesh m, int N, const double* occ, const double* vext_q, double mix, double* U,
                     double* lambda, const paro_params* p, paro_stats* s) {
  TRY(check_common(m, N));
  if (!occ || !vext_q || !U || !lambda) return fail(m, PARO_ERR_ARG, "null pointer");
  if (!(mix > 0.0 && mix <= 1.0)) return fail(m, PARO_ERR_ARG, "mix must be in (0, 1]");
  paro_params pp;
  if (p) pp = *p;
  else paro_default_params(&pp);
  const int Np = (N + 3) / 4 * 4;
  TRY(ensure_workspace(m, Np));
  TRY(ensure_ks(m));
  TRY(upload_occ(m, N, occ));
  CallScope cs(m, s, pp.profile);
  const double sigma = m->sigma;
  LAUNCH(1, launch_pack(m->g, N, Np, U, m->u, m->st));
  // start: Rayleigh-Ritz on span(U) with V_ext alone; its density is the first rho_in
  TRY(paro_set_potential(m, vext_q, sigma));
  std::vector<double> lam(N), lam_new(N);
  TRY(rr_packed(m, N, m->u, m->x, lam.data(), kRRFP64));
  CK(cudaMemcpyAsync(m->u, m->x, sizeof(double) * m->g.G * Np, cudaMemcpyDeviceToDevice, m->st));
  LAUNCH(1, launch_density(m->g, N, Np, m->u, m->ks_occ, m->ks_rho, m->st));
  const int limit = pp.fixed_outer > 0 ? pp.fixed_outer : pp.max_outer;
  const int nchk = (pp.n_check > 0 && pp.n_check < N) ? pp.n_check : N;  // Algorithm 3.2: occupied only
  int outer = 0, rc = PARO_ERR_NOT_CONVERGED;
  double dl = INFINITY;
  RRMode rr_mode = kRRFast;
  while (outer < limit) {
    // V from rho_in, used in both Step 3 and Step 4 of this iteration.  Mixed
    // handles solve the Hartree problem only as accurately as the SCF state needs
    // (the mixing corrects an early inexact potential): min(1e-4, 1e-2 |delta
    // lambda| of the previous iteration), never below solve_tol; float64 handles
    // solve to solve_tol every time.
    paro_params ph = pp;
    if (m->precision == PARO_MIXED) ph.solve_tol = std::fmax(pp.solve_tol, std::fmin(1e-4, 1e-2 * dl));
    TRY(ks_potential(m, m->ks_rho, vext_q, m->ks_v, nullptr, ph));
    TRY(paro_set_potential(m, m->ks_v, sigma));
    {
      Timer t(m, s ? &s->ms_solve : nullptr);
      int r1 = solve_packed(m, N, lam.data(), pp, s, true);
      if (r1 != PARO_OK) return r1;
    }
    {
      Timer t(m, s ? &s->ms_rr : nullptr);
      TRY(rr_packed(m, N, m->x, m->u, lam_new.data(), rr_mode, nullptr, m->x_split_valid));
    }
    LAUNCH(1, launch_density(m->g, N, Np, m->u, m->ks_occ, m->ks_rho2, m->st));
    LAUNCH(1, launch_mix(gauss_count(m->g), mix, m->ks_rho, m->ks_rho2, m->st));
    dl = 0.0;
    for (int i = 0; i < nchk; ++i) dl = std::fmax(dl, std::fabs(lam_new[i] - lam[i]));
    lam = lam_new;
    rr_mode = next_rr_mode(m, rr_mode, dl, lam);
    ++outer;
    if (pp.fixed_outer <= 0 && dl < pp.tol) {
      rc = PARO_OK;
      break;
    }
  }
  if (pp.fixed_outer > 0) rc = PARO_OK;
  if (s) {
    s->outer_iters = outer;
    s->max_dlambda = dl;
  }
  for (int i = 0; i < N; ++i) lambda[i] = lam[i];
  LAUNCH(1, launch_unpack(m->g, N, Np, m->u, U, m->st));
  CK(cudaStreamSynchronize(m->st));
  if (rc != PARO_OK) m->err = "paro_scf_iterate: max_outer reached before tol";
  return rc;
}

int paro_ks_energy(paro_mesh m, int N, const double* occ, const double* lambda, const double* U,
                   const paro_params* p, double* energy) {
  TRY(check_common(m, N));
  if (!occ || !lambda || !U || !energy) return fail(m, PARO_ERR_ARG, "null pointer");
  paro_params pp;
  if (p) pp = *p;
  else paro_default_params(&pp);
  const int Np = (N + 3) / 4 * 4;
  TRY(ensure_workspace(m, Np));
  TRY(ensure_ks(m));
  TRY(upload_occ(m, N, occ));
  CallScope cs(m, nullptr, 0);
  // rho of the given orbitals (in the rho_out buffer: rho_in of an SCF run is kept)
  LAUNCH(1, launch_pack(m->g, N, Np, U, m->u, m->st));
  LAUNCH(1, launch_density(m->g, N, Np, m->u, m->ks_occ, m->ks_rho2, m->st));
  TRY(ks_potential(m, m->ks_rho2, nullptr, nullptr, m->ks_vh, pp));
  LAUNCH(2, launch_energy_terms(m->g, m->ks_rho2, m->ks_vh, m->ks_part, m->ks_energy, m->st));
  CK(cudaMemcpyAsync(m->h_dbl, m->ks_energy, sizeof(double) * 3, cudaMemcpyDeviceToHost, m->st));
  CK(cudaStreamSynchronize(m->st));
  double band = 0.0;
  for (int i = 0; i < N; ++i) band += occ[i] * lambda[i];
  *energy = band - 0.5 * m->h_dbl[0] - m->h_dbl[1] + m->h_dbl[2];
  return PARO_OK;
}

int paro_ks_density_in(paro_mesh m, double* rho_q) {
  if (!m) return PARO_ERR_ARG;
  if (!rho_q) return fail(m, PARO_ERR_ARG, "null pointer");
  if (!m->ks_rho) return fail(m, PARO_ERR_STATE, "no Kohn-Sham run on this handle");
  CK(cudaMemcpyAsync(rho_q, m->ks_rho, sizeof(double) * gauss_count(m->g), cudaMemcpyDeviceToDevice, m->st));
  CK(cudaStreamSynchronize(m->st));
  return PARO_OK;
}

long long paro_interior_nodes(paro_mesh m) { return m ? (long long)m->g.nI : (long long)PARO_ERR_ARG; }

const char* paro_last_error(paro_mesh m) {
  if (!m) return g_create_err.c_str();
  return m->err.c_str();
}

}  // extern "C"
