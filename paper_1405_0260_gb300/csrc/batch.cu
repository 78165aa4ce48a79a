// Batches of independent systems: many meshes, each with its own orbital block,
// advanced to convergence by paro_iterate (Algorithm A.1 per system).
//
// Batched mode (the default): every system runs its loop in a host thread of
// its own, and the float32 correction solves of all mixed-precision, Jacobi
// systems run as one batched launch per refinement sweep (a coordinator in
// api.cu gathers them; cg2b.cu is the kernel), so the GPU streams the work of
// every system still iterating at once.  The rest of each loop runs on the
// system's own stream.  Other systems (float64, multigrid) iterate alone in
// their threads.
//
// Pool mode: a pool of n_workers host threads runs paro_iterate per system,
// largest first (interior nodes x orbitals), each system's kernels on its own
// stream, so that systems overlap on the GPU and one system's host-side waits
// hide behind the others' kernels.
#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "../../include/paro.h"

namespace paro {
int batch_cg_begin(const std::vector<paro_mesh>& ms, const std::vector<int>& Ns, const std::vector<paro_params>& ps,
                   void** coord, std::string* err);
void batch_cg_leave(paro_mesh m);
long long batch_cg_finish(void* coord);
void batch_cg_destroy(void* coord);
}  // namespace paro

struct paro_batch_s {
  struct System {
    paro_mesh m;
    int N;
    double* U;
    double* lambda;
    paro_params p;
    long long work;  // interior nodes x orbitals
  };
  std::vector<System> sys;
  int workers = 1;
  int fused = 1;               // batched correction solves (else the pool of workers)
  long long fused_launches = 0;  // batched launches of the last paro_batch_iterate
  std::string err;
  void* coord = nullptr;  // the batched-solve coordinator, kept across calls
};

extern "C" {

int paro_batch_create(paro_batch* out, int n_workers) {
  if (!out || n_workers < 1 || n_workers > 256) return PARO_ERR_ARG;
  paro_batch b = new paro_batch_s();
  b->workers = n_workers;
  *out = b;
  return PARO_OK;
}

int paro_batch_add(paro_batch b, paro_mesh m, int N, double* U, double* lambda, const paro_params* p) {
  if (!b || !m || !U || !lambda || N < 1) return PARO_ERR_ARG;
  for (const auto& s : b->sys)
    if (s.m == m) return PARO_ERR_ARG;  // one entry per handle: a handle is used by one thread at a time
  paro_batch_s::System s;
  s.m = m;
  s.N = N;
  s.U = U;
  s.lambda = lambda;
  if (p) s.p = *p;
  else paro_default_params(&s.p);
  s.work = paro_interior_nodes(m) * N;
  b->sys.push_back(s);
  return (int)b->sys.size() - 1;
}

int paro_batch_size(paro_batch b) { return b ? (int)b->sys.size() : PARO_ERR_ARG; }

static int batch_iterate_pool(paro_batch b, int* rc, paro_stats* stats) {
  const int n = (int)b->sys.size();
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return b->sys[a].work > b->sys[c].work; });
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n) return;
      const int i = order[k];
      auto& s = b->sys[i];
      paro_stats local{};
      rc[i] = paro_iterate(s.m, s.N, s.U, s.lambda, &s.p, stats ? &local : nullptr);
      if (stats) stats[i] = local;
    }
  };
  const int nw = std::min(b->workers, std::max(n, 1));
  std::vector<std::thread> pool;
  pool.reserve(nw);
  for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  return PARO_OK;
}

// One host thread per system; the coordinator batches the correction solves of
// the systems it accepted (the others solve alone).
static int batch_iterate_fused(paro_batch b, int* rc, paro_stats* stats) {
  const int n = (int)b->sys.size();
  std::vector<paro_mesh> ms(n);
  std::vector<int> Ns(n);
  std::vector<paro_params> ps(n);
  for (int i = 0; i < n; ++i) {
    ms[i] = b->sys[i].m;
    Ns[i] = b->sys[i].N;
    ps[i] = b->sys[i].p;
  }
  const int rcb = paro::batch_cg_begin(ms, Ns, ps, &b->coord, &b->err);
  if (rcb != PARO_OK) return rcb;
  std::vector<std::thread> th;
  th.reserve(n);
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i]() {
      auto& s = b->sys[i];
      paro_stats local{};
      rc[i] = paro_iterate(s.m, s.N, s.U, s.lambda, &s.p, stats ? &local : nullptr);
      paro::batch_cg_leave(s.m);  // also after an error: the others must not wait for it
      if (stats) stats[i] = local;
    });
  for (auto& t : th) t.join();
  b->fused_launches = paro::batch_cg_finish(b->coord);
  return PARO_OK;
}

int paro_batch_iterate(paro_batch b, int* rc, paro_stats* stats) {
  if (!b || !rc) return PARO_ERR_ARG;
  const int n = (int)b->sys.size();
  b->fused_launches = 0;
  b->err.clear();
  const int r = b->fused && n > 1 ? batch_iterate_fused(b, rc, stats) : batch_iterate_pool(b, rc, stats);
  if (r != PARO_OK) return r;
  for (int i = 0; i < n; ++i)
    if (rc[i] != PARO_OK) return rc[i];
  return PARO_OK;
}

int paro_batch_set_fused(paro_batch b, int on) {
  if (!b || (on != 0 && on != 1)) return PARO_ERR_ARG;
  b->fused = on;
  return PARO_OK;
}

long long paro_batch_fused_launches(paro_batch b) { return b ? b->fused_launches : (long long)PARO_ERR_ARG; }

const char* paro_batch_last_error(paro_batch b) { return b ? b->err.c_str() : "null batch"; }

int paro_batch_destroy(paro_batch b) {
  if (!b) return PARO_ERR_ARG;
  paro::batch_cg_destroy(b->coord);
  delete b;
  return PARO_OK;
}

}  // extern "C"
