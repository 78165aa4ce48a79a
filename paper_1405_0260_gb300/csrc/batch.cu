// Batches of independent systems: many meshes, each with its own orbital block,
// advanced to convergence by paro_iterate (Algorithm A.1 per system) from a pool
// of host worker threads.  Every system is a mesh handle with its own CUDA
// stream, so the kernels of different systems overlap on the GPU and the
// host-side waits of one system (the |delta lambda| test, the refinement
// sweeps' active counts) hide behind the other systems' kernels.  Systems are
// taken largest first (interior nodes x orbitals) so that the long ones start
// early.
#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "../../include/paro.h"

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

int paro_batch_iterate(paro_batch b, int* rc, paro_stats* stats) {
  if (!b || !rc) return PARO_ERR_ARG;
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
  for (int i = 0; i < n; ++i)
    if (rc[i] != PARO_OK) return rc[i];
  return PARO_OK;
}

int paro_batch_destroy(paro_batch b) {
  if (!b) return PARO_ERR_ARG;
  delete b;
  return PARO_OK;
}

}  // extern "C"
