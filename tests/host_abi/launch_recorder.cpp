// TEST INFRASTRUCTURE: stand-ins for the kernel launchers, so the host side
// of the C ABI (hm_api.cu: parameter checks, planner, chain image, arena,
// state machine, batching) can be exercised on a machine without a GPU.
// Each launcher only records what it was handed (the runtime calls are in
// cuda_runtime_stub.cpp).  Nothing here computes any step of the method;
// the product library never links it.
#include <cstring>
#include <vector>

#include "../../paper_1910_09142_gb300/csrc/hm_internal.h"

namespace {
enum Kind { K_EVOLVE64 = 0, K_EVOLVE_MIXED, K_MEASURE, K_COLLAPSE, K_RESET, K_SUSCEPT };
struct Launch {
  int kind, n, t0, t1, extra;     // extra: draw_initial (reset) or chi_cap (mixed)
  std::vector<const hm::ChainDev*> chains;
};
std::vector<Launch> g_log;

int record(int kind, const hm::BatchArg& b, int extra) {
  Launch l{kind, b.n, b.t0, b.t1, extra, {}};
  for (int i = 0; i < b.n; ++i) l.chains.push_back(b.c[i]);
  g_log.push_back(l);
  return HM_OK;
}
}  // namespace

namespace hm {
int launch_evolve_fp64(const BatchArg& b, const OutArg&, void*) { return record(K_EVOLVE64, b, 0); }
int launch_evolve_mixed(const BatchArg& b, const OutArg&, int chi_cap, int, void*) {
  return record(K_EVOLVE_MIXED, b, chi_cap);
}
int launch_measure_fp64(const BatchArg& b, const OutArg&, void*) { return record(K_MEASURE, b, 0); }
int launch_collapse_fp64(const BatchArg& b, const OutArg&, void*) { return record(K_COLLAPSE, b, 0); }
int launch_reset(const BatchArg& b, const OutArg&, int draw_initial, void*) {
  return record(K_RESET, b, draw_initial);
}
int launch_susceptibility_fp64(const BatchArg& b, const OutArg&, void*) { return record(K_SUSCEPT, b, 0); }
}  // namespace hm

// Accessors for the tests (ctypes).
extern "C" {
void hmtest_clear(void) { g_log.clear(); }
int hmtest_n_launches(void) { return (int)g_log.size(); }
int hmtest_launch(int i, int* kind, int* n, int* t0, int* t1, int* extra) {
  if (i < 0 || i >= (int)g_log.size()) return -1;
  const Launch& l = g_log[i];
  *kind = l.kind, *n = l.n, *t0 = l.t0, *t1 = l.t1, *extra = l.extra;
  return 0;
}
const void* hmtest_launch_chain(int i, int j) { return g_log[i].chains[j]; }
int hmtest_chain_ints(const void* p, int32_t* out8) {
  const hm::ChainDev* c = (const hm::ChainDev*)p;
  out8[0] = c->n_sites, out8[1] = c->n_ops, out8[2] = c->n_gates, out8[3] = c->n_env;
  out8[4] = c->counters[0], out8[5] = c->counters[1], out8[6] = c->basis_zx, out8[7] = c->chi_max;
  return 0;
}
const void* hmtest_chain_ops(const void* p) { return ((const hm::ChainDev*)p)->ops; }
const double* hmtest_chain_gates(const void* p) { return ((const hm::ChainDev*)p)->gates; }
const int32_t* hmtest_chain_env(const void* p) { return ((const hm::ChainDev*)p)->env_out; }
int32_t* hmtest_chain_chi(const void* p) { return ((const hm::ChainDev*)p)->chi; }
}
