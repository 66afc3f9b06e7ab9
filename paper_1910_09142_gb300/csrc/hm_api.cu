// Host side of the C ABI declared in include/hmetts.h: parameter checks, the
// ladder site map and Trotter/swap schedule planner, the gate table, the
// arena allocator and the entry points.  All device work is in hm_fp64.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "hm_internal.h"

using namespace hm;

namespace {

thread_local std::string g_err;   // message of the last failed context-free call

int fail(std::string* where, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  (where ? *where : g_err) = buf;
  return code;
}

// ---------------------------------------------------------------------------
// Site map, bonds and schedule (Sec. I.C Fig. 4, Sec. II Eq. H, Sec. I.A).
// ---------------------------------------------------------------------------

struct Bond {
  int i, j;
  double J;
};

struct Layout {
  int Lx = 0, two_W = 0, n_sites = 0, n_env = 0, first_cluster = -1;
  std::vector<int32_t> kind;          // per MPS site
  std::vector<int> phys;              // (2 x + y) -> MPS index
  std::vector<int> cluster_cols;
  std::vector<Bond> bonds;            // sorted by (i, j)
  std::vector<Bond> meas;             // measured bonds, sorted
  std::vector<int32_t> region;        // physical sites of the measured columns, sorted
  int n_steps = 0;
  double tau_eff = 0.0;
  bool fused = false;                 // HM_SCHED_FUSED
};

int check_params(const hm_params* p, std::string* err) {
  if (!p) return fail(err, HM_ERR_ARG, "null parameter block");
  if (p->Lx < 1 || p->Lx > 4096) return fail(err, HM_ERR_ARG, "Lx must be in [1, 4096]");
  if (p->two_W < 0 || (p->two_W & 1) || p->two_W > 2 * p->Lx)
    return fail(err, HM_ERR_ARG, "two_W must be even and in [0, 2 Lx]");
  if (!(p->beta >= 0.0) || !std::isfinite(p->beta)) return fail(err, HM_ERR_ARG, "beta must be finite and >= 0");
  if (!(p->tau > 0.0) || !std::isfinite(p->tau)) return fail(err, HM_ERR_ARG, "tau must be finite and > 0");
  if (!std::isfinite(p->J_leg) || !std::isfinite(p->J_rung)) return fail(err, HM_ERR_ARG, "couplings must be finite");
  if (p->chi_max < 1 || p->chi_max > 4096) return fail(err, HM_ERR_ARG, "chi_max must be in [1, 4096]");
  if (!(p->cutoff >= 0.0) || !(p->cutoff < 1.0)) return fail(err, HM_ERR_ARG, "cutoff must be in [0, 1)");
  if (p->precision != HM_FP64 && p->precision != HM_MIXED && p->precision != HM_MIXED32)
    return fail(err, HM_ERR_ARG, "unsupported precision %d", p->precision);
  if (p->basis_schedule != HM_ZX_ALTERNATE && p->basis_schedule != HM_Z_ONLY)
    return fail(err, HM_ERR_ARG, "unknown basis schedule");
  if (p->schedule != HM_SCHED_PLAIN && p->schedule != HM_SCHED_FUSED)
    return fail(err, HM_ERR_ARG, "unknown op schedule %d", p->schedule);
  if (p->no_susceptibility != 0 && p->no_susceptibility != 1)
    return fail(err, HM_ERR_ARG, "no_susceptibility must be 0 or 1");
  const bool dflt = p->meas_col_lo == -1 && p->meas_col_hi == -1;
  if (!dflt && (p->meas_col_lo < 0 || p->meas_col_hi > p->Lx || p->meas_col_lo >= p->meas_col_hi))
    return fail(err, HM_ERR_ARG, "measured columns must satisfy 0 <= lo < hi <= Lx");
  if (p->beta / (2.0 * p->tau) > 1e7) return fail(err, HM_ERR_ARG, "beta / (2 tau) too large");
  return HM_OK;
}

Layout make_layout(const hm_params& p) {
  Layout L;
  L.Lx = p.Lx;
  L.two_W = p.two_W;
  const int wc = p.two_W / 2;
  const int x0 = (p.Lx - wc) / 2;
  for (int x = x0; x < x0 + wc; ++x) L.cluster_cols.push_back(x);
  auto in_cluster = [&](int x) { return x >= x0 && x < x0 + wc; };
  L.phys.assign(2 * p.Lx, -1);
  for (int x = 0; x < p.Lx; ++x) {
    for (int y = 0; y < 2; ++y) {
      L.phys[2 * x + y] = (int)L.kind.size();
      if (in_cluster(x)) {
        if (L.first_cluster < 0) L.first_cluster = (int)L.kind.size();
        L.kind.push_back(SITE_CPHYS);
        L.kind.push_back(SITE_ANC);
      } else {
        L.kind.push_back(SITE_ENV);
        ++L.n_env;
      }
    }
  }
  L.n_sites = (int)L.kind.size();
  for (int x = 0; x < p.Lx; ++x) L.bonds.push_back({L.phys[2 * x], L.phys[2 * x + 1], p.J_rung});
  for (int x = 0; x + 1 < p.Lx; ++x)
    for (int y = 0; y < 2; ++y) L.bonds.push_back({L.phys[2 * x + y], L.phys[2 * (x + 1) + y], p.J_leg});
  std::sort(L.bonds.begin(), L.bonds.end(),
            [](const Bond& a, const Bond& b) { return a.i != b.i ? a.i < b.i : a.j < b.j; });
  int lo = p.meas_col_lo, hi = p.meas_col_hi;
  if (lo == -1 && hi == -1) {
    if (wc > 0) {
      lo = x0;
      hi = x0 + wc;
    } else {
      lo = 0;
      hi = p.Lx;
    }
  }
  std::vector<char> inside(L.n_sites, 0);
  for (int x = lo; x < hi; ++x)
    for (int y = 0; y < 2; ++y) inside[L.phys[2 * x + y]] = 1;
  for (const Bond& b : L.bonds)
    if (inside[b.i] && inside[b.j]) L.meas.push_back(b);
  for (int k = 0; k < L.n_sites; ++k)
    if (inside[k]) L.region.push_back(k);
  if (p.beta == 0.0) {
    L.n_steps = 0;
    L.tau_eff = p.tau;
  } else {
    L.n_steps = std::max(1, (int)std::floor(p.beta / (2.0 * p.tau) + 0.5));
    L.tau_eff = p.beta / (2.0 * L.n_steps);
  }
  L.fused = p.schedule == HM_SCHED_FUSED;
  return L;
}

// Op schedule of one evolution by beta/2 (second order: forward sweep of the
// sorted bonds, then the reversed sweep, each with exp(-(tau/2) J h)).
// Forward gate (i, j): centre at i, swap site i right to j-1, gate on
// (j-1, j), swap back.  Reverse gate: the mirror image around j.  The last
// split of each gate points the centre at the next gate's start; exact
// centre moves (identity gate, no truncation) cover the rest.
std::vector<OpDev> plan(const Layout& L) {
  struct Entry {
    int b;
    bool fwd;
  };
  std::vector<Entry> seq;
  const int nb = (int)L.bonds.size();
  for (int s = 0; s < L.n_steps; ++s) {
    for (int b = 0; b < nb; ++b) seq.push_back({b, true});
    for (int b = nb - 1; b >= 0; --b) seq.push_back({b, false});
  }
  auto start_of = [&](const Entry& e) { return e.fwd ? L.bonds[e.b].i : L.bonds[e.b].j; };
  std::vector<OpDev> ops;
  int c = 0;
  for (size_t t = 0; t < seq.size(); ++t) {
    const Bond& bd = L.bonds[seq[t].b];
    const int tgt = start_of(seq[t]);
    for (; c < tgt; ++c) ops.push_back({c, GATE_ID, 1, 1});
    for (; c > tgt; --c) ops.push_back({c - 1, GATE_ID, 0, 1});
    const int g = GATE_BOND0 + seq[t].b;
    if (seq[t].fwd) {
      for (int k = bd.i; k <= bd.j - 2; ++k) ops.push_back({k, GATE_SWAP, 1, 0});
      ops.push_back({bd.j - 1, g, 0, 0});
      for (int k = bd.j - 2; k >= bd.i; --k) ops.push_back({k, GATE_SWAP, 0, 0});
    } else {
      for (int k = bd.j - 1; k >= bd.i + 1; --k) ops.push_back({k, GATE_SWAP, 0, 0});
      ops.push_back({bd.i, g, 1, 0});
      for (int k = bd.i + 1; k <= bd.j - 1; ++k) ops.push_back({k, GATE_SWAP, 1, 0});
    }
    const int next = t + 1 < seq.size() ? start_of(seq[t + 1]) : 0;
    OpDev& last = ops.back();
    last.absorb = next <= last.k ? 0 : 1;
    c = last.absorb == 0 ? last.k : last.k + 1;
  }
  for (; c > 0; --c) ops.push_back({c - 1, GATE_ID, 0, 1});
  return ops;
}

// exp(-coef h) for h = S_i.S_j of two spin-1 (eigenvalues -2, -1, +1), as a
// sum of spectral projectors P_lambda = prod_{mu != lambda} (h - mu)/(lambda - mu).
void heisenberg_gate(double coef, double G[81]) {
  const double r2 = std::sqrt(2.0);
  double sz[9] = {1, 0, 0, 0, 0, 0, 0, 0, -1};
  double sp[9] = {0, r2, 0, 0, 0, r2, 0, 0, 0};
  double sm[9] = {0, 0, 0, r2, 0, 0, 0, r2, 0};
  double h[81];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d)
          h[(3 * a + b) * 9 + 3 * c + d] =
              sz[a * 3 + c] * sz[b * 3 + d] + 0.5 * (sp[a * 3 + c] * sm[b * 3 + d] + sm[a * 3 + c] * sp[b * 3 + d]);
  auto matmul = [](const double* x, const double* y, double* z) {
    for (int i = 0; i < 9; ++i)
      for (int j = 0; j < 9; ++j) {
        double s = 0.0;
        for (int k = 0; k < 9; ++k) s += x[i * 9 + k] * y[k * 9 + j];
        z[i * 9 + j] = s;
      }
  };
  const double lam[3] = {-2.0, -1.0, 1.0};
  for (int i = 0; i < 81; ++i) G[i] = 0.0;
  for (int l = 0; l < 3; ++l) {
    double P[81], T[81], F[81];
    for (int i = 0; i < 81; ++i) P[i] = (i % 10 == 0) ? 1.0 : 0.0;
    for (int m = 0; m < 3; ++m) {
      if (m == l) continue;
      for (int i = 0; i < 81; ++i) F[i] = (h[i] - ((i % 10 == 0) ? lam[m] : 0.0)) / (lam[l] - lam[m]);
      matmul(P, F, T);
      std::memcpy(P, T, sizeof T);
    }
    const double w = std::exp(-coef * lam[l]);
    for (int i = 0; i < 81; ++i) G[i] += w * P[i];
  }
}

std::vector<double> gate_table(const Layout& L) {
  std::vector<double> g(81 * (GATE_BOND0 + L.bonds.size()), 0.0);
  for (int i = 0; i < 9; ++i) g[GATE_ID * 81 + i * 10] = 1.0;
  for (int s1 = 0; s1 < 3; ++s1)
    for (int s2 = 0; s2 < 3; ++s2) g[GATE_SWAP * 81 + (3 * s2 + s1) * 9 + 3 * s1 + s2] = 1.0;
  for (size_t b = 0; b < L.bonds.size(); ++b)
    heisenberg_gate(0.5 * L.tau_eff * L.bonds[b].J, &g[(GATE_BOND0 + b) * 81]);
  return g;
}

// Ops plus the gate table they index (entries of gate_table first) and each
// entry's GI_* bits: GI_EXCHANGE for an odd number of SWAP letters (the two
// sites' contents change places), GI_MIXING when a bond gate is among the
// letters (the entry then conserves only m1 + m2, Sec. II.C).
struct Schedule {
  std::vector<OpDev> ops;
  std::vector<double> gates;          // n_gates * 81
  std::vector<int32_t> info;          // n_gates
  int32_t n_gates() const { return (int32_t)(gates.size() / 81); }
};

std::vector<int32_t> gate_info_table(const Layout& L) {
  std::vector<int32_t> info(GATE_BOND0 + L.bonds.size(), GI_MIXING);
  info[GATE_ID] = 0;
  info[GATE_SWAP] = GI_EXCHANGE;
  return info;
}

// HM_SCHED_FUSED: one pass over the plain op list with a stack.  A
// truncating split on the pair (k, k+1) that directly follows another
// truncating split on the same pair is folded into it: the gate word grows by
// one letter, and the absorb side becomes the later op's.  Two SWAPs at the
// end of a word annihilate.  When a word empties, its ops vanish; an exact
// centre move replaces them if they had moved the centre.  The folded op can
// then fold into the op below it on the stack.  Each word of two or more
// letters becomes a gate table entry holding the product, the later letters
// on the left.  The gates act on the physical legs only (Sec. I.A), so the
// product of gates on one pair is itself a two-site gate; the state without
// truncation is unchanged.
void fuse_schedule(Schedule& s) {
  struct Item {
    OpDev op;
    int c0;                           // centre before the op
    std::vector<int32_t> word;        // gate letters, first applied first
  };
  std::vector<Item> st;
  int c = 0;
  for (const OpDev& op : s.ops) {
    const int c1 = op.absorb ? op.k + 1 : op.k;
    if (!op.exact && !st.empty() && !st.back().op.exact && st.back().op.k == op.k) {
      Item it = std::move(st.back());
      st.pop_back();
      it.word.push_back(op.gate);
      const size_t n = it.word.size();
      if (n >= 2 && it.word[n - 1] == GATE_SWAP && it.word[n - 2] == GATE_SWAP) it.word.resize(n - 2);
      if (!it.word.empty()) {
        it.op.absorb = op.absorb;
        st.push_back(std::move(it));
      } else if (it.c0 != c1) {
        st.push_back({{op.k, GATE_ID, c1 == op.k + 1 ? 1 : 0, 1}, it.c0, {GATE_ID}});
      }
      c = c1;
      continue;
    }
    st.push_back({op, c, {op.gate}});
    c = c1;
  }
  std::map<std::vector<int32_t>, int32_t> entry;
  std::vector<OpDev> ops;
  ops.reserve(st.size());
  for (Item& it : st) {
    if (it.word.size() > 1) {
      auto f = entry.find(it.word);
      if (f == entry.end()) {
        double P[81], T[81];
        std::memcpy(P, &s.gates[(size_t)it.word[0] * 81], sizeof P);
        for (size_t q = 1; q < it.word.size(); ++q) {
          const double* G = &s.gates[(size_t)it.word[q] * 81];
          for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) {
              double acc = 0.0;
              for (int t = 0; t < 9; ++t) acc += G[i * 9 + t] * P[t * 9 + j];
              T[i * 9 + j] = acc;
            }
          std::memcpy(P, T, sizeof P);
        }
        f = entry.emplace(it.word, s.n_gates()).first;
        s.gates.insert(s.gates.end(), P, P + 81);
        int32_t inf = 0;
        for (int32_t g : it.word) {
          if (s.info[g] & GI_EXCHANGE) inf ^= GI_EXCHANGE;
          inf |= s.info[g] & GI_MIXING;
        }
        s.info.push_back(inf);
      }
      it.op.gate = f->second;
    } else {
      it.op.gate = it.word[0];
    }
    ops.push_back(it.op);
  }
  s.ops.swap(ops);
}

Schedule make_schedule(const Layout& L) {
  Schedule s{plan(L), gate_table(L), gate_info_table(L)};
  if (L.fused) fuse_schedule(s);
  return s;
}

// ---------------------------------------------------------------------------
// Memory plan of one chain (all inside one arena block).
// ---------------------------------------------------------------------------

struct MemPlan {
  std::vector<int64_t> bmax;         // n_sites + 1 bond caps
  std::vector<int64_t> slot_off;     // byte offsets of site slots
  int64_t ws_cap = 0, env_cap = 0;
  int32_t sv_cap = 0, chi_cap = 0;
  size_t off_desc, off_ops, off_gates, off_kind, off_mi, off_mj, off_mJ, off_ms, off_reg, off_xb, off_siteptr, off_chi,
      off_env, off_cnt, off_stats, off_status, off_theta, off_W, off_V, off_sig, off_perm, off_envws,
      off_ginfo, off_qn, off_sgn, off_meta, off_X, off_slots, total;
};

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// chi_cap x chi_cap matrices the susceptibility kernel keeps in env_ws.
int64_t susceptibility_matrices(const Layout& L) { return 20 + 4 * (int64_t)L.region.size(); }

MemPlan mem_plan(const hm_params& p, const Layout& L, size_t n_ops, size_t n_gates) {
  MemPlan m;
  const int n = L.n_sites;
  m.bmax.resize(n + 1);
  for (int i = 0; i <= n; ++i) {
    int64_t cap = 1;
    const int e = std::min(i, n - i);
    for (int t = 0; t < e && cap < p.chi_max; ++t) cap *= 3;
    m.bmax[i] = std::min<int64_t>(cap, p.chi_max);
    // a Bell pair (cluster physical site i-1, ancilla i) starts at bond dim 3
    if (i > 0 && i < n && L.kind[i - 1] == SITE_CPHYS) m.bmax[i] = std::max<int64_t>(m.bmax[i], 3);
  }
  for (int i = 0; i <= n; ++i) m.chi_cap = std::max<int32_t>(m.chi_cap, (int32_t)m.bmax[i]);
  for (int k = 0; k + 1 < n; ++k) {
    const int64_t mm = 3 * m.bmax[k], nn = 3 * m.bmax[k + 2];
    m.ws_cap = std::max(m.ws_cap, mm * nn);
    m.sv_cap = std::max<int32_t>(m.sv_cap, (int32_t)std::min(mm, nn));
  }
  // theta doubles as the split's value lists (4 sv_cap + 1 doubles)
  m.ws_cap = std::max<int64_t>(m.ws_cap, 4 * (int64_t)m.sv_cap + 8);
  if (n == 1) m.ws_cap = 64, m.sv_cap = 3;
  // transfer workspace: 10 chi x chi matrices + one right environment per
  // distinct measured end site (measure); the collapse uses the first 7
  std::vector<int> ends;
  for (const Bond& b : L.meas)
    if (std::find(ends.begin(), ends.end(), b.j) == ends.end()) ends.push_back(b.j);
  // the susceptibility sweeps use 20 matrices + 4 stored per region site
  const int64_t sus = p.no_susceptibility ? 0 : susceptibility_matrices(L);
  m.env_cap = std::max<int64_t>(10 + (int64_t)ends.size(), sus) * m.chi_cap * m.chi_cap;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  m.off_desc = take(sizeof(ChainDev));
  m.off_ops = take(std::max<size_t>(n_ops, 1) * sizeof(OpDev));
  m.off_gates = take(81 * sizeof(double) * n_gates);
  m.off_ginfo = take(n_gates * sizeof(int32_t));
  m.off_kind = take(n * sizeof(int32_t));
  m.off_mi = take(std::max<size_t>(L.meas.size(), 1) * sizeof(int32_t));
  m.off_mj = take(std::max<size_t>(L.meas.size(), 1) * sizeof(int32_t));
  m.off_mJ = take(std::max<size_t>(L.meas.size(), 1) * sizeof(double));
  m.off_ms = take(std::max<size_t>(L.meas.size(), 1) * sizeof(int32_t));
  m.off_reg = take(std::max<size_t>(L.region.size(), 1) * sizeof(int32_t));
  m.off_xb = take(9 * sizeof(double));
  m.off_siteptr = take(n * sizeof(double*));
  m.off_chi = take((n + 1) * sizeof(int32_t));
  m.off_env = take(std::max(L.n_env, 1) * sizeof(int32_t));
  m.off_cnt = take(8 * sizeof(int32_t));
  m.off_stats = take(ST_N * sizeof(double));
  m.off_status = take(2 * sizeof(int32_t));
  m.off_theta = take(m.ws_cap * sizeof(double));
  m.off_W = take(m.ws_cap * sizeof(double));
  m.off_V = take(m.ws_cap * sizeof(double));
  m.off_sig = take(m.sv_cap * sizeof(double));
  m.off_perm = take(m.sv_cap * sizeof(int32_t));
  m.off_envws = take(m.env_cap * sizeof(double));
  m.off_qn = take((size_t)(n + 1) * m.chi_cap * sizeof(int16_t));
  m.off_sgn = take(n * sizeof(int32_t));
  m.off_meta = take(kMetaBytes);
  // binary32 Jacobi of a charge block too large for shared memory (mixed)
  m.off_X = p.precision != HM_FP64 ? take(m.ws_cap * sizeof(double)) : 0;
  m.slot_off.resize(n);
  for (int s = 0; s < n; ++s) m.slot_off[s] = take(m.bmax[s] * 3 * m.bmax[s + 1] * sizeof(double));
  m.total = off;
  return m;
}

// ---------------------------------------------------------------------------
// Arena: first-fit free list over the caller's device buffer.
// ---------------------------------------------------------------------------

struct Arena {
  std::map<size_t, size_t> free_;    // offset -> size
  size_t size = 0;
  void init(size_t bytes) {
    size = bytes;
    free_.clear();
    if (bytes) free_[0] = bytes;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t noff = it->first + bytes;
        free_.erase(it);
        if (rest) free_[noff] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t largest() const {
    size_t m = 0;
    for (auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }
};

struct Chain {
  hm_params p;
  Layout L;
  MemPlan mp;
  std::vector<OpDev> ops;
  int32_t n_gates = 0;              // gate table entries on the device
  double cost = 0.0;                // dense-SVD flops of all ops at the bond caps
  size_t off = 0;
  ChainDev* dev = nullptr;          // device address of the descriptor
  int phase = 0;                    // 0 initial state, 1 evolved
  int cursor = 0;                   // ops done by hm_evolve_partial (mirror of counters[4])
  int n_obs = 0;
};

}  // namespace

struct hm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  char* base = nullptr;
  Arena arena;
  std::map<int64_t, Chain*> chains;
  int64_t next_id = 1;
  std::string err;
  int32_t* err_word = nullptr;      // device
  size_t err_off = 0;
};

namespace {

int cuda_fail(hm_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx ? &ctx->err : nullptr, HM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define HM_CUDA(ctx, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

int lookup(hm_ctx* ctx, const hm_chain* ids, int32_t n, std::vector<Chain*>* out) {
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  if (n < 0 || (n > 0 && !ids)) return fail(&ctx->err, HM_ERR_ARG, "bad chain list");
  out->clear();
  for (int32_t i = 0; i < n; ++i) {
    auto it = ctx->chains.find(ids[i]);
    if (it == ctx->chains.end()) return fail(&ctx->err, HM_ERR_ARG, "unknown chain handle %lld", (long long)ids[i]);
    out->push_back(it->second);
  }
  return HM_OK;
}

// Reads and clears the context's device error word (synchronising).
int check_device_error(hm_ctx* ctx) {
  int32_t code = 0;
  HM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  HM_CUDA(ctx, cudaMemcpy(&code, ctx->err_word, sizeof code, cudaMemcpyDeviceToHost));
  if (code != 0) {
    const int32_t zero = 0;
    HM_CUDA(ctx, cudaMemcpy(ctx->err_word, &zero, sizeof zero, cudaMemcpyHostToDevice));
    return fail(&ctx->err, code, "device step failed (%s)",
                code == HM_ERR_NUMERIC ? "SVD not converged or non-finite probability" : "device error");
  }
  return HM_OK;
}

template <typename F>
int for_batches(const std::vector<Chain*>& cs, F&& f) {
  for (size_t s = 0; s < cs.size(); s += kMaxBatch) {
    BatchArg b{};
    b.n = (int32_t)std::min<size_t>(kMaxBatch, cs.size() - s);
    for (int i = 0; i < b.n; ++i) b.c[i] = cs[s + i]->dev;
    const int rc = f(b, (int)s);
    if (rc != HM_OK) return rc;
  }
  return HM_OK;
}

struct Scratch {   // temporary arena block for host-output calls
  hm_ctx* ctx;
  size_t off = 0, bytes = 0;
  char* ptr = nullptr;
  int get(size_t nbytes) {
    if (!ctx->arena.alloc(nbytes, &off)) return fail(&ctx->err, HM_ERR_NOMEM, "arena full (staging)");
    bytes = nbytes;
    ptr = ctx->base + off;
    return HM_OK;
  }
  ~Scratch() {
    if (ptr) ctx->arena.release(off, bytes);
  }
};

}  // namespace

void hm::set_global_error(const char* msg) { g_err = msg; }

namespace {
// Named NVTX range over one entry point (a no-op unless a profiler attaches).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};
}  // namespace

extern "C" {

int hm_create(hm_ctx** out, int device, void* dev_mem, size_t bytes, void* cuda_stream) {
  if (!out || !dev_mem || bytes < 4096) return fail(nullptr, HM_ERR_ARG, "hm_create: bad arguments");
  if (reinterpret_cast<uintptr_t>(dev_mem) % 256) return fail(nullptr, HM_ERR_ARG, "arena must be 256-byte aligned");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
  hm_ctx* ctx = new hm_ctx;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->base = (char*)dev_mem;
  ctx->arena.init(bytes);
  if (!ctx->arena.alloc(256, &ctx->err_off)) {
    delete ctx;
    return fail(nullptr, HM_ERR_NOMEM, "arena too small");
  }
  ctx->err_word = (int32_t*)(ctx->base + ctx->err_off);
  e = cudaMemsetAsync(ctx->err_word, 0, 256, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail(nullptr, e, "hm_create");
  }
  *out = ctx;
  return HM_OK;
}

int hm_destroy(hm_ctx* ctx) {
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->chains) delete kv.second;
  delete ctx;
  return HM_OK;
}

// Limits a chain's kernels place on its bond caps: the mixed evolve stages
// column blocks in shared memory, so its footprint at the largest cap must
// fit what one CTA may opt into.
static int check_kernel_limits(const hm_params& p, const MemPlan& m, std::string* err) {
  int bcols = 0;
  if (p.precision != HM_FP64 && mixed_smem_bytes(m.chi_cap, &bcols) > kMaxSharedOptIn)
    return fail(err, HM_ERR_ARG, "chi cap %d needs %zu bytes of shared memory in the mixed evolve (max %zu)",
                m.chi_cap, mixed_smem_bytes(m.chi_cap, &bcols), kMaxSharedOptIn);
  return HM_OK;
}

int hm_query_memory(const hm_params* p, size_t* bytes_out) {
  int rc = check_params(p, nullptr);
  if (rc) return rc;
  if (!bytes_out) return fail(nullptr, HM_ERR_ARG, "null output");
  const Layout L = make_layout(*p);
  const Schedule sc = make_schedule(L);
  const MemPlan m = mem_plan(*p, L, sc.ops.size(), sc.gates.size() / 81);
  rc = check_kernel_limits(*p, m, nullptr);
  if (rc) return rc;
  *bytes_out = m.total;
  return HM_OK;
}

int hm_num_obs(const hm_params* p, int32_t* n_obs) {
  int rc = check_params(p, nullptr);
  if (rc) return rc;
  if (!n_obs) return fail(nullptr, HM_ERR_ARG, "null output");
  *n_obs = 1 + 2 * (int32_t)make_layout(*p).meas.size();
  return HM_OK;
}

int hm_num_env(const hm_params* p, int32_t* n_env) {
  int rc = check_params(p, nullptr);
  if (rc) return rc;
  if (!n_env) return fail(nullptr, HM_ERR_ARG, "null output");
  *n_env = make_layout(*p).n_env;
  return HM_OK;
}

int hm_plan(const hm_params* p, int32_t* ops, int32_t cap, int32_t* n_ops_out) {
  int rc = check_params(p, nullptr);
  if (rc) return rc;
  if (!n_ops_out) return fail(nullptr, HM_ERR_ARG, "null output");
  const std::vector<OpDev> v = make_schedule(make_layout(*p)).ops;
  *n_ops_out = (int32_t)v.size();
  if (ops) {
    if (cap < (int32_t)v.size()) return fail(nullptr, HM_ERR_ARG, "op buffer too small (%zu ops)", v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      ops[4 * i] = v[i].k;
      ops[4 * i + 1] = v[i].gate;
      ops[4 * i + 2] = v[i].absorb;
      ops[4 * i + 3] = v[i].exact;
    }
  }
  return HM_OK;
}

int hm_gates(const hm_params* p, double* out, int32_t cap, int32_t* n_gates_out) {
  int rc = check_params(p, nullptr);
  if (rc) return rc;
  if (!n_gates_out) return fail(nullptr, HM_ERR_ARG, "null output");
  const std::vector<double> g = make_schedule(make_layout(*p)).gates;
  *n_gates_out = (int32_t)(g.size() / 81);
  if (out) {
    if ((size_t)cap * 81 < g.size()) return fail(nullptr, HM_ERR_ARG, "gate buffer too small");
    std::memcpy(out, g.data(), g.size() * sizeof(double));
  }
  return HM_OK;
}

// Allocation and first initial state of a chain; next_sample > 0 resumes a
// checkpoint: the counters start at (n = next_sample, basis of sample n - 1).
static int init_chain_impl(hm_ctx* ctx, const hm_params* p, const int8_t* env_init, int64_t next_sample,
                           hm_chain* out) {
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  int rc = check_params(p, &ctx->err);
  if (rc) return rc;
  if (!out) return fail(&ctx->err, HM_ERR_ARG, "null output handle");
  HM_CUDA(ctx, cudaSetDevice(ctx->device));
  Chain* ch = new Chain;
  ch->p = *p;
  ch->L = make_layout(*p);
  Schedule sched = make_schedule(ch->L);
  ch->ops = std::move(sched.ops);
  ch->n_gates = sched.n_gates();
  ch->mp = mem_plan(*p, ch->L, ch->ops.size(), sched.gates.size() / 81);
  for (const OpDev& op : ch->ops) {
    const double m = 3.0 * ch->mp.bmax[op.k], q = 3.0 * ch->mp.bmax[op.k + 2];
    const double M = std::max(m, q), N = std::min(m, q);
    ch->cost += 4.0 * M * M * N + 8.0 * M * N * N + 9.0 * N * N * N;
  }
  ch->n_obs = 1 + 2 * (int)ch->L.meas.size();
  rc = check_kernel_limits(*p, ch->mp, &ctx->err);
  if (rc) {
    delete ch;
    return rc;
  }
  {
    // at most 8 measured bonds may start on one site (measure kernel buffer)
    std::map<int, int> starts;
    for (const Bond& b : ch->L.meas)
      if (++starts[b.i] > 8) {
        delete ch;
        return fail(&ctx->err, HM_ERR_ARG, "too many measured bonds on one site");
      }
  }
  if (env_init)
    for (int e = 0; e < ch->L.n_env; ++e)
      if (env_init[e] < 0 || env_init[e] > 2) {
        delete ch;
        return fail(&ctx->err, HM_ERR_ARG, "env_init values must be 0, 1 or 2");
      }
  const MemPlan& mp = ch->mp;
  if (!ctx->arena.alloc(mp.total, &ch->off)) {
    delete ch;
    return fail(&ctx->err, HM_ERR_NOMEM, "arena cannot hold the chain (%zu bytes needed, largest free %zu)",
                mp.total, ctx->arena.largest());
  }
  char* base = ctx->base + ch->off;
  // host image of the static part [0, off_theta)
  std::vector<char> img(mp.off_theta, 0);
  ChainDev d{};
  const Layout& L = ch->L;
  d.n_sites = L.n_sites;
  d.n_ops = (int32_t)ch->ops.size();
  d.chi_max = p->chi_max;
  d.n_env = L.n_env;
  d.n_meas = (int32_t)L.meas.size();
  d.n_gates = sched.n_gates();
  d.basis_zx = p->basis_schedule == HM_ZX_ALTERNATE;
  d.first_cluster = L.first_cluster;
  d.seed_lo = (uint32_t)(p->seed & 0xFFFFFFFFu);
  d.seed_hi = (uint32_t)(p->seed >> 32);
  d.chain_id = p->chain_id;
  d.cutoff = p->cutoff;
  d.ops = (const OpDev*)(base + mp.off_ops);
  d.gates = (const double*)(base + mp.off_gates);
  d.site_kind = (const int32_t*)(base + mp.off_kind);
  d.meas_i = (const int32_t*)(base + mp.off_mi);
  d.meas_j = (const int32_t*)(base + mp.off_mj);
  d.meas_J = (const double*)(base + mp.off_mJ);
  d.meas_slot = (const int32_t*)(base + mp.off_ms);
  d.region = (const int32_t*)(base + mp.off_reg);
  d.n_region = (int32_t)L.region.size();
  d.xbasis = (const double*)(base + mp.off_xb);
  d.site = (double**)(base + mp.off_siteptr);
  d.chi = (int32_t*)(base + mp.off_chi);
  d.env_out = (int32_t*)(base + mp.off_env);
  d.counters = (int32_t*)(base + mp.off_cnt);
  d.stats = (double*)(base + mp.off_stats);
  d.status = (int32_t*)(base + mp.off_status);
  d.err_where = d.status + 1;
  d.theta = (double*)(base + mp.off_theta);
  d.W = (double*)(base + mp.off_W);
  d.V = (double*)(base + mp.off_V);
  d.sig = (double*)(base + mp.off_sig);
  d.perm = (int32_t*)(base + mp.off_perm);
  d.env_ws = (double*)(base + mp.off_envws);
  d.gate_info = (const int32_t*)(base + mp.off_ginfo);
  d.qn = (int16_t*)(base + mp.off_qn);
  d.sgn = (int32_t*)(base + mp.off_sgn);
  d.meta = base + mp.off_meta;
  d.X = p->precision != HM_FP64 ? (float*)(base + mp.off_X) : nullptr;
  d.ws_cap = mp.ws_cap;
  d.env_cap = mp.env_cap;
  d.sv_cap = mp.sv_cap;
  d.chi_cap = mp.chi_cap;
  std::memcpy(img.data() + mp.off_desc, &d, sizeof d);
  if (!ch->ops.empty()) std::memcpy(img.data() + mp.off_ops, ch->ops.data(), ch->ops.size() * sizeof(OpDev));
  std::memcpy(img.data() + mp.off_gates, sched.gates.data(), sched.gates.size() * sizeof(double));
  std::memcpy(img.data() + mp.off_ginfo, sched.info.data(), sched.info.size() * sizeof(int32_t));
  std::memcpy(img.data() + mp.off_kind, L.kind.data(), L.kind.size() * sizeof(int32_t));
  std::vector<int> ends;
  for (size_t q = 0; q < L.meas.size(); ++q) {
    ((int32_t*)(img.data() + mp.off_mi))[q] = L.meas[q].i;
    ((int32_t*)(img.data() + mp.off_mj))[q] = L.meas[q].j;
    ((double*)(img.data() + mp.off_mJ))[q] = L.meas[q].J;
    auto it = std::find(ends.begin(), ends.end(), L.meas[q].j);
    if (it == ends.end()) {
      ends.push_back(L.meas[q].j);
      it = ends.end() - 1;
    }
    ((int32_t*)(img.data() + mp.off_ms))[q] = (int32_t)(it - ends.begin());
  }
  if (!L.region.empty())
    std::memcpy(img.data() + mp.off_reg, L.region.data(), L.region.size() * sizeof(int32_t));
  const double r = 1.0 / std::sqrt(2.0);
  const double xb[9] = {0.5, r, 0.5, r, 0.0, -r, 0.5, -r, 0.5};
  std::memcpy(img.data() + mp.off_xb, xb, sizeof xb);
  for (int s = 0; s < L.n_sites; ++s) ((double**)(img.data() + mp.off_siteptr))[s] = (double*)(base + mp.slot_off[s]);
  if (env_init)
    for (int e = 0; e < L.n_env; ++e) ((int32_t*)(img.data() + mp.off_env))[e] = env_init[e];
  {
    int32_t* cnt = (int32_t*)(img.data() + mp.off_cnt);
    cnt[0] = (int32_t)next_sample;
    cnt[1] = (next_sample > 0 && p->basis_schedule == HM_ZX_ALTERNATE && ((next_sample - 1) & 1)) ? 1 : 0;
  }
  cudaError_t e = cudaMemcpyAsync(base, img.data(), img.size(), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    ctx->arena.release(ch->off, mp.total);
    delete ch;
    return cuda_fail(ctx, e, "hm_init_chain upload");
  }
  ch->dev = (ChainDev*)(base + mp.off_desc);
  BatchArg b{};
  b.n = 1;
  b.c[0] = ch->dev;
  OutArg o{};
  o.ctx_err = ctx->err_word;
  rc = launch_reset(b, o, env_init ? 0 : 1, ctx->stream);
  if (rc != HM_OK) {
    ctx->arena.release(ch->off, mp.total);
    delete ch;
    return fail(&ctx->err, rc, "reset kernel launch failed");
  }
  const hm_chain id = ctx->next_id++;
  ctx->chains[id] = ch;
  *out = id;
  return HM_OK;
}

int hm_init_chain(hm_ctx* ctx, const hm_params* p, const int8_t* env_init, hm_chain* out) {
  return init_chain_impl(ctx, p, env_init, 0, out);
}

int hm_resume_chain(hm_ctx* ctx, const hm_params* p, const int8_t* env_out, int64_t next_sample,
                    hm_chain* out) {
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  if (next_sample < 1 || next_sample > INT32_MAX)
    return fail(&ctx->err, HM_ERR_ARG, "next_sample must be in [1, 2^31 - 1] (hm_init_chain starts at 0)");
  if (!env_out) return fail(&ctx->err, HM_ERR_ARG, "a resumed chain needs its environment outcomes");
  return init_chain_impl(ctx, p, env_out, next_sample, out);
}

int hm_free_chain(hm_ctx* ctx, hm_chain chain) {
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  auto it = ctx->chains.find(chain);
  if (it == ctx->chains.end()) return fail(&ctx->err, HM_ERR_ARG, "unknown chain handle");
  HM_CUDA(ctx, cudaSetDevice(ctx->device));
  HM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->arena.release(it->second->off, it->second->mp.total);
  delete it->second;
  ctx->chains.erase(it);
  return HM_OK;
}

// Evolve launches of a chain list: one group per precision, costliest chains
// first, batches of <= kMaxBatch; budget 0 runs whole op lists (in chunks of
// 4096 ops), budget > 0 advances every chain's own cursor by <= budget ops.
static int evolve_launches(hm_ctx* ctx, const std::vector<Chain*>& cs, int budget) {
  OutArg o{};
  o.ctx_err = ctx->err_word;
  for (int prec : {HM_FP64, HM_MIXED, HM_MIXED32}) {
    std::vector<Chain*> group;
    int chi_cap = 1;
    for (Chain* c : cs)
      if (c->p.precision == prec) {
        group.push_back(c);
        chi_cap = std::max<int>(chi_cap, c->mp.chi_cap);
      }
    // Costliest chains first: CTAs start roughly in index order, so an
    // uneven batch ends closer to its average load (longest processing time
    // first), and each launch of <= kMaxBatch chains holds similar costs.
    // Equal costs keep the caller's order.
    std::stable_sort(group.begin(), group.end(), [](const Chain* a, const Chain* b) { return a->cost > b->cost; });
    const int rc = for_batches(group, [&](BatchArg& b, int s) {
      auto launch = [&]() {
        return prec == HM_FP64 ? launch_evolve_fp64(b, o, ctx->stream)
                               : launch_evolve_mixed(b, o, chi_cap, prec == HM_MIXED, ctx->stream);
      };
      if (budget > 0) {
        b.budget = budget;
        return launch();
      }
      const int chunk = 4096;
      int batch_ops = 0;                          // this launch's longest op list
      for (int i = 0; i < b.n; ++i) batch_ops = std::max<int>(batch_ops, (int)group[s + i]->ops.size());
      for (int t0 = 0; t0 < batch_ops; t0 += chunk) {
        b.t0 = t0;
        b.t1 = t0 + chunk;
        const int r = launch();
        if (r != HM_OK) return r;
      }
      return HM_OK;
    });
    if (rc != HM_OK) return fail(&ctx->err, rc, "evolve launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
  return HM_OK;
}

int hm_evolve_partial(hm_ctx* ctx, const hm_chain* ids, int32_t n, int32_t max_ops, int32_t* done_out) {
  Range range("hm_evolve_partial");
  std::vector<Chain*> cs;
  int rc = lookup(ctx, ids, n, &cs);
  if (rc) return rc;
  if (max_ops < 1) return fail(&ctx->err, HM_ERR_ARG, "max_ops must be >= 1");
  for (Chain* c : cs)
    if (c->phase != 0) return fail(&ctx->err, HM_ERR_STATE, "hm_evolve_partial needs a chain that is not yet evolved");
  HM_CUDA(ctx, cudaSetDevice(ctx->device));
  rc = evolve_launches(ctx, cs, max_ops);
  if (rc) return rc;
  for (int32_t i = 0; i < n; ++i) {
    Chain* c = cs[i];
    c->cursor = std::min<int>(c->cursor + max_ops, (int)c->ops.size());
    const int done = c->cursor >= (int)c->ops.size();
    if (done) {
      c->phase = 1;
      c->cursor = 0;
    }
    if (done_out) done_out[i] = done;
  }
  return HM_OK;
}

int hm_evolve(hm_ctx* ctx, const hm_chain* ids, int32_t n) {
  Range range("hm_evolve");
  std::vector<Chain*> cs;
  int rc = lookup(ctx, ids, n, &cs);
  if (rc) return rc;
  for (Chain* c : cs)
    if (c->phase != 0 || c->cursor != 0)
      return fail(&ctx->err, HM_ERR_STATE, "hm_evolve needs a chain in its initial state");
  HM_CUDA(ctx, cudaSetDevice(ctx->device));
  rc = evolve_launches(ctx, cs, 0);
  if (rc) return rc;
  for (Chain* c : cs) c->phase = 1;
  return HM_OK;
}

static int measure_impl(hm_ctx* ctx, const hm_chain* ids, int32_t n, double* out_dev, int32_t n_obs,
                        std::vector<Chain*>& cs) {
  int rc = lookup(ctx, ids, n, &cs);
  if (rc) return rc;
  for (Chain* c : cs) {
    if (c->phase != 1) return fail(&ctx->err, HM_ERR_STATE, "measure needs an evolved chain");
    if (c->n_obs != n_obs) return fail(&ctx->err, HM_ERR_ARG, "n_obs %d does not match the chain's %d", n_obs, c->n_obs);
  }
  HM_CUDA(ctx, cudaSetDevice(ctx->device));
  OutArg o{};
  o.ctx_err = ctx->err_word;
  o.n_obs = n_obs;
  rc = for_batches(cs, [&](BatchArg& b, int s) {
    o.obs = out_dev + (size_t)s * n_obs;
    return launch_measure_fp64(b, o, ctx->stream);
  });
  if (rc != HM_OK) return fail(&ctx->err, rc, "measure launch failed");
  return HM_OK;
}

int hm_measure_cluster_device(hm_ctx* ctx, const hm_chain* ids, int32_t n, double* out_dev, int32_t n_obs) {
  Range range("hm_measure_cluster_device");
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  if (!out_dev && n > 0) return fail(&ctx->err, HM_ERR_ARG, "null output");
  std::vector<Chain*> cs;
  return measure_impl(ctx, ids, n, out_dev, n_obs, cs);
}

int hm_measure_cluster(hm_ctx* ctx, const hm_chain* ids, int32_t n, double* out, int32_t n_obs) {
  Range range("hm_measure_cluster");
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  if (!out && n > 0) return fail(&ctx->err, HM_ERR_ARG, "null output");
  if (n == 0) return HM_OK;
  Scratch sc{ctx};
  int rc = sc.get((size_t)n * n_obs * sizeof(double));
  if (rc) return rc;
  std::vector<Chain*> cs;
  rc = measure_impl(ctx, ids, n, (double*)sc.ptr, n_obs, cs);
  if (rc) return rc;
  HM_CUDA(ctx, cudaMemcpyAsync(out, sc.ptr, (size_t)n * n_obs * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return check_device_error(ctx);
}

int hm_measure_susceptibility(hm_ctx* ctx, const hm_chain* ids, int32_t n, double* out) {
  Range range("hm_measure_susceptibility");
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  if (n == 0) return HM_OK;
  if (!out) return fail(&ctx->err, HM_ERR_ARG, "null output");
  std::vector<Chain*> cs;
  int rc = lookup(ctx, ids, n, &cs);
  if (rc) return rc;
  for (Chain* c : cs) {
    if (c->phase != 1) return fail(&ctx->err, HM_ERR_STATE, "the susceptibility needs an evolved chain");
    // the kernel assumes its workspace: never launch it on a chain without one
    if (c->mp.env_cap < susceptibility_matrices(c->L) * c->mp.chi_cap * c->mp.chi_cap)
      return fail(&ctx->err, HM_ERR_ARG, "chain was created with no_susceptibility = 1");
  }
  HM_CUDA(ctx, cudaSetDevice(ctx->device));
  Scratch sc{ctx};
  rc = sc.get((size_t)n * sizeof(double));
  if (rc) return rc;
  OutArg o{};
  o.ctx_err = ctx->err_word;
  o.n_obs = 1;
  rc = for_batches(cs, [&](BatchArg& b, int s) {
    o.obs = (double*)sc.ptr + s;
    return launch_susceptibility_fp64(b, o, ctx->stream);
  });
  if (rc != HM_OK) return fail(&ctx->err, rc, "susceptibility launch failed");
  std::vector<double> raw(n);
  HM_CUDA(ctx, cudaMemcpyAsync(raw.data(), sc.ptr, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  rc = check_device_error(ctx);
  if (rc) return rc;
  for (int32_t i = 0; i < n; ++i) {
    const double nr = (double)cs[i]->L.region.size();
    out[2 * i] = cs[i]->p.beta / 3.0 * raw[i] / nr;
    out[2 * i + 1] = raw[i];
  }
  return HM_OK;
}

static int collapse_impl(hm_ctx* ctx, const hm_chain* ids, int32_t n, int8_t* env_dev, double* logp_dev,
                         std::vector<Chain*>& cs, double* cond_dev = nullptr) {
  int rc = lookup(ctx, ids, n, &cs);
  if (rc) return rc;
  int n_env = -1;
  for (Chain* c : cs) {
    if (c->phase != 1) return fail(&ctx->err, HM_ERR_STATE, "collapse needs an evolved chain");
    if ((env_dev || cond_dev) && n_env >= 0 && c->L.n_env != n_env)
      return fail(&ctx->err, HM_ERR_ARG, "chains of one collapse call must share n_env when env_out is given");
    n_env = c->L.n_env;
  }
  HM_CUDA(ctx, cudaSetDevice(ctx->device));
  OutArg o{};
  o.ctx_err = ctx->err_word;
  o.n_env = std::max(n_env, 0);
  rc = for_batches(cs, [&](BatchArg& b, int s) {
    o.env = env_dev ? env_dev + (size_t)s * o.n_env : nullptr;
    o.logp = logp_dev ? logp_dev + s : nullptr;
    o.cond = cond_dev ? cond_dev + (size_t)s * o.n_env * 3 : nullptr;
    return launch_collapse_fp64(b, o, ctx->stream);
  });
  if (rc != HM_OK) return fail(&ctx->err, rc, "collapse launch failed");
  for (Chain* c : cs) c->phase = 0;
  return HM_OK;
}

int hm_collapse_device(hm_ctx* ctx, const hm_chain* ids, int32_t n, int8_t* env_out_dev, double* logp_out_dev) {
  Range range("hm_collapse_device");
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  std::vector<Chain*> cs;
  return collapse_impl(ctx, ids, n, env_out_dev, logp_out_dev, cs);
}

int hm_collapse(hm_ctx* ctx, const hm_chain* ids, int32_t n, int8_t* env_out, double* logp_out) {
  Range range("hm_collapse");
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  if (n == 0) return HM_OK;
  if (!env_out && !logp_out) {
    std::vector<Chain*> cs;
    return collapse_impl(ctx, ids, n, nullptr, nullptr, cs);
  }
  std::vector<Chain*> cs;
  int rc = lookup(ctx, ids, n, &cs);
  if (rc) return rc;
  const size_t n_env = cs.empty() ? 0 : (size_t)cs[0]->L.n_env;
  const size_t env_bytes = align_up(std::max<size_t>((size_t)n * n_env, 1));
  Scratch sc{ctx};
  rc = sc.get(env_bytes + (size_t)n * sizeof(double));
  if (rc) return rc;
  int8_t* env_dev = (int8_t*)sc.ptr;
  double* logp_dev = (double*)(sc.ptr + env_bytes);
  rc = collapse_impl(ctx, ids, n, env_out ? env_dev : nullptr, logp_out ? logp_dev : nullptr, cs);
  if (rc) return rc;
  if (env_out && n_env)
    HM_CUDA(ctx, cudaMemcpyAsync(env_out, env_dev, (size_t)n * n_env, cudaMemcpyDeviceToHost, ctx->stream));
  if (logp_out)
    HM_CUDA(ctx, cudaMemcpyAsync(logp_out, logp_dev, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return check_device_error(ctx);
}

int hm_collapse_conditionals(hm_ctx* ctx, const hm_chain* ids, int32_t n, int8_t* env_out, double* logp_out,
                             double* cond_out) {
  Range range("hm_collapse_conditionals");
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  if (n == 0) return HM_OK;
  if (!env_out || !logp_out || !cond_out) return fail(&ctx->err, HM_ERR_ARG, "null output");
  std::vector<Chain*> cs;
  int rc = lookup(ctx, ids, n, &cs);
  if (rc) return rc;
  const size_t n_env = (size_t)cs[0]->L.n_env;
  const size_t env_bytes = align_up(std::max<size_t>((size_t)n * n_env, 1));
  const size_t cond_bytes = align_up(std::max<size_t>((size_t)n * n_env * 3 * sizeof(double), 8));
  Scratch sc{ctx};
  rc = sc.get(env_bytes + cond_bytes + (size_t)n * sizeof(double));
  if (rc) return rc;
  int8_t* env_dev = (int8_t*)sc.ptr;
  double* cond_dev = (double*)(sc.ptr + env_bytes);
  double* logp_dev = (double*)(sc.ptr + env_bytes + cond_bytes);
  rc = collapse_impl(ctx, ids, n, env_dev, logp_dev, cs, cond_dev);
  if (rc) return rc;
  if (n_env) {
    HM_CUDA(ctx, cudaMemcpyAsync(env_out, env_dev, (size_t)n * n_env, cudaMemcpyDeviceToHost, ctx->stream));
    HM_CUDA(ctx, cudaMemcpyAsync(cond_out, cond_dev, (size_t)n * n_env * 3 * sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->stream));
  }
  HM_CUDA(ctx, cudaMemcpyAsync(logp_out, logp_dev, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return check_device_error(ctx);
}

int hm_chain_stats(hm_ctx* ctx, hm_chain chain, double* out) {
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  auto it = ctx->chains.find(chain);
  if (it == ctx->chains.end() || !out) return fail(&ctx->err, HM_ERR_ARG, "unknown chain or null output");
  HM_CUDA(ctx, cudaSetDevice(ctx->device));
  HM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  HM_CUDA(ctx, cudaMemcpy(out, ctx->base + it->second->off + it->second->mp.off_stats, ST_N * sizeof(double),
                          cudaMemcpyDeviceToHost));
  return check_device_error(ctx);
}

int hm_get_mps(hm_ctx* ctx, hm_chain chain, int32_t* dims_out, int32_t dims_cap, double* buf, size_t cap,
               int32_t* n_sites_out, size_t* n_doubles_out) {
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  auto it = ctx->chains.find(chain);
  if (it == ctx->chains.end()) return fail(&ctx->err, HM_ERR_ARG, "unknown chain handle");
  Chain* c = it->second;
  const int n = c->L.n_sites;
  if (n_sites_out) *n_sites_out = n;
  if (!dims_out || dims_cap < n + 1) return fail(&ctx->err, HM_ERR_ARG, "dims buffer needs %d entries", n + 1);
  HM_CUDA(ctx, cudaSetDevice(ctx->device));
  HM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  char* base = ctx->base + c->off;
  HM_CUDA(ctx, cudaMemcpy(dims_out, base + c->mp.off_chi, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
  for (int i = 0; i <= n; ++i)   // never size a copy from a bond dim outside its slot
    if (dims_out[i] < 1 || dims_out[i] > c->mp.bmax[i])
      return fail(&ctx->err, HM_ERR_NUMERIC, "bond %d holds dim %d outside [1, %lld]", i, dims_out[i],
                  (long long)c->mp.bmax[i]);
  size_t tot = 0;
  for (int s = 0; s < n; ++s) tot += (size_t)dims_out[s] * 3 * dims_out[s + 1];
  if (n_doubles_out) *n_doubles_out = tot;
  if (!buf) return HM_OK;
  if (cap < tot) return fail(&ctx->err, HM_ERR_ARG, "buffer needs %zu doubles", tot);
  size_t o = 0;
  for (int s = 0; s < n; ++s) {
    const size_t sz = (size_t)dims_out[s] * 3 * dims_out[s + 1];
    HM_CUDA(ctx, cudaMemcpy(buf + o, base + c->mp.slot_off[s], sz * sizeof(double), cudaMemcpyDeviceToHost));
    o += sz;
  }
  int32_t cnt[4];
  HM_CUDA(ctx, cudaMemcpy(cnt, base + c->mp.off_cnt, sizeof cnt, cudaMemcpyDeviceToHost));
  if (cnt[2] == 1) {
    // the chain stores an S^x-basis sample with every leg rotated by R
    // (rows: the S^x eigenvectors; R = R^T = R^-1); return it unrotated
    const double r = 1.0 / std::sqrt(2.0);
    const double R[9] = {0.5, r, 0.5, r, 0.0, -r, 0.5, -r, 0.5};
    o = 0;
    for (int s = 0; s < n; ++s) {
      const int cl = dims_out[s], cr = dims_out[s + 1];
      for (int l = 0; l < cl; ++l)
        for (int x = 0; x < cr; ++x) {
          double* a = buf + o + (size_t)l * 3 * cr + x;
          const double a0 = a[0], a1 = a[cr], a2 = a[2 * cr];
          a[0] = R[0] * a0 + R[1] * a1 + R[2] * a2;
          a[cr] = R[3] * a0 + R[4] * a1 + R[5] * a2;
          a[2 * cr] = R[6] * a0 + R[7] * a1 + R[8] * a2;
        }
      o += (size_t)cl * 3 * cr;
    }
  }
  return check_device_error(ctx);
}

int hm_set_mps(hm_ctx* ctx, hm_chain chain, const int32_t* dims, int32_t n_sites, const double* buf,
               size_t n_doubles, int32_t centre, int32_t evolved) {
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  auto it = ctx->chains.find(chain);
  if (it == ctx->chains.end()) return fail(&ctx->err, HM_ERR_ARG, "unknown chain handle");
  Chain* c = it->second;
  const int n = c->L.n_sites;
  if (!dims || !buf || n_sites != n) return fail(&ctx->err, HM_ERR_ARG, "expected %d sites", n);
  if (dims[0] != 1 || dims[n] != 1) return fail(&ctx->err, HM_ERR_ARG, "boundary bond dims must be 1");
  size_t tot = 0;
  for (int i = 0; i <= n; ++i)
    if (dims[i] < 1 || dims[i] > c->mp.bmax[i]) return fail(&ctx->err, HM_ERR_ARG, "bond %d exceeds its cap %lld", i, (long long)c->mp.bmax[i]);
  for (int s = 0; s < n; ++s) tot += (size_t)dims[s] * 3 * dims[s + 1];
  if (tot != n_doubles) return fail(&ctx->err, HM_ERR_ARG, "expected %zu doubles", tot);
  if (centre != 0) return fail(&ctx->err, HM_ERR_ARG, "the orthogonality centre must be on site 0");
  HM_CUDA(ctx, cudaSetDevice(ctx->device));
  HM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  char* base = ctx->base + c->off;
  HM_CUDA(ctx, cudaMemcpy(base + c->mp.off_chi, dims, (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
  size_t o = 0;
  for (int s = 0; s < n; ++s) {
    const size_t sz = (size_t)dims[s] * 3 * dims[s + 1];
    HM_CUDA(ctx, cudaMemcpy(base + c->mp.slot_off[s], buf + o, sz * sizeof(double), cudaMemcpyHostToDevice));
    o += sz;
  }
  // the state is stored as given (frame 0) and carries no charge labels:
  // the chain evolves in dense mode (one block per split) until its next
  // collapse resets it to a charge-labelled initial state
  int32_t cnt[8];
  HM_CUDA(ctx, cudaMemcpy(cnt, base + c->mp.off_cnt, sizeof cnt, cudaMemcpyDeviceToHost));
  cnt[2] = 0;
  cnt[3] = 1;
  cnt[4] = 0;
  c->cursor = 0;
  HM_CUDA(ctx, cudaMemcpy(base + c->mp.off_cnt, cnt, sizeof cnt, cudaMemcpyHostToDevice));
  const std::vector<int16_t> q0((size_t)(n + 1) * c->mp.chi_cap, 0);
  const std::vector<int32_t> s0(n, 0);
  HM_CUDA(ctx, cudaMemcpy(base + c->mp.off_qn, q0.data(), q0.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
  HM_CUDA(ctx, cudaMemcpy(base + c->mp.off_sgn, s0.data(), s0.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  c->phase = evolved ? 1 : 0;
  return HM_OK;
}

int hm_apply_ops(hm_ctx* ctx, hm_chain chain, const int32_t* ops, int32_t n_ops) {
  if (!ctx) return fail(nullptr, HM_ERR_ARG, "null context");
  auto it = ctx->chains.find(chain);
  if (it == ctx->chains.end()) return fail(&ctx->err, HM_ERR_ARG, "unknown chain handle");
  Chain* c = it->second;
  if (n_ops <= 0) return HM_OK;
  if (!ops) return fail(&ctx->err, HM_ERR_ARG, "null op list");
  const int ng = c->n_gates;
  std::vector<OpDev> v(n_ops);
  for (int i = 0; i < n_ops; ++i) {
    v[i] = {ops[4 * i], ops[4 * i + 1], ops[4 * i + 2], ops[4 * i + 3]};
    if (v[i].k < 0 || v[i].k + 1 >= c->L.n_sites || v[i].gate < 0 || v[i].gate >= ng || (v[i].absorb & ~1) ||
        (v[i].exact & ~1))
      return fail(&ctx->err, HM_ERR_ARG, "invalid op %d", i);
  }
  HM_CUDA(ctx, cudaSetDevice(ctx->device));
  Scratch sc{ctx};
  int rc = sc.get(v.size() * sizeof(OpDev));
  if (rc) return rc;
  HM_CUDA(ctx, cudaMemcpyAsync(sc.ptr, v.data(), v.size() * sizeof(OpDev), cudaMemcpyHostToDevice, ctx->stream));
  BatchArg b{};
  b.n = 1;
  b.c[0] = c->dev;
  b.t0 = 0;
  b.t1 = n_ops;
  b.ops_override = (const OpDev*)sc.ptr;
  b.n_override = n_ops;
  OutArg o{};
  o.ctx_err = ctx->err_word;
  rc = c->p.precision == HM_FP64 ? launch_evolve_fp64(b, o, ctx->stream)
                                  : launch_evolve_mixed(b, o, c->mp.chi_cap, c->p.precision == HM_MIXED, ctx->stream);
  if (rc != HM_OK) return fail(&ctx->err, rc, "apply_ops launch failed");
  return check_device_error(ctx);   // the scratch op list must outlive the kernel
}

const char* hm_last_error(const hm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

}  // extern "C"
