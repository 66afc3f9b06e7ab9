// TEST INFRASTRUCTURE: the runtime behind simt_prelude.h (see there).
//
// A launch runs its blocks one after another.  A block's threads are
// cooperative fibers (POSIX ucontext) on the calling host thread: each fiber
// runs until it reaches a barrier or returns, then the next one runs.  When
// every live fiber of the block waits at __syncthreads (or every live fiber
// of a warp at a warp barrier), they are released together.  A fiber that
// returns leaves the barriers it would have joined.  If no fiber can run and
// no barrier can open, the block's barriers do not match: the launch stops
// with a message instead of hanging.  Fibers make a run deterministic.
//
// SIMT_ORDER picks the order in which runnable fibers run within a phase:
// "forward" (default), "reverse", or "random:<seed>" (a new permutation on
// every pass).  A kernel without data races gives bit-identical results in
// every order, because nothing orders two threads between barriers; a
// result that changes with the order exposes a missing barrier.
#include <ucontext.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>
#include <vector>

#include "simt_prelude.h"

namespace simt {
namespace {

enum State { RUNNABLE, AT_BLOCK, AT_WARP, AT_NAMED, DONE };

struct Fiber {
  ucontext_t ctx;
  std::unique_ptr<char[]> stack;
  State state = RUNNABLE;
  Idx tid{0, 0, 0};
  int bar_id = 0, bar_count = 0;      // named barrier this fiber waits at
};

constexpr size_t kStack = 256 * 1024;
ucontext_t g_main;
std::vector<Fiber> g_fibers;
Fiber* g_cur = nullptr;
Idx g_bid{0, 0, 0}, g_bdim{1, 1, 1}, g_gdim{1, 1, 1};
std::vector<unsigned char> g_smem;
std::vector<uint64_t> g_xbuf;                 // per-thread exchange slots
const std::function<void()>* g_body = nullptr;

void wait(State s) {
  g_cur->state = s;
  swapcontext(&g_cur->ctx, &g_main);
}

void entry() {
  (*g_body)();
  g_cur->state = DONE;
  swapcontext(&g_cur->ctx, &g_main);
}

// Opens every barrier whose live fibers all wait at it; false if none.
bool release() {
  bool any = false;
  bool all_block = true, some_block = false;
  for (const Fiber& f : g_fibers) {
    if (f.state == DONE) continue;
    if (f.state == AT_BLOCK) some_block = true;
    else all_block = false;
  }
  if (some_block && all_block) {
    for (Fiber& f : g_fibers)
      if (f.state == AT_BLOCK) f.state = RUNNABLE;
    return true;
  }
  // a named barrier (id, count) opens when `count` fibers wait at it
  for (int id = 1; id < 16; ++id) {
    int waiting = 0, count = -1;
    for (const Fiber& f : g_fibers)
      if (f.state == AT_NAMED && f.bar_id == id) {
        ++waiting;
        if (count >= 0 && f.bar_count != count) {
          std::fprintf(stderr, "simt: named barrier %d waited on with counts %d and %d\n", id, count, f.bar_count);
          std::abort();
        }
        count = f.bar_count;
      }
    if (waiting > 0 && waiting == count) {
      for (Fiber& f : g_fibers)
        if (f.state == AT_NAMED && f.bar_id == id) f.state = RUNNABLE;
      any = true;
    }
  }
  const size_t n = g_fibers.size();
  for (size_t w0 = 0; w0 < n; w0 += 32) {
    bool all = true, some = false;
    for (size_t i = w0; i < std::min(n, w0 + 32); ++i) {
      if (g_fibers[i].state == DONE) continue;
      if (g_fibers[i].state == AT_WARP) some = true;
      else all = false;
    }
    if (some && all) {
      for (size_t i = w0; i < std::min(n, w0 + 32); ++i)
        if (g_fibers[i].state == AT_WARP) g_fibers[i].state = RUNNABLE;
      any = true;
    }
  }
  return any;
}

}  // namespace

Idx tid() { return g_cur->tid; }
Idx bid() { return g_bid; }
Idx bdim() { return g_bdim; }
Idx gdim() { return g_gdim; }
void sync() { wait(AT_BLOCK); }
void syncwarp() { wait(AT_WARP); }
void named_sync(int id, int count) {
  g_cur->bar_id = id;
  g_cur->bar_count = count;
  wait(AT_NAMED);
}
uint64_t exchange(uint64_t bits, int lane_xor) {
  const unsigned t = g_cur->tid.x, w0 = t & ~31u;
  g_xbuf[t] = bits;
  wait(AT_WARP);
  const uint64_t out = g_xbuf[w0 + (((t - w0) ^ (unsigned)lane_xor) & 31u)];
  wait(AT_WARP);
  return out;
}
void* dynamic_smem() { return g_smem.data(); }

// Fiber order of one pass: forward, reversed, or a fresh pseudorandom
// permutation (a 64-bit linear congruential generator, Knuth's MMIX constants).
struct Order {
  int mode = 0;                       // 0 forward, 1 reverse, 2 random
  uint64_t state = 0;
  std::vector<unsigned> idx;
  void init(unsigned n) {
    const char* e = std::getenv("SIMT_ORDER");
    mode = 0;
    if (e && std::strcmp(e, "reverse") == 0) mode = 1;
    if (e && std::strncmp(e, "random:", 7) == 0) {
      mode = 2;
      state = std::strtoull(e + 7, nullptr, 10) * 2 + 1;
    }
    idx.resize(n);
    std::iota(idx.begin(), idx.end(), 0u);
    if (mode == 1) std::reverse(idx.begin(), idx.end());
  }
  void next_pass() {
    if (mode != 2) return;
    for (size_t i = idx.size(); i > 1; --i) {          // Fisher-Yates
      state = state * 6364136223846793005ULL + 1442695040888963407ULL;
      std::swap(idx[i - 1], idx[(state >> 33) % i]);
    }
  }
};

void launch(unsigned grid, unsigned block, size_t smem, const std::function<void()>& body) {
  Order order;
  order.init(block);
  g_bdim = {block, 1, 1};
  g_gdim = {grid, 1, 1};
  g_smem.assign(smem + 16, 0);
  g_xbuf.assign(block, 0);
  g_body = &body;
  g_fibers.clear();
  g_fibers.resize(block);
  for (Fiber& f : g_fibers) f.stack.reset(new char[kStack]);
  for (unsigned b = 0; b < grid; ++b) {
    g_bid = {b, 0, 0};
    for (unsigned t = 0; t < block; ++t) {
      Fiber& f = g_fibers[t];
      f.state = RUNNABLE;
      f.tid = {t, 0, 0};
      getcontext(&f.ctx);
      f.ctx.uc_stack.ss_sp = f.stack.get();
      f.ctx.uc_stack.ss_size = kStack;
      f.ctx.uc_link = nullptr;
      makecontext(&f.ctx, entry, 0);
    }
    for (;;) {
      bool ran = false, live = false;
      order.next_pass();
      for (unsigned i : order.idx) {
        Fiber& f = g_fibers[i];
        if (f.state == DONE) continue;
        live = true;
        if (f.state != RUNNABLE) continue;
        g_cur = &f;
        swapcontext(&g_main, &f.ctx);
        ran = true;
      }
      if (!live) break;
      if (!ran && !release()) {
        std::fprintf(stderr, "simt: block %u: barriers do not match (no fiber can run)\n", b);
        std::abort();
      }
    }
  }
  g_cur = nullptr;
}

}  // namespace simt
