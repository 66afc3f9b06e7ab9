// TEST INFRASTRUCTURE: compiles the library's CUDA kernels as host C++ so
// their logic can be checked against the oracle on a machine without a GPU.
// Included before each kernel source (-include).  A launch runs its blocks
// one after another; each block is blockDim host threads.  __syncthreads is
// a barrier of the block's threads, a warp shuffle exchanges through a
// per-warp buffer between two warp barriers, and __shared__ variables are
// function statics (one block runs at a time).  Intrinsics are written from
// their documented meaning.  Nothing here is part of the product.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>

#undef __global__
#undef __device__
#undef __shared__
#undef __launch_bounds__
#define __global__
#define __device__
#define __shared__ static
#define __launch_bounds__(...)
#define HM_HOST_EMULATION 1

namespace simt {
struct Idx {
  unsigned x, y, z;
};
Idx tid();
Idx bid();
Idx bdim();
Idx gdim();
void sync();
void syncwarp();
void named_sync(int id, int count);     // bar.sync id, count (count in threads)
uint64_t exchange(uint64_t bits, int lane_xor);
void* dynamic_smem();
void launch(unsigned grid, unsigned block, size_t smem, const std::function<void()>& body);
}  // namespace simt

#define threadIdx (simt::tid())
#define blockIdx (simt::bid())
#define blockDim (simt::bdim())
#define gridDim (simt::gdim())

inline void __syncthreads() { simt::sync(); }
inline void __syncwarp(unsigned = 0xffffffffu) { simt::syncwarp(); }

template <class T>
inline T __shfl_xor_sync(unsigned, T v, int lane_mask, int = 32) {
  static_assert(sizeof(T) <= 8, "shuffle of a type wider than 64 bits");
  uint64_t bits = 0;
  std::memcpy(&bits, &v, sizeof(T));
  bits = simt::exchange(bits, lane_mask);
  T out;
  std::memcpy(&out, &bits, sizeof(T));
  return out;
}

inline int __any_sync(unsigned mask, int pred) {
  int v = pred != 0;
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(mask, v, o);
  return v;
}

inline long long __double_as_longlong(double d) {
  long long r;
  std::memcpy(&r, &d, sizeof r);
  return r;
}
inline int __float_as_int(float f) {
  int r;
  std::memcpy(&r, &f, sizeof r);
  return r;
}
inline unsigned __float_as_uint(float f) {
  unsigned r;
  std::memcpy(&r, &f, sizeof r);
  return r;
}
inline float __uint_as_float(unsigned i) {
  float r;
  std::memcpy(&r, &i, sizeof r);
  return r;
}
inline float __int_as_float(int i) {
  float r;
  std::memcpy(&r, &i, sizeof r);
  return r;
}
// high 32 bits of the 64-bit product
inline unsigned __umulhi(unsigned a, unsigned b) { return (unsigned)(((unsigned long long)a * b) >> 32); }

// returns the old value, like the device atomics
inline int atomicCAS(int* p, int compare, int value) {
  std::atomic_ref<int> r(*p);
  r.compare_exchange_strong(compare, value);
  return compare;
}
inline int atomicMax(int* p, int value) {
  std::atomic_ref<int> r(*p);
  int old = r.load();
  while (old < value && !r.compare_exchange_weak(old, value)) {
  }
  return old;
}
inline int atomicMin(int* p, int value) {
  std::atomic_ref<int> r(*p);
  int old = r.load();
  while (old > value && !r.compare_exchange_weak(old, value)) {
  }
  return old;
}
inline unsigned atomicMax(unsigned* p, unsigned value) {
  std::atomic_ref<unsigned> r(*p);
  unsigned old = r.load();
  while (old < value && !r.compare_exchange_weak(old, value)) {
  }
  return old;
}
inline unsigned long long atomicMax(unsigned long long* p, unsigned long long value) {
  std::atomic_ref<unsigned long long> r(*p);
  unsigned long long old = r.load();
  while (old < value && !r.compare_exchange_weak(old, value)) {
  }
  return old;
}

// Global-namespace functions device code sees (float and double overloads).
using std::isfinite;
using std::copysign;
using std::fabs;
using std::fma;
using std::fmax;
using std::sqrt;
inline int min(int a, int b) { return a < b ? a : b; }
inline int max(int a, int b) { return a > b ? a : b; }
inline unsigned min(unsigned a, unsigned b) { return a < b ? a : b; }
inline unsigned max(unsigned a, unsigned b) { return a > b ? a : b; }
inline long long min(long long a, long long b) { return a < b ? a : b; }
inline long long max(long long a, long long b) { return a > b ? a : b; }
inline float min(float a, float b) { return std::fmin(a, b); }
inline float max(float a, float b) { return std::fmax(a, b); }
inline double min(double a, double b) { return std::fmin(a, b); }
inline double max(double a, double b) { return std::fmax(a, b); }
inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
inline float __fdividef(float a, float b) { return a / b; }
inline int __double2hiint(double x) {
  unsigned long long b;
  std::memcpy(&b, &x, 8);
  return (int)(unsigned)(b >> 32);
}
inline int __double2loint(double x) {
  unsigned long long b;
  std::memcpy(&b, &x, 8);
  return (int)(unsigned)(b & 0xffffffffull);
}
using std::frexp;
using std::ldexp;

template <class T>
inline cudaError_t cudaFuncSetAttribute(T* entry, cudaFuncAttribute attr, int value) {
  return cudaFuncSetAttribute((const void*)entry, attr, value);
}
