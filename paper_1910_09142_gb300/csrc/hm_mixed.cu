// Mixed-precision evolve (step 2 of Sec. I.C.1) for GB300.
//
// GB300 runs binary32 FMA about 58x faster than binary64 (measured 69.9 vs
// 1.2 TFLOP/s on 152 SMs), so this path forms the two-site tensor and applies
// the 9x9 gate in binary32 and runs the one-sided Jacobi sweeps of every
// charge block (Sec. II.C, hm_block.cuh) in binary32.  HM_MIXED then finishes
// each block with one binary64 sweep (the singular values and left vectors
// become binary64-accurate for that tensor); HM_MIXED32 stops at the binary32
// sweeps.  The truncation weights (Sec. II), the renormalisation of the kept
// singular values and the stored site tensors stay binary64.  Measurement
// and collapse (steps 3-4) are the binary64 kernels of hm_fp64.cu.
//
// One CTA owns one chain: 512 threads, one CTA per SM, or (hm_mixed_pair.cu)
// 256 threads, two CTAs per SM, for batches wider than the GPU.  The blocks
// of a split that fit in shared memory together form a wave and are
// decomposed at once, each by its own warp group; a block too large for
// shared memory keeps W and V in global memory and works on pairs of column
// blocks staged in shared memory (intra-block pairs once per sweep, then
// every cross pair of two staged blocks).
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "hm_block.cuh"
#include "hm_internal.h"

namespace hm {

namespace {

// This file builds the kernel twice: one CTA of 512 threads per SM (210 KB
// of shared memory), and, from hm_mixed_pair.cu, two CTAs of 256 threads per
// SM (108 KB each) for batches with more chains than SMs.
#ifndef HM_MIXED_NT
#define HM_MIXED_NT 512
#define HM_MIXED_CTAS_PER_SM 1
#endif
constexpr int NT = HM_MIXED_NT;
constexpr int kCtasPerSm = HM_MIXED_CTAS_PER_SM;
constexpr int kMaxSweeps = 60;
constexpr int GM = kMixedGM, GN = kMixedGN, GK = kMixedGK;   // binary32 GEMM tile (2x4 or 4x4 outputs a thread)

struct Scal {
  double red[NT / 32][2];
  double dval[4];
  int32_t ival[4];
};

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Rotate the column pair (x, y) of length q (W) and (vx, vy) of length p (V)
// so that x . y = 0 (Hestenes).  Warp-cooperative; returns 1 if rotated.
__device__ __forceinline__ int rotate_pair(float* x, float* y, int q, float* vx, float* vy, int p, float tol,
                                           int lane, float* rmax) {
  float al = 0.f, be = 0.f, ga = 0.f;
  for (int i = lane; i < q; i += 32) {
    const float a = x[i], b = y[i];
    al = fmaf(a, a, al);
    be = fmaf(b, b, be);
    ga = fmaf(a, b, ga);
  }
  al = warp_sumf(al);
  be = warp_sumf(be);
  ga = warp_sumf(ga);
  if (!(ga != 0.f && al > 0.f && be > 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be))) return 0;
  *rmax = fmaxf(*rmax, fabsf(ga) / (sqrtf(al) * sqrtf(be)));
  const float zeta = (be - al) / (2.f * ga);
  float t;
  if (fabsf(zeta) > 1e18f) t = 0.5f / zeta;
  else t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  const float cs = rsqrtf(1.f + t * t), sn = cs * t;
  for (int i = lane; i < q; i += 32) {
    const float a = x[i], b = y[i];
    x[i] = cs * a - sn * b;
    y[i] = sn * a + cs * b;
  }
  for (int i = lane; i < p; i += 32) {
    const float a = vx[i], b = vy[i];
    vx[i] = cs * a - sn * b;
    vy[i] = sn * a + cs * b;
  }
  return 1;
}

// Stage columns [c0, c0 + nc) of W (stride q) and V (stride p) into smem.
__device__ void stage(const float* W, const float* V, int q, int p, int c0, int nc, float* sw, float* sv) {
  for (int e = threadIdx.x; e < nc * q; e += NT) sw[e] = W[(size_t)c0 * q + e];
  for (int e = threadIdx.x; e < nc * p; e += NT) sv[e] = V[(size_t)c0 * p + e];
}

__device__ void unstage(float* W, float* V, int q, int p, int c0, int nc, const float* sw, const float* sv) {
  for (int e = threadIdx.x; e < nc * q; e += NT) W[(size_t)c0 * q + e] = sw[e];
  for (int e = threadIdx.x; e < nc * p; e += NT) V[(size_t)c0 * p + e] = sv[e];
}

// Cross pairs of the block Jacobi with the I column in registers: in every
// round t warp w pairs column I_w with J_{(w+t) mod b}, so warp w keeps I_w
// (and its V column) in registers for all later blocks J and only the J
// column crosses shared memory (one load and one store per element of W and
// of V).  Column norms are cached in `norm` (recomputed here first), so each
// rotation needs one dot product.  q <= 32 QL.
template <int QL>
__device__ void cross_phase_reg(float* W, float* V, int q, int p, int b, int nb, float* swJ, float* svJ,
                                float* norm, float tol, int& rot, float& rmax) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nwarps = NT / 32;
  for (int j = warp; j < p; j += nwarps) {
    const float* cj = W + (size_t)j * q;
    float s2 = 0.f;
    for (int i = lane; i < q; i += 32) s2 = fmaf(cj[i], cj[i], s2);
    s2 = warp_sumf(s2);
    if (lane == 0) norm[j] = s2;
  }
  __syncthreads();
  for (int I = 0; I + 1 < nb; ++I) {
    const int cI = I * b, nI = min(b, p - cI);
    const bool own = warp < nI;
    const int col = cI + warp;
    float xr[QL], vr[QL];
    float nx = 0.f;
#pragma unroll
    for (int k = 0; k < QL; ++k) {
      xr[k] = 0.f;
      vr[k] = 0.f;
    }
    if (own) {
      const float* xw = W + (size_t)col * q;
      const float* vw = V + (size_t)col * p;
#pragma unroll
      for (int k = 0; k < QL; ++k) {
        if (32 * k >= q) break;               // warp-uniform: only live chunks
        const int i = lane + 32 * k;
        xr[k] = i < q ? xw[i] : 0.f;
        vr[k] = i < p ? vw[i] : 0.f;
      }
      nx = norm[col];
    }
    for (int J = I + 1; J < nb; ++J) {
      const int cJ = J * b, nJ = min(b, p - cJ);
      for (int e = tid; e < nJ * q; e += NT) swJ[e] = W[(size_t)cJ * q + e];
      for (int e = tid; e < nJ * p; e += NT) svJ[e] = V[(size_t)cJ * p + e];
      __syncthreads();
      for (int t = 0; t < b; ++t) {
        const int j = (warp + t) % b;
        if (own && j < nJ) {
          float* y = swJ + (size_t)j * q;
          float* vy = svJ + (size_t)j * p;
          float yr[QL];
          float ga = 0.f;
#pragma unroll
          for (int k = 0; k < QL; ++k) {
            if (32 * k >= q) break;
            const int i = lane + 32 * k;
            yr[k] = i < q ? y[i] : 0.f;
            ga = fmaf(xr[k], yr[k], ga);
          }
          ga = warp_sumf(ga);
          const float be = norm[cJ + j];
          if (ga != 0.f && nx > 0.f && be > 0.f && fabsf(ga) > tol * sqrtf(nx) * sqrtf(be)) {
            rmax = fmaxf(rmax, fabsf(ga) / (sqrtf(nx) * sqrtf(be)));
            const float zeta = (be - nx) / (2.f * ga);
            float tt;
            if (fabsf(zeta) > 1e18f) tt = 0.5f / zeta;
            else tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
            const float cs = rsqrtf(1.f + tt * tt), sn = cs * tt;
#pragma unroll
            for (int k = 0; k < QL; ++k) {
              if (32 * k >= q) break;
              const int i = lane + 32 * k;
              const float a = xr[k], bb = yr[k];
              xr[k] = cs * a - sn * bb;
              if (i < q) y[i] = sn * a + cs * bb;
            }
#pragma unroll
            for (int k = 0; k < QL; ++k) {
              if (32 * k >= p) break;
              const int i = lane + 32 * k;
              if (i < p) {
                const float a = vr[k], bb = vy[i];
                vr[k] = cs * a - sn * bb;
                vy[i] = sn * a + cs * bb;
              }
            }
            nx -= tt * ga;
            __syncwarp();
            if (lane == 0) norm[cJ + j] = be + tt * ga;
            rot = 1;
          }
        }
        __syncthreads();
      }
      for (int e = tid; e < nJ * q; e += NT) W[(size_t)cJ * q + e] = swJ[e];
      for (int e = tid; e < nJ * p; e += NT) V[(size_t)cJ * p + e] = svJ[e];
      __syncthreads();
    }
    if (own) {
      float* xw = W + (size_t)col * q;
      float* vw = V + (size_t)col * p;
#pragma unroll
      for (int k = 0; k < QL; ++k) {
        if (32 * k >= q) break;
        const int i = lane + 32 * k;
        if (i < q) xw[i] = xr[k];
        if (i < p) vw[i] = vr[k];
      }
      if (lane == 0) norm[col] = nx;
    }
    __syncthreads();
  }
}

// Block one-sided Jacobi on W (q x p column-major, q >= p) with V (p x p).
// smem holds two blocks of b columns of W and of V.  Returns sweeps or -1.
// tmp: q p + p p floats of scratch (used once, to order the columns).
__device__ int cta_jacobi_f32(float* W, int q, int p, float* V, int b, float* smem, Scal& sc, float* tmp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nwarps = NT / 32;
  for (int e = tid; e < p * p; e += NT) V[e] = (e % (p + 1) == 0) ? 1.f : 0.f;
  __syncthreads();
  float* swI = smem;
  float* swJ = swI + (size_t)b * q;
  float* svI = swJ + (size_t)b * q;
  float* svJ = svI + (size_t)b * p;
  const float tol = sqrtf((float)q) * FLT_EPSILON;
  const int nb = (p + b - 1) / b;
  int done = 0;
  bool converged = false;
  if (tmp) {
    // order the columns by decreasing norm before the first sweep (W and V
    // permuted together, so W = X V still holds): the graded two-site
    // matrices converge in ~1 sweep fewer (12.3 -> 11.3 for 256 < p <= 512)
    float* nrm = svJ + (size_t)b * p;
    int* rk = reinterpret_cast<int*>(swI);
    for (int j = warp; j < p; j += nwarps) {
      const float* cj = W + (size_t)j * q;
      float s2 = 0.f;
      for (int i = lane; i < q; i += 32) s2 = fmaf(cj[i], cj[i], s2);
      s2 = warp_sumf(s2);
      if (lane == 0) nrm[j] = s2;
    }
    __syncthreads();
    for (int j = tid; j < p; j += NT) {
      const float nj = nrm[j];
      int r = 0;
      for (int i = 0; i < p; ++i) r += (nrm[i] > nj) || (nrm[i] == nj && i < j);
      rk[j] = r;
    }
    __syncthreads();
    float* tW = tmp;
    float* tV = tmp + (size_t)q * p;
    for (int e = tid; e < q * p; e += NT) tW[(size_t)rk[e / q] * q + e % q] = W[e];
    for (int e = tid; e < p * p; e += NT) tV[(size_t)rk[e / p] * p + e % p] = V[e];
    __syncthreads();
    for (int e = tid; e < q * p; e += NT) W[e] = tW[e];
    for (int e = tid; e < p * p; e += NT) V[e] = tV[e];
    __syncthreads();
  }
  while (done < kMaxSweeps) {
    if (tid == 0) {
      sc.ival[0] = 0;
      sc.ival[2] = 0;                   // largest rotation ratio of the sweep (float bits)
    }
    __syncthreads();
    int rot = 0;
    float rmax = 0.f;
    // intra-block pairs: round-robin tournament inside each block
    for (int I = 0; I < nb; ++I) {
      const int c0 = I * b, nc = min(b, p - c0);
      stage(W, V, q, p, c0, nc, swI, svI);
      __syncthreads();
      const int n2 = nc + (nc & 1);
      for (int r = 0; r < n2 - 1; ++r) {
        for (int pi = warp; pi < n2 / 2; pi += nwarps) {
          int a, bb;
          if (pi == 0) { a = r; bb = n2 - 1; } else { a = (r + pi) % (n2 - 1); bb = (r - pi + n2 - 1) % (n2 - 1); }
          if (a >= nc || bb >= nc) continue;
          rot |= rotate_pair(swI + (size_t)a * q, swI + (size_t)bb * q, q, svI + (size_t)a * p, svI + (size_t)bb * p,
                             p, tol, lane, &rmax);
        }
        __syncthreads();
      }
      unstage(W, V, q, p, c0, nc, swI, svI);
      __syncthreads();
    }
    // cross pairs of two different blocks: round t pairs column i of I with
    // column (i + t) mod b of J, b disjoint pairs per round
    if (q > 128 && q <= 32 * 24 && b <= nwarps) {
      cross_phase_reg<24>(W, V, q, p, b, nb, swJ, svJ, svJ + (size_t)b * p, tol, rot, rmax);
    } else
    for (int I = 0; I < nb; ++I) {
      const int cI = I * b, nI = min(b, p - cI);
      stage(W, V, q, p, cI, nI, swI, svI);
      for (int J = I + 1; J < nb; ++J) {
        const int cJ = J * b, nJ = min(b, p - cJ);
        stage(W, V, q, p, cJ, nJ, swJ, svJ);
        __syncthreads();
        for (int t = 0; t < b; ++t) {
          for (int i = warp; i < nI; i += nwarps) {
            const int j = (i + t) % b;
            if (j >= nJ) continue;
            rot |= rotate_pair(swI + (size_t)i * q, swJ + (size_t)j * q, q, svI + (size_t)i * p, svJ + (size_t)j * p,
                               p, tol, lane, &rmax);
          }
          __syncthreads();
        }
        unstage(W, V, q, p, cJ, nJ, swJ, svJ);
        __syncthreads();
      }
      unstage(W, V, q, p, cI, nI, swI, svI);
      __syncthreads();
    }
    if (rot && lane == 0) sc.ival[0] = 1;
    if (lane == 0) atomicMax(&sc.ival[2], __float_as_int(rmax));
    __syncthreads();
    const int any = sc.ival[0];
    const float rm = __int_as_float(sc.ival[2]);
    __syncthreads();
    ++done;
    // no rotation: converged; all rotations tiny: quadratic convergence puts
    // the next sweep's off-diagonals (O(rm^2)) below the tolerance
    if (!any || rm < 2e-4f) {
      converged = true;
      break;
    }
  }
  return converged ? done : -1;
}

__device__ void set_error(const ChainDev* c, int code, int where, int32_t* ctx_err) {
  if (threadIdx.x == 0) {
    if (atomicCAS(c->status, 0, code) == 0) *c->err_where = where;
    if (ctx_err) atomicCAS(ctx_err, 0, code);
  }
}

// Column scales 1 / |v_j| of V (binary32, leading dimension ldv) into scale.
// A binary32 Givens rotation with a small angle t has cs = 1 exactly once
// 1 + t^2 rounds to 1, so it stretches both columns by sqrt(1 + t^2): a bias
// that never cancels, and after the ~10^3 rotations a column sees it leaves
// V's columns longer than 1 by ~1e-5.  Left in, each kept singular vector
// would be weighted by its column's stretch, a systematic energy error of
// ~2e-5 in every sample (measured on GB300).  The rotations stay conformal,
// and W = theta V holds column by column, so scaling a column of W and of V
// by the same factor removes the stretch.  One warp per column.
__device__ void column_scales(const float* V32, int ldv, int p, double* scale) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < p; j += NT / 32) {
    const float* v = V32 + (size_t)j * ldv;
    double s2 = 0.0;
    for (int i = lane; i < p; i += 32) s2 = fma((double)v[i], (double)v[i], s2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) scale[j] = s2 > 0.0 ? 1.0 / sqrt(s2) : 1.0;
  }
  __syncthreads();
}

// After the binary32 sweeps: W64 = W32 with unit-column scales, V32 scaled
// in place to unit columns (a binary32 product: V32 holds binary32 values
// anyway, and the binary64 pipe is GB300's scarce one).  scale: p doubles.
__device__ void promote_w(const float* W32, int ldw, float* V32, int ldv, int q, int p, double* W64, double* scale) {
  column_scales(V32, ldv, p, scale);
  for (int e = threadIdx.x; e < q * p; e += NT) W64[e] = (double)W32[(size_t)(e / q) * ldw + e % q] * scale[e / q];
  for (int e = threadIdx.x; e < p * p; e += NT) V32[(size_t)(e / p) * ldv + e % p] *= (float)scale[e / p];
}

// After the polish: V64 = V32 with unit columns, W64 scaled alike (the
// binary64 sweep's rotations are binary32 in V).  Without a polish V32 has
// unit columns from promote_w already and is only widened.
__device__ void promote_v(const float* V32, int ldv, int q, int p, double* W64, double* V64, double* scale,
                          int rescale) {
  if (!rescale) {
    for (int e = threadIdx.x; e < p * p; e += NT) V64[e] = (double)V32[(size_t)(e / p) * ldv + e % p];
    return;
  }
  column_scales(V32, ldv, p, scale);
  for (int e = threadIdx.x; e < q * p; e += NT) W64[e] *= scale[e / q];
  for (int e = threadIdx.x; e < p * p; e += NT) V64[e] = (double)V32[(size_t)(e / p) * ldv + e % p] * scale[e / p];
}

// Shared memory of the binary32 block Jacobi; the kernel's dynamic shared
// memory is at least this (and at least the staged fallback's plan).  Two
// CTAs per SM share the SM's 228 KB.
constexpr size_t kBlockSmem = kCtasPerSm == 1 ? 210 * 1024 : kPairBlockSmem;

// Stopping rule of the binary64 polish: a sweep whose largest rotation ratio
// is below this leaves off-diagonals of order its square for the next sweep.
// After the binary32 sweeps that ratio is ~1e-6, so one binary64 sweep ends
// the polish with off-diagonals of order 1e-12.
constexpr double kPolishStop = 1e-5;

// Stopping ratio of the binary32 sweeps (warp-group path): 2e-4 when they
// are the whole SVD (HM_MIXED32; the next sweep's off-diagonals would be
// ~4e-8, below binary32 resolution), 1e-3 when a binary64 sweep follows
// (HM_MIXED): the off-diagonals it inherits are then ~1e-6, below
// kPolishStop, so one binary64 sweep still ends the polish.
constexpr float kStop32 = 2e-4f, kStop32Polished = 1e-3f;

// One two-site op (step 2 of Sec. I.C.1) in charge blocks (Sec. II.C):
// theta and the gate in binary32 (operands rounded from the binary64 site
// tensors, binary32 accumulation, gate coefficients as binary32 pairs); the
// blocks of a split in waves that fit in shared memory, each block of a wave
// decomposed by its own warp group at the same time: a binary32 one-sided
// Jacobi as a preconditioner, then binary64 sweeps on the promoted W and V
// until the binary64 stopping rule holds, so the singular values and the kept
// vectors are binary64-accurate for that theta.  A block too large for
// shared memory runs alone, its binary32 sweeps on column blocks staged from
// global memory.  Then the truncation rule (Sec. II), renormalisation and
// absorb in binary64.
__device__ void two_site_op_mixed(ChainDev* c, const OpDev op, int t, int bcols, int polish, float* smem, Scal& sc,
                                  blk::SplitSh& ss, blk::WaveSh& wv, blk::GroupSh& gs, int32_t* ctx_err) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (!blk::prepare<NT>(c, op, ss)) blk::prepare<NT>(c, op, ss);
  float* theta = reinterpret_cast<float*>(c->theta);
  blk::theta_blocks<NT, GM, GN, GK, float>(c, op.k, ss, theta, smem);
  const blk::Meta* M = reinterpret_cast<const blk::Meta*>(c->meta);
  int sw32 = 0, sw64 = 0;
  int64_t cost = -1;
  constexpr int64_t cap = (int64_t)(kBlockSmem / sizeof(float));
  for (int b0 = 0; b0 < ss.nblk;) {
    if (tid == 0) {
      // as many consecutive blocks as fit in shared memory (at most 15 and
      // one warp each); a block that does not fit alone takes the global path
      int64_t used = 0;
      int n = 0, p[15];
      while (b0 + n < ss.nblk && n < 15 && n < NT / 32) {
        const blk::BlockRec& r = M->b[b0 + n];
        const int64_t need = (int64_t)r.p * (r.q | 1) + (int64_t)r.p * (r.p | 1) + r.p;
        if (used + need > cap) break;
        wv.off[n] = (int32_t)used;
        p[n] = r.p;
        used += need;
        ++n;
      }
      wv.b0 = b0;
      wv.n = n;
      if (n > 0) blk::assign_warps(p, n, NT / 32, wv.w0, wv.nw);
    }
    __syncthreads();
    const int n = wv.n;
    if (n == 0) {
      const blk::BlockRec& r = M->b[b0];
      float* W32 = c->X;
      float* V32 = c->X + (size_t)r.q * r.p;
      blk::gather_block<NT, float, float>(c, op.k, ss, r, theta, W32, r.q, V32, r.p);
      __syncthreads();
      const int sw = cta_jacobi_f32(W32, r.q, r.p, V32, bcols, smem, sc, nullptr);
      if (sw < 0) {
        set_error(c, HM_ERR_NUMERIC, t, ctx_err);
        return;
      }
      double* W64 = c->W + r.woff;
      double* V64 = c->V + r.voff;
      promote_w(W32, r.q, V32, r.p, r.q, r.p, W64, c->sig);
      __syncthreads();
      const int s64 = polish ? blk::jacobi_group<double, float, 2>(W64, r.q, r.q, r.p, V32, r.p, c->sig, warp, NT / 32,
                                                                1, 0, gs, kPolishStop, kMaxSweeps)
                             : 0;
      __syncthreads();
      promote_v(V32, r.p, r.q, r.p, W64, V64, c->sig, polish);
      if (s64 < 0) {
        set_error(c, HM_ERR_NUMERIC, t, ctx_err);
        return;
      }
      const int64_t cb = (int64_t)r.q * r.p * r.p;
      if (cb > cost) cost = cb, sw32 = sw, sw64 = s64;
      b0 += 1;
      continue;
    }
    for (int i = 0; i < n; ++i) {
      const blk::BlockRec& r = M->b[b0 + i];
      float* W32 = smem + wv.off[i];
      float* V32 = W32 + (size_t)r.p * (r.q | 1);
      blk::gather_block<NT, float, float>(c, op.k, ss, r, theta, W32, r.q | 1, V32, r.p | 1);
    }
    __syncthreads();
    const int g = blk::my_group(wv, warp);
    if (g >= 0) {
      const blk::BlockRec& r = M->b[b0 + g];
      float* W32 = smem + wv.off[g];
      float* V32 = W32 + (size_t)r.p * (r.q | 1);
      const int sw = blk::jacobi_group<float>(W32, r.q, r.q | 1, r.p, V32, r.p | 1, V32 + (size_t)r.p * (r.p | 1),
                                              warp - wv.w0[g], wv.nw[g], g + 1, g, gs,
                                              polish ? kStop32Polished : kStop32, kMaxSweeps);
      if (warp == wv.w0[g] && (tid & 31) == 0) wv.sw[g] = sw;
    }
    __syncthreads();
    for (int i = 0; i < n; ++i) {
      const blk::BlockRec& r = M->b[b0 + i];
      const float* W32 = smem + wv.off[i];
      float* V32 = smem + wv.off[i] + (size_t)r.p * (r.q | 1);
      promote_w(W32, r.q | 1, V32, r.p | 1, r.q, r.p, c->W + r.woff, c->sig + r.svoff);
      __syncthreads();
    }
    if (polish && g >= 0) {
      // binary64 polish by the same groups: W in binary64 (global), V stays
      // in shared memory in binary32; norms of block g in c->sig
      const blk::BlockRec& r = M->b[b0 + g];
      float* V32 = smem + wv.off[g] + (size_t)r.p * (r.q | 1);
      const int s64 = blk::jacobi_group<double, float, 2>(c->W + r.woff, r.q, r.q, r.p, V32, r.p | 1, c->sig + r.svoff,
                                                       warp - wv.w0[g], wv.nw[g], g + 1, g, gs, kPolishStop,
                                                       kMaxSweeps);
      if (warp == wv.w0[g] && (tid & 31) == 0) wv.sw[g] = wv.sw[g] < 0 ? -1 : (s64 < 0 ? -1 : wv.sw[g] + 1000 * s64);
    }
    __syncthreads();
    for (int i = 0; i < n; ++i) {
      const blk::BlockRec& r = M->b[b0 + i];
      const float* V32 = smem + wv.off[i] + (size_t)r.p * (r.q | 1);
      promote_v(V32, r.p | 1, r.q, r.p, c->W + r.woff, c->V + r.voff, c->sig + r.svoff, polish);
      __syncthreads();
    }
    for (int i = 0; i < n; ++i) {
      const int code = wv.sw[i];
      if (code < 0) {
        set_error(c, HM_ERR_NUMERIC, t, ctx_err);
        return;
      }
      const blk::BlockRec& r = M->b[b0 + i];
      const int64_t cb = (int64_t)r.q * r.p * r.p;
      if (cb > cost) cost = cb, sw32 = code % 1000, sw64 = code / 1000;
    }
    b0 += n;
    __syncthreads();
  }
  blk::finish<NT>(c, op, t, ss, c->theta, ctx_err, sw32, sw64);
  if (threadIdx.x == 0 && ss.kk > 0) {
    double k1 = 0.0;
    for (int i = 0; i < ss.nin; ++i) {
      const int Q = M->qin[i];
      double rows = 0.0, cols = 0.0;
      for (int u = 0; u < 3; ++u) {
        rows += blk::seg_of(M, 0, ss.qbase, Q - ss.sk * blk::mval(u)).len;
        cols += blk::seg_of(M, 2, ss.qbase, Q + ss.sk1 * blk::mval(u)).len;
      }
      k1 += 2.0 * rows * blk::seg_of(M, 1, ss.qbase, Q).len * cols;
    }
    c->stats[ST_K1] += k1;
    c->stats[ST_K2] += 2.0 * 81.0 * c->chi[op.k] * c->chi[op.k + 2];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT, kCtasPerSm) evolve_mixed_kernel(BatchArg b, OutArg o, int bcols, int polish) {
  extern __shared__ float smem[];
  __shared__ Scal sc;
  __shared__ blk::SplitSh ss;
  __shared__ blk::WaveSh wv;
  __shared__ blk::GroupSh gs;
  ChainDev* c = b.c[blockIdx.x];
  const OpDev* ops = b.ops_override ? b.ops_override : c->ops;
  const int n_ops = b.ops_override ? b.n_override : c->n_ops;
  const int t0 = b.budget > 0 ? c->counters[4] : b.t0;
  const int t1 = b.budget > 0 ? min(t0 + b.budget, n_ops) : (b.t1 < n_ops ? b.t1 : n_ops);
  __syncthreads();                                           // every thread has read the cursor
  if (b.budget > 0 && threadIdx.x == 0) c->counters[4] = t1;
  for (int t = t0; t < t1; ++t) {
    if (*(volatile int32_t*)c->status != 0) return;
    __syncthreads();
    two_site_op_mixed(c, ops[t], t, bcols, polish, smem, sc, ss, wv, gs, o.ctx_err);
    __syncthreads();
  }
}

// Opt-in to the kernel's dynamic shared memory (per device, cached, under a
// lock: serving workers may launch from several host threads), then launch.
int launch_kernel(const BatchArg& b, const OutArg& o, int chi_cap, int polish, void* stream) {
  int bcols = 16;
  const size_t plan = mixed_smem_bytes(chi_cap, &bcols, kBlockSmem);
  const size_t smem = plan > kBlockSmem ? plan : kBlockSmem;
  static std::mutex mu;
  static size_t configured[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HM_ERR_CUDA;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64 || smem > configured[dev]) {
      if (cudaFuncSetAttribute(evolve_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
        return HM_ERR_CUDA;
      if (dev >= 0 && dev < 64) configured[dev] = smem;
    }
  }
  evolve_mixed_kernel<<<b.n, NT, smem, (cudaStream_t)stream>>>(b, o, bcols, polish);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

#if HM_MIXED_CTAS_PER_SM == 1
// SMs of the current device (cached per device ordinal).
int sm_count() {
  static std::mutex mu;
  static int count[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lock(mu);
  if (count[dev] == 0 && cudaDeviceGetAttribute(&count[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    count[dev] = 0;
  return count[dev];
}
#endif

}  // namespace

#if HM_MIXED_CTAS_PER_SM == 1
// A batch with more chains than SMs whose charge blocks fit half an SM's
// shared memory runs two chains per SM (hm_mixed_pair.cu): all of them are
// resident at once, and each SM interleaves two independent CTAs.
int launch_evolve_mixed(const BatchArg& b, const OutArg& o, int chi_cap, int polish, void* stream) {
  if (b.n <= 0) return HM_OK;
  const int sms = sm_count();
  if (chi_cap <= kPairChiCap && sms > 0 && b.n > sms) return launch_evolve_mixed_pair(b, o, chi_cap, polish, stream);
  return launch_kernel(b, o, chi_cap, polish, stream);
}
#else
int launch_evolve_mixed_pair(const BatchArg& b, const OutArg& o, int chi_cap, int polish, void* stream) {
  if (b.n <= 0) return HM_OK;
  return launch_kernel(b, o, chi_cap, polish, stream);
}
#endif

}  // namespace hm
