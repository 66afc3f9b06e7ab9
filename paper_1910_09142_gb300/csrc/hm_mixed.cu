// Mixed-precision evolve (step 2 of Sec. I.C.1) for GB300.
//
// GB300 runs binary32 FMA about 58x faster than binary64 (measured 69.9 vs
// 1.2 TFLOP/s on 152 SMs), so this path performs the two-site contraction,
// the 9x9 gate and the one-sided Jacobi SVD in binary32, while the
// truncation weights (Sec. II), the renormalisation of the kept singular
// values and the stored site tensors stay binary64.  Measurement and
// collapse (steps 3-4) are the binary64 kernels of hm_fp64.cu.
//
// One CTA owns one chain.  The Jacobi keeps W (q x p) and V (p x p) in the
// chain's global workspace and works on pairs of column blocks staged in
// shared memory: intra-block pairs once per sweep, then every cross pair of
// two blocks while both blocks sit in shared memory, so each staged column
// is reused by b rotations.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "hm_internal.h"

namespace hm {

namespace {

constexpr int NT = 512;
constexpr int kMaxSweeps = 60;
constexpr int GM = kMixedGM, GN = kMixedGN, GK = kMixedGK;   // binary32 GEMM tile (512 threads, 2x4 outputs each)

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

__device__ __forceinline__ double warp_sumd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// C (M x N, row-major binary32) = A (M x K, row-major binary64) * B (K x N,
// row-major binary64), operands rounded to binary32 on load.
__device__ void cta_gemm_f32(int M, int N, int K, const double* __restrict__ A, int lda,
                             const double* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                             float* sm) {
  float* sa = sm;               // [GK][GM]
  float* sb = sm + GK * GM;     // [GK][GN]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;   // 16 x 32 threads: rows ty + 32 r (r < 2), cols tx + 16 c (c < 4)
  for (int i0 = 0; i0 < M; i0 += GM) {
    for (int j0 = 0; j0 < N; j0 += GN) {
      float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
      for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = tid; e < GM * GK; e += NT) {
          const int kk = e % GK, ii = e / GK;
          const int gi = i0 + ii, gk = k0 + kk;
          sa[kk * GM + ii] = (gi < M && gk < K) ? (float)A[(size_t)gi * lda + gk] : 0.f;
        }
        for (int e = tid; e < GN * GK; e += NT) {
          const int jj = e % GN, kk = e / GN;
          const int gj = j0 + jj, gk = k0 + kk;
          sb[kk * GN + jj] = (gj < N && gk < K) ? (float)B[(size_t)gk * ldb + gj] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
          float a[2], b[4];
#pragma unroll
          for (int r = 0; r < 2; ++r) a[r] = sa[kk * GM + ty + 32 * r];
#pragma unroll
          for (int c = 0; c < 4; ++c) b[c] = sb[kk * GN + tx + 16 * c];
#pragma unroll
          for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int i = i0 + ty + 32 * r;
        if (i >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int j = j0 + tx + 16 * c;
          if (j < N) C[(size_t)i * ldc + j] = acc[r][c];
        }
      }
    }
  }
  __syncthreads();
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
  {
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

__device__ int truncation_rank(const double* s, int n, int chi_max, double cutoff, double* tail, double* total_out) {
  tail[n] = 0.0;
  for (int q = n - 1; q >= 0; --q) tail[q] = tail[q + 1] + s[q] * s[q];
  const double total = tail[0];
  *total_out = total;
  int k = n;
  for (int kk = 1; kk <= n; ++kk) {
    if (tail[kk] <= cutoff * total) {
      k = kk;
      break;
    }
  }
  if (k > chi_max) k = chi_max;
  while (k > 1 && k < n && s[k] >= s[k - 1] * (1.0 - 1e-8)) --k;
  return k;
}

__device__ void two_site_op_mixed(ChainDev* c, const OpDev op, int t, int bcols, float* smem, Scal& sc,
                                  int32_t* ctx_err) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = op.k;
  const int chil = c->chi[k], chim = c->chi[k + 1], chir = c->chi[k + 2];
  const int m = 3 * chil, n = 3 * chir;
  double* Ak = c->site[k];
  double* Ak1 = c->site[k + 1];
  float* theta = reinterpret_cast<float*>(c->theta);
  float* W = reinterpret_cast<float*>(c->W);
  float* V = reinterpret_cast<float*>(c->V);

  cta_gemm_f32(m, n, chim, Ak, chim, Ak1, n, theta, n, smem);

  const bool trans = n > m;
  const int q = trans ? n : m, p = trans ? m : n;
  const double* Gd = c->gates + (size_t)op.gate * 81;
  float* G = smem;
  for (int e = tid; e < 81; e += NT) G[e] = (float)Gd[e];
  __syncthreads();
  for (int e = tid; e < chil * chir; e += NT) {
    const int l = e / chir, r = e % chir;
    float th[9];
#pragma unroll
    for (int s1 = 0; s1 < 3; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < 3; ++s2) th[3 * s1 + s2] = theta[(size_t)(3 * l + s1) * n + s2 * chir + r];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        float x = 0.f;
#pragma unroll
        for (int u = 0; u < 9; ++u) x = fmaf(G[(3 * a + b) * 9 + u], th[u], x);
        const int row = 3 * l + a, col = b * chir + r;
        if (!trans) W[(size_t)col * q + row] = x;
        else W[(size_t)row * q + col] = x;
      }
  }
  __syncthreads();

  const int sweeps = cta_jacobi_f32(W, q, p, V, bcols, smem, sc, theta);   // theta is free here
  if (sweeps < 0) {
    set_error(c, HM_ERR_NUMERIC, t, ctx_err);
    return;
  }
  // singular values (norms accumulated in binary64), rank sort, truncation
  double* sig_raw = c->theta;       // theta is free now (binary64 view)
  double* tail = c->theta + p;
  for (int j = warp; j < p; j += NT / 32) {
    const float* cj = W + (size_t)j * q;
    double s2 = 0.0;
    for (int i = lane; i < q; i += 32) s2 = fma((double)cj[i], (double)cj[i], s2);
    s2 = warp_sumd(s2);
    if (lane == 0) sig_raw[j] = sqrt(s2);
  }
  __syncthreads();
  for (int j = tid; j < p; j += NT) {
    const double sj = sig_raw[j];
    int rank = 0;
    for (int i = 0; i < p; ++i) {
      const double si = sig_raw[i];
      rank += (si > sj) || (si == sj && i < j);
    }
    c->sig[rank] = sj;
    c->perm[rank] = j;
  }
  __syncthreads();
  if (tid == 0) {
    const double* s = c->sig;
    double total, nrm = 1.0;
    int kk;
    if (!op.exact) {
      kk = truncation_rank(s, p, c->chi_max, c->cutoff, tail, &total);
      if (!(total > 0.0) || !isfinite(total)) kk = -1;
      else {
        double kept = 0.0;
        for (int i = 0; i < kk; ++i) kept += s[i] * s[i];
        nrm = 1.0 / sqrt(kept);
        c->stats[ST_DISC] += tail[kk] / total;
      }
    } else {
      kk = 0;
      while (kk < p && kk < chim && s[kk] > 0.0) ++kk;
      if (kk == 0) kk = -1;
    }
    sc.ival[1] = kk;
    sc.dval[0] = nrm;
    if (kk > 0) {
      const double mm = (double)(m > n ? m : n), nn = (double)(m > n ? n : m);
      c->stats[ST_K1] += 2.0 * chil * 3.0 * chim * 3.0 * chir;
      c->stats[ST_K2] += 2.0 * 81.0 * chil * chir;
      c->stats[ST_SVD] += 4.0 * mm * mm * nn + 8.0 * mm * nn * nn + 9.0 * nn * nn * nn;
      c->stats[ST_SWEEPS] += sweeps;
      c->stats[ST_SPLITS] += 1.0;
      if (kk > c->stats[ST_MAXCHI]) c->stats[ST_MAXCHI] = kk;
    }
  }
  __syncthreads();
  const int kk = sc.ival[1];
  const double nrm = sc.dval[0];
  if (kk <= 0) {
    set_error(c, HM_ERR_NUMERIC, t, ctx_err);
    return;
  }
  const bool absorb_left = op.absorb == 0;
  for (int e = tid; e < m * kk; e += NT) {
    const int row = e / kk, i = e % kk;
    const int j = c->perm[i];
    const double sg = c->sig[i];
    double v;
    if (!trans) {
      const double w = W[(size_t)j * q + row];
      v = absorb_left ? w * nrm : w / sg;
    } else {
      const double u = V[(size_t)j * p + row];
      v = absorb_left ? u * sg * nrm : u;
    }
    Ak[e] = v;
  }
  for (int e = tid; e < kk * n; e += NT) {
    const int i = e / n, col = e % n;
    const int j = c->perm[i];
    const double sg = c->sig[i];
    double v;
    if (!trans) {
      const double u = V[(size_t)j * p + col];
      v = absorb_left ? u : u * sg * nrm;
    } else {
      const double w = W[(size_t)j * q + col];
      v = absorb_left ? w / sg : w * nrm;
    }
    Ak1[e] = v;
  }
  __syncthreads();
  if (tid == 0) c->chi[k + 1] = kk;
  __syncthreads();
}

__global__ void __launch_bounds__(NT) evolve_mixed_kernel(BatchArg b, OutArg o, int bcols) {
  extern __shared__ float smem[];
  __shared__ Scal sc;
  ChainDev* c = b.c[blockIdx.x];
  const OpDev* ops = b.ops_override ? b.ops_override : c->ops;
  const int n_ops = b.ops_override ? b.n_override : c->n_ops;
  const int t1 = b.t1 < n_ops ? b.t1 : n_ops;
  for (int t = b.t0; t < t1; ++t) {
    if (*(volatile int32_t*)c->status != 0) return;
    __syncthreads();
    two_site_op_mixed(c, ops[t], t, bcols, smem, sc, o.ctx_err);
    __syncthreads();
  }
}

}  // namespace

int launch_evolve_mixed(const BatchArg& b, const OutArg& o, int chi_cap, void* stream) {
  if (b.n <= 0) return HM_OK;
  int bcols = 16;
  const size_t smem = mixed_smem_bytes(chi_cap, &bcols);
  // the shared-memory opt-in is per device: cache it per device ordinal,
  // under a lock (serving workers may launch from several host threads)
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
  evolve_mixed_kernel<<<b.n, NT, smem, (cudaStream_t)stream>>>(b, o, bcols);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace hm
