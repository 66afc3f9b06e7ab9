// FP64 path of the hybrid purification-METTS sampler (arXiv:1910.09142).
//
// One CTA owns one Markov chain for the whole call: every two-site op of the
// Trotter schedule, the cluster measurement and the environment collapse run
// as a device-side loop over that chain's data.  On GB300 the binary64 pipe
// (about 2 DFMA per clock per SM) is the bound of every step here, so the
// design keeps all SMs busy with independent chains rather than tiling for
// bandwidth: a batch of >= 152 chains fills the chip.
//
// Steps (Sec. I.C.1): evolve (step 2) = theta GEMM + 9x9 gate + one-sided
// Jacobi SVD + truncation (Sec. II) + absorb, all in S^z charge blocks
// (Sec. II.C, hm_block.cuh); measure (step 3) = transfer matrices with S^z /
// S^+ / S^- insertions (Eq. H), contracted by charge block; collapse + reset
// (step 4, Eq. detailbalance1, Bell pairs of Sec. I.C), the reset writing the
// next initial state with its charges.  An S^x-basis sample is stored with
// every leg rotated by R (rows: the S^x eigenvectors), which exchanges S^x
// and S^z and leaves the gates and the Bell pairs unchanged, so it is blocked
// too; counters[2] records that frame for the measurement and the collapse.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "hm_block.cuh"
#include "hm_internal.h"

namespace hm {

namespace {

constexpr int NT = 256;          // threads per CTA
constexpr int kMaxSweeps = 60;   // one-sided Jacobi sweep budget
constexpr int TM = 64, TN = 64, TK = 16;

struct GemmSmem {
  double a[TK][TM + 1];
  double b[TK][TN + 1];
};

struct Shared {
  GemmSmem g;
  double red[NT / 32][4];
  double scal[8];
  int32_t ival[8];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of up to 3 values; result broadcast to every thread.
__device__ void block_sum3(double& x, double& y, double& z, Shared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  x = warp_sum(x);
  y = warp_sum(y);
  z = warp_sum(z);
  __syncthreads();
  if (lane == 0) {
    sh.red[warp][0] = x;
    sh.red[warp][1] = y;
    sh.red[warp][2] = z;
  }
  __syncthreads();
  double a = 0, b = 0, c = 0;
  for (int w = 0; w < NT / 32; ++w) {
    a += sh.red[w][0];
    b += sh.red[w][1];
    c += sh.red[w][2];
  }
  x = a;
  y = b;
  z = c;
  __syncthreads();
}

// C[M x N] = alpha op(A) op(B) (+ beta C), row-major.  TA: A stored K x M.
// TB: B stored N x K.  Whole CTA cooperates; ends with a barrier.
template <bool TA, bool TB>
__device__ void cta_gemm(int M, int N, int K, double alpha, const double* __restrict__ A, int lda,
                         const double* __restrict__ B, int ldb, double beta, double* __restrict__ C,
                         int ldc, GemmSmem& sm) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (int i0 = 0; i0 < M; i0 += TM) {
    for (int j0 = 0; j0 < N; j0 += TN) {
      double acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
      for (int k0 = 0; k0 < K; k0 += TK) {
        for (int e = tid; e < TM * TK; e += NT) {
          int ii, kk;
          if (TA) { ii = e % TM; kk = e / TM; } else { kk = e % TK; ii = e / TK; }
          const int gi = i0 + ii, gk = k0 + kk;
          double v = 0.0;
          if (gi < M && gk < K) v = TA ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
          sm.a[kk][ii] = v;
        }
        for (int e = tid; e < TN * TK; e += NT) {
          int jj, kk;
          if (TB) { kk = e % TK; jj = e / TK; } else { jj = e % TN; kk = e / TN; }
          const int gj = j0 + jj, gk = k0 + kk;
          double v = 0.0;
          if (gj < N && gk < K) v = TB ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj];
          sm.b[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
          double a[4], b[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) a[r] = sm.a[kk][ty + 16 * r];
#pragma unroll
          for (int c = 0; c < 4; ++c) b[c] = sm.b[kk][tx + 16 * c];
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty + 16 * r;
        if (i >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int j = j0 + tx + 16 * c;
          if (j >= N) continue;
          double v = alpha * acc[r][c];
          if (beta != 0.0) v += beta * C[(size_t)i * ldc + j];
          C[(size_t)i * ldc + j] = v;
        }
      }
    }
  }
  __syncthreads();
}

__device__ void set_error(const ChainDev* c, int code, int where, int32_t* ctx_err) {
  if (threadIdx.x == 0) {
    if (atomicCAS(c->status, 0, code) == 0) *c->err_where = where;
    if (ctx_err) atomicCAS(ctx_err, 0, code);
  }
}

// ---------------------------------------------------------------------------
// Step 2: one two-site op (Sec. I.A gates, Sec. II truncated SVD).
// ---------------------------------------------------------------------------

// One-sided (Hestenes) Jacobi on the q x p column-major matrix W (q >= p),
// accumulating the rotations in V (p x p).  Columns are paired by the
// round-robin tournament so that each round's pairs are disjoint; each warp
// rotates one pair at a time.  Returns sweeps used, or -1 if not converged.
__device__ int cta_jacobi(double* __restrict__ W, int q, int p, double* __restrict__ V, Shared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = NT / 32;
  for (int e = tid; e < p * p; e += NT) V[e] = (e % (p + 1) == 0) ? 1.0 : 0.0;
  const double tol = sqrt((double)q) * 2.220446049250313e-16;
  const int p2 = p + (p & 1);
  int done = 0;
  bool converged = false;
  double rmax = 0.0;
  while (done < kMaxSweeps) {
    if (tid == 0) {
      sh.ival[0] = 0;
      sh.scal[5] = 0.0;                 // largest rotation ratio of the sweep
    }
    __syncthreads();
    rmax = 0.0;
    for (int r = 0; r < p2 - 1; ++r) {
      for (int pi = warp; pi < p2 / 2; pi += nwarps) {
        int a, b;
        if (pi == 0) {
          a = r;
          b = p2 - 1;
        } else {
          a = (r + pi) % (p2 - 1);
          b = (r - pi + (p2 - 1)) % (p2 - 1);
        }
        if (a >= p || b >= p) continue;
        double* ca = W + (size_t)a * q;
        double* cb = W + (size_t)b * q;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < q; i += 32) {
          const double x = ca[i], y = cb[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.0 && al > 0.0 && be > 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          rmax = fmax(rmax, fabs(ga) / (sqrt(al) * sqrt(be)));
          const double zeta = (be - al) / (2.0 * ga);
          double t;
          if (fabs(zeta) > 1e150) t = 0.5 / zeta;
          else t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
          for (int i = lane; i < q; i += 32) {
            const double x = ca[i], y = cb[i];
            ca[i] = cs * x - sn * y;
            cb[i] = sn * x + cs * y;
          }
          double* va = V + (size_t)a * p;
          double* vb = V + (size_t)b * p;
          for (int i = lane; i < p; i += 32) {
            const double x = va[i], y = vb[i];
            va[i] = cs * x - sn * y;
            vb[i] = sn * x + cs * y;
          }
          if (lane == 0) sh.ival[0] = 1;
        }
      }
      __syncthreads();
    }
    if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(&sh.scal[5]),
                             (unsigned long long)__double_as_longlong(rmax));
    __syncthreads();
    const int rotated = sh.ival[0];
    const double rm = sh.scal[5];
    __syncthreads();
    ++done;
    // no rotation: converged; all rotations tiny: quadratic convergence puts
    // the next sweep's off-diagonals (O(rm^2)) far below the tolerance
    if (!rotated || rm < 1e-9) {
      converged = true;
      break;
    }
  }
  return converged ? done : -1;
}

// Truncation rule (Sec. II): smallest k >= 1 whose discarded weight
// sum_{q>=k} s_q^2 / sum s^2 <= cutoff, then min(k, chi_max), then lowered to
// the nearest gap s_{k} < s_{k-1} (1 - 1e-8).  Runs on thread 0.
__device__ int truncation_rank(const double* s, int n, int chi_max, double cutoff, double* tail,
                               double* total_out) {
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

__device__ void two_site_op(ChainDev* c, const OpDev op, int t, Shared& sh, int32_t* ctx_err) {
  const int tid = threadIdx.x;
  const int k = op.k;
  const int chil = c->chi[k], chim = c->chi[k + 1], chir = c->chi[k + 2];
  const int m = 3 * chil, n = 3 * chir;
  double* Ak = c->site[k];
  double* Ak1 = c->site[k + 1];
  double* theta = c->theta;
  double* W = c->W;
  double* V = c->V;

  // theta[(l s1), (s2 r)] = sum_m A_k[(l s1), m] A_{k+1}[m, (s2 r)]
  cta_gemm<false, false>(m, n, chim, 1.0, Ak, chim, Ak1, n, 0.0, theta, n, sh.g);

  // Gate on the physical legs, written column-oriented for the Jacobi:
  // trans = 0: W (m x n col-major) = X;  trans = 1: W (n x m col-major) = X^T.
  const bool trans = n > m;
  const int q = trans ? n : m, p = trans ? m : n;
  const double* G = c->gates + (size_t)op.gate * 81;
  for (int e = tid; e < chil * chir; e += NT) {
    const int l = e / chir, r = e % chir;
    double th[9];
#pragma unroll
    for (int s1 = 0; s1 < 3; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < 3; ++s2) th[3 * s1 + s2] = theta[(size_t)(3 * l + s1) * n + s2 * chir + r];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        double x = 0.0;
#pragma unroll
        for (int u = 0; u < 9; ++u) x = fma(G[(3 * a + b) * 9 + u], th[u], x);
        const int row = 3 * l + a, col = b * chir + r;
        if (!trans) W[(size_t)col * q + row] = x;
        else W[(size_t)row * q + col] = x;
      }
  }
  __syncthreads();

  const int sweeps = cta_jacobi(W, q, p, V, sh);
  if (sweeps < 0) {
    set_error(c, HM_ERR_NUMERIC, t, ctx_err);
    return;
  }

  // column norms (singular values), then rank-sort descending
  double* sig_raw = theta;               // theta is free now
  double* tail = theta + p;              // p + 1 doubles
  const int lane = tid & 31, warp = tid >> 5;
  for (int j = warp; j < p; j += NT / 32) {
    const double* cj = W + (size_t)j * q;
    double s2 = 0.0;
    for (int i = lane; i < q; i += 32) s2 = fma(cj[i], cj[i], s2);
    s2 = warp_sum(s2);
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
    double total;
    int kk;
    double nrm = 1.0;
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
    sh.ival[1] = kk;
    sh.scal[0] = nrm;
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
  const int kk = sh.ival[1];
  const double nrm = sh.scal[0];
  if (kk <= 0) {
    set_error(c, HM_ERR_NUMERIC, t, ctx_err);
    return;
  }
  const bool absorb_left = op.absorb == 0;
  // A_k[(l s), i] and A_{k+1}[i, (s r)] from the sorted singular triplets
  for (int e = tid; e < m * kk; e += NT) {
    const int row = e / kk, i = e % kk;
    const int j = c->perm[i];
    const double sg = c->sig[i];
    double v;
    if (!trans) {
      const double w = W[(size_t)j * q + row];   // = U sigma
      v = absorb_left ? w * nrm : w / sg;
    } else {
      const double u = V[(size_t)j * p + row];   // left vector
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
      const double u = V[(size_t)j * p + col];   // right vector
      v = absorb_left ? u : u * sg * nrm;
    } else {
      const double w = W[(size_t)j * q + col];   // = V sigma
      v = absorb_left ? w / sg : w * nrm;
    }
    Ak1[e] = v;
  }
  __syncthreads();
  if (tid == 0) c->chi[k + 1] = kk;
  __syncthreads();
}

// One two-site op of a chain, block by block in the S^z charge of the new
// middle bond (Sec. II.C): theta by block GEMMs, the gate within its
// conserved sectors, a binary64 one-sided Jacobi per block, then one
// truncation over the union of the blocks' singular values (Sec. II).  The
// blocks take the whole CTA in turn: the binary64 pipe (about 2 FMA per
// clock per SM on GB300) is the bound, and every warp of the CTA is needed
// to hide the latency of the global-memory rotations (splitting the warps
// over the blocks of a split measured 1.7x slower).
__device__ void two_site_op_blocked(ChainDev* c, const OpDev op, int t, Shared& sh, blk::SplitSh& ss,
                                    blk::GroupSh& gs, int32_t* ctx_err) {
  if (!blk::prepare<NT>(c, op, ss)) blk::prepare<NT>(c, op, ss);
  blk::theta_blocks<NT, TM, TN, TK, double>(c, op.k, ss, c->theta, &sh.g.a[0][0]);
  const blk::Meta* M = reinterpret_cast<const blk::Meta*>(c->meta);
  int sweeps = 0;
  int64_t cost = -1;
  for (int b = 0; b < ss.nblk; ++b) {
    const blk::BlockRec& r = M->b[b];
    blk::gather_block<NT, double, double>(c, op.k, ss, r, c->theta, c->W + r.woff, r.q, c->V + r.voff, r.p);
    __syncthreads();
    const int sw = blk::jacobi_group<double, double, 2>(c->W + r.woff, r.q, r.q, r.p, c->V + r.voff, r.p, c->sig,
                                             threadIdx.x >> 5, NT / 32, 1, 0, gs, 1e-9, kMaxSweeps);
    if (sw < 0) {
      set_error(c, HM_ERR_NUMERIC, t, ctx_err);
      return;
    }
    const int64_t cb = (int64_t)r.q * r.p * r.p;   // sweeps of the costliest block
    if (cb > cost) cost = cb, sweeps = sw;
    __syncthreads();
  }
  blk::finish<NT>(c, op, t, ss, c->theta, ctx_err, sweeps, 0);
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

__global__ void __launch_bounds__(NT) evolve_fp64_kernel(BatchArg b, OutArg o) {
  __shared__ Shared sh;
  __shared__ blk::SplitSh ss;
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
    two_site_op_blocked(c, ops[t], t, sh, ss, gs, o.ctx_err);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Transfer matrices (steps 3 and 4).
// ---------------------------------------------------------------------------

// Eout[cr x cr] = sum_{s,t} O[s][t] A^{sT} Ein A^t   (O == nullptr: identity).
// Z: cl x 3cr scratch.  Ein/Eout are row-major, bra index first.
__device__ void cta_transfer(const double* Ein, const double* A, int cl, int cr, const double* O,
                             double* Eout, double* Z, Shared& sh) {
  if (threadIdx.x == 0) sh.scal[4] += 6.0 * cl * cl * cr + 6.0 * cl * cr * cr;
  cta_gemm<false, false>(cl, 3 * cr, cl, 1.0, Ein, cl, A, 3 * cr, 0.0, Z, 3 * cr, sh.g);
  if (O) {
    for (int e = threadIdx.x; e < cl * cr; e += NT) {
      const int i = e / cr, r = e % cr;
      double* z = Z + (size_t)i * 3 * cr + r;
      const double z0 = z[0], z1 = z[cr], z2 = z[2 * cr];
      z[0] = O[0] * z0 + O[1] * z1 + O[2] * z2;
      z[cr] = O[3] * z0 + O[4] * z1 + O[5] * z2;
      z[2 * cr] = O[6] * z0 + O[7] * z1 + O[8] * z2;
    }
    __syncthreads();
  }
  cta_gemm<true, false>(cr, cr, 3 * cl, 1.0, A, cr, Z, cr, 0.0, Eout, cr, sh.g);
}

__device__ __constant__ double kSz[9] = {1, 0, 0, 0, 0, 0, 0, 0, -1};
// S+ = sqrt(2) (|+1><0| + |0><-1|); S- its transpose (basis m = +1, 0, -1)
__device__ __constant__ double kSp[9] = {0, 1.4142135623730951, 0, 0, 0, 1.4142135623730951, 0, 0, 0};
__device__ __constant__ double kSm[9] = {0, 0, 0, 1.4142135623730951, 0, 0, 0, 1.4142135623730951, 0};
// Right environment through one site: Rout[i, j] = sum_s A^s Rin A^{sT}
// (Rin cr x cr, Rout cl x cl).  Y: 3cl x cr scratch.
__device__ void cta_rtransfer(const double* Rin, const double* A, int cl, int cr, double* Rout, double* Y,
                              Shared& sh) {
  if (threadIdx.x == 0) sh.scal[4] += 12.0 * cl * cr * cr;
  cta_gemm<false, false>(3 * cl, cr, cr, 1.0, A, cr, Rin, cr, 0.0, Y, cr, sh.g);
  cta_gemm<false, true>(cl, cl, 3 * cr, 1.0, Y, 3 * cr, A, 3 * cr, 0.0, Rout, cl, sh.g);
}

// Charge blocks of the transfer matrices (Sec. II.C).  A bond's indices are
// grouped by S^z charge, so a charge is one run [start, start + len) of the
// bond.  For a state of definite total S^z an environment E[i, j] (bra i,
// ket j) is nonzero only where q_i - q_j = D, its charge shift: 0 for the
// plain environment, sigma for one S^+ inserted on a leg of sign sigma,
// -sigma for S^-.  Dense-mode chains have every charge 0: one run, D = 0,
// and these reduce to the plain dense transfers.
__device__ void charge_run(const int16_t* q, int n, int Q, int* start, int* len) {
  int lo = 0, hi = n;
  while (lo < hi) {                       // first index with q >= Q
    const int mid = (lo + hi) >> 1;
    if (q[mid] < Q) lo = mid + 1;
    else hi = mid;
  }
  int e = lo;
  while (e < n && q[e] == Q) ++e;
  *start = lo;
  *len = e - lo;
}

// Left environment through site pos with operator O (nullptr: identity;
// O[s][t] = <s|O|t>, nonzero only for m(s) - m(t) = dO):
// Eout[i', j'] = sum_{s,t} O[s][t] sum_{i,j} A[i,s,i'] Ein[i,j] A[j,t,j'],
// computed only on the charge blocks it can fill.  Ein has shift D; the
// result has shift D + sigma dO (returned).  Z: scratch of cl x cr doubles.
__device__ int cta_transfer_blk(const ChainDev* c, int pos, const double* Ein, int D, const double* O, int dO,
                                double* Eout, double* Z, Shared& sh) {
  const int cl = c->chi[pos], cr = c->chi[pos + 1];
  const double* A = c->site[pos];
  const int16_t* qL = c->qn + (size_t)pos * c->chi_cap;
  const int16_t* qR = qL + c->chi_cap;
  const int sg = c->sgn[pos];
  const int D2 = D + sg * dO;
  for (int e = threadIdx.x; e < cr * cr; e += NT) Eout[e] = 0.0;
  __syncthreads();
  double fl = 0.0;
  for (int b0 = 0; b0 < cr;) {
    int bs, bl;
    charge_run(qR, cr, qR[b0], &bs, &bl);     // bra run of the right bond
    const int Qb = qR[b0], Qk = Qb - D2;
    b0 = bs + bl;
    int ks, kl;
    charge_run(qR, cr, Qk, &ks, &kl);         // ket run
    if (kl == 0) continue;
    for (int s1 = 0; s1 < 3; ++s1) {
      int is, il;
      charge_run(qL, cl, Qb - sg * (1 - s1), &is, &il);
      if (il == 0) continue;
      bool first = true;
      for (int t1 = 0; t1 < 3; ++t1) {
        const double w = O ? O[3 * s1 + t1] : (s1 == t1 ? 1.0 : 0.0);
        if (w == 0.0) continue;
        int js, jl;
        charge_run(qL, cl, Qk - sg * (1 - t1), &js, &jl);
        if (jl == 0) continue;
        // Z (il x kl) (+)= w Ein[i-run, j-run] A[j-run, t1, k-run]
        cta_gemm<false, false>(il, kl, jl, w, Ein + (size_t)is * cl + js, cl, A + (size_t)(3 * js + t1) * cr + ks,
                               3 * cr, first ? 0.0 : 1.0, Z, kl, sh.g);
        fl += 2.0 * il * jl * kl;
        first = false;
      }
      if (first) continue;
      // Eout[b-run, k-run] += A[i-run, s1, b-run]^T Z
      cta_gemm<true, false>(bl, kl, il, 1.0, A + (size_t)(3 * is + s1) * cr + bs, 3 * cr, Z, kl, 1.0,
                            Eout + (size_t)bs * cr + ks, cr, sh.g);
      fl += 2.0 * il * bl * kl;
    }
  }
  if (threadIdx.x == 0) sh.scal[4] += fl;
  __syncthreads();
  return D2;
}

// Plain right environment through site pos (shift 0):
// Rout[i, j] = sum_s sum_{a,b} A[i,s,a] Rin[a,b] A[j,s,b], block by block.
// Y: scratch of cl x cr doubles.
__device__ void cta_rtransfer_blk(const ChainDev* c, int pos, const double* Rin, double* Rout, double* Y, Shared& sh) {
  const int cl = c->chi[pos], cr = c->chi[pos + 1];
  const double* A = c->site[pos];
  const int16_t* qL = c->qn + (size_t)pos * c->chi_cap;
  const int16_t* qR = qL + c->chi_cap;
  const int sg = c->sgn[pos];
  for (int e = threadIdx.x; e < cl * cl; e += NT) Rout[e] = 0.0;
  __syncthreads();
  double fl = 0.0;
  for (int i0 = 0; i0 < cl;) {
    int is, il;
    charge_run(qL, cl, qL[i0], &is, &il);
    const int Q = qL[i0];
    i0 = is + il;
    for (int s1 = 0; s1 < 3; ++s1) {
      int as, al;
      charge_run(qR, cr, Q + sg * (1 - s1), &as, &al);
      if (al == 0) continue;
      // Y (il x al) = A[i-run, s1, a-run] Rin[a-run, a-run]
      cta_gemm<false, false>(il, al, al, 1.0, A + (size_t)(3 * is + s1) * cr + as, 3 * cr, Rin + (size_t)as * cr + as,
                             cr, 0.0, Y, al, sh.g);
      // Rout[i-run, i-run] += Y A[i-run, s1, a-run]^T
      cta_gemm<false, true>(il, il, al, 1.0, Y, al, A + (size_t)(3 * is + s1) * cr + as, 3 * cr, 1.0,
                            Rout + (size_t)is * cl + is, cl, sh.g);
      fl += 2.0 * il * al * al + 2.0 * il * il * al;
    }
  }
  if (threadIdx.x == 0) sh.scal[4] += fl;
  __syncthreads();
}

// sum_{k,l} X[k, l] Y[k, l] over n entries, block-wide.
__device__ double cta_dot(const double* X, const double* Y, int n, Shared& sh) {
  double acc = 0.0, d1 = 0.0, d2 = 0.0;
  for (int e = threadIdx.x; e < n; e += NT) acc = fma(X[e], Y[e], acc);
  block_sum3(acc, d1, d2, sh);
  return acc;
}

// Step 3 (Sec. I.C.1): <S_i.S_j> and <Sz_i Sz_j> on every measured bond.
// Right environments are built explicitly from the last site (no reliance on
// the canonical form), so <psi|psi> is the full contraction and every value
// is divided by it.
__global__ void __launch_bounds__(NT) measure_fp64_kernel(BatchArg b, OutArg o) {
  __shared__ Shared sh;
  ChainDev* c = b.c[blockIdx.x];
  const int tid = threadIdx.x;
  double* out = o.obs + (size_t)blockIdx.x * o.n_obs;
  if (*(volatile int32_t*)c->status != 0) {
    for (int e = tid; e < o.n_obs; e += NT) out[e] = NAN;
    return;
  }
  const int64_t cc = (int64_t)c->chi_cap * c->chi_cap;
  double* Lp[2] = {c->env_ws, c->env_ws + cc};
  double* Ep[2] = {c->env_ws + 2 * cc, c->env_ws + 3 * cc};
  double* Z = c->env_ws + 4 * cc;          // 3 cc
  double* Et = c->env_ws + 7 * cc;         // cc
  double* Rp[2] = {c->env_ws + 8 * cc, c->env_ws + 9 * cc};
  double* Rend = c->env_ws + 10 * cc;      // one cc slot per distinct measured end site
  if (tid == 0) {
    Rp[0][0] = 1.0;
    sh.scal[4] = 0.0;
  }
  __syncthreads();
  // right sweep: R(pos) = environment of sites >= pos; keep R(b + 1) per end b
  int rc = 0;
  for (int pos = c->n_sites - 1; pos >= 0; --pos) {
    for (int q = 0; q < c->n_meas; ++q) {
      if (c->meas_j[q] == pos) {            // R(pos + 1) is current
        const int slot = c->meas_slot[q];
        const int n2 = c->chi[pos + 1] * c->chi[pos + 1];
        for (int e = tid; e < n2; e += NT) Rend[(size_t)slot * cc + e] = Rp[rc][e];
      }
    }
    __syncthreads();
    cta_rtransfer_blk(c, pos, Rp[rc], Rp[rc ^ 1], Z, sh);
    rc ^= 1;
  }
  const double nrm = Rp[rc][0];            // <psi|psi>
  if (tid == 0) Lp[0][0] = 1.0;
  __syncthreads();
  int pos = 0, cur = 0;
  double E_est = 0.0;
  // A chain in frame 1 stores R^N |psi> (R exchanges S^x and S^z, R S^z R =
  // S^x): there <Sz_i Sz_j> of |psi> is <Sx_i Sx_j> of the stored state,
  // which for a state of definite total S^z is (<S+_i S-_j> + <S-_i S+_j>)/4;
  // S_i.S_j is invariant.  Passes: (Sz Sz), (S+ S-), (S- S+); operator
  // charge shifts dO = 0, +1, -1 and -dO.
  const int frame = c->counters[2];
  const double* ops1[3] = {kSz, kSp, kSm};
  const double* ops2[3] = {kSz, kSm, kSp};
  const int dop[3] = {0, 1, -1};
  int bi = 0;
  while (bi < c->n_meas) {
    const int a = c->meas_i[bi];
    int bend = bi;
    while (bend < c->n_meas && c->meas_i[bend] == a) ++bend;
    const int blast = c->meas_j[bend - 1];
    while (pos < a) {
      cta_transfer_blk(c, pos, Lp[cur], 0, nullptr, 0, Lp[cur ^ 1], Z, sh);
      cur ^= 1;
      ++pos;
    }
    double vals[3][8];   // up to 8 bonds per start site
    for (int o1 = 0; o1 < 3; ++o1) {
      int ec = 0;
      int D = cta_transfer_blk(c, a, Lp[cur], 0, ops1[o1], dop[o1], Ep[ec], Z, sh);
      for (int kk = a + 1; kk <= blast; ++kk) {
        for (int q = bi; q < bend; ++q) {
          if (c->meas_j[q] == kk) {
            cta_transfer_blk(c, kk, Ep[ec], D, ops2[o1], -dop[o1], Et, Z, sh);
            const int n2 = c->chi[kk + 1] * c->chi[kk + 1];
            vals[o1][q - bi] = cta_dot(Et, Rend + (size_t)c->meas_slot[q] * cc, n2, sh);
          }
        }
        if (kk < blast) {
          D = cta_transfer_blk(c, kk, Ep[ec], D, nullptr, 0, Ep[ec ^ 1], Z, sh);
          ec ^= 1;
        }
      }
    }
    if (tid == 0) {
      for (int q = bi; q < bend; ++q) {
        const double pm = (vals[1][q - bi] + vals[2][q - bi]) / nrm;
        const double ss = vals[0][q - bi] / nrm + 0.5 * pm;
        const double zz = frame ? 0.25 * pm : vals[0][q - bi] / nrm;
        out[1 + 2 * q] = ss;
        out[2 + 2 * q] = zz;
        E_est += c->meas_J[q] * ss;
      }
    }
    bi = bend;
  }
  if (tid == 0) {
    out[0] = E_est;
    c->stats[ST_TRANSFER] += sh.scal[4];
  }
}

// Right environment with an operator on this site, accumulated:
// Rout <- acc * Rout + sum_{s,t} O[s][t] A^s Rin A^{tT}  (O == nullptr: identity;
// bra index s first).  Rin cr x cr, Rout cl x cl, Y: 3cl x cr scratch.
__device__ void cta_rtransfer_op(const double* Rin, const double* A, int cl, int cr, const double* O, double* Rout,
                                 double* Y, double acc, Shared& sh) {
  if (threadIdx.x == 0) sh.scal[4] += 12.0 * cl * cr * cr;
  cta_gemm<false, false>(3 * cl, cr, cr, 1.0, A, cr, Rin, cr, 0.0, Y, cr, sh.g);
  if (O) {
    for (int e = threadIdx.x; e < cl * cr; e += NT) {
      const int i = e / cr, r = e % cr;
      double* y = Y + (size_t)i * 3 * cr + r;
      const double y0 = y[0], y1 = y[cr], y2 = y[2 * cr];
      y[0] = O[0] * y0 + O[3] * y1 + O[6] * y2;
      y[cr] = O[1] * y0 + O[4] * y1 + O[7] * y2;
      y[2 * cr] = O[2] * y0 + O[5] * y1 + O[8] * y2;
    }
    __syncthreads();
  }
  cta_gemm<false, true>(cl, cl, 3 * cr, 1.0, Y, 3 * cr, A, 3 * cr, acc, Rout, cl, sh.g);
}

// Left environment with an operator on this site, accumulated:
// Eout <- acc * Eout + sum_{s,t} O[s][t] A^{sT} Ein A^t.
__device__ void cta_transfer_acc(const double* Ein, const double* A, int cl, int cr, const double* O, double* Eout,
                                 double* Z, double acc, Shared& sh) {
  if (threadIdx.x == 0) sh.scal[4] += 6.0 * cl * cl * cr + 6.0 * cl * cr * cr;
  cta_gemm<false, false>(cl, 3 * cr, cl, 1.0, Ein, cl, A, 3 * cr, 0.0, Z, 3 * cr, sh.g);
  if (O) {
    for (int e = threadIdx.x; e < cl * cr; e += NT) {
      const int i = e / cr, r = e % cr;
      double* z = Z + (size_t)i * 3 * cr + r;
      const double z0 = z[0], z1 = z[cr], z2 = z[2 * cr];
      z[0] = O[0] * z0 + O[1] * z1 + O[2] * z2;
      z[cr] = O[3] * z0 + O[4] * z1 + O[5] * z2;
      z[2 * cr] = O[6] * z0 + O[7] * z1 + O[8] * z2;
    }
    __syncthreads();
  }
  cta_gemm<true, false>(cr, cr, 3 * cl, 1.0, A, cr, Z, cr, acc, Eout, cr, sh.g);
}

// Uniform susceptibility (Eq. sus, Sec. II.A): the double sum
// sum_{a in M} sum_{b physical} <S_a . S_b> / <psi|psi>, written to o.obs[chain].
// A right sweep carries the plain right environment R and the running sums
// R_z, R_-, R_+ of right environments with S^z, S^-, S^+ inserted on every
// physical site to the right, and keeps all four at each region site a
// (R(a+1)); a left sweep carries the mirrored sums L, L_z, L_+, L_- and
// closes, at each region site a, O_a on L against the right sums (b > a)
// and the left sums with O_a against R (b < a).  Linear in the chain length.
__global__ void __launch_bounds__(NT) susceptibility_fp64_kernel(BatchArg b, OutArg o) {
  __shared__ Shared sh;
  ChainDev* c = b.c[blockIdx.x];
  const int tid = threadIdx.x;
  double* out = o.obs + blockIdx.x;
  if (*(volatile int32_t*)c->status != 0) {
    if (tid == 0) *out = NAN;
    return;
  }
  const int64_t cc = (int64_t)c->chi_cap * c->chi_cap;
  double* Rc[4];
  double* Rn[4];
  double* Lc[4];
  double* Ln[4];
  for (int qq = 0; qq < 4; ++qq) {
    Rc[qq] = c->env_ws + qq * cc;
    Rn[qq] = c->env_ws + (4 + qq) * cc;
    Lc[qq] = c->env_ws + (8 + qq) * cc;
    Ln[qq] = c->env_ws + (12 + qq) * cc;
  }
  double* Z = c->env_ws + 16 * cc;         // 3 cc
  double* Et = c->env_ws + 19 * cc;
  double* store = c->env_ws + 20 * cc;     // 4 cc per region site
  // right sums carry S^z, S^-, S^+ ; left sums carry S^z, S^+, S^-
  const double* ropk[4] = {nullptr, kSz, kSm, kSp};
  const double* lopk[4] = {nullptr, kSz, kSp, kSm};
  if (tid == 0) {
    Rc[0][0] = 1.0;
    Rc[1][0] = Rc[2][0] = Rc[3][0] = 0.0;
    Lc[0][0] = 1.0;
    Lc[1][0] = Lc[2][0] = Lc[3][0] = 0.0;
    sh.scal[4] = 0.0;
  }
  __syncthreads();
  const int n = c->n_sites;
  int amax = -1;
  for (int s2 = 0; s2 < c->n_region; ++s2) amax = max(amax, c->region[s2]);
  for (int pos = n - 1; pos >= 0; --pos) {
    const int cl = c->chi[pos], cr = c->chi[pos + 1];
    int slot = -1;
    for (int s2 = 0; s2 < c->n_region; ++s2)
      if (c->region[s2] == pos) slot = s2;
    if (slot >= 0) {
      for (int qq = 0; qq < 4; ++qq)
        for (int e = tid; e < cr * cr; e += NT) store[(size_t)(4 * slot + qq) * cc + e] = Rc[qq][e];
      __syncthreads();
    }
    const double* A = c->site[pos];
    const bool phys = c->site_kind[pos] != SITE_ANC;
    cta_rtransfer_op(Rc[0], A, cl, cr, nullptr, Rn[0], Z, 0.0, sh);
    for (int qq = 1; qq < 4; ++qq) {
      cta_rtransfer_op(Rc[qq], A, cl, cr, nullptr, Rn[qq], Z, 0.0, sh);
      if (phys) cta_rtransfer_op(Rc[0], A, cl, cr, ropk[qq], Rn[qq], Z, 1.0, sh);
    }
    for (int qq = 0; qq < 4; ++qq) {
      double* t = Rc[qq];
      Rc[qq] = Rn[qq];
      Rn[qq] = t;
    }
  }
  const double nrm = Rc[0][0];             // <psi|psi>
  double total = 0.0;
  for (int pos = 0; pos <= amax; ++pos) {
    const int cl = c->chi[pos], cr = c->chi[pos + 1];
    const double* A = c->site[pos];
    int slot = -1;
    for (int s2 = 0; s2 < c->n_region; ++s2)
      if (c->region[s2] == pos) slot = s2;
    if (slot >= 0) {
      const double* R0 = store + (size_t)(4 * slot) * cc;
      const double* Rz = R0 + cc;
      const double* Rm = R0 + 2 * cc;
      const double* Rp = R0 + 3 * cc;
      const int n2 = cr * cr;
      // b > a: O_a on L, closed against the right sums
      cta_transfer_acc(Lc[0], A, cl, cr, kSz, Et, Z, 0.0, sh);
      total += cta_dot(Et, Rz, n2, sh);
      cta_transfer_acc(Lc[0], A, cl, cr, kSp, Et, Z, 0.0, sh);
      total += 0.5 * cta_dot(Et, Rm, n2, sh);
      cta_transfer_acc(Lc[0], A, cl, cr, kSm, Et, Z, 0.0, sh);
      total += 0.5 * cta_dot(Et, Rp, n2, sh);
      // b < a: left sums with O_a, closed against R
      cta_transfer_acc(Lc[1], A, cl, cr, kSz, Et, Z, 0.0, sh);
      total += cta_dot(Et, R0, n2, sh);
      cta_transfer_acc(Lc[2], A, cl, cr, kSm, Et, Z, 0.0, sh);
      total += 0.5 * cta_dot(Et, R0, n2, sh);
      cta_transfer_acc(Lc[3], A, cl, cr, kSp, Et, Z, 0.0, sh);
      total += 0.5 * cta_dot(Et, R0, n2, sh);
      total += 2.0 * nrm;                  // b = a: S.S = s(s+1) = 2
    }
    if (pos == amax) break;
    const bool phys = c->site_kind[pos] != SITE_ANC;
    cta_transfer_acc(Lc[0], A, cl, cr, nullptr, Ln[0], Z, 0.0, sh);
    for (int qq = 1; qq < 4; ++qq) {
      cta_transfer_acc(Lc[qq], A, cl, cr, nullptr, Ln[qq], Z, 0.0, sh);
      if (phys) cta_transfer_acc(Lc[0], A, cl, cr, lopk[qq], Ln[qq], Z, 1.0, sh);
    }
    for (int qq = 0; qq < 4; ++qq) {
      double* t = Lc[qq];
      Lc[qq] = Ln[qq];
      Ln[qq] = t;
    }
  }
  if (tid == 0) {
    *out = total / nrm;
    c->stats[ST_TRANSFER] += sh.scal[4];
  }
}

// ---------------------------------------------------------------------------
// Step 4: collapse and reset.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                             uint32_t k0, uint32_t k1) {
  const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
  const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
  const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
  c0 = n0;
  c1 = lo1;
  c2 = n2;
  c3 = lo0;
}

// Philox4x32-10 (Salmon et al., SC'11): counter (n, ordinal, seed_hi, 0),
// key (seed_lo, chain_id); u = ((x0 >> 5) 2^26 + (x1 >> 6)) 2^-53.
__device__ double philox_uniform(uint32_t n, uint32_t ordinal, uint32_t seed_hi, uint32_t seed_lo,
                                 uint32_t chain) {
  uint32_t c0 = n, c1 = ordinal, c2 = seed_hi, c3 = 0u;
  uint32_t k0 = seed_lo, k1 = chain;
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    philox_round(c0, c1, c2, c3, k0, k1);
  }
  return ((double)(c0 >> 5) * 67108864.0 + (double)(c1 >> 6)) * (1.0 / 9007199254740992.0);
}

// First b with u < cumulative p_b, else the last b with p_b > 0.
__device__ int choose3(const double p[3], double u) {
  double acc = 0.0;
  for (int b = 0; b < 3; ++b) {
    acc += p[b];
    if (u < acc) return b;
  }
  for (int b = 2; b >= 0; --b)
    if (p[b] > 0.0) return b;
  return -1;
}

__device__ void basis_rows(const ChainDev* c, int basis, double B[9]) {
  for (int i = 0; i < 9; ++i) B[i] = basis ? c->xbasis[i] : ((i % 4 == 0) ? 1.0 : 0.0);
}

// Sequential projective measurement of the environment, left to right, in the
// basis of sample n (Sec. I.C.1 step 4); cluster sites are traced out, which
// turns the boundary vector into a density matrix (Eq. detailbalance1).
__global__ void __launch_bounds__(NT) collapse_fp64_kernel(BatchArg b, OutArg o) {
  __shared__ Shared sh;
  ChainDev* c = b.c[blockIdx.x];
  const int tid = threadIdx.x;
  if (*(volatile int32_t*)c->status != 0) return;
  const int n_sample = c->counters[0];
  const int basis = (c->basis_zx && (n_sample & 1)) ? 1 : 0;
  // the measured basis as seen by the stored state: R maps the S^z basis to
  // the S^x basis and back (R e_b = v_b, R v_b = e_b), so a frame-1 state is
  // measured in the other basis; the outcome order is the same
  double B[9];
  basis_rows(c, basis ^ c->counters[2], B);
  const int64_t cc = (int64_t)c->chi_cap * c->chi_cap;
  double* R[2] = {c->env_ws, c->env_ws + cc};
  double* X = c->env_ws + 2 * cc;      // cl x 3cr
  double* At = c->env_ws + 5 * cc;     // cl x cr
  double* Y = c->env_ws + 6 * cc;      // cl x cr
  int cur = 0;
  bool vec_mode = true;
  if (tid == 0) {
    R[0][0] = 1.0;                     // v = [1]
    sh.scal[4] = 0.0;
  }
  __syncthreads();
  int e_ord = 0;
  double logp = 0.0;
  for (int k = 0; k < c->n_sites; ++k) {
    const double* A = c->site[k];
    const int cl = c->chi[k], cr = c->chi[k + 1];
    if (c->site_kind[k] == SITE_ENV) {
      double q[3] = {0.0, 0.0, 0.0};
      if (vec_mode) {
        // X[(s r)] = sum_l v[l] A[l, s, r]
        for (int e = tid; e < 3 * cr; e += NT) {
          double acc = 0.0;
          for (int l = 0; l < cl; ++l) acc = fma(R[cur][l], A[(size_t)l * 3 * cr + e], acc);
          X[e] = acc;
        }
        __syncthreads();
        for (int r = tid; r < cr; r += NT) {
          const double x0 = X[r], x1 = X[cr + r], x2 = X[2 * cr + r];
          for (int bb = 0; bb < 3; ++bb) {
            const double w = B[3 * bb] * x0 + B[3 * bb + 1] * x1 + B[3 * bb + 2] * x2;
            q[bb] = fma(w, w, q[bb]);
          }
        }
      } else {
        cta_gemm<false, false>(cl, 3 * cr, cl, 1.0, R[cur], cl, A, 3 * cr, 0.0, X, 3 * cr, sh.g);
        for (int e = tid; e < cl * cr; e += NT) {
          const int i = e / cr, r = e % cr;
          const double* a = A + (size_t)i * 3 * cr + r;
          const double* x = X + (size_t)i * 3 * cr + r;
          const double a0 = a[0], a1 = a[cr], a2 = a[2 * cr];
          const double x0 = x[0], x1 = x[cr], x2 = x[2 * cr];
          for (int bb = 0; bb < 3; ++bb) {
            const double at = B[3 * bb] * a0 + B[3 * bb + 1] * a1 + B[3 * bb + 2] * a2;
            const double yt = B[3 * bb] * x0 + B[3 * bb + 1] * x1 + B[3 * bb + 2] * x2;
            q[bb] = fma(at, yt, q[bb]);
          }
        }
      }
      block_sum3(q[0], q[1], q[2], sh);
      if (tid == 0) {
        const double tot = q[0] + q[1] + q[2];
        int pick = -1;
        double pb = 0.0;
        if (tot > 0.0 && isfinite(tot)) {
          const double p[3] = {q[0] / tot, q[1] / tot, q[2] / tot};
          if (o.cond)
            for (int bb = 0; bb < 3; ++bb) o.cond[((size_t)blockIdx.x * o.n_env + e_ord) * 3 + bb] = p[bb];
          const double u = philox_uniform((uint32_t)n_sample, (uint32_t)e_ord, c->seed_hi, c->seed_lo,
                                          c->chain_id);
          pick = choose3(p, u);
          if (pick >= 0) pb = p[pick];
        }
        sh.ival[2] = pick;
        sh.scal[1] = pick >= 0 ? q[pick] : 0.0;
        if (pick >= 0) logp += log(pb);
      }
      __syncthreads();
      const int pick = sh.ival[2];
      const double qb = sh.scal[1];
      if (pick < 0) {
        set_error(c, HM_ERR_NUMERIC, 100000 + k, o.ctx_err);
        return;
      }
      if (tid == 0) {
        c->env_out[e_ord] = pick;
        if (o.env) o.env[(size_t)blockIdx.x * o.n_env + e_ord] = (int8_t)pick;
      }
      const double b0 = B[3 * pick], b1 = B[3 * pick + 1], b2 = B[3 * pick + 2];
      if (vec_mode) {
        const double sc = 1.0 / sqrt(qb);
        for (int r = tid; r < cr; r += NT)
          R[cur ^ 1][r] = (b0 * X[r] + b1 * X[cr + r] + b2 * X[2 * cr + r]) * sc;
        __syncthreads();
      } else {
        for (int e = tid; e < cl * cr; e += NT) {
          const int i = e / cr, r = e % cr;
          const double* a = A + (size_t)i * 3 * cr + r;
          const double* x = X + (size_t)i * 3 * cr + r;
          At[e] = b0 * a[0] + b1 * a[cr] + b2 * a[2 * cr];
          Y[e] = b0 * x[0] + b1 * x[cr] + b2 * x[2 * cr];
        }
        __syncthreads();
        cta_gemm<true, false>(cr, cr, cl, 1.0 / qb, At, cr, Y, cr, 0.0, R[cur ^ 1], cr, sh.g);
        if (tid == 0) sh.scal[4] += 6.0 * cl * cl * cr + 2.0 * cl * cr * cr;
      }
      cur ^= 1;
      ++e_ord;
    } else {
      if (vec_mode) {
        // rho = v v^T
        for (int e = tid; e < cl * cl; e += NT) R[cur ^ 1][e] = R[cur][e / cl] * R[cur][e % cl];
        __syncthreads();
        cur ^= 1;
        vec_mode = false;
      }
      cta_transfer(R[cur], A, cl, cr, nullptr, R[cur ^ 1], X, sh);
      cur ^= 1;
    }
  }
  if (tid == 0) {
    if (o.logp) o.logp[blockIdx.x] = logp;
    c->counters[0] = n_sample + 1;
    c->counters[1] = basis;
    c->stats[ST_TRANSFER] += sh.scal[4];
  }
}

// Writes the initial state |i>_E |B>_C from env_out and counters[1]
// (Sec. I.C.1 step 1): environment sites (1,3,1) basis vectors, cluster
// physical sites delta(s, 2 - a)/sqrt(3) of shape (1,3,3), ancillas
// delta(2 - a, s) of shape (3,3,1) (the Bell bond ordered by ascending
// S^z charge).  An environment drawn in the S^x basis is stored in frame 1:
// every leg rotated by R (rows: the S^x eigenvectors), which maps the S^x
// eigenvector v_b to e_b and leaves the Bell pairs and the Heisenberg gates
// unchanged (R is real orthogonal and the gates commute with R (x) R), so
// every initial state is a product of S^z eigenstates and Bell pairs with
// definite total S^z, and every sample evolves in charge blocks (Sec. II.C).
// With draw_initial, first draws the environment in the Sz basis with
// p = 1/3 each and sample index n = -1.
__global__ void __launch_bounds__(NT) reset_kernel(BatchArg b, OutArg o, int draw_initial) {
  ChainDev* c = b.c[blockIdx.x];
  const int tid = threadIdx.x;
  if (*(volatile int32_t*)c->status != 0) return;
  if (draw_initial) {
    const double third = 1.0 / 3.0;
    const double p[3] = {third, third, third};
    for (int e = tid; e < c->n_env; e += NT) {
      const double u = philox_uniform(0xFFFFFFFFu, (uint32_t)e, c->seed_hi, c->seed_lo, c->chain_id);
      c->env_out[e] = choose3(p, u);
    }
    if (tid == 0) {
      c->counters[0] = 0;
      c->counters[1] = 0;
    }
    __syncthreads();
  }
  const double r3 = 1.0 / sqrt(3.0);
  // env ordinal of site k = number of env sites before k
  for (int k = tid; k < c->n_sites; k += NT) {
    double* A = c->site[k];
    const int kind = c->site_kind[k];
    if (kind == SITE_ENV) {
      int ord = 0;
      for (int s = 0; s < k; ++s) ord += c->site_kind[s] == SITE_ENV;
      const int pick = c->env_out[ord];
      for (int s = 0; s < 3; ++s) A[s] = s == pick ? 1.0 : 0.0;
      c->sgn[k] = 1;
    } else if (kind == SITE_CPHYS) {
      for (int e = 0; e < 9; ++e) A[e] = (e / 3 == 2 - e % 3) ? r3 : 0.0;     // A[0, s, a]
      c->sgn[k] = 1;
    } else {
      for (int e = 0; e < 9; ++e) A[e] = (e / 3 == 2 - e % 3) ? 1.0 : 0.0;    // A[a, s, 0]
      c->sgn[k] = -1;
    }
  }
  for (int i = tid; i <= c->n_sites; i += NT)
    c->chi[i] = (i > 0 && i < c->n_sites && c->site_kind[i - 1] == SITE_CPHYS) ? 3 : 1;
  if (tid == 0) {
    // bond charges: q_0 = 0, q_{k+1} = q_k + m(pick) after an environment
    // site; the Bell bond carries q_k + (-1, 0, +1); back to q_k after the ancilla
    const int cap = c->chi_cap;
    int q = 0, ord = 0;
    c->qn[0] = 0;
    for (int k = 0; k < c->n_sites; ++k) {
      const int kind = c->site_kind[k];
      int16_t* next = c->qn + (size_t)(k + 1) * cap;
      if (kind == SITE_ENV) {
        q += 1 - c->env_out[ord++];
        next[0] = (int16_t)q;
      } else if (kind == SITE_CPHYS) {
        next[0] = (int16_t)(q - 1);
        next[1] = (int16_t)q;
        next[2] = (int16_t)(q + 1);
      } else {
        next[0] = (int16_t)q;
      }
    }
    c->counters[2] = c->counters[1];
    c->counters[3] = 0;
    c->counters[4] = 0;
  }
}

}  // namespace

static int check_launch() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

int launch_evolve_fp64(const BatchArg& b, const OutArg& o, void* stream) {
  if (b.n <= 0) return HM_OK;
  evolve_fp64_kernel<<<b.n, NT, 0, (cudaStream_t)stream>>>(b, o);
  return check_launch();
}

int launch_measure_fp64(const BatchArg& b, const OutArg& o, void* stream) {
  if (b.n <= 0) return HM_OK;
  measure_fp64_kernel<<<b.n, NT, 0, (cudaStream_t)stream>>>(b, o);
  return check_launch();
}

int launch_susceptibility_fp64(const BatchArg& b, const OutArg& o, void* stream) {
  if (b.n <= 0) return HM_OK;
  susceptibility_fp64_kernel<<<b.n, NT, 0, (cudaStream_t)stream>>>(b, o);
  return check_launch();
}

int launch_collapse_fp64(const BatchArg& b, const OutArg& o, void* stream) {
  if (b.n <= 0) return HM_OK;
  collapse_fp64_kernel<<<b.n, NT, 0, (cudaStream_t)stream>>>(b, o);
  const int rc = check_launch();
  if (rc != HM_OK) return rc;
  reset_kernel<<<b.n, NT, 0, (cudaStream_t)stream>>>(b, o, 0);
  return check_launch();
}

int launch_reset(const BatchArg& b, const OutArg& o, int draw_initial, void* stream) {
  if (b.n <= 0) return HM_OK;
  reset_kernel<<<b.n, NT, 0, (cudaStream_t)stream>>>(b, o, draw_initial);
  return check_launch();
}

}  // namespace hm

// ---------------------------------------------------------------------------
// Allocation-free two-site update (hm_two_site_update_static).
//
// For callers that cannot allocate device memory: code running inside
// another library's memory pool, in a process whose allocator is owned by
// someone else, or on a path that must not allocate while it runs.  The scratch of the
// update (chain descriptor, site slots, theta, Jacobi matrices, singular
// values) lives in one file-scope device array of fixed size; every GPU that
// loads this library holds it until the process exits.  All calls share the
// array, so two calls whose kernels overlap on the GPU race on it.
// ---------------------------------------------------------------------------

namespace hm {
namespace {

constexpr int kStaticChi = 128;                                       // largest chi_l, chi_m, chi_r
constexpr int64_t kStaticSlot = (int64_t)kStaticChi * 3 * kStaticChi;  // one site tensor
constexpr int64_t kStaticWs = (int64_t)(3 * kStaticChi) * (3 * kStaticChi);
constexpr int kStaticSv = 3 * kStaticChi;
constexpr int64_t kStaticDoubles = 64 + 2 * kStaticSlot + 3 * kStaticWs + 2 * kStaticSv;

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];
static_assert(sizeof(ChainDev) + 2 * sizeof(double*) + 6 * sizeof(int32_t) <= 48 * sizeof(double),
              "descriptor and meta data must fit below the statistics slots");

__global__ void __launch_bounds__(NT)
two_site_static_kernel(double* scratch, const double* A, const double* B, int chi_l, int chi_m, int chi_r,
                       const double* gate, int chi_max, double cutoff, int absorb, double* A_out,
                       double* B_out, int32_t* k_out) {
  __shared__ Shared sh;
  ChainDev* c = reinterpret_cast<ChainDev*>(scratch);
  char* meta = reinterpret_cast<char*>(scratch) + sizeof(ChainDev);   // 64 doubles hold struct + meta
  double** sites = reinterpret_cast<double**>(meta);
  int32_t* chi = reinterpret_cast<int32_t*>(meta + 2 * sizeof(double*));
  int32_t* status = chi + 4;
  double* stats = scratch + 48;
  double* slotA = scratch + 64;
  double* slotB = slotA + kStaticSlot;
  double* ws = slotB + kStaticSlot;
  if (threadIdx.x == 0) {
    // everything that must start at zero is cleared here, every call
    ChainDev d = {};
    d.n_sites = 2;
    d.n_gates = 1;
    d.chi_max = chi_max;
    d.cutoff = cutoff;
    d.gates = gate;
    d.site = sites;
    d.chi = chi;
    d.stats = stats;
    d.status = status;
    d.err_where = status + 1;
    d.theta = ws;
    d.W = ws + kStaticWs;
    d.V = ws + 2 * kStaticWs;
    d.sig = ws + 3 * kStaticWs;
    d.perm = reinterpret_cast<int32_t*>(ws + 3 * kStaticWs + kStaticSv);
    d.ws_cap = kStaticWs;
    d.sv_cap = kStaticSv;
    d.chi_cap = kStaticChi;
    *c = d;
    sites[0] = slotA;
    sites[1] = slotB;
    chi[0] = chi_l;
    chi[1] = chi_m;
    chi[2] = chi_r;
    status[0] = status[1] = 0;
    for (int i = 0; i < ST_N; ++i) stats[i] = 0.0;
  }
  for (int e = threadIdx.x; e < chi_l * 3 * chi_m; e += NT) slotA[e] = A[e];
  for (int e = threadIdx.x; e < chi_m * 3 * chi_r; e += NT) slotB[e] = B[e];
  __syncthreads();
  const OpDev op = {0, 0, absorb, 0};
  two_site_op(c, op, 0, sh, nullptr);
  __syncthreads();
  const int code = *(volatile int32_t*)status;
  const int kk = chi[1];
  if (code != 0) {
    if (threadIdx.x == 0) *k_out = code;
    return;
  }
  for (int e = threadIdx.x; e < chi_l * 3 * kk; e += NT) A_out[e] = slotA[e];
  for (int e = threadIdx.x; e < kk * 3 * chi_r; e += NT) B_out[e] = slotB[e];
  if (threadIdx.x == 0) *k_out = kk;
}

}  // namespace

}  // namespace hm

#include <mutex>

namespace {

std::mutex g_static_mu;
double* g_static_ptr[64] = {};   // device address of g_static_scratch, per device

}  // namespace

extern "C" int hm_two_site_update_static(const double* A_dev, const double* B_dev, int32_t chi_l, int32_t chi_m,
                                         int32_t chi_r, const double* gate_dev, int32_t chi_max, double cutoff,
                                         int32_t absorb, double* A_out_dev, double* B_out_dev,
                                         int32_t* k_out_dev, void* cuda_stream) {
  using namespace hm;
  if (!A_dev || !B_dev || !gate_dev || !A_out_dev || !B_out_dev || !k_out_dev) {
    set_global_error("hm_two_site_update_static: null pointer argument");
    return HM_ERR_ARG;
  }
  if (chi_l < 1 || chi_m < 1 || chi_r < 1 || chi_max < 1 || chi_l > kStaticChi || chi_m > kStaticChi ||
      chi_r > kStaticChi || chi_max > kStaticChi) {
    set_global_error("hm_two_site_update_static: chi_l, chi_m, chi_r and chi_max must lie in [1, 128] "
                     "(the size of its fixed scratch array)");
    return HM_ERR_ARG;
  }
  if ((absorb != 0 && absorb != 1) || !(cutoff >= 0.0) || !(cutoff < 1.0)) {
    set_global_error("hm_two_site_update_static: absorb must be 0 or 1 and cutoff in [0, 1)");
    return HM_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    set_global_error("hm_two_site_update_static: no current CUDA device");
    return HM_ERR_CUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
      // one-time set-up on this device (the device is current here): the
      // host-side symbol is only a stand-in, the kernel needs the device address
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
        set_global_error("hm_two_site_update_static: cudaGetSymbolAddress of the scratch array failed");
        return HM_ERR_CUDA;
      }
      g_static_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_static_ptr[dev];
  }
  two_site_static_kernel<<<1, NT, 0, (cudaStream_t)cuda_stream>>>(scratch, A_dev, B_dev, chi_l, chi_m, chi_r,
                                                                  gate_dev, chi_max, cutoff, absorb, A_out_dev,
                                                                  B_out_dev, k_out_dev);
  if (cudaGetLastError() != cudaSuccess) {
    set_global_error("hm_two_site_update_static: kernel launch failed");
    return HM_ERR_CUDA;
  }
  return HM_OK;
}
