// Charge blocks of the two-site update, shared by the binary64 evolve
// (hm_fp64.cu) and the mixed-precision evolve (hm_mixed.cu).
//
// Sec. II.C ("Exploiting Conserved Quantum Numbers"): the gates exp(-tau J
// S_i.S_j) conserve S^z_i + S^z_j, and an initial state |i>_E |B>_C whose
// environment is a product of S^z eigenstates has a definite total S^z.  So
// every bond index carries a charge q, every position's leg a sign sigma
// (+1 for a spin, -1 for an ancilla: its Bell partner carries the opposite
// S^z, which makes each Bell pair neutral), and A[l, s, r] = 0 unless
// q(l) + sigma m(s) = q(r), with m = +1, 0, -1 for s = 0, 1, 2.  A SWAP
// moves a site's content, and with it its sign, to the other position.
//
// After the gate, the two-site tensor theta[(l a), (b r)] is block diagonal
// in the charge Q of the new middle bond: rows with q(l) + sigma_k m(a) = Q
// against columns with q(r) - sigma_{k+1} m(b) = Q.  Each block is decomposed
// on its own.  The singular values of theta are the union of the blocks'
// values, so the truncation rule (Sec. II) runs on that union and keeps the
// set a dense SVD keeps; each kept value's block labels its new bond index.
//
// Bond indices stay grouped by charge in ascending order, so one charge is
// one contiguous run of a bond, and a block's rows (and columns) are three
// runs, one per local state.  A chain in dense mode (every charge and sign 0)
// has a single block: the unblocked split.
//
// Entries outside the blocks are never computed: the block GEMMs write only
// entries whose row and column charges agree, the gate is applied only
// within its conserved sectors, and the absorb writes explicit zeros.  So the
// structure holds exactly, in any precision.
#pragma once

#include <cstdint>

#include "hm_internal.h"

namespace hm {
namespace blk {

constexpr int kWin = 512;                 // charges one split may span (window)
constexpr int kMaxBlocks = kWin;

// m(s) of the local basis s = 0, 1, 2 (m = +1, 0, -1).
__device__ __forceinline__ int mval(int s) { return 1 - s; }

// One output block of a split.
struct BlockRec {
  int32_t Q, mq, nq, trans;               // charge, rows (l a), columns (b r), W holds the transpose
  int32_t q, p, svoff, pad;               // W is q x p column-major, q >= p; first slot in the value list
  int32_t rst[3], rlen[3], roff[3];       // per a: first l, count, offset in the row list
  int32_t cst[3], clen[3], coff[3];       // per b: first r, count, offset in the column list
  int64_t woff, voff;                     // offsets (elements) of the block's W and V
};

// Split metadata in the chain's meta workspace.
struct Meta {
  int32_t tab[3][kWin][2];                // (start, length) of each charge's run: left, middle, right bond
  int32_t qin[kWin];                      // middle charges with rows and columns (theta blocks)
  BlockRec b[kMaxBlocks];
};

static_assert(sizeof(Meta) <= kMetaBytes, "meta workspace of a chain");

// Shared scalars of a split (CTA shared memory).
struct SplitSh {
  int32_t sk, sk1, osk, osk1;             // input and output leg signs of sites k, k+1
  int32_t qbase, qtop, nin, nblk, ok;
  int32_t mask[9];                        // per output (a b): input (s1 s2) of its conserved sector
  int32_t kk;
  double nrm;
  double G[81];
};

struct Seg {
  int32_t start, len;
};

__device__ __forceinline__ Seg seg_of(const Meta* M, int bond, int qbase, int q) {
  const int i = q - qbase;
  if (i < 0 || i >= kWin) return {0, 0};   // callers stay within [qbase, qtop + 3]
  return {M->tab[bond][i][0], M->tab[bond][i][1]};
}

// Marks a chain as having no usable charge structure from here on: every
// charge and sign 0 (one block per split).  Sec. II.C's blocking is an
// optimisation; the dense split computes the same decomposition.
template <int NT>
__device__ void go_dense(ChainDev* c) {
  const int nb = (c->n_sites + 1) * c->chi_cap;
  for (int e = threadIdx.x; e < nb; e += NT) c->qn[e] = 0;
  for (int e = threadIdx.x; e < c->n_sites; e += NT) c->sgn[e] = 0;
  if (threadIdx.x == 0) c->counters[3] = 1;
  __syncthreads();
}

// Phase A: signs, charge-run tables of the three bonds, the middle charges
// of the theta blocks and the output blocks with their workspace offsets.
// Returns false if the chain had to switch to dense mode first (then call again).
template <int NT>
__device__ bool prepare(ChainDev* c, const OpDev& op, SplitSh& s) {
  const int tid = threadIdx.x;
  const int k = op.k;
  const int chil = c->chi[k], chim = c->chi[k + 1], chir = c->chi[k + 2];
  const int16_t* qL = c->qn + (size_t)k * c->chi_cap;
  const int16_t* qM = qL + c->chi_cap;
  const int16_t* qR = qM + c->chi_cap;
  Meta* M = reinterpret_cast<Meta*>(c->meta);
  const int info = c->gate_info[op.gate];
  __shared__ int lo_sh, hi_sh, bad_sh;
  if (tid == 0) {
    lo_sh = 1 << 30;
    hi_sh = -(1 << 30);
    bad_sh = 0;
    const int a = c->sgn[k], b = c->sgn[k + 1];
    s.ok = 1;
    // a gate that is not a permutation conserves m1 + m2 only: on legs of
    // unequal sign (a spin next to an ancilla) it breaks the charge rule
    if ((info & 2) && a != b) s.ok = 0;
    s.sk = a;
    s.sk1 = b;
    s.osk = (info & 1) ? b : a;
    s.osk1 = (info & 1) ? a : b;
  }
  __syncthreads();
  {
    // charge range of the three bonds; each charge must be one run, ascending
    int lo = 1 << 30, hi = -(1 << 30), bad = 0;
    const int nall = chil + chim + chir;
    for (int e = tid; e < nall; e += NT) {
      int i;
      const int16_t* q;
      if (e < chil) i = e, q = qL;
      else if (e < chil + chim) i = e - chil, q = qM;
      else i = e - chil - chim, q = qR;
      lo = min(lo, (int)q[i]);
      hi = max(hi, (int)q[i]);
      if (i > 0 && q[i] < q[i - 1]) bad = 1;
    }
    if (lo <= hi) {
      atomicMin(&lo_sh, lo);
      atomicMax(&hi_sh, hi);
    }
    if (bad) atomicMax(&bad_sh, 1);
  }
  __syncthreads();
  if (tid == 0) {
    s.qbase = lo_sh - 3;
    s.qtop = hi_sh;
    if (hi_sh - lo_sh + 7 > kWin || bad_sh) s.ok = 0;
  }
  __syncthreads();
  if (!s.ok) {
    __syncthreads();
    if (c->counters[3]) return true;      // already dense: every charge is 0, cannot fail again
    go_dense<NT>(c);
    return false;
  }
  const int qb = s.qbase;
  const int span = s.qtop - qb + 4;        // window entries any lookup of this split reaches
  for (int e = tid; e < 3 * span; e += NT) {
    M->tab[e / span][e % span][0] = 0;
    M->tab[e / span][e % span][1] = 0;
  }
  __syncthreads();
  const int nall = chil + chim + chir;
  for (int e = tid; e < nall; e += NT) {
    int bond, i, n;
    const int16_t* q;
    if (e < chil) bond = 0, i = e, n = chil, q = qL;
    else if (e < chil + chim) bond = 1, i = e - chil, n = chim, q = qM;
    else bond = 2, i = e - chil - chim, n = chir, q = qR;
    if (i == 0 || q[i] != q[i - 1]) {
      int j = i + 1;
      while (j < n && q[j] == q[i]) ++j;
      M->tab[bond][q[i] - qb][0] = i;
      M->tab[bond][q[i] - qb][1] = j - i;
    }
  }
  for (int e = tid; e < 81; e += NT) s.G[e] = c->gates[(size_t)op.gate * 81 + e];
  __syncthreads();
  if (tid < 9) {
    const int a = tid / 3, b = tid % 3;
    int msk = 0;
    for (int u = 0; u < 9; ++u) {
      const int s1 = u / 3, s2 = u % 3;
      if (s.sk * mval(s1) + s.sk1 * mval(s2) == s.osk * mval(a) + s.osk1 * mval(b) && s.G[(3 * a + b) * 9 + u] != 0.0)
        msk |= 1 << u;
    }
    s.mask[tid] = msk;
  }
  if (tid == 0) {
    int nin = 0, nblk = 0;
    int64_t woff = 0, voff = 0;
    int svoff = 0;
    // candidate charges: [lowest - 2, highest + 2] of the three bonds
    for (int i = 1; i <= s.qtop - qb + 2; ++i) {
      const int Q = qb + i;
      // theta block of middle charge Q: rows (l s1) and columns (s2 r) exist
      int rows = 0, cols = 0;
      for (int t = 0; t < 3; ++t) {
        rows += seg_of(M, 0, qb, Q - s.sk * mval(t)).len;
        cols += seg_of(M, 2, qb, Q + s.sk1 * mval(t)).len;
      }
      if (rows > 0 && cols > 0) M->qin[nin++] = Q;
      // output block of new middle charge Q
      BlockRec r;
      int mq = 0, nq = 0;
      for (int t = 0; t < 3; ++t) {
        const Seg a = seg_of(M, 0, qb, Q - s.osk * mval(t));
        const Seg b = seg_of(M, 2, qb, Q + s.osk1 * mval(t));
        r.rst[t] = a.start, r.rlen[t] = a.len, r.roff[t] = mq;
        r.cst[t] = b.start, r.clen[t] = b.len, r.coff[t] = nq;
        mq += a.len;
        nq += b.len;
      }
      if (mq == 0 || nq == 0) continue;
      r.Q = Q;
      r.mq = mq;
      r.nq = nq;
      r.trans = nq > mq;
      r.q = r.trans ? nq : mq;
      r.p = r.trans ? mq : nq;
      r.svoff = svoff;
      r.pad = 0;
      r.woff = woff;
      r.voff = voff;
      woff += (int64_t)r.q * r.p;
      voff += (int64_t)r.p * r.p;
      svoff += r.p;
      M->b[nblk++] = r;
    }
    s.nin = nin;
    s.nblk = nblk;
  }
  __syncthreads();
  return true;
}

// Phase B: theta[(l s1), (s2 r)] = sum_m A_k[(l s1), m] A_{k+1}[m, (s2 r)] for
// every entry whose row charge q(l) + sigma_k m(s1) and column charge
// q(r) - sigma_{k+1} m(s2) agree (Sec. I.A two-site tensor), one GEMM per
// middle charge over that charge's run of the middle bond.  Entries of a
// charge absent from the middle bond are written as 0.  A, B are binary64
// site tensors; T is the accumulation and storage type of theta.
template <int NT, int TM, int TN, int TK, typename T>
__device__ void theta_blocks(const ChainDev* c, int k, const SplitSh& s, T* __restrict__ theta, T* smem) {
  const int tid = threadIdx.x;
  const int chim = c->chi[k + 1], chir = c->chi[k + 2];
  const int n = 3 * chir;
  const double* __restrict__ A = c->site[k];
  const double* __restrict__ B = c->site[k + 1];
  const Meta* M = reinterpret_cast<const Meta*>(c->meta);
  // thread tile: rows ty + TY a (a < RA), columns tx + TX b (b < 4)
  constexpr int RB = 4, TX = TN / RB, TY = NT / TX, RA = TM / TY;
  static_assert(TN % RB == 0 && NT % TX == 0 && TM % TY == 0, "tile must split evenly over the CTA");
  const int tx = tid % TX, ty = tid / TX;
  T* sa = smem;                            // [TK][TM + 1]
  T* sb = smem + TK * (TM + 1);            // [TK][TN + 1]
  for (int bi = 0; bi < s.nin; ++bi) {
    const int Q = M->qin[bi];
    int rst[3], roff[4], cst[3], coff[4];
    roff[0] = coff[0] = 0;
    for (int t = 0; t < 3; ++t) {
      const Seg a = seg_of(M, 0, s.qbase, Q - s.sk * mval(t));
      const Seg b = seg_of(M, 2, s.qbase, Q + s.sk1 * mval(t));
      rst[t] = a.start;
      roff[t + 1] = roff[t] + a.len;
      cst[t] = b.start;
      coff[t + 1] = coff[t] + b.len;
    }
    const Seg mid = seg_of(M, 1, s.qbase, Q);
    const int Mv = roff[3], Nv = coff[3], K = mid.len;
    for (int i0 = 0; i0 < Mv; i0 += TM) {
      for (int j0 = 0; j0 < Nv; j0 += TN) {
        T acc[RA][RB];
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
          for (int b = 0; b < RB; ++b) acc[a][b] = T(0);
        for (int k0 = 0; k0 < K; k0 += TK) {
          for (int e = tid; e < TM * TK; e += NT) {
            const int ii = e / TK, kk = e % TK;
            const int v = i0 + ii, g = k0 + kk;
            T x = T(0);
            if (v < Mv && g < K) {
              const int t = v >= roff[2] ? 2 : (v >= roff[1] ? 1 : 0);
              const int l = rst[t] + v - roff[t];
              x = (T)A[(size_t)(3 * l + t) * chim + mid.start + g];
            }
            sa[kk * (TM + 1) + ii] = x;
          }
          for (int e = tid; e < TN * TK; e += NT) {
            const int jj = e % TN, kk = e / TN;
            const int u = j0 + jj, g = k0 + kk;
            T x = T(0);
            if (u < Nv && g < K) {
              const int t = u >= coff[2] ? 2 : (u >= coff[1] ? 1 : 0);
              const int r = cst[t] + u - coff[t];
              x = (T)B[(size_t)(mid.start + g) * n + t * chir + r];
            }
            sb[kk * (TN + 1) + jj] = x;
          }
          __syncthreads();
#pragma unroll 4
          for (int kk = 0; kk < TK; ++kk) {
            T bv[RB];
#pragma unroll
            for (int b = 0; b < RB; ++b) bv[b] = sb[kk * (TN + 1) + tx + TX * b];
#pragma unroll
            for (int a = 0; a < RA; ++a) {
              const T av = sa[kk * (TM + 1) + ty + TY * a];
#pragma unroll
              for (int b = 0; b < RB; ++b) acc[a][b] = fma(av, bv[b], acc[a][b]);
            }
          }
          __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < RA; ++a) {
          const int v = i0 + ty + TY * a;
          if (v >= Mv) continue;
          const int t = v >= roff[2] ? 2 : (v >= roff[1] ? 1 : 0);
          const int row = 3 * (rst[t] + v - roff[t]) + t;
#pragma unroll
          for (int b = 0; b < RB; ++b) {
            const int u = j0 + tx + TX * b;
            if (u >= Nv) continue;
            const int tt = u >= coff[2] ? 2 : (u >= coff[1] ? 1 : 0);
            theta[(size_t)row * n + tt * chir + cst[tt] + u - coff[tt]] = acc[a][b];
          }
        }
      }
    }
  }
  __syncthreads();
}

// Phase C input: block b of theta after the gate (Sec. I.A: the gate acts on
// the physical legs only), written column-major into W (q x p, leading
// dimension ldw; the transpose when the block is wider than tall).  V = I.
template <int NT, typename TT, typename TW>
__device__ void gather_block(const ChainDev* c, int k, const SplitSh& s, const BlockRec& r,
                             const TT* __restrict__ theta, TW* __restrict__ W, int ldw, TW* __restrict__ V, int ldv) {
  const int chir = c->chi[k + 2];
  const int n = 3 * chir;
  const int total = r.mq * r.nq;
  for (int e = threadIdx.x; e < total; e += NT) {
    const int v = e / r.nq, u = e % r.nq;              // u fastest: r runs contiguously in theta
    const int a = v >= r.roff[2] ? 2 : (v >= r.roff[1] ? 1 : 0);
    const int b = u >= r.coff[2] ? 2 : (u >= r.coff[1] ? 1 : 0);
    const int l = r.rst[a] + v - r.roff[a];
    const int rr = r.cst[b] + u - r.coff[b];
    const int msk = s.mask[3 * a + b];
    TT x = TT(0), y = TT(0);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      if (msk & (1 << t)) {
        const int s1 = t / 3, s2 = t % 3;
        const TT th = theta[(size_t)(3 * l + s1) * n + s2 * chir + rr];
        const double g = s.G[(3 * a + b) * 9 + t];
        const TT ghi = (TT)g;
        x = fma(ghi, th, x);
        // a binary32 theta takes each coefficient as a binary32 pair
        // (hi + lo): rounding the gate itself would repeat the same relative
        // error at every application of that gate and add up coherently over
        // the evolution, while the rounding of the products does not
        if (sizeof(TT) < sizeof(double)) y = fma((TT)(g - (double)ghi), th, y);
      }
    }
    if (r.trans) W[(size_t)v * ldw + u] = (TW)(x + y);
    else W[(size_t)u * ldw + v] = (TW)(x + y);
  }
  for (int e = threadIdx.x; e < r.p * r.p; e += NT) {
    const int j = e / r.p, i = e % r.p;
    V[(size_t)j * ldv + i] = (i == j) ? TW(1) : TW(0);
  }
}

// Barrier of the nthreads threads (a multiple of 32) of a warp group; ids
// 1..15 (0 is __syncthreads).  HM_HOST_EMULATION: the kernels compiled as
// host C++ by the CPU emulation of the tests.
__device__ __forceinline__ void group_sync(int id, int nthreads) {
#if defined(__CUDA_ARCH__)
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
#elif defined(HM_HOST_EMULATION)
  simt::named_sync(id, nthreads);
#endif
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Tangent t of the Jacobi rotation that makes columns with Gram entries
// (a, g; g, b) orthogonal: t = sign(z) / (|z| + sqrt(1 + z^2)),
// z = (b - a) / (2 g) = d / (2 g).  It sits on the critical path of every
// pass, so it takes the short-latency binary32 forms (approximate divide and
// reciprocal square root, a few ulp): a rotation is exactly conformal
// whatever its angle, the stretch c^2 + s^2 - 1 is removed with the column
// scales when W and V are promoted, and an angle that is off by 1e-7
// relative leaves an off-diagonal 1e-7 times the one it removed, which the
// next sweep takes.  The binary64 kernels need it cheaply too:
// GB300 has few binary64 units, and a binary64 square root or divide is a
// sequence of them.  The rotation (c, s) = (1, t) / sqrt(1 + t^2) is
// orthogonal to binary64 rounding whatever t is, so t only has to be close:
// z is formed in binary32 from d and g scaled by the same power of two (z
// does not change; bits_to_float, integer instructions only), which leaves
// an off-diagonal of relative size ~1e-7 times the one it removes, for the
// next sweep.  Operands too far apart for binary32 take the binary64 formula.
// Squared column norm below which the binary32 sweeps leave a column alone:
// a normal number whose square root (1e-15) is far below binary32
// resolution against columns of order one.  With both norms above it, a
// rotated pair's |g| > tol sqrt(a b) > 1e-37 is normal too.
constexpr float kTiny32 = 1e-30f;

__device__ __forceinline__ float jacobi_tangent32(float d, float g) {
  const float z = __fdividef(d, 2.0f * g);
  if (fabsf(z) > 1e18f) return __fdividef(0.5f, z);
  const float w = 1.0f + z * z;
  return copysignf(__fdividef(1.0f, fabsf(z) + w * rsqrtf(w)), z);
}

// Biased binary64 exponent of x (0 for zero and subnormals).
__device__ __forceinline__ int bexp64(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

// x * 2^(1023 - e) as a binary32 number, built from the bits of x by integer
// instructions (no binary64 or conversion instruction): the top 23 bits of
// the mantissa, truncated (relative error < 2^-23).  0 when x is zero,
// subnormal, or 2^126 or more below 2^(e - 1023).  e >= the exponent of x.
__device__ __forceinline__ float bits_to_float(double x, int e) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int ex = (int)((hi >> 20) & 0x7ffu);
  const int ef = ex - e + 127;
  if (ex == 0 || ef <= 0) return 0.0f;
  return __uint_as_float((hi & 0x80000000u) | ((unsigned)ef << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

__device__ __forceinline__ double jacobi_tangent64(double d, double g) {
  const int e = max(bexp64(d), bexp64(g));
  const float gf = bits_to_float(g, e);
  if (fabsf(gf) >= 1e-30f) return (double)jacobi_tangent32(bits_to_float(d, e), gf);
  const double z = d / (2.0 * g);
  return fabs(z) > 1e150 ? 0.5 / z : copysign(1.0, z) / (fabs(z) + sqrt(1.0 + z * z));
}

// Per-group convergence words of a grouped Jacobi (shared memory).
struct GroupSh {
  int32_t flag[16];
  uint32_t rbits[16];                     // largest rotation ratio of the sweep, binary32 bits
};

// One pass: the L lanes of this lane's pair (a, b) (a < 0: no pair) take the
// dot product of the two columns, the rotation angle and the rotation of W
// and V, then the pair's first lane stores the two new norms.  Every lane of
// the warp takes part (the reductions are warp shuffles).  A lane moves its
// rows in batches of B, every load of a batch issued before the first store
// (a store to one column could alias the next load of the other, so the
// compiler keeps them in program order), and its first batch stays in
// registers from the dot product to the rotation: a pass waits on one memory
// latency per batch, not one per row.  Binary64 (T = double): the rotation
// tests and the tangent take binary32 values built from the operands' bits,
// so that a pass spends its binary64 instructions on the rotation itself
// (GB300 runs binary64 at about 1/64 of the binary32 rate).  rmax: largest
// ratio |g| / sqrt(a b) seen (binary64: 1 once some ratio reached `stop`);
// rot: set when a rotation was applied.
template <typename T, typename TV, int L, int B>
__device__ __forceinline__ void jacobi_pass(T* __restrict__ W, int q, int ldw, int p, TV* __restrict__ V, int ldv,
                                            T* __restrict__ nrm, int a, int b, int sl, T tol, T stop, T& rmax,
                                            int& rot) {
  constexpr bool SC = sizeof(T) == sizeof(double);   // binary64 form of the angle
          T* x = W + (size_t)(a < 0 ? 0 : a) * ldw;
          T* y = W + (size_t)(b < 0 ? 0 : b) * ldw;
          // rows sl + u L (u < B) of both columns stay in registers from the
          // dot product to the rotation; further rows go in batches of B whose
          // loads are all issued before any use (one memory latency a batch)
          T x0[B], y0[B], gacc[B];
  #pragma unroll
          for (int u = 0; u < B; ++u) {
            const int i = sl + u * L;
            const bool in = a >= 0 && i < q;
            x0[u] = in ? x[i] : T(0);
            y0[u] = in ? y[i] : T(0);
          }
  #pragma unroll
          for (int u = 0; u < B; ++u) gacc[u] = x0[u] * y0[u];
          if (a >= 0) {
            for (int i0 = sl + B * L; i0 < q; i0 += B * L) {
              T xr[B], yr[B];
  #pragma unroll
              for (int u = 0; u < B; ++u) {
                const int i = i0 + u * L;
                xr[u] = i < q ? x[i] : T(0);
                yr[u] = i < q ? y[i] : T(0);
              }
  #pragma unroll
              for (int u = 0; u < B; ++u) gacc[u] = fma(xr[u], yr[u], gacc[u]);
            }
          }
          T ga = gacc[0];
  #pragma unroll
          for (int u = 1; u < B; ++u) ga += gacc[u];
  #pragma unroll
          for (int o = L / 2; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
          bool done = false;
          T na = T(0), nb = T(0);
          if (a >= 0) {
            const T al = nrm[a], be = nrm[b];
            bool go;
            T ratio = T(0);
            float rf = 0.0f;
            if constexpr (SC) {
              // |g| / sqrt(a b) in binary32 from the operands' bits (integer
              // pipe), each scaled by its own power of two: a, b in [1, 2), g
              // by the mean exponent, so the ratio holds over the whole
              // binary64 range and no pair is skipped for its columns' sizes
              const int ea = bexp64(al), eb = bexp64(be);
              const float af = bits_to_float(al, ea), bf = bits_to_float(be, eb);
              rf = fabsf(bits_to_float(ga, (ea + eb) >> 1)) * rsqrtf(fmax(af * bf, 1.0f));
              if ((ea + eb) & 1) rf *= 0.70710678f;
              go = ga != T(0) && af > 0.0f && bf > 0.0f && rf > (float)tol;
            } else {
              // columns below kTiny32 are noise at binary32 resolution, and
              // the fast reciprocal square root flushes subnormal inputs to 0
              ratio = fabs(ga) * (rsqrtf(fmax(al, kTiny32)) * rsqrtf(fmax(be, kTiny32)));
              go = ga != T(0) && al > kTiny32 && be > kTiny32 && ratio > tol;
            }
            if (go) {
              T t, cs;
              if constexpr (SC) {
                // binary64 pipe: b - a, 1 + t^2, one rsqrt, s = c t
                if (rf >= (float)stop) rmax = T(1);
                t = jacobi_tangent64(be - al, ga);
                cs = rsqrt(T(1) + t * t);
              } else {
                rmax = fmax(rmax, ratio);
                t = jacobi_tangent32(be - al, ga);
                cs = rsqrtf(T(1) + t * t);
              }
              const T sn = cs * t;
  #pragma unroll
              for (int u = 0; u < B; ++u) {
                const int i = sl + u * L;
                if (i < q) {
                  x[i] = cs * x0[u] - sn * y0[u];
                  y[i] = sn * x0[u] + cs * y0[u];
                }
              }
              for (int i0 = sl + B * L; i0 < q; i0 += B * L) {
                T xr[B], yr[B];
  #pragma unroll
                for (int u = 0; u < B; ++u) {
                  const int i = i0 + u * L;
                  xr[u] = i < q ? x[i] : T(0);
                  yr[u] = i < q ? y[i] : T(0);
                }
  #pragma unroll
                for (int u = 0; u < B; ++u) {
                  const int i = i0 + u * L;
                  if (i < q) {
                    x[i] = cs * xr[u] - sn * yr[u];
                    y[i] = sn * xr[u] + cs * yr[u];
                  }
                }
              }
              TV* vx = V + (size_t)a * ldv;
              TV* vy = V + (size_t)b * ldv;
              const TV cv = (TV)cs, sv = (TV)sn;
              for (int i0 = sl; i0 < p; i0 += B * L) {
                TV xr[B], yr[B];
  #pragma unroll
                for (int u = 0; u < B; ++u) {
                  const int i = i0 + u * L;
                  xr[u] = i < p ? vx[i] : TV(0);
                  yr[u] = i < p ? vy[i] : TV(0);
                }
  #pragma unroll
                for (int u = 0; u < B; ++u) {
                  const int i = i0 + u * L;
                  if (i < p) {
                    vx[i] = cv * xr[u] - sv * yr[u];
                    vy[i] = sv * xr[u] + cv * yr[u];
                  }
                }
              }
              na = al - t * ga;
              nb = be + t * ga;
              done = true;
              rot = 1;
            }
          }
          __syncwarp();              // every lane of the pair has read the old norms
          if (done && sl == 0) {
            nrm[a] = na;
            nrm[b] = nb;
          }
}

// One-sided (Hestenes) Jacobi run by a group of nw warps (warp lw of the
// group, barrier id bar): W (q x p column-major, q >= p, leading dimension
// ldw), rotations accumulated into V (p x p, leading dimension ldv, holds the
// starting basis), column norms cached in nrm and recomputed at every sweep
// start.  Round-robin pairing: every round's pairs are disjoint.  L lanes
// work on one pair, so a warp rotates 32 / L pairs at once (more pairs in
// flight, shorter reductions; the rotations are latency-bound, not
// arithmetic-bound); each pair's work is one jacobi_pass.  Stops after a
// sweep with no rotation or whose largest ratio |g| / sqrt(a b) is below
// `stop` (the next sweep's off-diagonals are then of order stop^2).  Returns
// the sweeps, or -1 when max_sweeps ran out.
template <typename T, typename TV, int L, int B>
__device__ int jacobi_lanes(T* __restrict__ W, int q, int ldw, int p, TV* __restrict__ V, int ldv,
                            T* __restrict__ nrm, int lw, int nw, int bar, int g, GroupSh& gs, T stop, int max_sweeps) {
  constexpr int PPW = 32 / L;              // pairs per warp at once
  const int lane = threadIdx.x & 31;
  const int sub = lane / L, sl = lane % L;
  const int nthr = 32 * nw;
  const T eps = sizeof(T) == sizeof(double) ? T(2.220446049250313e-16) : T(1.1920928955078125e-07);
  const T tol = sqrt((T)q) * eps;
  const int p2 = p + (p & 1);
  const int npair = p2 / 2;
  for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
    for (int j = lw; j < p; j += nw) {
      const T* cj = W + (size_t)j * ldw;
      T s2 = T(0);
      for (int i = lane; i < q; i += 32) s2 = fma(cj[i], cj[i], s2);
      s2 = warp_sum_t(s2);
      if (lane == 0) nrm[j] = s2;
    }
    if (lw == 0 && lane == 0) {
      gs.flag[g] = 0;
      gs.rbits[g] = 0u;
    }
    group_sync(bar, nthr);
    T rmax = T(0);
    int rot = 0;
    for (int rd = 0; rd < p2 - 1; ++rd) {
      for (int base = lw * PPW; base < npair; base += nw * PPW) {   // warp-uniform
        const int pi = base + sub;
        int a = -1, b = -1;
        if (pi < npair) {
          const int m = p2 - 1;          // (rd +- pi) mod m, 0 <= rd < m, 0 < pi < m
          if (pi == 0) {
            a = rd;
            b = m;
          } else {
            a = rd + pi;
            if (a >= m) a -= m;
            b = rd - pi;
            if (b < 0) b += m;
          }
          if (a >= p || b >= p) a = b = -1;
        }
        jacobi_pass<T, TV, L, B>(W, q, ldw, p, V, ldv, nrm, a, b, sl, tol, stop, rmax, rot);
      }
      group_sync(bar, nthr);
    }
    // warp max of the ratios, then one atomic per warp
    float rm32 = (float)rmax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rm32 = fmaxf(rm32, __shfl_xor_sync(0xffffffffu, rm32, o));
    const int anyrot = __any_sync(0xffffffffu, rot);
    if (lane == 0) {
      if (anyrot) atomicMax(&gs.flag[g], 1);
      atomicMax(&gs.rbits[g], __float_as_uint(rm32));
    }
    group_sync(bar, nthr);
    const int any = gs.flag[g];
    const T rm = (T)__uint_as_float(gs.rbits[g]);
    group_sync(bar, nthr);
    if (!any || rm < stop) return sweep;
  }
  return -1;
}

// Block-ordered one-sided Jacobi for the binary32 sweeps.  The columns form
// super-columns of C = 4, and the round-robin tournament pairs the
// super-columns (ns2 - 1 super-rounds, ns2 = super-columns rounded up to
// even).  A warp owns the eight columns of its super-pair for a whole
// super-round.  It rotates every column of one super-column against every
// column of the other: four sub-rounds of four disjoint pairs, one pair per
// 8 lanes.  In the first super-round it also rotates the pairs inside both
// super-columns (three sub-rounds).  Only __syncwarp separates its
// sub-rounds.  A sweep still visits every pair once, as in jacobi_lanes,
// with the same passes per warp, but waits at ns2 - 1 group barriers
// instead of p - 1: the barrier, not the arithmetic, was what the sweeps
// waited on.  Same arguments, stopping rule and result as jacobi_lanes.
template <typename T, typename TV, int B>
__device__ int jacobi_blocks(T* __restrict__ W, int q, int ldw, int p, TV* __restrict__ V, int ldv,
                             T* __restrict__ nrm, int lw, int nw, int bar, int g, GroupSh& gs, T stop, int max_sweeps) {
  constexpr int L = 8, C = 4;              // 32 / L = C pairs per pass
  const int lane = threadIdx.x & 31;
  const int sub = lane / L, sl = lane % L;
  const int nthr = 32 * nw;
  const T eps = sizeof(T) == sizeof(double) ? T(2.220446049250313e-16) : T(1.1920928955078125e-07);
  const T tol = sqrt((T)q) * eps;
  const int ns = (p + C - 1) / C, ns2 = ns + (ns & 1), nsp = ns2 / 2;
  for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
    for (int j = lw; j < p; j += nw) {
      const T* cj = W + (size_t)j * ldw;
      T s2 = T(0);
      for (int i = lane; i < q; i += 32) s2 = fma(cj[i], cj[i], s2);
      s2 = warp_sum_t(s2);
      if (lane == 0) nrm[j] = s2;
    }
    if (lw == 0 && lane == 0) {
      gs.flag[g] = 0;
      gs.rbits[g] = 0u;
    }
    group_sync(bar, nthr);
    T rmax = T(0);
    int rot = 0;
    for (int sr = 0; sr < ns2 - 1; ++sr) {
      for (int sp = lw; sp < nsp; sp += nw) {                       // warp-uniform
        const int m = ns2 - 1;             // (sr +- sp) mod m, as for the columns
        int A, Bc;
        if (sp == 0) {
          A = sr;
          Bc = m;
        } else {
          A = sr + sp;
          if (A >= m) A -= m;
          Bc = sr - sp;
          if (Bc < 0) Bc += m;
        }
        const bool okA = A < ns, okB = Bc < ns;                     // ns2 > ns: one padding super-column
        if (sr == 0) {
          // pairs inside A (lanes 0-15) and inside B (lanes 16-31): the
          // round robin of four columns, (k, 3) and ((k + 1) % 3, (k + 2) % 3)
          const int base = (sub < 2 ? A : Bc) * C;
          const bool ok = sub < 2 ? okA : okB;
          for (int k = 0; k < C - 1; ++k) {
            int a = base + ((sub & 1) == 0 ? k : (k + 1) % (C - 1));
            int b = base + ((sub & 1) == 0 ? C - 1 : (k + 2) % (C - 1));
            if (!ok || a >= p || b >= p) a = b = -1;
            jacobi_pass<T, TV, L, B>(W, q, ldw, p, V, ldv, nrm, a, b, sl, tol, stop, rmax, rot);
            __syncwarp();                  // the norms stored by the pass are read by other lanes next
          }
        }
        if (okA && okB) {
          for (int k = 0; k < C; ++k) {
            int a = A * C + sub, b = Bc * C + ((sub + k) & (C - 1));
            if (a >= p || b >= p) a = b = -1;
            jacobi_pass<T, TV, L, B>(W, q, ldw, p, V, ldv, nrm, a, b, sl, tol, stop, rmax, rot);
            __syncwarp();
          }
        }
      }
      group_sync(bar, nthr);
    }
    float rm32 = (float)rmax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rm32 = fmaxf(rm32, __shfl_xor_sync(0xffffffffu, rm32, o));
    const int anyrot = __any_sync(0xffffffffu, rot);
    if (lane == 0) {
      if (anyrot) atomicMax(&gs.flag[g], 1);
      atomicMax(&gs.rbits[g], __float_as_uint(rm32));
    }
    group_sync(bar, nthr);
    const int any = gs.flag[g];
    const T rm = (T)__uint_as_float(gs.rbits[g]);
    group_sync(bar, nthr);
    if (!any || rm < stop) return sweep;
  }
  return -1;
}

// Lanes per pair from a latency model of one round: ceil(pairs / slots)
// passes, each a fixed cost (reduction over log2 L lanes, the rotation
// angle) plus the per-lane element work (about 3 q / L loads and FMAs).
__device__ __forceinline__ int lanes_per_pair(int q, int p, int nw) {
  int best = 32;
  long long bt = -1;
  for (int L = 32; L >= 8; L >>= 1) {
    const int slots = nw * (32 / L);
    const int passes = ((p + 1) / 2 + slots - 1) / slots;
    const int lg = L == 32 ? 5 : (L == 16 ? 4 : 3);
    const long long tcost = (long long)passes * (150 + 25 * lg + 12 * ((q + L - 1) / L));
    if (bt < 0 || tcost < bt) bt = tcost, best = L;
  }
  return best;
}

// One-sided Jacobi of one block by a warp group: the block ordering
// (jacobi_blocks) for binary32 blocks of 16 columns or more, otherwise the
// round-robin ordering with L lanes per pair from the latency model.
// TV: element type of V.  A binary64 polish of a binary32 result may keep V
// in binary32: V carries binary32 accuracy from the preconditioning sweeps
// anyway, and the polish's rotations are tiny (angles ~1e-6).
// B: rows per lane and batch (register budget: 4 B values of T in flight).
// A lane's rows are rounded up to a multiple of B, and on the binary64 pipe
// every issued instruction costs the same whatever the lanes' predicates, so
// the binary64 kernels take B = 2.
template <typename T, typename TV = T, int B = 4>
__device__ int jacobi_group(T* __restrict__ W, int q, int ldw, int p, TV* __restrict__ V, int ldv,
                            T* __restrict__ nrm, int lw, int nw, int bar, int g, GroupSh& gs, T stop, int max_sweeps) {
  if constexpr (sizeof(T) == sizeof(float)) {
    if (p >= 16) return jacobi_blocks<T, TV, B>(W, q, ldw, p, V, ldv, nrm, lw, nw, bar, g, gs, stop, max_sweeps);
  }
  const int L = lanes_per_pair(q, p, nw);
  if (L == 8) return jacobi_lanes<T, TV, 8, B>(W, q, ldw, p, V, ldv, nrm, lw, nw, bar, g, gs, stop, max_sweeps);
  if (L == 16) return jacobi_lanes<T, TV, 16, B>(W, q, ldw, p, V, ldv, nrm, lw, nw, bar, g, gs, stop, max_sweeps);
  return jacobi_lanes<T, TV, 32, B>(W, q, ldw, p, V, ldv, nrm, lw, nw, bar, g, gs, stop, max_sweeps);
}

// Warp groups for one wave of charge blocks: every block gets at least one
// warp, then warps go one at a time to the block whose sweep takes longest
// ((p - 1) rounds of ceil(p / (2 w)) pairs per warp), never beyond p / 2.
// nblk <= 15 and nblk <= nwarps.  Writes the first warp and the warp count
// of every block.  One thread.
__device__ inline void assign_warps(const int* p, int nblk, int nwarps, int* w0, int* nw) {
  int used = 0;
  for (int b = 0; b < nblk; ++b) nw[b] = 1, ++used;
  while (used < nwarps) {
    int best = -1;
    long long bt = -1;
    for (int b = 0; b < nblk; ++b) {
      const int cap = (p[b] + 1) / 2;
      if (nw[b] >= cap) continue;
      const long long t = (long long)(p[b] - 1) * ((p[b] + 2 * nw[b] - 1) / (2 * nw[b]));
      if (t > bt) bt = t, best = b;
    }
    if (best < 0) break;
    ++nw[best];
    ++used;
  }
  int w = 0;
  for (int b = 0; b < nblk; ++b) w0[b] = w, w += nw[b];
}

// One wave of a split's charge blocks: blocks [b0, b0 + n) decomposed at
// once, block i by warps [w0[i], w0[i] + nw[i]) (barrier id i + 1).
struct WaveSh {
  int32_t b0, n;
  int32_t w0[15], nw[15], sw[15];
  int32_t off[15];                        // shared-memory offset (elements) of block i
};

// Index of this warp's group in the wave, or -1 (an idle warp).
__device__ __forceinline__ int my_group(const WaveSh& wv, int warp) {
  for (int i = 0; i < wv.n; ++i)
    if (warp >= wv.w0[i] && warp < wv.w0[i] + wv.nw[i]) return i;
  return -1;
}

__device__ __forceinline__ double warp_sum64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Truncation rule (Sec. II): smallest k >= 1 whose discarded weight
// sum_{q>=k} s_q^2 / sum s^2 <= cutoff, then min(k, chi_max), then lowered to
// the nearest gap s_k < s_{k-1} (1 - 1e-8).  s sorted descending; one thread.
__device__ inline int trunc_rank(const double* s, int n, int chi_max, double cutoff, double* tail, double* total_out) {
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

// Dense-SVD flop count 4 M^2 N + 8 M N^2 + 9 N^3 of an m x n matrix (M >= N).
__device__ __forceinline__ double svd_count(double m, double n) {
  const double M = m > n ? m : n, N = m > n ? n : m;
  return 4.0 * M * M * N + 8.0 * M * N * N + 9.0 * N * N * N;
}

// Phase D: singular values of every block (column norms of its converged W,
// binary64), one descending order over all blocks, the truncation rule,
// renormalisation, then the new bond grouped by charge (ascending; by value
// within a charge), the absorb into A_k and A_{k+1} (zeros outside the
// blocks) and the new middle charges.  W and V hold every block's binary64
// result; `scratch` (the theta buffer) holds 4 per-value arrays.
template <int NT>
__device__ void finish(ChainDev* c, const OpDev& op, int t, SplitSh& s, double* __restrict__ scratch,
                       int32_t* ctx_err, int sweeps32, int sweeps64) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nwarps = NT / 32;
  const int k = op.k;
  const int chil = c->chi[k], chim = c->chi[k + 1], chir = c->chi[k + 2];
  const int m = 3 * chil, n = 3 * chir;
  const Meta* M = reinterpret_cast<const Meta*>(c->meta);
  const int nb = s.nblk;
  const BlockRec& last = M->b[nb - 1];
  const int P = last.svoff + last.p;                  // values over all blocks
  double* sraw = scratch;                             // P: value of slot
  int32_t* sblk = reinterpret_cast<int32_t*>(scratch + P);   // P: block of slot
  double* tail = scratch + 2 * P;                     // P + 1
  int32_t* newslot = reinterpret_cast<int32_t*>(scratch + 3 * P + 1);   // kk: slot of new index
  // column norms -> raw values, slot = svoff + column
  for (int b = 0; b < nb; ++b) {
    const BlockRec& r = M->b[b];
    const double* Wb = c->W + r.woff;
    for (int j = warp; j < r.p; j += nwarps) {
      const double* cj = Wb + (size_t)j * r.q;
      double s2 = 0.0;
      for (int i = lane; i < r.q; i += 32) s2 = fma(cj[i], cj[i], s2);
      s2 = warp_sum64(s2);
      if (lane == 0) {
        sraw[r.svoff + j] = sqrt(s2);
        sblk[r.svoff + j] = b;
      }
    }
  }
  __syncthreads();
  // descending rank (ties by slot): sig[rank] = value, perm[rank] = slot
  for (int j = tid; j < P; j += NT) {
    const double sj = sraw[j];
    int rank = 0;
    for (int i = 0; i < P; ++i) {
      const double si = sraw[i];
      rank += (si > sj) || (si == sj && i < j);
    }
    c->sig[rank] = sj;
    c->perm[rank] = j;
  }
  __syncthreads();
  if (tid == 0) {
    const double* sv = c->sig;
    double total, nrm = 1.0;
    int kk;
    if (!op.exact) {
      kk = trunc_rank(sv, P, c->chi_max, c->cutoff, tail, &total);
      if (!(total > 0.0) || !isfinite(total)) kk = -1;
      else {
        double kept = 0.0;
        for (int i = 0; i < kk; ++i) kept += sv[i] * sv[i];
        nrm = 1.0 / sqrt(kept);
        c->stats[ST_DISC] += tail[kk] / total;
      }
    } else {
      kk = 0;
      while (kk < P && kk < chim && sv[kk] > 0.0) ++kk;
      if (kk == 0) kk = -1;
    }
    s.kk = kk;
    s.nrm = nrm;
    if (kk > 0) {
      double svd = 0.0;
      for (int b = 0; b < nb; ++b) svd += svd_count(M->b[b].mq, M->b[b].nq);
      c->stats[ST_SVD] += svd;
      c->stats[ST_SVD_DENSE] += svd_count(m, n);
      c->stats[ST_SWEEPS] += sweeps32;
      c->stats[ST_SWEEPS64] += sweeps64;
      c->stats[ST_SPLITS] += 1.0;
      c->stats[ST_BLOCKS] += nb;
      if (kk > c->stats[ST_MAXCHI]) c->stats[ST_MAXCHI] = kk;
    }
  }
  __syncthreads();
  const int kk = s.kk;
  const double nrm = s.nrm;
  if (kk <= 0) {
    if (tid == 0) {
      if (atomicCAS(c->status, 0, HM_ERR_NUMERIC) == 0) *c->err_where = t;
      if (ctx_err) atomicCAS(ctx_err, 0, HM_ERR_NUMERIC);
    }
    return;
  }
  // new position of kept rank i: kept values of lower-charge blocks first,
  // then by rank within the block
  for (int i = tid; i < kk; i += NT) {
    const int slot = c->perm[i];
    const int b = sblk[slot];
    int pos = 0;
    for (int j = 0; j < kk; ++j) {
      const int bj = sblk[c->perm[j]];
      pos += (bj < b) || (bj == b && j < i);
    }
    newslot[pos] = slot;
  }
  __syncthreads();
  const bool absorb_left = op.absorb == 0;
  double* Ak = c->site[k];
  double* Ak1 = c->site[k + 1];
  // A_k[(l a), i]
  for (int e = tid; e < m * kk; e += NT) {
    const int row = e / kk, i = e % kk;
    const int slot = newslot[i];
    const BlockRec& r = M->b[sblk[slot]];
    const int j = slot - r.svoff;
    const int l = row / 3, a = row % 3;
    double v = 0.0;
    const int lo = l - r.rst[a];
    if (lo >= 0 && lo < r.rlen[a]) {
      const int rl = r.roff[a] + lo;
      const double sg = sraw[slot];
      if (!r.trans) {
        const double w = c->W[r.woff + (size_t)j * r.q + rl];   // = U sigma
        v = absorb_left ? w * nrm : w / sg;
      } else {
        const double u = c->V[r.voff + (size_t)j * r.p + rl];   // left vector
        v = absorb_left ? u * sg * nrm : u;
      }
    }
    Ak[e] = v;
  }
  // A_{k+1}[i, (b r)]
  for (int e = tid; e < kk * n; e += NT) {
    const int i = e / n, col = e % n;
    const int slot = newslot[i];
    const BlockRec& r = M->b[sblk[slot]];
    const int j = slot - r.svoff;
    const int b = col / chir, rr = col % chir;
    double v = 0.0;
    const int lo = rr - r.cst[b];
    if (lo >= 0 && lo < r.clen[b]) {
      const int cl = r.coff[b] + lo;
      const double sg = sraw[slot];
      if (!r.trans) {
        const double u = c->V[r.voff + (size_t)j * r.p + cl];   // right vector
        v = absorb_left ? u : u * sg * nrm;
      } else {
        const double w = c->W[r.woff + (size_t)j * r.q + cl];   // = V sigma
        v = absorb_left ? w / sg : w * nrm;
      }
    }
    Ak1[e] = v;
  }
  int16_t* qM = c->qn + (size_t)(k + 1) * c->chi_cap;
  for (int i = tid; i < kk; i += NT) qM[i] = (int16_t)M->b[sblk[newslot[i]]].Q;
  __syncthreads();
  if (tid == 0) {
    c->chi[k + 1] = kk;
    c->sgn[k] = s.osk;
    c->sgn[k + 1] = s.osk1;
  }
  __syncthreads();
}

}  // namespace blk
}  // namespace hm
