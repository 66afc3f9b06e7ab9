// Internal data structures shared by the host API (hm_api.cu) and the FP64
// kernels (hm_fp64.cu).  Nothing here is part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/hmetts.h"

namespace hm {

// Site kinds of the hybrid state (Sec. I.C, Fig. 4).
enum : int32_t { SITE_ENV = 0, SITE_CPHYS = 1, SITE_ANC = 2 };

// Gate table layout of the CUDA side: 0 identity, 1 SWAP, 2 + b bond b.
enum : int32_t { GATE_ID = 0, GATE_SWAP = 1, GATE_BOND0 = 2 };

// One two-site op: theta = A_k A_{k+1}, gate, SVD, truncate, absorb.
struct OpDev {
  int32_t k;       // left site of the pair
  int32_t gate;    // gate table index
  int32_t absorb;  // 0: A_k <- U S (centre k), 1: A_{k+1} <- S V^T (centre k+1)
  int32_t exact;   // 1: centre move (keep all nonzero s up to the old bond, no renorm)
};

// Per-chain statistics slots (doubles), see hm_chain_stats.
enum : int {
  ST_K1 = 0, ST_K2, ST_SVD, ST_TRANSFER, ST_DISC, ST_MAXCHI, ST_SWEEPS, ST_SPLITS,
  ST_SVD_DENSE, ST_SWEEPS64, ST_BLOCKS, ST_RESERVED, ST_N
};
static_assert(ST_N == HM_NUM_STATS, "statistics slots of the C ABI");

// Bits of a gate table entry's info word (ChainDev::gate_info).
enum : int32_t {
  GI_EXCHANGE = 1,   // moves the two sites' contents across (an odd number of SWAP letters)
  GI_MIXING = 2      // not a permutation: conserves m1 + m2 only (a bond gate or a product with one)
};

// Device-resident description and state of one chain.  Lives in the arena;
// every pointer is a device address inside the same chain block.
struct ChainDev {
  // static description
  int32_t n_sites, n_ops, chi_max, n_env, n_meas, n_gates;
  int32_t basis_zx, first_cluster;
  uint32_t seed_lo, seed_hi, chain_id, pad0;
  double cutoff;
  const OpDev* ops;          // n_ops
  const double* gates;       // n_gates * 81, row (3a+b), column (3 s1 + s2)
  const int32_t* site_kind;  // n_sites
  const int32_t* meas_i;     // n_meas, sorted by (i, j)
  const int32_t* meas_j;
  const double* meas_J;
  const int32_t* meas_slot;  // n_meas: index of meas_j among the distinct end sites
  const int32_t* region;     // n_region physical sites of the measured columns (sorted)
  int32_t n_region, pad1;
  const double* xbasis;      // 9: rows are the Sx eigenvectors (m=+1,0,-1 order)
  const int32_t* gate_info;  // n_gates: GI_* bits
  // mutable state
  double** site;             // n_sites device pointers (fixed slots)
  int32_t* chi;              // n_sites + 1 bond dims; site s is (chi[s], 3, chi[s+1])
  int32_t* env_out;          // n_env: basis index of the current environment state
  int32_t* counters;         // [0] sample index n, [1] basis of the current initial state,
                             // [2] frame of the stored state (0: as is, 1: every leg rotated by R,
                             //     which exchanges S^x and S^z), [3] dense mode (no charge labels),
                             // [4] op cursor of a partial evolution (hm_evolve_partial)
  double* stats;             // ST_N
  int32_t* status;           // 0 = ok, else a negative HM_ERR_* code
  int32_t* err_where;        // op index / site where the error happened
  // workspaces
  double* theta;             // ws_cap doubles: two-site tensor, then scratch
  double* W;                 // ws_cap: the matrix the one-sided Jacobi orthogonalises
  double* V;                 // ws_cap: accumulated rotations
  double* sig;               // sv_cap: sorted singular values
  int32_t* perm;             // sv_cap: sorted index -> Jacobi column
  double* env_ws;            // env_cap: transfer-matrix workspace (measure, collapse)
  int16_t* qn;               // (n_sites + 1) x chi_cap: S^z charge of every bond index (grouped, ascending)
  int32_t* sgn;              // n_sites: charge sign of each position's leg (+1 spin, -1 ancilla, 0 dense)
  void* meta;                // split metadata (charge runs, blocks), kMetaBytes
  float* X;                  // ws_cap doubles of binary32 scratch (mixed chains), or nullptr
  int64_t ws_cap, env_cap;
  int32_t sv_cap, chi_cap;
};

constexpr size_t kMetaBytes = 80 * 1024;   // >= sizeof(blk::Meta) (checked in hm_block.cuh)

constexpr int kMaxBatch = 448;   // chains per launch (kernel parameter block < 4 KB)

struct BatchArg {
  int32_t n;
  int32_t t0, t1;                // op range [t0, t1) for the evolve kernel
  int32_t n_override;            // op count of ops_override
  int32_t budget;                // > 0: each chain runs ops [cursor, cursor + budget) of its own
                                 // list from its counters[4] and advances it (t0, t1 unused)
  const OpDev* ops_override;     // explicit op list (debug / kernel parity) or nullptr
  ChainDev* c[kMaxBatch];
};

struct OutArg {
  double* obs;        // device, n * n_obs (measure) or nullptr
  int32_t n_obs;
  int32_t n_env;      // stride of env_out
  int8_t* env;        // device, n * n_env (collapse) or nullptr
  double* logp;       // device, n (collapse) or nullptr
  double* cond;       // device, n * n_env * 3 conditional probabilities (collapse) or nullptr
  int32_t* ctx_err;   // device error word shared by the context
};

// Kernel launchers (hm_fp64.cu).
int launch_evolve_fp64(const BatchArg& b, const OutArg& o, void* stream);
int launch_measure_fp64(const BatchArg& b, const OutArg& o, void* stream);
int launch_collapse_fp64(const BatchArg& b, const OutArg& o, void* stream);
int launch_reset(const BatchArg& b, const OutArg& o, int draw_initial, void* stream);
// Susceptibility double sum (Eq. sus), raw and unnormalised by beta: o.obs[i].
int launch_susceptibility_fp64(const BatchArg& b, const OutArg& o, void* stream);
// Message returned by hm_last_error(NULL) (hm_api.cu).
void set_global_error(const char* msg);

// Mixed-precision evolve (hm_mixed.cu); chi_cap = largest bond cap in the
// batch; polish != 0 finishes every SVD with binary64 sweeps (HM_MIXED).
// A batch of more chains than SMs with chi_cap <= kPairChiCap goes to
// launch_evolve_mixed_pair (hm_mixed_pair.cu): two CTAs of 256 threads per
// SM with kPairBlockSmem of shared memory each.  kPairChiCap: on the S=1
// ladder at chi = 256 the largest charge block measured needs 106 KB in the
// binary32 layout (p (q + 1) + p (p + 1) + p values; oracle U(1) chain,
// Lx = 16, 2W = 8, beta = 1, three samples); a larger block takes the
// staged global-memory path of the same kernel.
int launch_evolve_mixed(const BatchArg& b, const OutArg& o, int chi_cap, int polish, void* stream);
int launch_evolve_mixed_pair(const BatchArg& b, const OutArg& o, int chi_cap, int polish, void* stream);
constexpr int kPairChiCap = 256;
constexpr size_t kPairBlockSmem = 108 * 1024;

// Binary32 GEMM tile of the mixed evolve kernel, and the dynamic shared
// memory one CTA may opt into on sm_100-class parts (227 KB).
constexpr int kMixedGM = 64, kMixedGN = 64, kMixedGK = 16;
constexpr size_t kMaxSharedOptIn = 227 * 1024;

// Dynamic shared memory of the mixed evolve kernel at bond cap chi_cap: two
// column blocks of b columns of the q + p <= 6 chi_cap row panel, plus the
// cached column norms; b = 16, halved (down to 2) while that exceeds the
// budget (210 KB, or kPairBlockSmem with two CTAs per SM).
// The GEMM tile is the floor.  Writes b to *bcols.
inline size_t mixed_smem_bytes(int chi_cap, int* bcols, size_t budget = 210 * 1024) {
  const size_t qp = 6 * (size_t)chi_cap;
  int b = 16;
  while (b > 2 && (2 * (size_t)b * qp + 3 * (size_t)chi_cap) * sizeof(float) > budget) b /= 2;
  *bcols = b;
  const size_t bytes = (2 * (size_t)b * qp + 3 * (size_t)chi_cap) * sizeof(float);
  const size_t gemm = 2 * (size_t)kMixedGK * kMixedGM * sizeof(float);
  return bytes > gemm ? bytes : gemm;
}

}  // namespace hm
