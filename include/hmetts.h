/*
 * hmetts.h -- C ABI of the GB300 (sm_103a) hybrid purification-METTS sampler.
 *
 * One Markov step of the hybrid METTS-ancilla method of Chen & Stoudenmire,
 * arXiv:1910.09142, Sec. I.C.1 ("Markov Chain Sampling Algorithm"):
 *   1. initial state |i_n>_E |B>_C: environment sites in a product state,
 *      cluster physical sites each in a Bell pair with an ancilla (Sec. I.C);
 *   2. imaginary-time evolution by beta/2 of the physical legs with
 *      second-order Trotter gates on an MPS, each two-site update split by a
 *      truncated SVD (Sec. I.A, Sec. II "sources of error");
 *   3. cluster observables <<A>>_n = <psi|A|psi> (Sec. I.C.1 step 3, Sec. II.A);
 *   4. projective collapse of the environment and reset of the cluster to Bell
 *      pairs (Sec. I.C.1 step 4, Eq. detailbalance1).
 * The model is the S=1 Heisenberg two-leg ladder of Sec. II, Eq. H.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: HM_OK (0) or a negative HM_ERR_* code; hm_last_error()
 *   gives a one-line message.  A failed call leaves no partially initialised
 *   chain behind.
 * - Memory: the caller hands one device buffer to hm_create(); the library
 *   sub-allocates every chain and workspace inside it and never calls
 *   cudaMalloc itself.  Host pointers passed in are owned by the caller and
 *   only need to stay valid until the call returns.  Calls with HOST outputs
 *   (hm_measure_cluster, hm_collapse with an output pointer,
 *   hm_measure_susceptibility) and hm_apply_ops stage through a temporary
 *   arena block of their output size (n * n_obs doubles; n * n_env bytes
 *   plus n doubles; n doubles; the op list), released before they return.
 *   They fail with HM_ERR_NOMEM when the arena has no such block free; the
 *   _device variants need none.
 * - Streams: all device work of a context is issued on the CUDA stream given
 *   to hm_create() (NULL = legacy default stream).  Calls that return host
 *   data synchronise that stream before returning; the others are
 *   asynchronous.  One context must not be used from two host threads at once.
 * - Data layout: an MPS site tensor A[k] has shape (chi_{k-1}, 3, chi_k),
 *   row-major FP64, local basis m = +1, 0, -1.  Bond dims live on the device.
 * - Precision: HM_FP64 runs every step in IEEE binary64.  HM_MIXED forms
 *   the two-site tensor and applies the gate in binary32 (binary64 site
 *   tensors rounded on load, gate coefficients as binary32 hi + lo pairs),
 *   decomposes each charge block with binary32 one-sided Jacobi sweeps, then
 *   finishes with binary64 sweeps so the singular values and vectors are
 *   binary64-accurate for that tensor; truncation, renormalisation, stored
 *   tensors, measurement and collapse are binary64.  HM_MIXED32 is HM_MIXED
 *   without the binary64 sweeps.  Measured on GB300 against HM_FP64 (same
 *   chains, same draws): per-sample energies within ~1e-6 relative for both
 *   mixed forms (the tests state 1e-5).
 */
#ifndef HMETTS_H
#define HMETTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HM_OK 0
#define HM_ERR_ARG (-1)      /* invalid argument or handle                         */
#define HM_ERR_NOMEM (-2)    /* arena cannot hold the chain (admission refused)    */
#define HM_ERR_CUDA (-3)     /* a CUDA runtime call failed                         */
#define HM_ERR_NUMERIC (-4)  /* SVD not converged, non-finite value, p_total <= 0  */
#define HM_ERR_TIMEOUT (-5)  /* a device-side iteration budget ran out             */
#define HM_ERR_STATE (-6)    /* call out of order (e.g. evolve twice, no collapse) */

#define HM_FP64 0            /* every step in binary64                              */
#define HM_MIXED 1           /* evolve: contraction and gate in binary32, Jacobi SVD */
                             /* in binary32 then binary64 sweeps; truncation,        */
                             /* renormalisation, stored tensors, measurement and     */
                             /* collapse in binary64                                 */
#define HM_MIXED32 2         /* HM_MIXED with the SVD left at its binary32 sweeps    */

#define HM_ZX_ALTERNATE 0    /* collapse sample n in the Sz basis (n even) or Sx basis (n odd) */
#define HM_Z_ONLY 1          /* collapse every sample in the Sz basis              */

#define HM_NUM_STATS 12      /* doubles written by hm_chain_stats                   */

#define HM_SCHED_PLAIN 0     /* every gate and SWAP of the schedule is its own split */
#define HM_SCHED_FUSED 1     /* consecutive splits on one site pair become one split */
                             /* with the product gate; SWAP SWAP pairs drop out      */

typedef struct hm_ctx hm_ctx;
typedef int64_t hm_chain;

/*
 * Parameters of one Markov chain (Sec. II, Eq. H; Sec. I.A; Sec. I.C).
 *   Lx            ladder length (columns); 2*Lx physical spin-1 sites, Lx >= 1.
 *   two_W         cluster physical sites (even, 0..2*Lx): the central
 *                 two_W/2 columns, x0 = floor((Lx - two_W/2)/2).  0 = METTS,
 *                 2*Lx = ancilla (purification) method.
 *   J_leg, J_rung couplings J and J_perp of Eq. H.
 *   beta, tau     inverse temperature and Trotter step; M = floor(beta/(2 tau) + 1/2)
 *                 (at least 1 when beta > 0) steps of size beta/(2M) are taken
 *                 (Sec. I.A).
 *   chi_max       bond dimension cap of every truncated SVD (>= 1; under
 *                 HM_MIXED / HM_MIXED32 the largest cap must be <= 2150, the shared memory
 *                 the binary32 evolve stages its column blocks in; larger
 *                 caps are refused with HM_ERR_ARG at admission).
 *   cutoff        truncation error target: the smallest kept count whose
 *                 discarded weight sum s^2 / total s^2 <= cutoff (Sec. II).
 *   precision     HM_FP64, HM_MIXED or HM_MIXED32.
 *   seed          Philox4x32-10 key word 0 (low 32 bits) and counter word 2
 *                 (high 32 bits).
 *   chain_id      Philox key word 1: independent random stream per chain.
 *   basis_schedule HM_ZX_ALTERNATE or HM_Z_ONLY.
 *   meas_col_lo/hi measured columns [lo, hi); -1/-1 = the cluster (or the
 *                 whole ladder when two_W = 0).  Every rung and leg bond with
 *                 both ends inside is measured.
 *   schedule      HM_SCHED_PLAIN or HM_SCHED_FUSED.  Both apply the same
 *                 product of gates (Sec. I.A, second-order steps of Sec. II);
 *                 the fused schedule merges the two half-step gates that meet
 *                 at a step's turning points into one gate, and each bond gate
 *                 into the SWAP next to it on the same site pair, and drops
 *                 SWAP SWAP pairs.  Without truncation the evolved state is
 *                 the same.  With truncation it truncates less often: on the
 *                 Lx = 16, two_W = 8, chi = 256 ladder it runs 16% fewer
 *                 two-site splits, worth 5% of the dense-SVD flop count
 *                 (the fused splits are mostly small environment ones).
 *   no_susceptibility 0: reserve the transfer workspace hm_measure_susceptibility
 *                 needs, (20 + 4 |M|) chi_cap^2 doubles (about a fifth of a
 *                 Lx = 16, chi = 256 chain); 1: do not, so more chains fit,
 *                 and hm_measure_susceptibility refuses the chain (HM_ERR_ARG).
 */
typedef struct {
  int32_t Lx, two_W;
  double J_leg, J_rung, beta, tau;
  int32_t chi_max;
  double cutoff;
  int32_t precision;
  uint64_t seed;
  uint32_t chain_id;
  int32_t basis_schedule;
  int32_t meas_col_lo, meas_col_hi;
  int32_t schedule;
  int32_t no_susceptibility;
} hm_params;

/* Create a context on CUDA device `device`, sub-allocating from the caller's
 * device buffer [dev_mem, dev_mem + bytes) (256-byte aligned, owned by the
 * caller, must outlive the context).  `cuda_stream` is a cudaStream_t or NULL. */
int hm_create(hm_ctx** out, int device, void* dev_mem, size_t bytes, void* cuda_stream);

/* Destroy a context (synchronises its stream).  The device buffer is not freed. */
int hm_destroy(hm_ctx* ctx);

/* Upper bound of the arena bytes one chain with these parameters needs
 * (site tensors at their maximal bond dims, SVD and contraction workspaces).
 * Used for admission: hm_init_chain fails with HM_ERR_NOMEM, without side
 * effects, when the arena has fewer free bytes. */
int hm_query_memory(const hm_params* p, size_t* bytes_out);

/* Number of observables hm_measure_cluster writes per chain:
 * 1 + 2 * (measured bonds).  Layout: [0] E_est = sum_b J_b <S_i.S_j>_b,
 * then per measured bond b (bonds sorted by MPS index): <S_i.S_j>, <Sz_i Sz_j>. */
int hm_num_obs(const hm_params* p, int32_t* n_obs);

/* Number of environment sites (collapse outcomes per sample). */
int hm_num_env(const hm_params* p, int32_t* n_env);

/* Allocate a chain and write its first initial state (step 1).  env_init:
 * host array of n_env outcomes in {0,1,2} (Sz basis: m = +1, 0, -1), or NULL
 * to draw them from the chain's Philox stream with sample index n = -1.
 * Synchronises the stream (the chain image is uploaded from the host).
 * HM_ERR_NOMEM, with nothing allocated, when the arena cannot hold it. */
int hm_init_chain(hm_ctx* ctx, const hm_params* p, const int8_t* env_init, hm_chain* out);

/* Resume a chain from its checkpoint (no counterpart in the paper; the
 * state a chain carries between samples is only this, because step 4 resets
 * the cluster to Bell pairs).  Allocates the chain like hm_init_chain and
 * writes the initial state of sample `next_sample` (>= 1): env_out (host,
 * n_env values in {0,1,2}) are the outcomes the collapse of sample
 * next_sample - 1 returned, read in that sample's basis (Sz for an even
 * index or under HM_Z_ONLY, Sx for an odd one).  The resumed chain then
 * draws exactly what the uninterrupted chain would: same Philox counters,
 * same bases.  Errors: HM_ERR_ARG for next_sample < 1 (use hm_init_chain),
 * a NULL or out-of-range env_out, or any hm_init_chain error. */
int hm_resume_chain(hm_ctx* ctx, const hm_params* p, const int8_t* env_out, int64_t next_sample,
                    hm_chain* out);

/* Release a chain's arena memory (synchronises the stream). */
int hm_free_chain(hm_ctx* ctx, hm_chain chain);

/* Step 2 for n chains: evolve each chain's initial state by beta/2 with the
 * second-order Trotter schedule; leaves the orthogonality centre on site 0.
 * Asynchronous.  Requires the chain to be in its initial state. */
int hm_evolve(hm_ctx* ctx, const hm_chain* ids, int32_t n);

/* Step 2 in slices, for schedulers that bound the work of one call (a
 * serving tick): advances each chain's evolution by at most max_ops ops of
 * its schedule (hm_plan), from where the previous call on it stopped.  A
 * chain whose schedule is complete is evolved (ready for measure and
 * collapse), exactly as after hm_evolve; done_out (HOST, n, nullable)
 * receives 1 for those chains and 0 for the others.  The slices give the
 * same state as one hm_evolve.  HM_ERR_STATE for an evolved chain, and
 * hm_evolve refuses a chain whose evolution is under way.  Asynchronous. */
int hm_evolve_partial(hm_ctx* ctx, const hm_chain* ids, int32_t n, int32_t max_ops, int32_t* done_out);

/* Step 3: n_obs observables per chain into the HOST array out[n * n_obs]
 * (row i = chain ids[i]).  Synchronises.  Requires an evolved chain. */
int hm_measure_cluster(hm_ctx* ctx, const hm_chain* ids, int32_t n, double* out, int32_t n_obs);

/* Step 3, device variant: out is a DEVICE array of n * n_obs doubles.
 * Asynchronous. */
int hm_measure_cluster_device(hm_ctx* ctx, const hm_chain* ids, int32_t n, double* out_dev,
                              int32_t n_obs);

/* Uniform susceptibility estimator of Eq. sus (Sec. II.A) for n evolved
 * chains: out[2 i] = chi_M = (beta / 3) (1 / |M|) sum_{j in M} sum_i <S_j . S_i>
 * and out[2 i + 1] = the double sum itself, where M is the set of physical
 * sites of the measured columns (see meas_col_lo/hi; the paper averages over
 * the central 6 x 2 sites) and i runs over every physical site, environment
 * included (<S_j . S_j> = 2).  HOST output (2 n doubles); binary64; no
 * canonical-form assumption.  Synchronises. */
int hm_measure_susceptibility(hm_ctx* ctx, const hm_chain* ids, int32_t n, double* out);

/* Step 4: collapse the environment of n evolved chains, left to right, in the
 * basis of their sample index, then reset each chain to the new initial state
 * |i_{n+1}>_E |B>_C.  env_out (HOST, n * n_env, nullable): basis indices of
 * the outcomes; logp_out (HOST, n, nullable): log-probability of the drawn
 * outcome string.  Synchronises when an output pointer is given. */
int hm_collapse(hm_ctx* ctx, const hm_chain* ids, int32_t n, int8_t* env_out, double* logp_out);

/* Step 4, device variant: env_out_dev (int8, n * n_env) and logp_out_dev
 * (double, n) are DEVICE arrays or NULL.  Asynchronous. */
int hm_collapse_device(hm_ctx* ctx, const hm_chain* ids, int32_t n, int8_t* env_out_dev,
                       double* logp_out_dev);

/* Step 4 with its intermediate results, for parity checks: as hm_collapse,
 * and cond_out (HOST, n * n_env * 3 doubles) receives, per environment site
 * in collapse order, the conditional probabilities p(b | outcomes before it)
 * of the three basis states of that sample's basis (Eq. detailbalance1: the
 * probability of the drawn string is their product along the outcomes).
 * The chains must share n_env.  env_out, logp_out and cond_out must not be
 * NULL.  Synchronises; stages through an arena block like hm_collapse. */
int hm_collapse_conditionals(hm_ctx* ctx, const hm_chain* ids, int32_t n, int8_t* env_out, double* logp_out,
                             double* cond_out);

/* Per-chain counters since init, to HOST out[HM_NUM_STATS]:
 * [0] flops of the two-site contractions, counted block by block
 *     (2 rows x inner x columns of every charge block, Sec. II.C),
 * [1] gate flops (2 * 81 chi_l chi_r),
 * [2] SVD flops of the blocked decompositions: the dense count
 *     4 M^2 N + 8 M N^2 + 9 N^3 (M >= N) of every charge block,
 * [3] measurement + collapse transfer-matrix flops,
 * [4] sum of discarded weights, [5] largest bond dimension seen,
 * [6] Jacobi sweeps (largest block of each split; binary32 sweeps under
 *     HM_MIXED), [7] two-site splits,
 * [8] the dense-SVD count of the same splits without blocking (what one
 *     unblocked SVD per split would be charged), [9] binary64 polish sweeps
 *     (HM_MIXED), [10] charge blocks decomposed, [11] reserved.
 * Synchronises. */
int hm_chain_stats(hm_ctx* ctx, hm_chain chain, double* out);

/* Copy the chain's current MPS to the host: dims_out[n_sites + 1] bond dims
 * and the site tensors concatenated into buf (capacity `cap` doubles);
 * *n_sites_out = sites, *n_doubles_out = doubles written.  Synchronises. */
int hm_get_mps(hm_ctx* ctx, hm_chain chain, int32_t* dims_out, int32_t dims_cap,
               double* buf, size_t cap, int32_t* n_sites_out, size_t* n_doubles_out);

/* Replace the chain's MPS (dims[n_sites + 1], tensors concatenated as in
 * hm_get_mps; the orthogonality centre must be on `centre`).  Marks the chain
 * as "initial" (ready for hm_evolve) or, with evolved != 0, as evolved (ready
 * for measure / collapse).  For checkpoint restore and debugging. */
int hm_set_mps(hm_ctx* ctx, hm_chain chain, const int32_t* dims, int32_t n_sites,
               const double* buf, size_t n_doubles, int32_t centre, int32_t evolved);

/* Run an explicit list of n_ops two-site ops on one chain (debugging and
 * kernel-level parity).  ops[4 i ..]: (site k, gate, absorb, exact) with gate
 * index into the chain's gate table (0 = identity, 1 = SWAP, 2 + b = bond b
 * of the sorted bond list at tau/2, then a fused chain's product gates; see
 * hm_gates), absorb 0 = left (A_k <- U S), 1 = right (A_{k+1} <- S V^T),
 * exact 1 = keep every nonzero singular value up to the old bond dim without
 * renormalising (a centre move).  The op list is staged in the arena, so the
 * call synchronises the stream; HM_ERR_ARG for an op outside the chain or
 * the table. */
int hm_apply_ops(hm_ctx* ctx, hm_chain chain, const int32_t* ops, int32_t n_ops);

/* The op schedule of hm_evolve (host planner; no GPU needed): writes up to
 * `cap` ops as 4 int32 each (k, gate, absorb, exact) and *n_ops_out. */
int hm_plan(const hm_params* p, int32_t* ops, int32_t cap, int32_t* n_ops_out);

/* Gate table of a chain (no GPU needed): n_gates * 81 doubles, row index
 * 3 a + b (output legs), column 3 s1 + s2.  Entry 0 is the identity, 1 the
 * SWAP, 2 + b the gate of bond b; under HM_SCHED_FUSED the products used by
 * fused ops follow, in order of first use.  *n_gates_out = the entry count. */
int hm_gates(const hm_params* p, double* out, int32_t cap, int32_t* n_gates_out);

/* ---- Allocation-free entry point -------------------------------------------
 * The paper has no counterpart: this is a library convenience.  It serves
 * callers that cannot call cudaMalloc (code running inside another
 * framework's memory pool, processes whose device allocator belongs to
 * someone else, paths that must not allocate while they run): it performs ONE two-site update of
 * step 2 -- theta = A B, the 9x9 gate, the binary64 one-sided Jacobi SVD,
 * the truncation rule and the absorb -- with all scratch in a fixed device
 * array of the library (about 4.3 MB, kept by every GPU that loads the
 * library until the process exits).  It never allocates or frees memory.
 *   A_dev     (chi_l, 3, chi_m) binary64, device; B_dev (chi_m, 3, chi_r).
 *   gate_dev  81 binary64 on the device, row 3a+b, column 3 s1 + s2.
 *   chi_l, chi_m, chi_r, chi_max must lie in [1, 128]; larger values return
 *             HM_ERR_ARG (the fixed scratch cannot hold them).
 *   A_out_dev (chi_l, 3, k) and B_out_dev (k, 3, chi_r) with room for
 *             k = min(3 chi_l, 3 chi_r, chi_max); k_out_dev: one int32 that
 *             receives k, or a negative HM_ERR_* code if the SVD failed.
 *   absorb    0: A_out = U S (centre left), 1: B_out = S V^T (centre right).
 * Asynchronous on cuda_stream.  The first call on each device looks up the
 * device address of the scratch array (set-up; make that first call before
 * any stream capture).  Every call shares the one array and leaves its
 * contents behind; calls whose kernels overlap on the GPU race on it, so
 * issue them on one stream or serialise them. */
int hm_two_site_update_static(const double* A_dev, const double* B_dev, int32_t chi_l, int32_t chi_m,
                              int32_t chi_r, const double* gate_dev, int32_t chi_max, double cutoff,
                              int32_t absorb, double* A_out_dev, double* B_out_dev, int32_t* k_out_dev,
                              void* cuda_stream);

/* The message of the last failed call on ctx (or of the last failed
 * context-free call when ctx is NULL). */
const char* hm_last_error(const hm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HMETTS_H */
