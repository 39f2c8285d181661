/*
 * afqmc.h - C ABI of the GB300 ph-AFQMC walker-step library (libafqmc.so).
 *
 * The library propagates a population of Slater-determinant walkers in
 * imaginary time with the phaseless auxiliary-field QMC step of Shee et al.
 * (arXiv:1804.03310): force bias, auxiliary-field draw and hybrid weight with
 * the phaseless cut (Sec. II), the one-body operator sum_g x_g L_g and its
 * Taylor exponential applied to the walker orbitals (Sec. II, Eq. 2-3,
 * Thouless propagation by matrix products), overlaps and Green's functions
 * from batched small inverses and Sherman-Morrison-Woodbury updates for
 * multi-determinant trials (Sec. III, Eq. 4), the local energy through the
 * precomputed trial-contracted tensor (Sec. III, Eq. 5), walker
 * orthonormalisation and comb population control (Sec. IV.A, Sec. V).
 *
 * Conventions for every call:
 *  - Matrices are row-major, double precision, on the HOST unless a
 *    parameter says "device". Complex numbers are two doubles (re, im).
 *  - Inputs are copied during the call; the caller keeps ownership of all
 *    buffers it passes. Outputs go to caller-allocated host buffers.
 *  - Every call returns an afqmc_status. Nothing aborts, traps or exits.
 *    After a failure afqmc_last_error(ctx) describes it. A context that hit
 *    AFQMC_E_CUDA is poisoned: only afqmc_last_error and afqmc_destroy are
 *    then accepted.
 *  - All GPU work of a context is issued on its stream (the caller's stream
 *    when one is given at creation). Calls returning host data synchronise
 *    that stream. Calls on one context are not thread-safe.
 *  - All device memory a context uses is allocated in afqmc_create and freed
 *    in afqmc_destroy; propagation allocates nothing.
 */
#ifndef AFQMC_H
#define AFQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afqmc_ctx afqmc_ctx;

typedef enum {
  AFQMC_OK = 0,
  AFQMC_E_INVALID = 1,    /* bad argument or unsupported size */
  AFQMC_E_OOM = 2,        /* device allocation failed */
  AFQMC_E_CUDA = 3,       /* a CUDA call failed; the context is poisoned */
  AFQMC_E_POPULATION = 4, /* every walker weight is zero (comb impossible) */
  AFQMC_E_TIMEOUT = 5,    /* a bounded device-side wait gave up */
  AFQMC_E_NUMERIC = 6,    /* non-finite setup quantity (e.g. trial energy) */
  AFQMC_E_STATE = 7       /* checkpoint buffer does not match the context */
} afqmc_status;

/* Arithmetic of the walker step.
 * FP64:    complex128 walkers, every contraction in FP64.
 * FP32:    complex64 walkers, FP32 SIMT contractions.
 * TF32:    complex64 walkers, dense contractions on tcgen05 tensor cores with
 *          TF32 operands and FP32 accumulation.
 * TF32X3:  as TF32 with split (hi + lo) operands, three products per term;
 *          the tensor core accumulates at most 128 K values before the sum
 *          continues in FP32 registers.
 * BF16X3:  the propagation (Taylor series and both half steps) with BF16
 *          hi + lo operands, three BF16 products per term, FP32
 *          accumulation; the force-bias, one-body-operator and energy
 *          contractions, which feed the weights and the energy directly,
 *          as in TF32X3.
 * The reduced modes keep FP64 for walker weights, the accumulation of
 * log-determinants and ln det R, the population-control prefix sums and the
 * energy shift E_T; params.fp64_islands moves the QR (Sec. IV.A), and
 * optionally the small inverse, to FP64 arithmetic as well. */
typedef enum {
  AFQMC_FP64 = 0,
  AFQMC_FP32 = 1,
  AFQMC_TF32 = 2,
  AFQMC_TF32X3 = 3,
  AFQMC_BF16X3 = 4
} afqmc_precision;

/* Weight update after each step (Sec. II), both with the phaseless cut
 * max(0, cos(dtheta)), dtheta the phase of the walker's overlap ratio
 * <Psi_T|phi'>/<Psi_T|phi> (times the mean-field scalar factor when
 * mf_subtract is set):
 * HYBRID:        W <- W |I| cut, I = ratio * exp(sum_g x_g xbar_g -
 *                xbar_g^2/2) * exp(dtau (E_T - E_0)); E_0 = -1/2 sum_g
 *                lbar_g^2 with the mean field subtracted, else 0.
 * LOCAL_ENERGY:  W <- W exp(-dtau (Re E_L - E_T)) cut, E_L the local energy
 *                of the walker before the move (one energy evaluation per
 *                step). One-determinant trials only (AFQMC_E_INVALID
 *                otherwise): the walkers start at the reference
 *                determinant, where a multi-determinant trial's
 *                per-determinant energies are 0/0 limits. */
typedef enum {
  AFQMC_WEIGHT_HYBRID = 0,
  AFQMC_WEIGHT_LOCAL_ENERGY = 1
} afqmc_weight_mode;

typedef struct {
  int32_t M;             /* orbitals (one-particle basis size), 1..256 */
  int32_t n_up, n_dn;    /* electrons per spin, 0..M each, n_up + n_dn >= 1 */
  int32_t n_chol;        /* Cholesky / density-fitting vectors L_g, >= 1 */
  int32_t n_det;         /* determinants in the trial, >= 1 */
  int32_t n_walkers;     /* walkers, >= 1 */
  double dtau;           /* imaginary-time step (Ha^-1), > 0 */
  uint64_t seed;         /* Philox key for the field draws and the comb */
  int32_t run_id;        /* Philox stream tag, 0 .. 2^29-1 */
  int32_t precision;     /* afqmc_precision */
  int32_t ortho_every;   /* orthonormalise after every k-th step (0: never) */
  int32_t measure_every; /* local-energy measurement cadence (0: never) */
  int32_t pc_every;      /* comb population-control cadence (0: never) */
  int32_t taylor_order;  /* terms of the exponential's Taylor series, 1..12 */
  double fb_cap;         /* cap on |xbar_g|; <= 0 disables the cap */
  double e_shift;        /* energy shift E_T; NaN: local energy of the reference determinant */
  int32_t fp64_islands;  /* reduced-precision modes: 1 = Gauss-Jordan inverse and
                            Gram-Schmidt (QR) arithmetic in FP64; 2 = the QR
                            alone in FP64; 0 (default) = FP32 arithmetic
                            there, with the log-determinant and ln det R
                            sums still accumulated in FP64. Other values:
                            AFQMC_E_INVALID */
  int32_t graphs;        /* 1: afqmc_propagate replays whole periods of the
                            ortho / measure / comb cadence as CUDA graphs
                            (same kernels, same results); 0: plain launches */
  int32_t autotune;      /* tensor-core modes: 1 = time the launch shapes
                            (afqmc_tuning) on this system at creation and keep
                            the fastest, cached per shape for the process;
                            0 = fixed heuristics */
  int32_t weight_cap;    /* 0 (default): no cap, the paper's hybrid weights.
                            k > 0: after each step a walker's weight is capped
                            at k times the reference weight, the common weight
                            of the last comb (1, since the comb divides it out,
                            see afqmc_log_weight_scale; 1 before the first
                            comb; a restored checkpoint takes the mean of its
                            positive weights). Guards long runs against
                            a walker near a node of the trial taking a runaway
                            weight, at the price of a bias that vanishes as k
                            grows. */
  int32_t cs_group;      /* correlated sampling (Sec. V): 0 = none. Runs
                            that share seed and run_id draw the same fields
                            walker by walker (the Philox counter depends on
                            nothing else), so a neutral/cation pair given the
                            same seed, run_id, n_chol and n_walkers samples
                            the same auxiliary-field paths and their energy
                            difference loses most of its variance. A server
                            admits the runs submitted with the same nonzero
                            cs_group together, once all cs_size of them have
                            arrived; outside a server the field is only
                            validated. */
  int32_t cs_size;       /* runs in the group, 2..16 (0 when cs_group is 0) */
  int32_t weight_mode;   /* afqmc_weight_mode (Sec. II): 0 = hybrid
                            importance factor, 1 = local-energy form */
  int32_t mf_subtract;   /* 1: subtract the mean field lbar_g = <L_g> of the
                            reference determinant from the Cholesky
                            operators (the propagator's exact form is
                            unchanged; the phaseless cut sees smaller
                            phases); 0: none */
  int32_t block_sparse;  /* Cholesky vectors that are block-diagonal in a
                            common partition of the basis (every L_g zero
                            between different blocks, as for basis shells of
                            an atom): the one-body operator V = sum s_g L_g
                            is then block-diagonal too, is built on the
                            blocks' entries only and its Taylor series is
                            applied block by block, between the two dense
                            half steps (same arithmetic, far fewer
                            operations). 0 (default): use it when the
                            partition has at least two blocks, none larger
                            than 32, and at most M^2/4 entries; 1: require
                            it (AFQMC_E_INVALID otherwise); 2: dense */
  int32_t reserved[3];   /* must be zero */
} afqmc_params;

/* Fill *p with defaults: taylor_order 6, fb_cap 1, e_shift NaN, FP64,
 * ortho_every 2, measure_every 20, pc_every 20, graphs 1, autotune 1,
 * everything else zero. */
void afqmc_params_default(afqmc_params* p);

/* Create a context: copy the Hamiltonian and trial to the device, precompute
 * the one-body remainder H1' = h1 - 1/2 sum_g L_g L_g (two-body term of Eq. 1
 * written as -1/2 sum_g v_g^2, Sec. II), B_half = exp(-dtau/2 H1') (symmetric
 * Trotter split), the half-rotated vectors D^H L_g, the exchange part of the
 * Eq. 5 tensor, and initialise every walker to the reference determinant with
 * weight 1. Setup is not part of the propagation time (Sec. III).
 *
 *  h1      [M*M]            symmetric one-body matrix T_ij of Eq. 1
 *  L       [n_chol*M*M]     each L_g symmetric; V_ijkl = sum_g L_g,ik L_g,jl
 *  C_up    [M*M]            orbitals for spin up, column p = orbital p
 *  C_dn    [M*M]            orbitals for spin down
 *  occ_up  [n_det*n_up]     orbital indices of each determinant; row 0 is the
 *  occ_dn  [n_det*n_dn]     reference. Determinants must be orthonormal
 *                           (orthonormal C, distinct occupation rows).
 *  ci      [2*n_det]        CI coefficients (re, im); |Psi_T> = sum_i c_i |D_i>
 *  stream  cudaStream_t of the caller, or NULL for a stream the context owns.
 *  out     receives the context.
 * Returns AFQMC_E_INVALID for sizes outside the documented ranges or a
 * non-orthonormal trial, AFQMC_E_OOM when device memory is short. */
afqmc_status afqmc_create(const afqmc_params* params, const double* h1,
                          const double* L, const double* C_up,
                          const double* C_dn, const int32_t* occ_up,
                          const int32_t* occ_dn, const double* ci,
                          void* stream, afqmc_ctx** out);

/* Advance every walker by n_steps imaginary-time steps (Sec. II): force
 * bias, field draw, propagation, new overlap and hybrid phaseless weight;
 * after step count s (1-based) orthonormalise when s % ortho_every == 0,
 * measure the local energy when s % measure_every == 0, comb when
 * s % pc_every == 0. Asynchronous on the context's stream; a later call that
 * returns host data reports AFQMC_E_POPULATION if a comb found all weights 0. */
afqmc_status afqmc_propagate(afqmc_ctx* ctx, int32_t n_steps);

/* Orthonormalise every walker now: the QR factor Q with R's diagonal real
 * and positive (the factorisation modified Gram-Schmidt produces), computed
 * from the Cholesky factor of the Gram matrix; ln det R is accumulated in
 * FP64 and the log-overlap drops by it (Sec. IV.A). */
afqmc_status afqmc_orthonormalize(afqmc_ctx* ctx);

/* Comb population control now (Sec. V final comments); offset drawn from
 * Philox stream 1 at the current step counter. Every walker leaves with
 * weight 1; the common weight S/n goes to afqmc_log_weight_scale. */
afqmc_status afqmc_population_control(afqmc_ctx* ctx);

/* Local energy E_L = <Psi_T|H|phi>/<Psi_T|phi> of every walker (Sec. II,
 * via Eq. 5). e_loc [2*n_walkers] (re, im) or NULL; e_mixed receives
 * sum_w W Re E_L / sum_w W (NaN if all weights are 0), or NULL. */
afqmc_status afqmc_local_energy(afqmc_ctx* ctx, double* e_loc, double* e_mixed);

/* Walker weights [n_walkers] and, if log_ovlp is not NULL, the
 * log-overlaps ln <Psi_T|phi> [2*n_walkers] (re, im). */
afqmc_status afqmc_weights(afqmc_ctx* ctx, double* w, double* log_ovlp);

/* Mixed Green's functions G_ij = <c+_i c_j> of one walker, [2*M*M] each
 * (re, im interleaved, row-major); either pointer may be NULL. */
afqmc_status afqmc_green(afqmc_ctx* ctx, int32_t walker, double* G_up,
                         double* G_dn);

/* Self-test of failure detection (no counterpart in the paper): runs on the
 * context's stream one kernel whose single thread waits, with the bounded
 * wait every tensor-core pipeline uses, on an mbarrier that nothing ever
 * completes, giving up after about limit_cycles SM clock cycles (0..4e9);
 * no copy or MMA is in flight. Returns AFQMC_E_TIMEOUT, the status a
 * timed-out pipeline wait reports, and leaves the context usable. */
afqmc_status afqmc_selftest_wait_timeout(afqmc_ctx* ctx, int64_t limit_cycles);

/* The energy shift E_T in use (Sec. II): params.e_shift, or when that is NaN
 * the energy of the reference determinant <D_0|H|D_0>, evaluated in FP64 at
 * creation whatever the step precision. */
afqmc_status afqmc_energy_shift(afqmc_ctx* ctx, double* e_shift);

/* Log of the factor the weights have been divided by. Each comb (Sec. V)
 * gives every walker the common weight S/n (S the total weight, n the
 * walkers); the library divides it out, so every walker restarts at weight
 * 1, and adds ln(S/n) here, so that a population far below E_T cannot
 * overflow. The absolute weight of walker i is w_i * exp(*log_scale);
 * estimators are ratios of weights and need no correction. Counts from
 * creation or from the last afqmc_set_state (whose image carries absolute
 * weights). Synchronises the context's stream. */
afqmc_status afqmc_log_weight_scale(afqmc_ctx* ctx, double* log_scale);

/* Force bias xbar of the last step, [n_walkers * n_chol * 2] (re, im). */
afqmc_status afqmc_force_bias(afqmc_ctx* ctx, double* xbar);

/* Mixed energies recorded by measurements inside afqmc_propagate:
 * up to max_n pairs (step count, energy) into out[2*i], out[2*i+1];
 * *n receives the number recorded so far (history keeps the last 4096). */
afqmc_status afqmc_energy_history(afqmc_ctx* ctx, double* out, int32_t max_n,
                                  int32_t* n);

/* Checkpoint. With buf == NULL, *bytes receives the size needed. Otherwise
 * writes a self-describing image (header, walker orbitals as complex128
 * [n_walkers][n_up+n_dn][M], weights, log-overlaps, step counter) of at most
 * *bytes bytes and sets *bytes to the size written. */
afqmc_status afqmc_get_state(afqmc_ctx* ctx, void* buf, size_t* bytes);

/* Restore an image written by afqmc_get_state for a context of the same
 * sizes (precision may differ). AFQMC_E_STATE if it does not match. The
 * Philox counter is a pure function of (seed, run, step, walker, field), so
 * a resumed run draws exactly the fields the uninterrupted run would. */
afqmc_status afqmc_set_state(afqmc_ctx* ctx, const void* buf, size_t bytes);

/* Wait for all work of the context. */
afqmc_status afqmc_synchronize(afqmc_ctx* ctx);

/* Per-kernel device timing, for roofline accounting. When enabled, CUDA
 * events bracket every launch of the kernels listed below on the context's
 * stream. afqmc_kernel_stats returns for kernel id k the number of launches,
 * the summed device time in ms, and the algorithmic work per launch (flops
 * for contractions, bytes for bandwidth-bound kernels; *is_bytes says which).
 * Ids: 0 force bias, 1 field draw, 2 one-body operator, 3 propagation,
 * 4 overlap/Green's, 5 weights, 6 orthonormalisation, 7 energy contraction,
 * 8 comb. Returns AFQMC_E_INVALID for an unknown id. */
afqmc_status afqmc_set_kernel_timing(afqmc_ctx* ctx, int32_t enable);
afqmc_status afqmc_kernel_stats(afqmc_ctx* ctx, int32_t kernel_id,
                                int64_t* launches, double* total_ms,
                                double* work_per_launch, int32_t* is_bytes);
#define AFQMC_N_KERNEL_IDS 9

/* Number of kernel launches issued since creation (all of this library's),
 * counting each kernel of a replayed graph. */
int64_t afqmc_launch_count(const afqmc_ctx* ctx);

/* Launch shapes of the tensor-core modes (TF32, TF32X3, BF16X3). Shapes change the
 * numerics only through the order of FP32 sums (split K) and through the
 * propagation path (taylor_fused below);
 * every choice meets the same tolerance against the FP64 path. In the FP64
 * and FP32 modes get returns xsplit 1 and zeros, and set accepts only that. */
typedef struct {
  int32_t xsplit;         /* K ranges of the force-bias contraction, 1..8 */
  int32_t bn_force_bias;  /* output tile width (64 or 128) of the force-bias, */
  int32_t bn_one_body;    /*   one-body-operator, energy and half-step */
  int32_t bn_energy;      /*   contractions */
  int32_t bn_half_step;
  int32_t taylor_fused;   /* propagation path: 0 = series on the CUDA cores,
                             half steps as contractions; 1 = one fused
                             tensor-core kernel for B_half exp_T(V) B_half
                             with the operator held on chip; 2 = series on
                             the tensor cores, half steps as separate
                             contractions (1 and 2 need M <= 64); 3 = one
                             fused tensor-core kernel with the operator
                             streamed from memory by TMA (needs M > 64);
                             4 = the block-diagonal series of
                             params.block_sparse (the only path, and only
                             there, when the context uses it) */
  int32_t reserved[2];    /* zero */
} afqmc_tuning;
afqmc_status afqmc_get_tuning(afqmc_ctx* ctx, afqmc_tuning* out);
afqmc_status afqmc_set_tuning(afqmc_ctx* ctx, const afqmc_tuning* t);

/* Device memory of a context with these parameters: *resident bytes held
 * from afqmc_create to afqmc_destroy (what afqmc_device_bytes reports), and
 * *setup_peak further bytes of FP64 staging held during afqmc_create only.
 * occ_up / occ_dn as for afqmc_create (they fix the active orbitals of a
 * multi-determinant trial; may be NULL when n_det == 1). Host-only: needs no
 * GPU. AFQMC_E_INVALID for parameters afqmc_create would reject by size. */
afqmc_status afqmc_footprint(const afqmc_params* params, const int32_t* occ_up,
                             const int32_t* occ_dn, size_t* resident,
                             size_t* setup_peak);

/* Device bytes allocated by the context (equals the footprint's resident). */
size_t afqmc_device_bytes(const afqmc_ctx* ctx);

/* Blocks of steps captured as CUDA graphs so far (0 when graphs are off or
 * the stream could not be captured, in which case propagation falls back to
 * plain launches). */
int32_t afqmc_graph_count(const afqmc_ctx* ctx);

/* ------------------------------------------------------------------------
 * Multi-system batching (no counterpart in the paper, whose runs are one
 * system per GPU).
 *
 * A batch advances several contexts of uneven sizes (M, electrons, n_chol,
 * walkers, precision, trial) together. Each block of steps_per_block steps
 * is ONE CUDA graph launch on the batch's stream: the graph holds every
 * member's captured block as an independent branch, so the systems run
 * concurrently on the GPU and the host issues one launch per block, not one
 * per kernel. Each member advances exactly as afqmc_propagate(ctx,
 * steps_per_block) would (same kernels, same Philox counters, same
 * results). The batch orders its work after all work already issued on the
 * members' streams and the members' later work after the batch's, so the
 * contexts remain usable one by one between batch calls. Members must stay
 * alive while the batch exists; kernel timing must be off on them.
 * Errors are described by afqmc_last_error(NULL).
 * ------------------------------------------------------------------------ */
typedef struct afqmc_batch afqmc_batch;
afqmc_status afqmc_batch_create(afqmc_ctx* const* ctxs, int32_t n,
                                int32_t steps_per_block, afqmc_batch** out);
afqmc_status afqmc_batch_propagate(afqmc_batch* b, int32_t n_blocks);
/* Number of graph launches issued by the batch so far. */
int64_t afqmc_batch_launches(const afqmc_batch* b);
afqmc_status afqmc_batch_synchronize(afqmc_batch* b);
void afqmc_batch_destroy(afqmc_batch* b);

/* ------------------------------------------------------------------------
 * Serving loop (no counterpart in the paper).
 *
 * A server accepts independent ph-AFQMC runs (each a full afqmc_create
 * input plus n_blocks blocks of steps_per_block steps) and runs them on one
 * GPU with continuous batching: a native scheduler thread admits queued runs
 * in arrival order as soon as a slot is free and the HBM budget holds the
 * run's footprint (resident + setup staging, afqmc_footprint), and a later
 * run that fits may overtake a head run that does not (the head is overtaken
 * at most 8 times, then admission waits for it). Each admitted run gets its
 * own stream; its walkers stay on the device from admission to its last
 * block; blocks are captured as CUDA graphs and kept two deep in each run's
 * stream, so the work of all admitted runs overlaps on the GPU. A finished
 * run's memory is freed at once. A run's results depend only on its own
 * inputs (its Philox counters are keyed by its seed and run_id), so they are
 * the same alone and in any mix.
 * Errors of these calls are described by afqmc_last_error(NULL).
 * ------------------------------------------------------------------------ */
typedef struct afqmc_server afqmc_server;

typedef struct {
  size_t hbm_budget;   /* device bytes for runs; 0: 90% of the free memory */
  int32_t max_active;  /* runs on the GPU at once, 1..256 (0: 64) */
  int32_t device;      /* CUDA device ordinal */
  int32_t reserved[4]; /* zero */
} afqmc_server_config;

enum { AFQMC_RUN_QUEUED = 0, AFQMC_RUN_ACTIVE = 1, AFQMC_RUN_DONE = 2,
       AFQMC_RUN_FAILED = 3 };

typedef struct {
  int32_t state;        /* AFQMC_RUN_* */
  int32_t status;       /* afqmc_status of a failed run, else AFQMC_OK */
  int32_t n_blocks, blocks_done;
  double t_submit;      /* host seconds since the server started; -1 if */
  double t_admit;       /*   the event has not happened yet */
  double t_done;
  size_t footprint;     /* resident + setup staging bytes used for admission */
  char message[160];    /* error text of a failed run */
} afqmc_run_info;

typedef struct {
  double t_start;       /* host seconds: the later of the block's enqueue and
                           the previous block's completion */
  double t_end;         /* host seconds: completion seen by the scheduler */
  double device_ms;     /* device time between the block's start and end */
  double e_mixed;       /* mixed energy of the latest measurement (NaN if none) */
  double weight_sum;    /* sum of walker weights at that measurement (in
                           units of the run's log weight scale) */
  int64_t step;         /* step count at the end of the block */
} afqmc_block_result;

typedef struct {
  int64_t submitted, admitted, completed, failed, blocks;
  double walker_steps;  /* walker-steps of all completed blocks */
  double p50_ms, p99_ms;/* block latency t_end - t_start over completed blocks */
  double elapsed_s;     /* host seconds since the server started */
  int32_t active, queued, max_active_seen, reserved0;
  size_t bytes_in_use, peak_bytes;  /* admitted footprints (resident only) */
} afqmc_server_stats;

afqmc_status afqmc_server_create(const afqmc_server_config* cfg, afqmc_server** out);
/* Queue a run. All inputs as for afqmc_create (copied during the call);
 * n_blocks >= 1 blocks of steps_per_block >= 1 steps. *run_id receives the
 * run's handle (not the Philox run_id, which stays params->run_id).
 * Correlated-sampling groups (params->cs_group != 0): every member must
 * match the group's first member in seed, run_id, n_chol, n_walkers, dtau,
 * the cadences, the Taylor order, cs_size, n_blocks and steps_per_block
 * (else AFQMC_E_INVALID), a group takes at most cs_size runs, and a group
 * id cannot be reused once its runs were admitted. */
afqmc_status afqmc_server_submit(afqmc_server* s, const afqmc_params* params,
                                 const double* h1, const double* L,
                                 const double* C_up, const double* C_dn,
                                 const int32_t* occ_up, const int32_t* occ_dn,
                                 const double* ci, int32_t n_blocks,
                                 int32_t steps_per_block, int64_t* run_id);
/* State of a run and up to max_blocks of its block results (blocks may be
 * NULL). AFQMC_E_INVALID for an unknown run. */
afqmc_status afqmc_server_poll(afqmc_server* s, int64_t run_id, afqmc_run_info* info,
                               afqmc_block_result* blocks, int32_t max_blocks);
/* Wait until the run (run_id >= 0) or every submitted run (run_id < 0) is
 * done or failed; AFQMC_E_TIMEOUT after timeout_s seconds (< 0: no limit). */
afqmc_status afqmc_server_wait(afqmc_server* s, int64_t run_id, double timeout_s);
afqmc_status afqmc_server_stats_get(afqmc_server* s, afqmc_server_stats* out);
/* Stop the scheduler (runs still queued or active are abandoned) and free
 * everything. */
void afqmc_server_destroy(afqmc_server* s);

/* Comb population control that allocates no device memory.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot call cudaMalloc: applications whose device memory is all owned by
 * another memory manager (a framework's caching allocator or a pool reserved
 * at start-up) and real-time or certified hosts that forbid device
 * allocation after initialisation. It runs the same blocked FP64 prefix sum
 * and comb as afqmc_population_control, but on the caller's device buffers,
 * with its scratch in a file-scope device array of
 * AFQMC_COMB_STATIC_MAX_WALKERS + 1 doubles (512 KB) that every GPU loading
 * the library holds until the process exits.
 *
 *  d_weight  [n_walkers] device, walker weights (read only)
 *  n_walkers 1 .. AFQMC_COMB_STATIC_MAX_WALKERS, else AFQMC_E_INVALID
 *  seed, run_id, step   Philox key, stream tag and step counter of the comb
 *            offset (stream 1), as in afqmc_population_control
 *  d_parent  [n_walkers] device, receives the parent index of each new walker
 *  d_wnew    [1] device, receives the common new weight sum(W)/n_walkers, or
 *            -1 (with d_parent the identity) when there is nothing to comb:
 *            every weight zero, or a NaN or infinite weight. That -1 is the
 *            call's only report of it (the kernel's own status word stays
 *            in the library's scratch array and is cleared by the next call)
 *  stream    cudaStream_t to run on (NULL: the legacy default stream)
 *
 * Asynchronous on `stream`; it calls no cudaMalloc, cudaFree or allocating
 * library routine. The first call on each device looks up the scratch
 * array's device address (with that device current) and should come before
 * any stream capture. All calls share the one array, which keeps the last
 * call's contents (the call clears what must start at zero), so calls that
 * overlap on the GPU race: serialise them, e.g. on one stream. Errors are
 * described by afqmc_last_error(NULL). */
#define AFQMC_COMB_STATIC_MAX_WALKERS 65536
afqmc_status afqmc_comb_static(const double* d_weight, int32_t n_walkers,
                               uint64_t seed, int32_t run_id, int64_t step,
                               int32_t* d_parent, double* d_wnew, void* stream);

/* Text of the last error on this context ("" if none); valid until the next
 * call on the context. ctx may be NULL for errors of afqmc_create and of the
 * context-free calls. */
const char* afqmc_last_error(const afqmc_ctx* ctx);

/* Free all device memory of the context and the stream it owns. */
void afqmc_destroy(afqmc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* AFQMC_H */
