/*
 * lise.h -- C ABI of the B300 two-component TDSLDA step (liblise.so).
 *
 * Method: arXiv:2009.00745 ("LISE"), reduced to one (u, v) pair per
 * quasiparticle state for spin-symmetric, spin-singlet pairing:
 *   i d/dt (u, v) = [[h, Delta], [Delta*, -h*]] (u, v)                 (Eq. tdslda)
 *   h = -(alpha/2) lap + beta (3 pi^2 n)^(2/3) / 2 - mu + V_ext(r, t),
 *   Delta = -g nu                                                  (Eq. pairingfield)
 *   n = 2 sum_k |v_k|^2,  nu = sum_k u_k v_k^*                    (Eqs. rho_t, nu_t)
 * on a periodic cubic lattice with spacing a (Sec. "Discretization"); the
 * Laplacian is spectral, D^(2) = F^-1[(ik)^2 F] with the Nyquist mode kept.
 * Time stepping: three steps of the order-4 series expansion with averaged
 * predictor/corrector densities (Sec. "TDSLDA / Time evolution"), then the
 * 5th-order Adams-Bashforth-Milne predictor-modifier-corrector of Eqs. p, m,
 * c, y, with 2 right-hand-side evaluations per step.  hbar = m = 1.
 *
 * Units and conventions
 *   - Lattice: nx = ny = nz = N with N in {8, 12, 16, 20, 24, 32, 40, 48, 64};
 *     site index r = (z * N + y) * N + x, x fastest.  V_ext's drive term uses
 *     z_c = (z - N/2) a.
 *   - State layout (host and device): psi[q][c][z][y][x] as interleaved
 *     (re, im) doubles, q < n_qp, c = 0 for u and c = 1 for v; that is
 *     n_qp * 2 * N^3 complex numbers, 16 bytes each.
 *   - Densities: n[r] (double), nu[r] as interleaved (re, im) doubles.
 *
 * Ownership and threading
 *   - The caller owns every host buffer passed in; the library reads or writes
 *     it only during the call (host copies complete before the call returns).
 *   - The context owns all device memory it allocates (lise_footprint_bytes
 *     tells how much); it allocates in lise_create (and lise_set_shard, which
 *     replaces the density partial-sum arrays).
 *   - A context is not thread-safe: do not use one context from two threads at
 *     once.  Different contexts are independent.
 *   - Work is enqueued on the context's stream.  lise_step returns after
 *     enqueueing; errors raised by device work are sticky and reported by the
 *     next call that synchronises (lise_sync, lise_get_state, lise_densities,
 *     lise_energy, lise_rhs) or by lise_step itself once detected.
 *
 * Status codes: every function returning int returns one of LISE_* below.
 */
#ifndef LISE_H
#define LISE_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LISE_OK 0
#define LISE_EINVAL 1     /* invalid argument (NULL pointer, unsupported lattice, dt mismatch, ...) */
#define LISE_ENOMEM 2     /* footprint above hbm_budget_bytes, or device allocation failed */
#define LISE_ECUDA 3      /* a CUDA runtime call or kernel launch failed */
#define LISE_ENONFINITE 4 /* a density or the input state is NaN or infinite */
#define LISE_ETIMEOUT 5   /* a bounded device wait ran out (the tensor-memory planes kernel's
                             wait for its MMAs, the staged pencils kernel's wait for its
                             tensor-memory-accelerator copies); sticky like LISE_ENONFINITE */
#define LISE_ESTATE 6     /* call out of order (e.g. lise_step before lise_set_state) */
#define LISE_EEXCHANGE 7  /* the shard exchange callback (lise_set_shard) returned non-zero */

#define LISE_FP64 0       /* FFTs, H psi, ABM history, densities: all in FP64 */
#define LISE_MIXED 1      /* FFTs and H psi in complex64 (FP32 accumulation), so the
                             derivatives y' are FP32 values (stored exactly in complex64);
                             the states y_n, y_{n-1}, Q and every sum with a state value
                             (y_{n+1} = Q + k1 m', Q = (y_n + y_{n-1})/2 + Y) in FP64; the
                             derivative combinations of Eqs. p, c (Y, R, p - c) and the
                             density products in FP32 (Kahan-compensated per thread, FP64
                             Neumaier across groups); m (the next H psi operand) in FP32 */
#define LISE_MIXED_STRICT 2 /* FFTs and H psi as LISE_MIXED; the whole ABM history and
                             state update in FP64: the derivative combinations as exact
                             integer sums of the FP32 derivatives rounded once to FP64, R and
                             p - c in complex128, P, Q, m and y_{n+1} in FP64 (m rounded to
                             FP32 only as the H psi operand), density products and sums in
                             FP64.  More bytes (R and p - c) and FP64 work than LISE_MIXED */

typedef struct lise_ctx lise_ctx;

typedef struct {
  int nx, ny, nz;           /* lattice; must be equal (cubic), see above */
  double dx;                /* lattice constant a > 0 */
  int n_qp;                 /* number of quasiparticle states, >= 1 */
  double alpha;             /* h contains -(alpha/2) lap */
  double beta;              /* U(n) = beta (3 pi^2 n)^(2/3) / 2 */
  double mu;                /* chemical potential (constant) */
  double g;                 /* Delta = -g nu */
  const double *v_static;   /* host array of N^3 doubles (static V_ext), or NULL; copied */
  double drive_A;           /* V_ext(r, t) += drive_A sin(drive_Omega t) z_c */
  double drive_Omega;
  int precision;            /* LISE_FP64, LISE_MIXED or LISE_MIXED_STRICT */
  int device;               /* CUDA device ordinal */
  size_t hbm_budget_bytes;  /* 0 = no limit; otherwise lise_create fails with LISE_ENOMEM
                               (allocating nothing) if the footprint exceeds it */
  void *stream;             /* cudaStream_t to enqueue on, or NULL for a stream owned by the context */
  int remove_phase;         /* 1: evolve i dpsi_k/dt = (H - eta_k) psi_k with eta_k = <psi_k|H|psi_k>
                               (trivial-phase removal, Eq. sp_en), in the right-hand sides and the
                               series start (eta_k of the step's starting state); 0: plain Eq. tdslda */
  double pair_alpha;        /* Eq. g0: g0(r) = g (1 - pair_alpha n(r) / pair_n0); 0 = constant g */
  double pair_n0;           /* reference density of Eq. g0 (> 0 when pair_alpha != 0) */
  int pair_lattice;         /* 1: lattice renormalisation of Eq. geff_3D,
                               1/g_eff = 1/g0(r) - meff (pi/dx) K / (4 pi^2), meff = 1/alpha,
                               K = 2.442749607806335; 0: g_eff = g0(r).  Delta = -g_eff nu; with a
                               density-dependent g_eff, U gains (d g_eff/dn) |nu|^2 and
                               E_pair = g_eff(n) |nu|^2 (Eq. pairing) */
  int renormalize;          /* 1: at the end of every ABM step each state is scaled to unit norm,
                               a^3 sum_r (|u|^2 + |v|^2) = 1, before its y' is formed (the optional
                               renormalisation the paper describes after Eq. sp_en); 0: off */
  double pair_ec;           /* > 0: the spherical momentum cutoff of Eq. geff at energy E_c = pair_ec,
                               1/g_eff(r) = 1/g0(r) - meff k_c/(2 pi^2) (1 - (k_F/2k_c) ln[(k_c+k_F)/(k_c-k_F)])
                               for k_F^2 >= 0 and (1 + (|k_F|/k_c) arctan(|k_F|/k_c)) for k_F^2 < 0, with
                               meff = 1/alpha, k_F^2 = 2 meff (mu - U_loc), k_c^2 = 2 meff (E_c + mu - U_loc),
                               U_loc(r) = U(n(r)) + V_ext(r, t); g_eff = g0 where k_c^2 <= 0.  U gains
                               (d g_eff/dn) |nu|^2 (through g0 and U(n)).  Requires alpha > 0,
                               pair_lattice = 0 and pair_ec <= alpha pi^2 / (2 dx^2) (the paper's bound:
                               Eq. geff does not apply above the natural cutoff of one axis); else
                               LISE_EINVAL.  0: off */
} lise_params;

/* Device bytes lise_create would allocate for these parameters (0 if invalid). */
size_t lise_footprint_bytes(const lise_params *p);

/* Validates p, allocates the device state and copies v_static.
 * Errors: LISE_EINVAL (bad parameters), LISE_ENOMEM, LISE_ECUDA. */
int lise_create(const lise_params *p, lise_ctx **out);

/* Sets y_0 = psi (host buffer, layout above) at time t0 and runs the start
 * procedure: 3 series-expansion steps of size dt (8 H psi each), storing
 * y'_k = f(t_k, y_k) for k = 0..3, so the context is at t0 + 3 dt and ready for
 * ABM steps.  dt may be negative (backward evolution) but not 0.
 * A sticky LISE_ENONFINITE or LISE_ETIMEOUT from earlier work is cleared first (the
 * new state replaces the whole history); LISE_ECUDA stays sticky.
 * Synchronises.  Errors: LISE_EINVAL, LISE_ENONFINITE (psi has NaN/Inf), LISE_ECUDA. */
int lise_set_state(lise_ctx *c, const double *psi, double t0, double dt);
/* Same with psi a device pointer (same layout) on the context's device. */
int lise_set_state_device(lise_ctx *c, const double *psi_dev, double t0, double dt);

/* Pencil-kernel tile autotuning.  The states per batch of the pencils kernel (2 or 4,
 * where the variant fits in shared memory, and 1 for the FP64 tensor-core kernel of
 * lattices with N a multiple of 16) are chosen per lattice size and precision
 * by timing the two pencils launches of an ABM step for each candidate, once per
 * process, on the first lise_set_state of that lattice and precision.  The choice
 * does not change any result (bitwise).  lise_pencil_batch returns the batch size in
 * use (the tuned one, else the default; 0 for an unsupported N or precision).
 * lise_set_pencil_batch forces qb (1, 2 or 4; LISE_EINVAL if that variant does not
 * exist) or, with qb = 0, clears the choice so that the next lise_set_state tunes. */
int lise_pencil_batch(int N, int precision);
int lise_set_pencil_batch(int N, int precision, int qb);
/* The same for the planes per block of the FFT planes kernel (the in-plane part T_xy on
 * lattices that do not use the tensor-core planes kernels: the mixed path, and FP64 with N
 * not a multiple of 16): candidates 1, 2, 4, 8 (line FFTs through shared memory) and, in the
 * FP32 compute precision with N <= 48, -1, -2, -4, -8 (the same transforms with each thread
 * holding whole lines in registers, -pb planes per block), where the variant fits in shared
 * memory and registers, tuned on the first lise_set_state of each lattice and precision;
 * results do not depend on it (the same operations in the same order for every plane).
 * lise_planes_per_block returns the value in use (0 for the tensor-core lattices or an
 * unsupported N); the setter forces pb or clears it with pb = 0 (LISE_EINVAL for a variant
 * that does not exist). */
int lise_planes_per_block(int N, int precision);
int lise_set_planes_per_block(int N, int precision, int pb);

/* Current density of Eq. j of the current state (spin factor 2):
 * j(r) = 2 sum_k Im(v_k grad v_k^*), with the spectral first derivative
 * F^-1[(ik) F] whose Nyquist coefficient is dropped (Sec. "Discretization").
 * j_out: host, 3 N^3 doubles [component x, y, z][z][y][x].  FP64 on the device
 * for both precisions; deterministic.  Synchronises.  Errors: LISE_ESTATE before
 * set_state, LISE_EINVAL (null), LISE_ENOMEM, LISE_ECUDA. */
int lise_currents(lise_ctx *c, double *j_out);

/* Boost (Eq. kick, Sec. "External boosts and external potentials"): every state
 * of the current state y(t) becomes u -> e^{i chi(r)} u, v -> e^{-i chi(r)} v, and
 * the ABM history restarts through the series start at t with the same dt (as
 * after lise_set_state; t advances by 3 dt).  chi: host, N^3 doubles [z][y][x]
 * (e.g. p.r for a velocity p/m; periodic on the lattice when p is a lattice
 * momentum).  Copies chi; synchronises.  Errors: LISE_ESTATE before set_state,
 * LISE_EINVAL (null or non-finite chi), LISE_ECUDA. */
int lise_kick(lise_ctx *c, const double *chi);

/* Enqueues n_steps >= 0 ABM steps (Eqs. p, m, c, y).  dt must equal the
 * set_state dt (the stored history is only valid for that step), else
 * LISE_EINVAL.  Errors: LISE_ESTATE before set_state, LISE_ECUDA. */
int lise_step(lise_ctx *c, int n_steps, double dt);

/* Copies the current state y_n to a host (or device) buffer.  Synchronises. */
int lise_get_state(lise_ctx *c, double *psi_out);
int lise_get_state_device(lise_ctx *c, double *psi_dev_out);

/* Current time t_n. */
int lise_get_time(lise_ctx *c, double *t);

/* Densities of the current state: n_out[N^3], nu_out[2 N^3] (host).  Synchronises. */
int lise_densities(lise_ctx *c, double *n_out, double *nu_out);

/* Energy and particle number of the current state at the current time:
 *   E = a^3 sum_r [(alpha/2) tau + (3/10) beta (3 pi^2)^(2/3) n^(5/3) + g_eff(n) |nu|^2 + V_ext n],
 *   tau = 2 sum_k |grad v_k|^2 (spectral, same Laplacian as the step; Eq. pairing
 *   gives the + g |nu|^2 term), N = a^3 sum_r n.  FP64 with compensated sums.
 * Synchronises. */
int lise_energy(lise_ctx *c, double *E, double *N);

/* One right-hand side f(t, psi) = -i H[psi](t) psi for an arbitrary host state
 * (same layout), with the potentials built from psi's own densities; written
 * to dpsi_out (host).  Uses the context's scratch arrays: it invalidates the
 * ABM history, so lise_set_state must be called again before lise_step.
 * Synchronises. */
int lise_rhs(lise_ctx *c, const double *psi, double t, double *dpsi_out);

/* Checkpoint / restart.  The paper restarts from saved wavefunctions with a new
 * series-expansion start (Sec. "Checkpoint and restart"); these calls save the
 * whole ABM history instead, so a run resumes bit-exactly:
 * y_n, y_{n-1}, y'_n..y'_{n-3}, m_{n+1}, p_n - c_n, Q, R, the potentials of
 * m_{n+1}, t and dt, behind a 64-byte header.  Host buffers; synchronise. */
size_t lise_checkpoint_bytes(const lise_ctx *c);
/* LISE_ESTATE before lise_set_state; LISE_EINVAL if bytes is too small. */
int lise_checkpoint_save(lise_ctx *c, void *buf, size_t bytes);
/* The checkpoint must come from a context with the same lattice, state count
 * and precision (else LISE_EINVAL); the physical parameters are the context's. */
int lise_checkpoint_load(lise_ctx *c, const void *buf, size_t bytes);

/* Serving: a request loop over one GPU.  Each request is an independent
 * evolution (parameters, initial state on the host, n_steps ABM steps).  A
 * worker thread admits queued requests in arrival order while the sum of their
 * footprints (lise_footprint_bytes) stays within hbm_budget_bytes and fewer
 * than max_active run; each admitted request keeps its state and ABM history
 * resident in its own context and stream; the worker enqueues steps_per_turn
 * steps at a time for every active request whose previous chunk finished, so
 * the work of different requests overlaps on the GPU.  A request's result does
 * not depend on what else runs (same deterministic kernels, own buffers). */
typedef struct lise_server lise_server;
typedef struct {
  int status;       /* LISE_OK, or the error that ended the request */
  double submit_s;  /* seconds since lise_server_create when submitted, */
  double admit_s;   /* admitted (context created, start procedure begun), */
  double done_s;    /* and finished (final state copied back) */
  double t;         /* final time of the evolution */
  double E, N;      /* energy and particle number of the final state */
} lise_request_info;
/* max_active >= 1, steps_per_turn >= 1, hbm_budget_bytes > 0. */
int lise_server_create(int device, size_t hbm_budget_bytes, int max_active, int steps_per_turn,
                       lise_server **out);
/* Copies psi (host, layout above) and queues the request; returns at once with
 * its id.  p->device, p->hbm_budget_bytes and p->stream are ignored (the server
 * sets them).  LISE_ENOMEM if the request alone exceeds the budget. */
int lise_server_submit(lise_server *s, const lise_params *p, const double *psi, double t0, double dt,
                       int n_steps, long *id);
/* Same without copying: the server reads the initial state from psi_in when it
 * admits the request and writes the final state to psi_out (may be NULL: no
 * state is copied back) when it finishes.  The caller keeps both buffers
 * (host, layout above) valid and unchanged until lise_server_wait returns for
 * this id; lise_server_wait's psi_out is then not used.  Submitting many large
 * requests this way costs no host copies and no extra host memory. */
int lise_server_submit_borrowed(lise_server *s, const lise_params *p, const double *psi_in, double *psi_out,
                                double t0, double dt, int n_steps, long *id);
/* Blocks until request id is done; copies its final state to psi_out (host;
 * may be NULL) and its timings to info (may be NULL); forgets the request.
 * Returns the request's status. */
int lise_server_wait(lise_server *s, long id, double *psi_out, lise_request_info *info);
/* Non-blocking: *done = 1 if request id has finished (lise_server_wait then
 * returns at once), else 0.  LISE_EINVAL for an unknown id. */
int lise_server_poll(lise_server *s, long id, int *done);
/* Admission order.  LISE_ADMIT_FIFO (the default): strictly in arrival order,
 * a request that does not fit the free budget holds back all later ones.
 * LISE_ADMIT_FIRST_FIT: the first queued request (in arrival order) that fits
 * is admitted; a request passed over max_skips times holds back later ones
 * until it is admitted (bounded waiting).  max_skips >= 0 (ignored for FIFO). */
#define LISE_ADMIT_FIFO 0
#define LISE_ADMIT_FIRST_FIT 1
int lise_server_set_admission(lise_server *s, int policy, int max_skips);
/* Batched stepping (off by default; set before the first submission, else LISE_ESTATE):
 * the active requests of each FP32 compute precision (LISE_MIXED, LISE_MIXED_STRICT;
 * without remove_phase or renormalize) are stepped together through one lise_batch,
 * rebuilt whenever a request joins (once its series start has finished) or leaves; the
 * others are stepped one by one.  Results are unchanged (bitwise). */
int lise_server_set_batching(lise_server *s, int enable);
/* Largest sum of admitted footprints and largest number of active requests seen. */
int lise_server_stats(lise_server *s, size_t *peak_used_bytes, int *peak_active);
/* Finishes every submitted request, stops the worker and frees the server. */
void lise_server_destroy(lise_server *s);

/* Batched evolutions: several contexts (any lattice sizes and state counts) of the FP32
 * compute precision (all LISE_MIXED or all LISE_MIXED_STRICT, on one device, without
 * remove_phase, renormalize or sharding), each after lise_set_state, stepped together.
 * Every kernel of an ABM step runs as one launch per lattice size over all evolutions of
 * that size (a device work table maps each block to an evolution and state group), and
 * four steps are captured as one CUDA graph; each evolution keeps its own dt, drive and
 * time.  The arguments are those lise_step uses, so every evolution's result is bitwise
 * the same as stepping its context alone.  No counterpart in the paper, which batches
 * the FFTs of one evolution's states (Sec. "FFT in batch").
 * lise_batch_create waits for the contexts' pending work and builds the work tables
 * (device memory owned by the batch).  While a context belongs to a live batch, use it
 * only through the batch until lise_batch_sync (or lise_batch_destroy) returns; after
 * that every context call works as usual (the contexts' times and histories have moved
 * on), and a context stepped on its own can no longer be stepped by the batch
 * (LISE_ESTATE).  lise_batch_step enqueues n_steps steps of every member on the batch's
 * stream; lise_batch_sync waits and reports the first member's sticky error.
 * Errors: LISE_EINVAL (null, duplicate or unsuitable contexts), LISE_ESTATE (a context
 * without a state, or moved on outside the batch), LISE_ENOMEM, LISE_ECUDA. */
typedef struct lise_batch lise_batch;
int lise_batch_create(lise_ctx *const *ctxs, int n, lise_batch **out);
int lise_batch_step(lise_batch *b, int n_steps);
int lise_batch_sync(lise_batch *b);
void lise_batch_destroy(lise_batch *b);

/* Per-launch timing.  Kernel classes of the path: */
#define LISE_KC_PLANES 0    /* in-plane 2D FFT -> kinetic multiply -> inverse (T_xy) */
#define LISE_KC_PENCILS 1   /* z-pencil FFT, BdG apply and the fused ABM / series epilogue */
#define LISE_KC_REDUCE 2    /* density reduction over state groups and the potentials */
#define LISE_KC_POINTWISE 3 /* start-up predictor, plain density and input checks */
#define LISE_KC_COUNT 4
/* enable = 1 records a CUDA event pair on the context's stream around every
 * kernel launch from now on (and clears earlier records); 0 stops recording. */
int lise_profile(lise_ctx *c, int enable);
/* Launch count and summed device time (ms) of one kernel class since profiling
 * was enabled.  Synchronises.  LISE_EINVAL for an unknown class. */
int lise_profile_read(lise_ctx *c, int kernel_class, long *launches, double *total_ms);
/* Name of a kernel class ("planes", "pencils", ...), or NULL. */
const char *lise_kernel_class_name(int kernel_class);

/* Waits for enqueued work and reports sticky errors. */
int lise_sync(lise_ctx *c);

/* Sharded densities: the states of one evolution split over several contexts (one per GPU
 * or process), as the paper splits the quasiparticle wavefunctions over GPUs and sums the
 * partial densities over all of them before the potentials are built (Sec. "CPU-GPU
 * hybrid structure"; Eqs. rho_t, nu_t are sums over all states).
 * Each context holds n_qp of the states.  Its density sums run in groups of group_size
 * states (the same on every shard); the groups of all shards, in the order of the states,
 * are numbered 0 .. n_groups_all - 1 and this context's are first_group ..
 * first_group + ceil(n_qp / group_size) - 1.  The partial sums are kept for all groups,
 * as three arrays [n_groups_all][N^3] (n, Re nu, Im nu) in one block `parts` of
 * 3 n_groups_all N^3 doubles.  Before every density reduction (two per ABM step, the
 * start, lise_densities, lise_energy, lise_currents, lise_rhs) the library calls
 *   exchange(user, parts, on_device, stream, N^3, first_group, n_local, n_groups_all)
 * on the calling thread, with this context's groups filled in; the callee fills in every
 * other group (from the other shards) and returns 0, or non-zero to fail the call with
 * LISE_EEXCHANGE.  on_device = 1: parts is the device block and the callee enqueues its
 * transfers (e.g. NCCL collectives) on `stream` (a cudaStream_t); capturable = 1 lets
 * lise_step capture them into its CUDA graphs.  on_device = 0: parts is a pinned host
 * copy (the library copies this context's groups out first and the whole block back
 * afterwards; stream is NULL) and lise_step uses no graphs.  Each group is summed in a
 * fixed order and the groups are reduced in their global order, so a sharded evolution
 * gives bit-for-bit the result of one context holding all states with the same
 * group_size.  With exchange = NULL the call only sets the group size (n_groups_all must
 * then equal this context's group count, first_group 0).
 * lise_set_shard replaces the partial-sum arrays (device, and pinned host memory for a host
 * exchange) and invalidates the history: call it before lise_set_state.  Every shard
 * must make the same sequence of calls.  Errors: LISE_EINVAL (group_size outside
 * 1..64, a group range outside 0..n_groups_all), LISE_ENOMEM, LISE_ECUDA. */
typedef int (*lise_exchange_fn)(void *user, double *parts, int on_device, void *stream, long nxyz,
                                int first_group, int n_groups_local, int n_groups_all);
typedef struct {
  int group_size;             /* states per density group, 1..64, equal on all shards */
  int first_group;            /* this context's first group among all shards' groups */
  int n_groups_all;           /* groups over all shards */
  lise_exchange_fn exchange;  /* NULL: no other shard (sets the group size only) */
  void *user;                 /* passed to exchange */
  int on_device;              /* 1: exchange works on the device block, 0: on a host copy */
  int capturable;             /* on_device only: 1 if the enqueued transfers can be graph-captured */
} lise_shard;
int lise_set_shard(lise_ctx *c, const lise_shard *s);

/* Bounded device waits.  The kernels that wait on the hardware (the tensor-memory planes
 * kernel for its MMAs, the staged pencils kernel for its tensor-memory-accelerator copies)
 * give up after a number of polls of their barrier, set the context's error word and
 * stop; the next synchronising call then reports LISE_ETIMEOUT.  polls > 0 sets that
 * number, polls == 0 makes every such wait give up at once (a way to exercise this error
 * path), polls < 0 restores the default (4194304 polls, far beyond any healthy wait).  A
 * block that gives up still lets the MMAs and copies it has in flight finish before it
 * frees its tensor memory and exits.  Applies to work enqueued after the call
 * (synchronises the context's stream when the limit changes).  Errors: LISE_EINVAL
 * (null context), LISE_ECUDA. */
int lise_set_wait_limit(lise_ctx *c, long polls);

/* Static description of a status code. */
const char *lise_strerror(int status);

/* Frees the context and its device memory (synchronises first).  NULL is a no-op. */
void lise_destroy(lise_ctx *c);

/* ---- Measurement (no counterpart in the paper) ----
 * FP64 fused multiply-add throughput of `device` under its current clock (TFLOP/s, an FMA
 * counts 2), timed with CUDA events on a kernel of independent FMA chains (best of 5
 * launches of about 10 ms after a warm-up): the denominator of the FP64-pipe fraction of
 * the benchmark's roofline.  Errors: LISE_EINVAL (null pointer, no such device), LISE_ECUDA. */
int lise_measure_fp64_peak(int device, double *tflops);

/* ---- Right-hand side without any allocation (no counterpart in the paper) ----
 * For callers that must not allocate device memory while they run: a host
 * framework whose caching allocator already holds the free device memory (a
 * stray cudaMalloc would fail or fragment its pool), latency-critical loops
 * that cannot afford cudaMalloc's implicit device synchronisation, plug-ins
 * that are handed only buffers and a stream.  It computes the same
 * f(t, psi) = -i H[psi](t) psi as lise_rhs, from the device buffer psi_dev to
 * the device buffer dpsi_dev (layout as above, on device p->device, enqueued on
 * p->stream, NULL = the default stream), with no context and no cudaMalloc,
 * cudaFree or other allocating call.  All scratch lives in one fixed device
 * array of LISE_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds
 * until the process exits.
 *   Capacity: 32 n_qp N^3 bytes (FP64; 16 for LISE_MIXED) for the in-plane
 *   kinetic part, 24 G N^3 for density partials (G = groups of <= 64 states),
 *   56 N^3 for densities, potentials and V_ext, plus small tables, each part
 *   rounded up to 256 bytes.  A problem that needs more returns LISE_ENOMEM
 *   (e.g. FP64 16^3 fits about 400 states, 32^3 about 50).
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current); make that first call
 *   before any stream capture.
 *   Sharing: every call reuses the same array and leaves its contents behind
 *   (the error word is cleared at the start of each call); calls that overlap
 *   on the GPU (other streams, other host threads) race on it, so serialise
 *   them.  p->hbm_budget_bytes is ignored.  Synchronises p->stream.
 *   Errors: LISE_EINVAL (the checks of lise_create, or a null buffer), LISE_ENOMEM (too
 *   large for the array), LISE_ECUDA, LISE_ENONFINITE (a density is NaN or infinite),
 *   LISE_ETIMEOUT (a bounded device wait ran out). */
#define LISE_NOALLOC_SCRATCH_BYTES (64u << 20)
int lise_rhs_noalloc(const lise_params *p, const double *psi_dev, double t, double *dpsi_dev);

#ifdef __cplusplus
}
#endif
#endif
