/*
 * nbody.h - C ABI of libnbody, a GB300 (sm_103a) implementation of the
 * fourth-order Hermite scheme with hierarchical (block) individual
 * timesteps of Tanikawa, Yoshikawa, Okamoto & Nitadori (arXiv:1104.2700),
 * Sec. 2, whose O(n_act * N) force evaluation (Sec. 3, Eqs. acc, jrk, pot)
 * runs in hand-written CUDA kernels.
 *
 * Conventions for every call
 *   - Every call returns an nb_status; nothing throws across the ABI.  After
 *     a failure nb_last_error() describes it.  A failure is sticky: every
 *     later call on the context returns the same status until
 *     nb_set_particles() or nb_set_state() reloads the system.
 *   - Host arrays are read or written during the call and never kept.
 *     Device arrays (on_device = 1) must be device memory of the context's
 *     device; the call is then stream-ordered on the context stream and may
 *     return before the GPU finishes (nb_synchronize() waits).
 *   - Vectors are n x 3 row-major doubles: component c of particle i is
 *     element 3*i + c.  Particle indices are int32 in [0, n).
 *   - A context is not thread-safe; different contexts are independent.
 *   - Units are whatever the caller uses; G is part of the configuration.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_ctx nb_ctx; /* opaque; owns all device memory it allocates */

typedef enum nb_status {
    NB_OK = 0,
    NB_EINVAL = 1,     /* bad argument (size, pointer, value out of range)   */
    NB_ECUDA = 2,      /* a CUDA runtime call failed                          */
    NB_ENOMEM = 3,     /* device or pinned host allocation failed             */
    NB_ENONFINITE = 4, /* a force, jerk or timestep came out NaN or infinite  */
    NB_EDTMIN = 5,     /* a timestep fell below dt_min                        */
    NB_ETIMEOUT = 6,   /* a bounded device-side wait gave up                  */
    NB_ESTATE = 7      /* call out of order (no particles, mismatched block)  */
} nb_status;

/* Precision of the force evaluation (Sec. 3.2 "Arithmetic precision").
 *   NB_FP64   every operation in double precision (the baseline path).
 *   NB_MIXED  the paper's mixed scheme on FP32 pipes: r_ij from double-single
 *             positions, the pair arithmetic in FP32 with a hardware rsqrt,
 *             FP32 partial sums per j tile folded into compensated
 *             (double-single) accumulators.  Fastest; per-particle relative
 *             errors follow the FP32 rounding of each pair.
 *   NB_DS     the same pair formulas in double-single (float-float)
 *             arithmetic built from error-free FP32 transforms.
 *   NB_HYBRID no counterpart in the paper: FP32 pairs (refined rsqrt, FP32
 *             runs of 16 j folded into double-single sums) except near pairs,
 *             whose acceleration or jerk term could exceed 10 % of the
 *             particle's own |a| or |j| (from its state a, j); those are
 *             evaluated in double-single.  A particle whose state has
 *             a = j = 0 (the evaluation inside nb_set_particles) treats every
 *             pair as near.  Errors stay well inside 1e-6 per particle on the
 *             measured workloads at ~2.5x the DS throughput.  Integration
 *             guard: each evaluation also stores a per-particle estimate of
 *             its FP32 far-field noise; a particle whose noise would reach
 *             3 % of the crackle scale of its step (eta |j| dt / 12) is
 *             evaluated entirely in DS next time, so the Aarseth timesteps
 *             keep the DS schedule.  The default.
 *   NB_MIXED_SPJ  NB_MIXED, except that the jerk is summed in plain FP32
 *             across each warp's whole run of j (up to all N), as the
 *             paper's production kernel does (Sec. 4, Fig. err_snp_djerk);
 *             acceleration and potential are bit-identical to NB_MIXED under
 *             the same launch shape.  For the accumulation study; its jerk
 *             error grows with N.
 *   NB_HYBRID_SPJ  NB_HYBRID, except that the jerk of the far pairs is summed
 *             in plain FP32 across each warp's whole run of j instead of in
 *             runs folded into double-single sums (the same accumulation
 *             study on the precision that integrates; near pairs and the
 *             acceleration and potential as in NB_HYBRID).
 *   NB_FP64_HERMITE6  not the paper's scheme but the sixth-order Hermite
 *             scheme beside it (Nitadori & Makino 2008), in FP64: the same
 *             block timesteps, the force evaluation also giving the snap
 *             (the second time derivative of Eq. acc along the predicted
 *             trajectories, from the predicted accelerations), the predictor
 *             carried to crackle, the corrector from the quintic Hermite
 *             interpolant of a(t), the timestep
 *             eta ((|a||s| + |j|^2) / (|c||x| + |d|^2))^(1/6) with c, d, x
 *             the interpolant's third to fifth derivatives.  eta near 0.1
 *             gives the energy error the fourth-order scheme reaches at
 *             eta = 0.02 in about a third of the steps.  One system only
 *             (no ensembles, no snapshots); nb_set_state needs every t_i
 *             equal; nb_correct takes the last nb_force results only. */
typedef enum nb_precision {
    NB_FP64 = 0,
    NB_MIXED = 1,
    NB_DS = 2,
    NB_HYBRID = 3,
    NB_MIXED_SPJ = 4,
    NB_HYBRID_SPJ = 5,
    NB_FP64_HERMITE6 = 6
} nb_precision;

typedef struct nb_config {
    int32_t precision;    /* nb_precision                                       */
    int32_t device;       /* CUDA device ordinal                                */
    double G;             /* gravitational constant (Eq. eom)                   */
    double eta_start;     /* first step: dt = eta_start |a|/|j|                 */
    double dt_max;        /* largest timestep; must be a power of two           */
    double dt_min;        /* smallest timestep allowed (NB_EDTMIN below it)     */
    void* stream;         /* cudaStream_t to run on; NULL = a private stream    */
    int32_t i_per_thread; /* force kernel register blocking; 0 = default        */
    int32_t ctas_per_sm;  /* persistent force CTAs per SM; 0 = default          */
    int32_t autotune;     /* 1: run nb_autotune after every load                */
    int32_t j_split;      /* lanes per i particle: the j range of each tile is
                           * split over 1, 2, 4 or 8 lanes of a warp and the
                           * partial sums are added with warp shuffles (a
                           * group then holds 32 / j_split i); 0 = default 1.
                           * Values above 1 need i_per_thread 0 or 1; any
                           * other value, or 2 i per thread with a split, is
                           * NB_EINVAL at nb_create.                        */
    int64_t wait_limit_cycles; /* GPU clock cycles a force kernel waits for
                              * one staged j tile before it gives up and the
                              * call fails with NB_ETIMEOUT; 0 = about one
                              * second.  Tests set it tiny to exercise the
                              * failure path without faulting the GPU. */
} nb_config;

/* Fill *cfg with the defaults: NB_HYBRID, device 0, G = 1, eta_start = 0.01,
 * dt_max = 1/16, dt_min = 2^-40, private stream, default launch shapes, no
 * autotuning. */
void nb_config_init(nb_config* cfg);

/* Launch shapes of the force kernel (i-tile per lane, j-split inside a warp
 * and over warps): blocks of fewer than nact_split active particles use the
 * "small" shape, others the "large" one.  When tiny_split > 0, a force call
 * whose block size the host knows (nb_force with n_act >= 0) on fewer than
 * tiny_split particles uses a third, "tiny" shape; a block step, whose size
 * is on the device, launches the small and the large shape as two parallel
 * branches (one returns at once) and never the tiny one, since a third
 * branch costs a block step more than the shape saves.  i_per_thread is the
 * i-tile per lane; j_split the lanes that share one i, each taking every
 * j_split-th j of a tile (an i-group is 32 * i_per_thread / j_split
 * particles); ctas_per_sm sets the persistent grid, which fixes how far each
 * i-group's j range is split across warps.  An ensemble context uses one
 * i-tile and one j split for both shapes (its force plan is cut once per
 * block) and no tiny shape.  An ensemble's force launch cuts its (i-group,
 * j tile) pairs into ens_chunks chunks per warp: with 1 each warp takes one
 * contiguous range; with more (by default 4 for the hybrid precisions,
 * whose tiles differ several-fold in cost), each warp's first chunk is its
 * own and the rest go to warps in the order they come free.  The *_us
 * fields give the force time the autotuner measured for the chosen shapes
 * on their probe blocks (tiny_us 0 without a tiny shape). */
typedef struct nb_tuning {
    int32_t small_i_per_thread;
    int32_t small_ctas_per_sm;
    int32_t large_i_per_thread;
    int32_t large_ctas_per_sm;
    int32_t nact_split;
    int32_t small_j_split;
    int32_t large_j_split;
    double small_us;
    double large_us;
    int32_t tiny_split;   /* 0: no tiny shape */
    int32_t tiny_i_per_thread;
    int32_t tiny_ctas_per_sm;
    int32_t tiny_j_split;
    double tiny_us;
    int32_t ens_chunks;   /* ensembles: stream-K chunks per warp, 1-4 (0: the
                           * default, 4 for the hybrid precisions, else 1) */
} nb_tuning;

/* Autotuner.  The paper compares blockings of its force loop (i by j
 * particles per AVX register) by measurement and fixes the fastest (Sec.
 * 3.3); this makes that comparison at run time, on the loaded workload.  It
 * times every candidate launch shape of the force kernel on probe blocks of
 * 32, 96, 256, 2048 and min(n, 65536) particles, spread evenly over the
 * context's stored order (nb_spatial_order) like the scattered members of a
 * block step (for the hybrid precision with the integration guard idle, as
 * in a steady integration), and keeps the fastest for each bucket, with the
 * bucket boundary nact_split at 1024 (probes up to 256 small) or 4096 (2048
 * small too), whichever gives the least total.  A single system then may
 * take a tiny shape (tiny_split 64: probe 32; 160: probes 32 and 96), kept
 * only when it beats the small shape on those probes by more than 0.5 us.
 * Predicts all particles to the time of particle 0 first, so call
 * nb_predict again before nb_force.  *out (may be NULL) receives the choice.
 * Blocks.  Errors: NB_ESTATE (nothing loaded), NB_ECUDA. */
nb_status nb_autotune(nb_ctx* ctx, nb_tuning* out);

/* Set the force launch shapes by hand (a fixed blocking, as Sec. 3.3
 * fixes its own), e.g. ones an earlier nb_autotune returned for the same
 * workload (its *_us fields are ignored).  Each shape
 * used (the tiny one only when tiny_split > 0) must name a built kernel
 * (i_per_thread 1 or 2, j_split 1, 2, 4 or 8; 2 i per thread only with j
 * split 1) and 1 to its occupancy of CTAs per SM; 0 <= tiny_split <
 * nact_split; 0 <= ens_chunks <= 4.  An ensemble context takes equal small
 * and large i-tiles and j splits and tiny_split 0.  The shapes hold until
 * the next nb_autotune (a context created with autotune = 1 retunes on
 * every load).  Errors:
 * NB_EINVAL (shape or boundary out of range; nothing changes), NB_ECUDA. */
nb_status nb_set_tuning(nb_ctx* ctx, const nb_tuning* tuning);

/* Self-test of failure detection (no counterpart in the paper): run one
 * force launch in which no warp stages its first j tile, so that tile's
 * bounded wait runs out (~0.1 ms), exactly as it would if a copy never
 * arrived.  Each warp then lets its other copies land and returns.  Returns
 * NB_ETIMEOUT when the kernel reported the timeout (the expected outcome),
 * NB_OK if it did not.  The context stays usable (status and counters are
 * cleared; the error is not sticky); the force outputs are not meaningful.
 * Blocks. */
nb_status nb_selftest_timeout(nb_ctx* ctx);

/* Create a context on cfg->device.  *out receives the handle.
 * Errors: NB_EINVAL (NULL pointer, dt_max not a power of two, unknown
 * precision), NB_ECUDA (no such device). */
nb_status nb_create(const nb_config* cfg, nb_ctx** out);

/* Release every resource of the context (NULL is accepted). */
nb_status nb_destroy(nb_ctx* ctx);

/* Load a system (Sec. 2 set-up): masses m[n], positions r[n][3] and
 * velocities v[n][3] (host arrays, copied), softening eps (Eq. eom) and the
 * Aarseth accuracy parameter eta (Eq. timestep).  Sets t_i = 0, evaluates
 * a, j on every particle (Eqs. acc, jrk) and the first timesteps
 * dt_i = pow2_floor(min(eta_start |a_i|/|j_i|, dt_max)).  Blocks until done.
 * Errors: NB_EINVAL (n < 1, n > 2^31 - 1, eps < 0, eta <= 0, NULL array),
 * NB_ENOMEM, NB_ENONFINITE (e.g. eps = 0 with two particles at one point). */
nb_status nb_set_particles(nb_ctx* ctx, int64_t n, const double* m, const double* r,
                           const double* v, double eps, double eta);

/* Load a full Hermite state: m[n], r, v, a, j [n][3], t[n], dt[n] (the
 * checkpoint/resume entry point).  Arrays are host memory, or device memory
 * when on_device = 1.  Every dt_i must be a power of two <= dt_max and t_i a
 * multiple of dt_i; this is the caller's responsibility.
 * Errors: NB_EINVAL, NB_ENOMEM. */
nb_status nb_set_state(nb_ctx* ctx, int64_t n, const double* m, const double* r,
                       const double* v, const double* a, const double* j,
                       const double* t, const double* dt, double eps, double eta,
                       int32_t on_device);

/* Copy the state out (any pointer may be NULL to skip that array).  Host
 * arrays block until written; device arrays are stream-ordered. */
nb_status nb_get_state(nb_ctx* ctx, double* r, double* v, double* a, double* j,
                       double* t, double* dt, int32_t on_device);

/* Sixth-order variant only (NB_FP64_HERMITE6): the snap s[n][3] and
 * crackle c[n][3] of every particle at its own time t_i (either pointer may
 * be NULL), host or device arrays as in nb_get_state.  Errors: NB_ESTATE
 * (another precision, or nothing loaded). */
nb_status nb_get_snap(nb_ctx* ctx, double* s, double* c, int32_t on_device);

/* Device snapshot of the whole Hermite state (no counterpart in the paper):
 * a rollback point that never leaves the GPU.  nb_snapshot_bytes() is the
 * size of one snapshot of the loaded system (0 if none is loaded).
 * nb_snapshot copies m, x, v, a, j, t, dt, the per-particle derived data
 * (next-time keys, hybrid noise estimates), the layout bounds and the
 * context's spatial order (nb_spatial_order) into the caller's device
 * buffer `buf` (at least nb_snapshot_bytes, 16-byte aligned); nb_restore
 * copies such a snapshot back.  Both are one kernel on
 * the context stream, asynchronous and capturable in a CUDA graph.  A
 * snapshot belongs to the system it was taken from (same n and, for an
 * ensemble, the same systems); restoring into another is undefined.
 * Errors: NB_ESTATE (nothing loaded), NB_EINVAL (NULL or misaligned buf). */
int64_t nb_snapshot_bytes(const nb_ctx* ctx);
nb_status nb_snapshot(nb_ctx* ctx, void* buf);
nb_status nb_restore(nb_ctx* ctx, const void* buf);

/* Steps 2-3 (Eqs. xpred, vpred): predict every particle to time t into the
 * layout the force kernel streams.  Asynchronous. */
nb_status nb_predict(nb_ctx* ctx, double t);

/* Step 1: t_next = min_i (t_i + dt_i) and the active block, every i with
 * t_i + dt_i == t_next, in ascending index order.  If t_next > t_end the
 * block is empty.  *t_next and *n_act are written (host); idx (host, may be
 * NULL, capacity n) receives the block.  Blocks until done. */
nb_status nb_select(nb_ctx* ctx, double t_end, double* t_next, int32_t* n_act,
                    int32_t* idx);

/* Step 4 (Eqs. acc, jrk, pot): acceleration acc[n_act][3], jerk
 * jerk[n_act][3] and potential pot[n_act] of the particles idx[0..n_act)
 * from every particle j != i at the last predicted time (nb_predict).  Any
 * output pointer may be NULL.  With on_device = 0, idx and the outputs are
 * host arrays and the call blocks; with on_device = 1 they are device arrays
 * and the call is stream-ordered.  The results are also kept for
 * nb_correct.
 * Order: the force kernel cuts its i-groups from the list as it receives
 * it.  A host list is first put in the context's spatial order
 * (nb_spatial_order), as the lists of nb_block_step are, and the outputs
 * are returned in the caller's order; a device list is processed in its own
 * order, so a device list in spatial order is the fast one (and gives the
 * same bits as the same particles given as a host list).  Results are
 * reproducible for a given list; another order of the same particles may
 * change the last bits.
 * Errors: NB_EINVAL (n_act < 0 or > n, bad index), NB_ESTATE (no particles
 * loaded). */
nb_status nb_force(nb_ctx* ctx, int32_t n_act, const int32_t* idx, double* acc,
                   double* jerk, double* pot, int32_t on_device);

/* Steps 5-8 for the block idx[0..n_act) whose particles are all due at time
 * t (t_i + dt_i == t): Hermite interpolation (snap, crackle), corrector,
 * a0 <- a1, j0 <- j1, t_i <- t, new power-of-two timestep from Eq. timestep.
 * acc/jerk are the new a1, j1 ([n_act][3], host or device per on_device);
 * NULL for both uses the last nb_force results (same n_act required).
 * Blocks when on_device = 0.  Errors: NB_EINVAL, NB_ESTATE, NB_ENONFINITE,
 * NB_EDTMIN (reported after the work completes). */
nb_status nb_correct(nb_ctx* ctx, double t, int32_t n_act, const int32_t* idx,
                     const double* acc, const double* jerk, int32_t on_device);

/* One block step (steps 1-8) entirely on the device, no host round trip:
 * select, predict, force, correct.  Does nothing once t_next > t_end.
 * Asynchronous; device errors surface at the next blocking call. */
nb_status nb_block_step(nb_ctx* ctx, double t_end);

/* Integrate (steps 1-9 of Sec. 2) until every particle reaches t_end; with
 * t_end a multiple of dt_max all particles end synchronised at t_end.
 * *n_steps / *n_interactions (may be NULL) receive the block steps and the
 * interactions (n_act * n per block, self pair counted) of this call.
 * Blocks.  Errors: NB_ENONFINITE, NB_EDTMIN, NB_ETIMEOUT. */
nb_status nb_step_until(nb_ctx* ctx, double t_end, uint64_t* n_steps,
                        uint64_t* n_interactions);

/* Energy diagnostic at a synchronised time: kinetic sum 1/2 m v^2 and
 * potential 1/2 sum m_i phi_i (Eq. pot).  With fp64_potential = 1 the
 * potential is summed in FP64 whatever the context precision.  Blocks. */
nb_status nb_energy(nb_ctx* ctx, int32_t fp64_potential, double* kin, double* pot);

/* Wait for all work queued on the context stream and report device errors. */
nb_status nb_synchronize(nb_ctx* ctx);

/* Load an ensemble of k independent systems (Sec. 2 set-up, applied to each
 * system on its own).  System q owns particles [offsets[q], offsets[q+1])
 * of the concatenated host arrays m[n], r[n][3], v[n][3] (n = offsets[k],
 * offsets[0] = 0, every system non-empty) and has softening eps[q]; all
 * share G (configuration) and eta.  Particles of different systems never
 * interact.  Each system keeps its own block schedule: one block step
 * (nb_block_step, nb_step_until) advances every system whose next block time
 * is within t_end by one block, all of them in the same kernel launches.
 * nb_force then needs idx strictly ascending; nb_correct is not available.
 * Errors: NB_EINVAL (k < 1, empty system, eps < 0, eta <= 0), NB_ENOMEM,
 * NB_ENONFINITE. */
nb_status nb_set_ensemble(nb_ctx* ctx, int32_t k, const int64_t* offsets, const double* m,
                          const double* r, const double* v, const double* eps, double eta);

/* Energy of each system at a synchronised time: kin[q] = sum 1/2 m v^2 and
 * pot[q] = 1/2 sum m phi over system q (Eq. pot), k entries each (one for a
 * single system).  fp64_potential as in nb_energy.  Blocks. */
nb_status nb_energy_systems(nb_ctx* ctx, int32_t fp64_potential, double* kin, double* pot);

/* Number of systems loaded (1 after nb_set_particles, k after
 * nb_set_ensemble, 0 before either). */
int32_t nb_num_systems(const nb_ctx* ctx);

/* j-partitioned force (the paper's parallel scheme splits the j sum of
 * Eqs. acc, jrk, pot over processes, Sec. 4-5): from this call on, every
 * force evaluation of the context precision (nb_force and the force step of
 * nb_block_step / nb_step_until) sums only over part `part` of `parts`
 * contiguous ranges of the j layout's tiles (tiles [T part / parts,
 * T (part + 1) / parts) of the T = ceil(n / 64) tiles, in the context's
 * stored order).  The parts of all `parts` contexts holding the same state
 * add up to the whole force; a distributed driver keeps the state
 * replicated, sums acc, jerk and pot over the parts (one all-reduce of
 * 7 n_act doubles per block step) and then corrects (nb_correct with the
 * summed acc / jerk).  nb_energy, nb_autotune and the load-time
 * evaluations always use every j.  With the hybrid precision each part
 * keeps its own far-field noise estimates (the integration guard acts on
 * its part).  part 0 of 1 (the default, restored by every load) is the
 * whole sum.  Errors: NB_EINVAL (part outside [0, parts), more parts than
 * tiles, an ensemble), NB_ESTATE (nothing loaded). */
nb_status nb_set_j_part(nb_ctx* ctx, int32_t part, int32_t parts);

/* The context's spatial order (no counterpart in the paper): the context
 * stores its particles in this order, order[k] being the caller's index of
 * the k-th stored particle (n host entries).  Within each system the
 * particles follow a space-filling (Morton) curve through the system's
 * bounding box, so consecutive particles are close in space; the force
 * kernel's j tiles and the i-groups it cuts from a list are then compact,
 * which the hybrid precision's far-tile path needs.  Every index the calls
 * take or return is the caller's; the order only changes the summation
 * order.  It is computed from the positions at every load and at the start
 * of every nb_step_until (a pure function of those positions, so a run
 * resumed from a checkpoint gets the order the original had), and
 * nb_restore restores the order stored with the snapshot.  Blocks.
 * Errors: NB_ESTATE (nothing loaded), NB_EINVAL (NULL order). */
nb_status nb_spatial_order(nb_ctx* ctx, int32_t* order);

/* Number of particles loaded (0 before nb_set_particles). */
int64_t nb_num_particles(const nb_ctx* ctx);

/* Description of the last failure on ctx ("" if none); valid until the
 * next call on ctx. */
const char* nb_last_error(const nb_ctx* ctx);

/* Static name of a status code. */
const char* nb_status_string(nb_status s);

/* Force evaluation that allocates no memory.  The paper has no counterpart:
 * this is a service for callers that cannot allocate device memory, for
 * example a host framework that owns every device allocation and forbids
 * others, or a process whose GPU memory is already fully reserved.
 * The calls above keep their buffers in a context that nb_set_particles
 * sizes with cudaMalloc; this one keeps nothing between calls and never
 * calls cudaMalloc, cudaFree or an allocating library routine.
 *
 * It computes what nb_force computes in NB_DS precision (Eqs. acc, jrk,
 * pot): acc[n_act][3], jerk[n_act][3] and pot[n_act] of the particles
 * idx[0..n_act) from every particle j != i, given masses m[n], positions
 * r[n][3] and velocities v[n][3] (already at the wanted time), softening
 * eps and constant G.  All pointers are device memory of the current
 * device; the work runs on `stream` (a cudaStream_t, NULL = legacy default)
 * and the call returns after it has finished.
 *
 * Its only working memory is one fixed device array of
 * NB_STATIC_SCRATCH_BYTES inside the library, held on each GPU where it has
 * been materialised until the process exits.  Limit: n <= NB_STATIC_MAX_N
 * on any GPU (the force kernel's grid is sized so that this holds whatever
 * the SM count); larger n returns NB_EINVAL with a message on stderr.
 *
 * First call on a device: a one-time set-up (the array's device address,
 * kernel attributes).  Under the CUDA runtime's default lazy module
 * loading, that is also when the driver loads this part of the library onto
 * the device and so reserves the array's NB_STATIC_SCRATCH_BYTES: a caller
 * that later reserves all remaining GPU memory must make its first call (a
 * call with n_act = 0 is enough) before it does so, and before any stream
 * capture.  Later calls allocate nothing.
 *
 * Every call synchronises `stream` to read back the kernel's status word, so
 * the call cannot be made while `stream` is being captured into a graph.
 * Every call shares the array: calls that overlap on the GPU (other
 * threads, other streams) race and must be serialised by the caller.
 * Errors: NB_EINVAL (sizes, NULL pointers, an index outside [0, n)),
 * NB_ECUDA, NB_ETIMEOUT. */
#define NB_STATIC_MAX_N 131072
#define NB_STATIC_SCRATCH_BYTES (32 * 1024 * 1024)
nb_status nb_force_static(int64_t n, const double* m, const double* r, const double* v,
                          double eps, double G, int32_t n_act, const int32_t* idx,
                          double* acc, double* jerk, double* pot, void* stream);

/* Calibration, with no counterpart in the paper: the measured FP32 and FP64
 * fused-multiply-add throughput of `device` in TFLOP/s (an FMA counts as 2
 * flop), from independent FMA chains on every SM, best of 3 timed launches
 * (~20 ms each on GB300).  These are the denominators for the
 * force kernels' ALU roofline.  Blocks; allocates and frees its own scratch;
 * restores the caller's current device.  Errors: NB_EINVAL (NULL output or
 * bad device), NB_ECUDA. */
nb_status nb_measure_peaks(int32_t device, double* fp32_tflops, double* fp64_tflops);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
