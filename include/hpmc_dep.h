/*
 * hpmc_dep.h — C ABI of the GB300 implicit-depletant hard-particle Monte Carlo
 * library (libhpmc_dep.so).
 *
 * The method is that of Glaser, Karas & Glotzer, "A parallel algorithm for
 * implicit depletant simulations" (arXiv:1508.07077):
 *   - N hard colloids in a cubic periodic box of side L, in a grand-canonical
 *     bath of ideal-gas (penetrable) depletants of diameter q and fugacity
 *     z_p, sampled with the semigrand weight exp(z_p V_f - beta H_cc)
 *     (Sec. III.A, Eq. 2);
 *   - single-colloid trial moves in a checkerboard of active cells
 *     (Sec. III.E); for each move a Poisson number of depletants is inserted
 *     in the circumsphere of the moved colloid's new pose (Sec. III.B-C), and
 *     the move is accepted with the configurational-bias weight (Sec. III.D,
 *     Eq. 12) or, for n_trial = 0, rejected on any blocking depletant.
 *
 * Conventions for every entry point:
 *   - Return value: HPMC_OK (0) or a negative HPMC_ERR_* code; nothing throws
 *     or aborts across this boundary.  hpmc_strerror() names the code.
 *   - Pointers are plain host or device addresses as each argument states;
 *     arguments with a `mem` flag accept either (HPMC_HOST / HPMC_DEVICE).
 *     Positions are row-major n x 3 doubles (x, y, z), orientations n x 4
 *     doubles (w, x, y, z) unit quaternions, body frame -> box frame.
 *   - The library owns all device memory it allocates; inputs are copied.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it unless stated.
 *   - Errors raised inside kernels (e.g. a neighbourhood larger than the
 *     on-chip capacity) are sticky and reported by the next synchronising
 *     call (hpmc_get_state, hpmc_sync) as HPMC_ERR_DEVICE.
 */
#ifndef HPMC_DEP_H
#define HPMC_DEP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HPMC_OK 0
#define HPMC_ERR_ARG (-1)      /* invalid argument or parameter combination */
#define HPMC_ERR_OVERLAP (-2)  /* the configuration has overlapping colloids */
#define HPMC_ERR_CUDA (-3)     /* a CUDA runtime call failed */
#define HPMC_ERR_TIMEOUT (-4)  /* a bounded device-side wait gave up */
#define HPMC_ERR_STATE (-5)    /* call not valid in the context's state */
#define HPMC_ERR_CAP (-6)      /* a size exceeds a documented capacity */
#define HPMC_ERR_DEVICE (-7)   /* a kernel recorded an error (sticky) */

#define HPMC_SPHERE 0          /* params: {diameter} */
#define HPMC_HEMISPHERE 1      /* params: {diameter}; reference point = centre of the flat face */
#define HPMC_SPHEROID 2        /* params: {a, c}: semi-axes a = b (equator), c (body z) */

#define HPMC_FP64 0            /* every overlap test in FP64 */
#define HPMC_FP32_RECHECK 1    /* FP32 tests with a certified margin, FP64 recheck near contact */

#define HPMC_V0_CIRCUMSPHERE 0 /* depletants sampled in the new pose's circumsphere (default) */
#define HPMC_V0_SHELL 1        /* spheres: in the shell that can hold the move's lens */
#define HPMC_V0_CUBE 2         /* in the cube of side 2 R_s around the circumsphere */

#define HPMC_HOST 0
#define HPMC_DEVICE 1

#define HPMC_PHASES_LAUNCHES 0    /* colour phases: one kernel launch per phase (default) */
#define HPMC_PHASES_PERSISTENT 1  /* colour phases: one persistent launch per sweep */

typedef struct hpmc_ctx hpmc_ctx;

/* Event counters, accumulated since creation or hpmc_reset_counters().
 * The first nine are a pure function of the trajectory and are identical
 * on every correct implementation of the method (dep_evaluated is defined in
 * depletant order, so it does not depend on which lane finds a blocking
 * depletant first); the rest depend on the evaluation order of the CB trials
 * or on the precision form. */
typedef struct hpmc_counters {
    uint64_t moves;            /* trial moves proposed */
    uint64_t accept;           /* accepted */
    uint64_t reject_cell;      /* proposal left its cell (Sec. III.E) */
    uint64_t reject_overlap;   /* colloid-colloid overlap at the new pose */
    uint64_t reject_depletant; /* n_trial = 0 and a depletant blocks the move */
    uint64_t reject_cb;        /* n_trial > 0: CB weight W = 0 or u >= W */
    uint64_t dep_drawn;        /* sum of Poisson counts N_p over moves that drew them */
    uint64_t translate;        /* translation (not rotation) proposals */
    uint64_t dep_evaluated;    /* depletants up to and including the first blocking
                                  one (all N_p when none blocks; n_trial = 0) */
    uint64_t dep_blocking;     /* blocking depletants found */
    uint64_t cb_fwd_ok;        /* successful forward CB reinsertions */
    uint64_t cb_rev_ok;        /* successful reverse CB reinsertions */
    uint64_t cap_hits;         /* attempt-stream caps reached (expected 0) */
    uint64_t rechecks;         /* FP32 decisions re-taken in FP64 (HPMC_FP32_RECHECK) */
    uint64_t reserved[2];
} hpmc_counters;

/* Create a context on CUDA device `device` for n colloids in a cubic box of
 * side box_l with positions pos (n x 3, each in [0, box_l)) and orientations
 * quat (n x 4, or NULL = identity), both in memory `mem`.  seed and replica
 * key the counter-based random streams (Philox4x32-10): a trajectory is a
 * pure function of (inputs, parameters, seed, replica, sweep index).
 * precision: HPMC_FP64 or HPMC_FP32_RECHECK.  Defaults: unit spheres, no
 * depletants (z_p = 0), translations d_max = 0.1.  Overlaps are checked at the
 * first hpmc_sweep.  *out receives the context (NULL on failure). */
int hpmc_init(hpmc_ctx **out, int n, double box_l, const double *pos,
              const double *quat, int mem, uint64_t seed, uint32_t replica,
              int precision, int device);

/* One replica of a batch: an independent system with its own state point.
 * Pointers are host memory, read during hpmc_init_batch only. */
typedef struct hpmc_replica_desc {
    int n;                  /* colloids */
    double box_l;           /* cubic box side */
    const double *pos;      /* n x 3, each coordinate in [0, box_l) */
    const double *quat;     /* n x 4 unit quaternions, or NULL = identity */
    double q, n_r;          /* depletant diameter and fugacity z_p */
    int n_trial;            /* configurational-bias reinsertions (0 = none) */
    double d_max, a_max, p_translate;  /* trial moves, as hpmc_set_moves */
    uint32_t replica;       /* key word of this replica's random streams */
    int n_cell;             /* checkerboard cells per side (even), 0 = largest valid */
} hpmc_replica_desc;

/* A batch of n_rep independent replica systems in one context, all of the
 * same shape (params as hpmc_set_shape), keyed by (seed, desc[r].replica).
 * Every hpmc_sweep advances all replicas by one sweep in one set of kernel
 * launches covering the whole batch; a replica's trajectory is identical to
 * that of the same system alone in its own context.  Positions of the batch
 * (hpmc_get_state / hpmc_set_state) are the replicas' arrays one after the
 * other in replica order; counters from hpmc_get_state are summed over
 * replicas.  The parameter setters below apply to every replica. */
int hpmc_init_batch(hpmc_ctx **out, int n_rep, const hpmc_replica_desc *desc, int shape,
                    const double *shape_params, int nparams, uint64_t seed, int precision,
                    int device);

/* Replica r of a batch: positions (n x 3), orientations (n x 4) and its own
 * counters, each optional (NULL), into host memory.  Synchronises. */
int hpmc_get_replica(hpmc_ctx *ctx, int r, double *pos, double *quat,
                     hpmc_counters *counters);

/* Trial-move parameters of replica r only (e.g. a step size tuned per
 * replica); as hpmc_set_moves otherwise. */
int hpmc_set_replica_moves(hpmc_ctx *ctx, int r, double d_max, double a_max,
                           double p_translate);

/* Colloid shape (Sec. II; hemisphere Sec. V.A; discoid = oblate spheroid
 * a = b, c < a, Sec. V.B).  params/nparams as listed at HPMC_SPHERE etc. */
int hpmc_set_shape(hpmc_ctx *ctx, int kind, const double *params, int nparams);

/* Penetrable ideal-gas depletants of diameter q (q >= 0) at reservoir number
 * density / fugacity n_r = z_p (Sec. III.A; phi_p^r = (pi/6) q^3 z_p), and
 * n_trial configurational-bias reinsertions per blocking depletant
 * (Sec. III.D, Eq. 12; 0 = plain rejection).  The mean number of depletants
 * per move, lambda = z_p (4 pi / 3) (R_circ + q/2)^3, must not exceed 700. */
int hpmc_set_depletant(hpmc_ctx *ctx, double q, double n_r, int n_trial);

/* Trial moves: translation uniform in [-d_max, d_max]^3, rotation by at most
 * a_max radians about a uniformly random axis (anisotropic shapes only),
 * translation chosen with probability p_translate when both are enabled.
 * d_max must be below the cell width. */
int hpmc_set_moves(hpmc_ctx *ctx, double d_max, double a_max, double p_translate);

/* Checkerboard cells per box side (even, width >= 2 R_circ + q), or 0 for the
 * largest valid count.  Part of the trajectory's definition (Sec. III.E). */
int hpmc_set_cells(hpmc_ctx *ctx, int n_cell);

/* Launch shape: warps cooperating on one moved colloid's depletants and
 * colloid tests in the colour-phase kernels (1..8, default 1), and the
 * schedule of the eight colour phases of a sweep (Sec. III.E):
 * HPMC_PHASES_LAUNCHES (default) runs one kernel launch per phase, each waiting
 * for the previous one (programmatic dependent launch lets a phase's
 * set-up overlap the previous one's tail); HPMC_PHASES_PERSISTENT runs all
 * eight in one
 * persistent launch whose one-warp CTAs take the non-empty active cells in
 * phase order from a ticket counter, each cell waiting only until the
 * non-empty cells of its 27-cell neighbourhood that belong to earlier phases
 * of the sweep are done (per-cell readiness counters; every wait is bounded,
 * see hpmc_set_wait_limit).  The persistent schedule applies to the
 * HPMC_FP32_RECHECK form of spheres with one warp per colloid; other
 * combinations use the launches.  Performance knobs only: results are
 * identical for every value.  HPMC_ERR_ARG for an unknown schedule. */
int hpmc_set_launch(hpmc_ctx *ctx, int warps_per_colloid, int phase_schedule);

/* Grid of each colour-phase launch (HPMC_PHASES_LAUNCHES, HPMC_FP32_RECHECK
 * form of spheres, one warp per colloid): 0 launches one CTA per cell of the
 * phase; 1..64 launches that many waves of resident one-warp CTAs, each
 * taking every grid-th non-empty cell of the phase in turn (fewer CTA
 * launches where a phase has many cells per SM, at 24 instead of 32
 * resident CTAs per SM); -1 (the default) chooses 2 for hard interactions
 * without CB when a phase has more cells than one wave of the
 * one-CTA-per-cell grid, else 0.  A performance knob only:
 * results are identical for every value.  Takes effect at the next sweep.
 * HPMC_ERR_ARG outside -1..64. */
int hpmc_set_phase_waves(hpmc_ctx *ctx, int waves);

/* Bound of every device-side wait of the persistent colour phases, in
 * seconds of GPU global time (default 1; 1e-6 .. 60).  A wait that runs out
 * records HPMC_ERR_TIMEOUT (reported by the next synchronising call, as
 * hpmc_sync or hpmc_get_state) and its cell is left unmoved for that sweep;
 * the kernel still finishes, and the context stays usable (hpmc_set_state
 * clears the error).  Takes effect at the next sweep. */
int hpmc_set_wait_limit(hpmc_ctx *ctx, double seconds);

/* Testing aid for the bounded waits: the persistent colour phases never
 * publish global cell `cell` as done (-1, the default: none), so the waits of
 * its neighbours in later phases run out.  Host-side fault injection only;
 * the device is never made to fault or hang.  Takes effect at the next sweep.
 * HPMC_ERR_ARG for cell < -1. */
int hpmc_debug_withhold_cell(hpmc_ctx *ctx, int cell);

/* Autotuner: time every combination of warps_per_colloid in warps[0..nw)
 * and cells per side in cells[0..nc) (0 = the largest valid count) over
 * n_sweeps sweeps each (after one untimed sweep), on the context's own
 * systems, and keep the fastest.  The configuration, sweep index and
 * counters are restored afterwards, so the trajectory continues as if the
 * tuning had not run; the chosen cell count is part of the trajectory's
 * definition from then on (hpmc_set_cells).  A candidate the library rejects
 * (e.g. a cell width below 2 R_circ + q) is skipped.  Writes the choice to
 * *best_warps, *best_cells (either may be NULL) and its milliseconds per
 * sweep to *best_ms (may be NULL).  Synchronous.  HPMC_ERR_ARG if no
 * candidate is valid. */
int hpmc_autotune(hpmc_ctx *ctx, const int *warps, int nw, const int *cells, int nc,
                  int n_sweeps, int *best_warps, int *best_cells, double *best_ms);

/* FP32 form only: margin on squared distances inside which an FP32 decision
 * is re-taken in FP64.  0 selects the derived certified bound (default);
 * a value below that bound is rejected with HPMC_ERR_ARG at the next sweep.
 * For the anisotropic shapes a value above the derived distance margins of
 * the depletant tests and of the pair certificates replaces them as well;
 * with the shell V_0 it also widens the FP32 shell-acceptance band by that
 * fraction of r^4 (1 sends every shell decision to FP64).
 * Larger margins only move more decisions to the exact FP64 path. */
int hpmc_set_fp32_margin(hpmc_ctx *ctx, double margin);

/* Depletant sampling region V_0 (Sec. III.C).  HPMC_V0_CIRCUMSPHERE (default):
 * N_p ~ Poisson(z_p |V_0|) depletants uniform in the circumsphere of
 * diameter d_colloid + d_depletant around the moved colloid's new pose.
 * HPMC_V0_SHELL (spheres only; the restriction to the excluded-volume shell
 * the paper remarks on): a translation by D only needs the shell
 * R_s - t_k <= |e - x'| < R_s, where t_k = k sqrt(3) d_max / 32 + 1e-9 R_s is
 * the thickness of level k (1..32), the smallest whose integer rule bounds
 * |D| from the move's random words; N_p ~ Poisson(z_p |shell_k|).  A shell
 * point takes attempt t's words: v = (s11(w0), s11(w1), s11(w2)),
 * r = R_in + t_k u01(w3), accepted iff |v|^6 R_s^4 < r^4, e = v r / |v|.
 * Acceptance probabilities are those of the circumsphere (the blocking
 * depletants form the same Poisson process), so the sampled ensemble is the
 * same; the trajectory and the counters dep_drawn and dep_evaluated are
 * those of the shell.  HPMC_V0_CUBE (every shape): the axis-aligned cube
 * [-R_s, R_s)^3 around the new reference point, N_p ~ Poisson(z_p (2 R_s)^3),
 * depletant k = attempt k (no rejection step); those outside the new pose's
 * excluded volume are irrelevant.  HPMC_ERR_ARG for the shell with an
 * anisotropic shape or an unknown mode.  Takes effect at the next sweep. */
int hpmc_set_v0(hpmc_ctx *ctx, int mode);

/* Soft colloid-depletant interaction (the paper's closing remark that the
 * scheme generalises to soft potentials such as the Hertz potential).
 * eps > 0: u(r) = eps (1 - r/s)^(5/2) kT for r < s = (d_colloid +
 * d_depletant) / 2, else 0, in place of the hard colloid-depletant overlap
 * (colloids stay hard among themselves).  A depletant at x blocks a move with
 * probability e^(-U_others(x)) max(0, e^(-u_old(x)) - e^(-u_new(x))), decided
 * by u01 of the fourth word of its attempt (U_others summed over the other
 * colloids in ascending index; e^(-y) by Cody-Waite reduction and the
 * degree-14 Taylor polynomial, the same bits on every side).  Spheres,
 * n_trial = 0 and the circumsphere or cube V_0 (HPMC_ERR_ARG at the next
 * sweep otherwise); both forms (HPMC_FP32_RECHECK takes each depletant's two
 * early exits, r_new >= r_old and u01 >= e^(-u_old) - e^(-u_new), and its
 * blocking test in FP32 outside certified bands, the FP64 statement inside
 * them: the same decisions).  eps = 0 (default): hard. */
int hpmc_set_soft(hpmc_ctx *ctx, double eps);

/* Colloids in use.  Replica r keeps its colloids in its slots 0..n_live-1
 * (the RNG stream of a colloid is its slot); slots beyond are not moved,
 * binned or tested.  hpmc_set_live sets the count of one replica (0..its
 * number of slots; spheres; re-validated at the next sweep); hpmc_get_live
 * writes every replica's count to n_live[0..n_rep).  Both synchronise the
 * device.  Without these calls every slot is in use. */
int hpmc_set_live(hpmc_ctx *ctx, int replica, int n_live);
int hpmc_get_live(hpmc_ctx *ctx, int *n_live);

/* Gibbs-ensemble colloid exchange (Sec. IV.B, coexistence; spheres).
 * Replicas 2p and 2p + 1 are the two boxes of pair p (they must share q,
 * n_r and n_trial: one depletant reservoir).  Each call makes n_attempts
 * exchange attempts per pair, one after another, all pairs in parallel
 * (one CTA per pair), on `stream`.  Attempt s of pair p (s counts the
 * pair's attempts from 0) draws from box 2p's key with stream word
 * 0xFFFFFFFE and counter s: purpose 1 sub 0 picks the source box (top bit
 * of word 0) and its slot floor(w_1 n_src / 2^32); purpose 1 sub 1 the new
 * position L_dst u01(w_d); purpose 7 sub 1 the Metropolis test
 * u53 < N_src V_dst / ((N_dst + 1) V_src); then the hard-core test in the
 * new box and the depletants of Sec. III.B at the new position (purposes
 * 3, 4), a depletant overlapping the inserted colloid and no other colloid
 * of its box blocking the move, or with n_trial > 0 entering the weight of
 * Eq. 12 with forward trials around the old position in the old box and
 * n_trial - 1 reverse trials around the new one (purposes 5, 6 with the
 * depletant index as sub; accept with purpose 7 sub 0, u53 < W).  On
 * acceptance the new box's slot n_dst takes the colloid and the old box's
 * last colloid moves into the vacated slot.  The exchange's depletant
 * counters go to the source box's counters.  FP64 decisions (the FP32 form
 * takes its point tests in FP32 with certified margins, FP64 inside them).
 * HPMC_ERR_ARG for an odd replica count, a non-sphere shape, unequal
 * depletant parameters, the shell or cube V_0 or a soft interaction. */
int hpmc_gibbs_exchange(hpmc_ctx *ctx, int n_attempts, void *stream);

/* Pair p's attempt count and its counters (attempts, accepted, rejected:
 * empty source box, Gibbs ratio, overlap, depletant, CB; depletants drawn).
 * Synchronises; HPMC_ERR_DEVICE for a recorded kernel error. */
int hpmc_get_gibbs(hpmc_ctx *ctx, int pair, uint64_t *step, uint64_t counters[8]);

/* Per-kernel timing.  While on, hpmc_sweep launches its kernels one by one
 * (no graph) with CUDA events around the cell-list kernels and around every
 * colour-phase kernel.  hpmc_get_timing synchronises and returns the summed
 * milliseconds and launch counts for kinds 0 = cell list and schedule,
 * 1 = colour-phase kernel, 2 = depletant lens kernel (FP32 form), then clears
 * them.  ms/launches may be NULL; nkinds is the length of both arrays (up to 3
 * are filled). */
int hpmc_set_timing(hpmc_ctx *ctx, int on);
int hpmc_get_timing(hpmc_ctx *ctx, double *ms, uint64_t *launches, int nkinds);

/* Enqueue n_sweeps checkerboard sweeps (each colloid gets one trial move per
 * sweep) on `stream`.  The first call after a parameter change validates the
 * configuration (synchronously: HPMC_ERR_OVERLAP if colloids overlap) and
 * records the sweep as a CUDA graph. */
int hpmc_sweep(hpmc_ctx *ctx, int n_sweeps, void *stream);

/* Copy the state out (synchronises `stream`): positions (n x 3) and
 * orientations (n x 4, may be NULL) into memory `mem`; *sweep (may be NULL)
 * receives the next sweep index; *counters (may be NULL) the counters.
 * Returns HPMC_ERR_DEVICE if a kernel recorded an error. */
int hpmc_get_state(hpmc_ctx *ctx, double *pos, double *quat, int mem,
                   uint64_t *sweep, hpmc_counters *counters, void *stream);

/* Replace positions / orientations (quat may be NULL to keep them) and the
 * sweep index (checkpoint / resume: bit-exact continuation).  Synchronises
 * `stream`: the buffers are consumed on return, and the new configuration
 * is checked in the same round trip (positions in the box, no overlaps; a
 * failed check is reported by the next hpmc_sweep, as HPMC_ERR_OVERLAP or
 * HPMC_ERR_ARG).  After a parameter change the check runs at the next sweep
 * instead. */
int hpmc_set_state(hpmc_ctx *ctx, const double *pos, const double *quat, int mem,
                   uint64_t sweep, void *stream);

/* Zero the counters. */
int hpmc_reset_counters(hpmc_ctx *ctx);

/* Block until all work of the context has finished; report sticky errors. */
int hpmc_sync(hpmc_ctx *ctx);

/* Standalone checkerboard cell list of one sweep (Sec. III.E): the grid shift
 * of sweep `sweep` under (seed, replica), cells of width box_l / n_cell.
 * pos_dev: device n x 3 doubles in [0, box_l).  Outputs (device):
 * cell_start[n_cell^3 + 1] (exclusive prefix of counts), cell_idx[n] (the
 * colloids of each cell in ascending index).  Allocates its scratch (cell
 * counts and per-colloid cell ids) with cudaMallocAsync / cudaFreeAsync on
 * `stream`. */
int hpmc_cell_list(int n, double box_l, int n_cell, const double *pos_dev,
                   uint64_t seed, uint32_t replica, uint64_t sweep,
                   int *cell_start_dev, int *cell_idx_dev, void *stream);

/* The same cell list as hpmc_cell_list, for callers that cannot allocate
 * device memory at the time they need it (a loop with a fixed memory budget
 * after start-up, code running while another component owns the allocator, a
 * framework that hands out memory only from its own pool).  The paper has no
 * counterpart: this is a service of the library, not a step of the method.
 * It calls no cudaMalloc / cudaFree or any other allocating routine; its
 * scratch is a file-scope device array of 1.25 MB that every GPU which loads
 * the library holds until the process exits.
 *   - Limits: n_cell <= 40 (n_cell^3 <= 65536 cells) and n <= 262144
 *     colloids; n_cell in 41..1024 or a larger n returns HPMC_ERR_CAP without
 *     doing anything (n_cell > 1024, odd or < 2 is HPMC_ERR_ARG, as for
 *     hpmc_cell_list).
 *   - The first call on a device looks up the array's device address for that
 *     device (cudaGetSymbolAddress, with the device current) and keeps it for
 *     the life of the process; make that first call before any stream capture
 *     on the device.  cudaDeviceReset on that device invalidates the kept
 *     address (the module is reloaded at another address): do not call this
 *     entry point on a device after resetting it.
 *   - Every call on a device shares the one array, which keeps the last
 *     call's contents (the counts are cleared at the start of each call):
 *     calls whose work overlaps on the GPU (different streams, no ordering)
 *     race and give wrong lists.  Order them on one stream or with events.
 * Arguments, outputs and errors as for hpmc_cell_list. */
int hpmc_cell_list_noalloc(int n, double box_l, int n_cell, const double *pos_dev,
                           uint64_t seed, uint32_t replica, uint64_t sweep,
                           int *cell_start_dev, int *cell_idx_dev, void *stream);

/* Depletant free volume (Sec. IV.A observable): of n_probe points uniform in
 * replica `replica`'s box, how many overlap none of its colloids as a
 * depletant of diameter q (at the current positions, FP64 tests).  Probe m
 * draws Philox4x32-10 under the key (seed_lo, seed_hi) with counter
 * (sample, m_lo, 8 << 24 | m_hi, 0) and sits at box_l * ((w_d + 1/2) 2^-32);
 * alpha = n_free / n_probe, and phi_p = alpha * eta_r.  Synchronous.  Uses
 * stream-ordered scratch on the context's own stream. */
int hpmc_free_volume(hpmc_ctx *ctx, int replica, double q, uint64_t seed, uint32_t sample,
                     uint64_t n_probe, uint64_t *n_free);

/* The architecture the library's kernels were compiled for, as the CUDA
 * runtime reports it for the current device (cudaFuncGetAttributes of one of
 * them): *binary_version (103 for sm_103a) and *ptx_version (0 when the
 * library carries no PTX); either pointer may be NULL, not both.  A library
 * service, not a step of the method. */
int hpmc_kernel_arch(int *binary_version, int *ptx_version);

/* The library's own device Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
 * SC'11: the counter-based generator every random stream of the method draws
 * from, the reading of the paper's unspecified random numbers) applied to n
 * (counter, key) pairs, so that the device generator can be checked against
 * the published known-answer vectors.  ctr_dev: n x 4 words, key_dev: n x 2
 * words (k0, k1), out_dev: n x 4 words, all device memory owned by the
 * caller.  variant 0: the rounds with the key bumped by the Weyl constants
 * each round; 1: the same with the ten round keys precomputed (the form the
 * depletant loops use).  Enqueued on `stream`; HPMC_ERR_ARG for n < 0, an
 * unknown variant or a NULL buffer with n > 0. */
int hpmc_philox(int n, const uint32_t *ctr_dev, const uint32_t *key_dev, uint32_t *out_dev,
                int variant, void *stream);

/* Colloid slots of the context (*n_total: the rows of the pos / quat
 * buffers of hpmc_get_state and hpmc_set_state) and replicas (*n_rep); either
 * pointer may be NULL.  A pinned host buffer is read or written in place by
 * the device (no staging copy), so it must hold that many rows. */
int hpmc_get_size(hpmc_ctx *ctx, int *n_total, int *n_rep);

/* Human-readable name of an HPMC_* code. */
const char *hpmc_strerror(int code);

/* Free the context and its device memory (synchronises its work). */
void hpmc_destroy(hpmc_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HPMC_DEP_H */
