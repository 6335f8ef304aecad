/* respa3b -- GB300 (sm_103a) r-RESPA molecular dynamics with Lennard-Jones
 * pair forces on every inner step and cutoff Axilrod-Teller-Muto (ATM)
 * three-body forces only on outer steps.
 *
 * Method: arXiv 2507.11172 (Martin, Newcome, Muehlhaeusser, Mishra, Gratl,
 * Bungartz), "The Multiple Time-Stepping Method for 3-Body Interactions in
 * High Performance Molecular Dynamics Simulations".
 *   - potentials: LJ 12-6 and ATM, Sec. 2.1;
 *   - cutoff: a pair counts iff r <= r_c; a triplet counts iff all three of
 *     its pair distances are <= r_c (Fig. 2 caption, Sec. 4.2.2); plain
 *     truncation, no shift;
 *   - integrator: the single-loop r-RESPA of Algorithm 2 (Sec. 4.1), with the
 *     step-size factor s = k_inner and the paper's dt = dt_outer / k_inner;
 *   - Newton's third law (Sec. 2.2; the paper's outlook in Sec. 5): the default triplet
 *     kernel evaluates each triplet once and gives all three members their forces;
 *     LJ pairs are evaluated from both members (no scatter), as a GPU trade-off.
 *
 * Units are reduced LJ units (Sec. 4.2, Table 1): the caller chooses eps,
 * sigma, nu and the mass; k_B = 1.  The box is a periodic cube of side L
 * with minimum-image distances, and L must exceed 3 * max(r_c, r_c + skin)
 * (a precondition that keeps every cutoff sphere inside one image).
 *
 * Conventions for every entry point
 *   - Returns md_status; nothing is thrown across the boundary.
 *   - Host arrays are caller-owned, read or written only during the call,
 *     and always in the caller's original particle order (the library keeps
 *     its own cell-sorted order internally).  Vectors are n x 3 row-major
 *     (x0 y0 z0 x1 y1 z1 ...), IEEE double.
 *   - Device memory is owned by the library; handles are not thread-safe:
 *     one thread at a time per handle.
 *   - Calls are synchronous: when a call returns, its GPU work has finished.
 */
#ifndef RESPA3B_H
#define RESPA3B_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_system md_system;
typedef struct md_batch md_batch;

typedef enum {
  MD_OK = 0,
  MD_ERR_ARG = -1,            /* invalid argument (n < 3, dt <= 0, k < 1, eps/sigma/r_c <= 0, NULL) */
  MD_ERR_OOM = -2,            /* device memory (or the batch's memory budget) exhausted */
  MD_ERR_BOX_TOO_SMALL = -3,  /* L <= 3 * max(r_c2 + skin, r_c3): minimum image not unique */
  MD_ERR_NONFINITE = -4,      /* a position, velocity, force or energy became NaN/Inf */
  MD_ERR_DEVICE_TIMEOUT = -5, /* a kernel's bounded wait for its own asynchronous shared-memory copies
                                gave up (cell-tile LJ kernel); no kernel waits on another launch or on
                                the host */
  MD_ERR_CUDA = -6,           /* a CUDA runtime call failed (message via md_last_error) */
  MD_ERR_STATE = -7,          /* call not valid in this state (e.g. ticket unknown) */
  MD_ERR_CAPACITY = -8,       /* a cell, neighbour list or triplet list exceeded its capacity */
  MD_ERR_CANCELLED = -9       /* batch request cancelled by md_batch_cancel */
} md_status;

enum { MD_FP32 = 0, MD_FP64 = 1 };
/* OR into md_create_system's precision: keep the state on the host and allocate device
 * memory only at first use or when a batch admits the system (serving by memory budget). */
enum { MD_DEFERRED = 0x100 };

/* Per-handle counters; all fields refer to the system's lifetime unless noted. */
typedef struct {
  uint64_t triplets_last;      /* interacting triplets found by the last ATM evaluation */
  uint64_t triplets_total;     /* interacting triplets summed over all ATM evaluations */
  uint64_t atm_evals;          /* ATM evaluations (one per outer step, plus initial) */
  uint64_t lj_evals;           /* LJ evaluations (one per inner step, plus initial) */
  uint64_t outer_steps;        /* outer r-RESPA steps completed */
  uint64_t replays;            /* calls replayed because a particle moved more than skin / 2 */
  uint64_t guard_rechecks;     /* cutoff tests re-decided in FP64 (guard band) */
  double atm_ms_total;         /* summed ATM kernel time from CUDA events (profiling on) */
  uint64_t atm_timed;          /* number of ATM launches in atm_ms_total */
  int32_t max_cell_count;      /* largest cell occupancy seen at the last binning */
  int32_t cells_per_side;      /* binning grid */
  int32_t atm_kernel;          /* triplet kernel in use: 0 cell, 1 per-particle, 2 rotation, -1 not chosen yet */
  int32_t atm_bases_per_warp;  /* rotation kernel: consecutive bases per warp in a work item (autotuned) */
  uint64_t near_triplets_last; /* distance classes: near-class triplets found by the last near evaluation */
  int32_t lj_block;            /* LJ kernel: particles (threads) per block (autotuned: 32, 64 or 128) */
  int32_t list_warps;          /* pair-list build: warps per CTA (autotuned: 2, 4 or 8) */
  int32_t tuned_from_cache;    /* 1 if the last tuning reused the choices of an earlier system with the same
                                  key (N bucket, density bucket, r_c2, r_c3, skin, precision, classes) */
  int32_t lj_kernel;           /* LJ kernel in use: 0 row kernel (one thread per particle, neighbour positions
                                  gathered from global memory), 1 cell-tile kernel, 2 team kernel
                                  (md_set_lj_kernel) */
  int32_t lj_team;             /* team kernel: lanes per particle (autotuned: 4, 8 or 16) */
  int32_t reserved_;
} md_stats;

/* Create a system of n >= 3 particles in a periodic cube of side box_L: the input x0, v0 of
 * Algorithm 2 (Sec. 4.1) and the periodic cutoff setting of Sec. 4.2.
 * pos: n x 3, caller order, any finite values (folded into [0, L));
 * vel: n x 3 or NULL for zeros; mass > 0 and finite (the paper's m, usually 1); box_L > 0 and finite.
 * precision: MD_FP32 (FP32 forces; LJ per-particle sums compensated (TwoSum), triplet forces summed
 * per particle in 64-bit fixed point (exact, order-independent); FP64 positions, velocities, energies)
 * or MD_FP64 (everything in FP64).  Non-finite pos / vel: MD_ERR_NONFINITE.
 * cuda_stream: a cudaStream_t to run on, or NULL for a library-owned stream.
 * Potentials default to eps = sigma = 1, r_c2 = 2.5, nu = 0, r_c3 = 2.5
 * until md_set_potentials.  On error *out is NULL. */
md_status md_create_system(md_system **out, int64_t n, double box_L, const double *pos, const double *vel,
                           double mass, int precision, void *cuda_stream);

/* LJ 12-6 (eps, sigma, pair cutoff rc_pair) and ATM (nu, triplet cutoff
 * rc_triplet), Sec. 2.1; the cutoff rules of the Fig. 2 caption and Sec. 4.2.2.
 * All five finite; eps, sigma, the cutoffs > 0, nu >= 0 (else MD_ERR_ARG); nu = 0
 * disables the three-body force.  Invalidates the cached forces (Algorithm 2
 * recomputes F2b(x0) and F3b(x0)). */
md_status md_set_potentials(md_system *s, double lj_eps, double lj_sigma, double rc_pair, double atm_nu,
                            double rc_triplet);

/* Verlet-list skin for the pair list of the linked-cell neighbour search (Sec. 2.2, Sec. 4.1: the
 * paper's linked cells; the skin is this library's, default 0.3 sigma, thinner for boxes below
 * 3 (r_c2 + 0.3) at creation).  The pair list is rebuilt at every outer step; if
 * any particle moves more than skin/2 within one, the call is replayed from its
 * start with a rebuild before every inner step at which some particle has moved
 * more than skin/2 since the last rebuild (decided on the device), so results
 * never depend on the skin.  The next calls start that way too; the plain plan is
 * retried after 4 calls, then after 8, 16, ... (up to 64) while replays recur
 * (md_stats.replays counts them).  Batches do the same per cycle. */
md_status md_set_skin(md_system *s, double skin);

/* Advance n_outer >= 0 outer steps of k_inner >= 1 inner steps each:
 * Algorithm 2 with s = k_inner and dt = dt_outer / k_inner.  Positions and
 * velocities are updated in place; forces are cached between calls. */
md_status md_respa_step(md_system *s, int n_outer, int k_inner, double dt_outer);

/* Current forces (caller order, n x 3), F = -grad Phi (Eq. 1-3): f2 = LJ, f3 = ATM (Sec. 2.1),
 * the F2b and F3b of Algorithm 2 at the current positions; either may be NULL.
 * Evaluates them first if they are not cached.  MD_ERR_STATE while the system is in a batch. */
md_status md_get_forces(md_system *s, double *f2, double *f3);

/* Energies at the current state (a full step of Algorithm 2; only full iterations are meaningful,
 * Sec. 4.1): kinetic 0.5 m sum v^2, LJ energy, ATM energy (Eq. 2-3, Sec. 2.1; the total energy of the
 * RVITE metric, Eq. 4) and the virial W = sum over interactions of sum r_a . F_a (pressure
 * P = (2 e_kin + W) / (3 L^3), the pressure of Sec. 4.2.2).  Reduced in FP64.  Any pointer may be
 * NULL. */
md_status md_get_energy(md_system *s, double *e_kin, double *u2, double *u3, double *virial);

/* Radial distribution function pair counts at the current positions (the RDF of
 * Sec. 4.2.2, before normalisation): counts[b] = number of unordered pairs {i, j}
 * with b * dr <= r_ij < (b + 1) * dr, dr = r_max / nbins, r_ij the minimum-image
 * distance computed in IEEE double as sqrt((dx*dx + dy*dy) + dz*dz) (the integer
 * counts equal a plain CPU histogram of the positions md_get_state returns).
 * 1 <= nbins <= 8192; 0 < r_max <= r_c2 + skin (the pair-list radius), else
 * MD_ERR_ARG.  counts: host array of nbins, caller-owned.  g(r) for bin b is
 * counts[b] / (n / 2 * (n / L^3) * 4/3 pi ((b+1)^3 - b^3) dr^3).  Evaluates the
 * forces first if they are not cached (the counts then refer to the same positions). */
md_status md_get_rdf(md_system *s, int nbins, double r_max, uint64_t *counts);

/* Copy positions (folded into [0, L)) and velocities out / in, caller order,
 * n x 3 each; either may be NULL: the input x0, v0 and output of Algorithm 2 ("positions and
 * velocities updated in place", Sec. 4.1), also the checkpoint / resume pair.  md_set_state
 * invalidates cached forces; it
 * returns MD_ERR_NONFINITE, with nothing changed, if an input value is NaN/Inf.
 * Both copy straight between the caller's buffers and the device (pinned caller
 * memory moves by DMA) and permute to and from the sorted layout on the device. */
md_status md_get_state(md_system *s, double *pos, double *vel);
md_status md_set_state(md_system *s, const double *pos, const double *vel);

/* Distance classes for the three-body force (the multiple-time-stepping outlook of Sec. 5, after the
 * intermediate-cutoff splitting of Nakano et al. cited in Sec. 3): an intermediate cutoff r_a splits
 * the ATM triplets into a near class (all three pair distances <= r_a) and a far class (the other
 * triplets with all three distances <= r_c3).  md_respa_step then integrates three levels in one
 * loop, in the manner of Algorithm 2: LJ every inner step dt, the near class with step-size factor
 * s_near (kicks s_near dt / 2 F3near / m around every block of s_near inner steps), the far class
 * with the outer step (kicks dt_outer / 2 (F3 - F3near) / m).  k_inner must be a multiple of s_near
 * (MD_ERR_ARG otherwise); s_near = k_inner, or r_a below every pair distance, is Algorithm 2 again.
 * Requires 0 < r_a <= min(r_c2, r_c3); single systems only (md_batch_submit rejects them,
 * MD_ERR_ARG).  r_a <= 0 turns the classes off.  Reallocates the handle's device memory (state kept)
 * and invalidates the cached forces.  At every binning each particle keeps as near-class candidates
 * its neighbours above it (the triplet ownership order) within r_a + skin; more than 64 give
 * MD_ERR_CAPACITY.  Every near evaluation re-decides r_a exactly at the current positions. */
md_status md_set_distance_classes(md_system *s, double r_a, int s_near);

/* Cached near-class ATM forces F3near (n x 3, caller order) at the current positions (the near distance
 * class of the Sec. 5 outlook, ATM of Sec. 2.1); md_get_forces' f3 is the whole ATM force (near + far).
 * MD_ERR_STATE if the classes are off. */
md_status md_get_near_forces(md_system *s, double *f3near);

/* Counters (see md_stats; the triplet counts are those of the cutoff rule of the Fig. 2 caption, the
 * step counts those of Algorithm 2).  profile = 1 launches a call's kernels one by one
 * (instead of replaying a captured CUDA graph) with CUDA events recorded on
 * the system's stream around every ATM launch (atm_ms_total / atm_timed). */
md_status md_get_stats(md_system *s, md_stats *out);
md_status md_set_profiling(md_system *s, int profile);

/* Triplet-kernel choice (an autotuning knob, like the paper's node-level autotuning in AutoPas,
 * Sec. 4.1; results agree within the FP tolerance):
 *   0  one CTA per base cell, shared-memory staging, each triplet evaluated once with
 *      Newton-3 scatter of the three forces;
 *   1  one warp per particle, neighbours from the pair list, only the force on that
 *      particle per evaluation (each triplet evaluated from each member, no scatter);
 *   2  one warp per particle and its half list (its neighbours within r_c3 above it in the
 *      order: cell layer along z, fixed-point z, sorted index), every neighbour pair visited
 *      once by a cyclic rotation across the lanes, each triplet evaluated once (Newton 3)
 *      with its forces kept as edge weights; per-neighbour terms added to per-particle sums
 *      in 64-bit fixed point (FP32 path: bitwise reproducible) or with FP64 atomics (FP64);
 *      1 and 2 need r_c3 <= r_c2 + skin, else 0 is used;
 *  -1  (default) time the allowed kernels (the rotation kernel with 4, 8 and 16 bases per warp in
 *      a work item) on the system's first evaluation and keep the fastest.  A batch uses its
 *      members' common choice, else 2 where allowed, else 0.
 * The same autotuner picks the LJ block size and the pair-list build's warps per CTA (md_stats), and
 * caches every choice for the process under the key (device, N in half-octave buckets, density in
 * steps of 0.025, r_c2, r_c3, skin, precision, distance classes on/off): a later system with the same
 * key takes the cached choices without trials (md_stats.tuned_from_cache = 1). */
md_status md_set_atm_kernel(md_system *s, int variant);

/* Launch shapes fixed instead of autotuned (no counterpart in the paper; an autotuning knob like
 * md_set_atm_kernel): lj_block 32, 64 or 128 particles per LJ block, list_warps 2, 4 or 8 warps per
 * CTA of the pair-list build, rot_bases_per_warp 4, 8 or 16 (rotation kernel work items); 0 leaves a
 * shape to the autotuner.  Every shape gives the same forces bit for bit.  Applied at the next call
 * that evaluates forces; MD_ERR_ARG for other values, MD_ERR_STATE while the system is in a batch. */
md_status md_set_shapes(md_system *s, int lj_block, int list_warps, int rot_bases_per_warp);

/* LJ kernel choice for the pair forces of Sec. 2.1 (LJ 12-6, every inner step of Algorithm 2; an
 * autotuning knob like md_set_atm_kernel; both give the forces of the pair list within FP rounding):
 *   0  row kernel: one thread per particle walks its pair-list row and gathers the neighbours'
 *      positions from global memory (md_set_shapes' lj_block particles per block);
 *   1  cell-tile kernel: one CTA per block of 2 x 2 x 2 cells copies the positions of the 4 x 4 x 4
 *      cells around it into shared memory (bulk asynchronous copies completing on an mbarrier, waited
 *      on with a bounded poll: MD_ERR_DEVICE_TIMEOUT if it gives up), then one thread per particle
 *      walks its pair-list row against shared memory; used where that staging fits in shared memory
 *      (about 52 cap_cell particles), else 0;
 *   2  team kernel: 4, 8 or 16 adjacent lanes per particle share its row (consecutive entries read
 *      together, neighbour positions gathered from global memory), their compensated partial sums
 *      combined by TwoSum; more warps resident than with one thread per particle;
 *  -1  (default) time all of them (the row kernel with 32, 64 and 128 particles per block, the team
 *      kernel with 4, 8 and 16 lanes per particle) on the system's first evaluation and keep the
 *      fastest (cached per key with the other choices).  Batches use the row kernel.
 * Applied at the next call that evaluates forces (the cached forces are recomputed); MD_ERR_ARG for
 * other values, MD_ERR_STATE while the system is in a batch. */
md_status md_set_lj_kernel(md_system *s, int variant);

/* Failure-detection test knob (no counterpart in the paper): from the next call on, the cell-tile LJ
 * kernel (md_set_lj_kernel 1) announces `bytes` more to its copy barrier than its bulk copies deliver,
 * so that barrier never completes; every copy it issues still completes, the kernel's bounded wait
 * (0.1-0.3 s) runs out, the call fails with MD_ERR_DEVICE_TIMEOUT and the state is restored to the call's
 * start, while the CUDA context stays usable.  0 <= bytes <= 4096 (MD_ERR_ARG otherwise); 0, the
 * default, turns it off.  For tests of the timeout path only. */
md_status md_inject_copy_shortfall(md_system *s, int bytes);

/* Number of particles, box side and precision of a handle (the inputs of Algorithm 2). */
md_status md_get_info(md_system *s, int64_t *n, double *box_L, int *precision);

/* Device memory of a handle in bytes: what it holds, or for a deferred system (MD_DEFERRED) what it
 * will hold once resident -- the figure md_batch_create's budget admission counts.  No counterpart in
 * the paper (serving, the batched ensemble of this library). */
md_status md_get_memory(md_system *s, size_t *device_bytes);

/* Release all device memory of the handle (the end of the run of Algorithm 2); NULL is accepted. */
md_status md_destroy_system(md_system *s);

/* Static string for a status code (no counterpart in the paper: error reporting of this C ABI). */
const char *md_status_string(md_status st);
/* Message of this thread's last failing call (the failing CUDA call for MD_ERR_CUDA, the exceeded limit
 * for MD_ERR_CAPACITY, ...); "" if none.  No counterpart in the paper. */
const char *md_last_error(void);

/* ---------------- batched ensemble / continuous serving ----------------
 * No counterpart in the paper, which runs one system at a time: many independent replicas of
 * Algorithm 2 (Sec. 4.1), each exactly as md_respa_step would advance it.
 * A batch advances many independent systems together: on every inner "tick"
 * one launch per kernel covers all resident systems (uneven sizes, different
 * k_inner), captured as a CUDA graph per batch composition.  Systems are
 * created with md_create_system (same precision for all members) and lent to
 * the batch; their device state stays resident.
 *
 * md_batch_create: hbm_budget_bytes bounds the device memory of admitted
 *   systems (0 = no bound beyond the device).
 * md_batch_submit: queue n_outer outer steps of (k_inner, dt_outer) for s;
 *   returns a ticket.  The system joins the batch at the next md_batch_run
 *   call (admission) if it fits in the budget, else it waits.
 * md_batch_run: advance every admitted request by up to max_ticks inner
 *   ticks (<= 0: until every admitted request has finished); finished
 *   requests leave the batch and queued ones are admitted as memory frees.
 * md_batch_poll: *done = 1 once the ticket's request has finished.
 * md_batch_latency: per-outer-step wall-clock latency samples (ms) of the
 *   ticket's request, measured from its admission; *count in/out.
 * md_batch_destroy: release the batch (systems stay valid; NULL accepted). */
md_status md_batch_create(md_batch **out, size_t hbm_budget_bytes);
/* Bound the particles of the resident systems (0, the default: no bound beyond the memory budget).
 * Every resident system advances one outer step per cycle, so the particles resident set the time of
 * a cycle and with it every request's outer-step latency; queued requests wait (in order) while the
 * head of the queue would take the resident particles past the bound, and a request larger than the
 * bound by itself runs alone.  Applies from the next admission.  MD_ERR_ARG for a negative bound.  No
 * counterpart in the paper (serving). */
md_status md_batch_set_limits(md_batch *b, int64_t max_resident_particles);
md_status md_batch_submit(md_batch *b, md_system *s, int n_outer, int k_inner, double dt_outer, uint64_t *ticket);
md_status md_batch_run(md_batch *b, int max_ticks);
md_status md_batch_poll(md_batch *b, uint64_t ticket, int *done);
md_status md_batch_latency(md_batch *b, uint64_t ticket, double *ms, int *count);
md_status md_batch_pending(md_batch *b, int *queued, int *resident);
/* Cycles run so far and how many of them were replayed from their start (a member's particle left its
 * skin, or a capacity grew); either pointer may be NULL.  No counterpart in the paper (serving
 * monitoring of the batched ensemble). */
md_status md_batch_cycles(md_batch *b, uint64_t *cycles, uint64_t *replayed);
/* Cancel a request (call between md_batch_run calls).  A queued request is dropped and its system is
 * left as it was; a resident one finishes the outer step it is in (so its state is a full step of
 * Algorithm 2; md_batch_latency counts the steps done) and leaves at the end of the next cycle.  The
 * ticket then polls done with MD_ERR_CANCELLED.  MD_ERR_STATE for an unknown ticket or one that has
 * already finished, failed or been cancelled. */
md_status md_batch_cancel(md_batch *b, uint64_t ticket);
md_status md_batch_destroy(md_batch *b);

/* ---------------- all-triplet (DirectSum) ATM forces ----------------
 * The reference method of the paper's energy studies (Sec. 4.1, "DirectSum"):
 * every unordered triplet of n distinct particles, open boundaries (no periodic
 * images), no cutoff.  pos: host, n x 3 (caller order); f3: host n x 3 output;
 * u3: host output or NULL.  precision: MD_FP32 (FP32 triplet arithmetic, the
 * per-particle sums compensated, combined in FP64) or MD_FP64.  cuda_stream:
 * cudaStream_t or NULL.  Every triplet is evaluated from each of its three
 * members (3 C(n, 3) evaluations, no scatter).  Capacity: all particles' positions
 * fit in one CTA's shared memory (n <= 14464 FP32, 7232 FP64), else
 * MD_ERR_CAPACITY.  Allocates and frees its device buffers; synchronous. */
md_status md_atm_direct(const double *pos, int64_t n, double atm_nu, int precision, double *f3, double *u3,
                        void *cuda_stream);

/* ---------------- arithmetic peaks of the device ----------------
 * No counterpart in the paper (it reports no throughput): the FP32 and FP64 fused multiply-add throughput of the current device,
 * the denominators of the triplet kernel's roofline fraction (its work is plain FP32 arithmetic, not a
 * dense contraction).  kind: 0 FP32 FMA, 1 packed FP32x2 FMA (two per instruction), 2 FP64 FMA.  Every
 * resident thread of one full wave runs 8 independent FMA chains; the trip count grows until one launch
 * lasts at least min_ms (0 < min_ms <= 1e4), then the best of three timed launches (CUDA events) gives
 * *flops_per_s (2 flop per FMA) and *ms_out (may be NULL).  Runs on its own stream; allocates 4 bytes;
 * synchronous.  Reads no clock setting and changes none: the rate is the one at the clock of the moment. */
md_status md_measure_fma_peak(int kind, double min_ms, double *flops_per_s, double *ms_out);

/* ---------------- allocation-free ATM forces ----------------
 * No counterpart in the paper (the forces are those of Sec. 2.1 with the cutoff of the Fig. 2
 * caption): an entry point for callers that cannot
 * allocate device memory (code living inside another framework's memory
 * pool, a process whose device allocator is locked down, or a caller that
 * must not trigger the device-wide synchronisation of cudaMalloc/cudaFree).
 *
 * Computes the ATM forces F3 (and energy, triplet count) of one configuration
 * with FP32 triplet arithmetic: the binning sort and the cell triplet kernel
 * (md_set_atm_kernel variant 0; md_get_forces defaults to the autotuned choice,
 * usually the rotation kernel), whose per-stencil partial forces are combined
 * per particle with TwoSum and added in FP64.  It allocates nothing: every
 * intermediate array lives in a file-scope __device__ array of 8.8 MiB (at most
 * 9 MiB) that each GPU loading the library holds until the process exits.
 *   d_pos: device, n x 3 doubles, caller order;  d_f3: device, n x 3 output;
 *   box_L, atm_nu >= 0, rc_triplet > 0: finite (MD_ERR_ARG otherwise);
 *   u3, triplets: host outputs or NULL;  cuda_stream: cudaStream_t or NULL.
 * Limits: 3 <= n <= MD_NOALLOC_MAX_N, L > 3 r_c (MD_ERR_BOX_TOO_SMALL), at most
 * 32^3 cells (coarser cells beyond that).  n above the limit returns
 * MD_ERR_CAPACITY before any device work.  Messages of failing calls go to md_last_error.
 * The first call on a device looks up the arrays' device addresses and
 * uploads the pair table (a synchronous copy), so make that first call before
 * any stream capture.  All calls share the arrays: calls that overlap on the
 * GPU (other threads or streams) race; serialise them.  Synchronous: returns
 * after the forces are written. */
#define MD_NOALLOC_MAX_N 16384
md_status md_atm_forces_noalloc(const double *d_pos, int64_t n, double box_L, double atm_nu, double rc_triplet,
                                double *d_f3, double *u3, uint64_t *triplets, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* RESPA3B_H */
