/*
 * lbm_metaball.h -- C ABI of the GB300 (sm_103a) lattice sweep of the coupled
 * metaball-DEM / lattice-Boltzmann method of Zhang et al., arXiv 2206.11634.
 *
 * One handle holds one lattice (D3Q19, or the paper's D3Q15 of §2.2), its
 * node flags and a set of metaball particles.  lbm_step() advances it by whole
 * LBM steps, each of which runs on the GPU, in order:
 *   1. node classification (§2.3.1, Eq. (26)): a node is solid when
 *      M_j(x) = sum_i K_i/|x - x_i|^2 >= c0 for a particle j (Eq. (4)), owned
 *      by the particle with the largest M_j (ties to the lower index);
 *      nodes a particle uncovered since the last step are refilled (§2.3.3,
 *      Eq. (30));
 *   2. the fused stream/collide sweep (§2.2, Eqs. (14)-(18), BGK with Guo
 *      forcing) with velocity-interpolated bounce-back on particle links
 *      (§2.3.1, Eqs. (19)-(25), q from Eq. (27)), halfway bounce-back on box
 *      walls and where VIBB lacks a second fluid node (§2.3.5 item 1), the
 *      Galilean-invariant momentum exchange (§2.3.2, Eqs. (28)-(29)) and the
 *      missing-force-point terms (§2.3.5 item 2, Eqs. (31)-(32));
 *   3. a deterministic reduction of the per-link force and torque into one
 *      total per particle: FP64 partials summed in a fixed order on FP64
 *      lattices; below FP64 an exact sum of the FP32 link terms in 64-bit
 *      fixed point (units of 2^-40), read out as FP64;
 *   4. n_sub DEM sub-steps (§2.3.4) with the hydrodynamic load frozen:
 *      metaball-metaball and metaball-wall contacts (§2.1.3-2.1.4, Eqs.
 *      (5)-(13)), the contact law of §2.1.1 (Eqs. (2)-(3)), velocity Verlet
 *      and Euler's equations in the body frame (Eq. (1)).  By default the
 *      rigid-body integrator is FP64, and so is the contact geometry on FP64
 *      lattices; below FP64 the contact geometry is FP32 (lbm_config.dem_mode
 *      gives the choices).
 *
 * Units are lattice units: dx = dt = C = 1, c_s^2 = 1/3.  Node (i,j,k) sits
 * at position (i,j,k); a non-periodic face is a resting no-slip wall halfway
 * between the last node and the next (at -1/2 and n-1/2).
 *
 * Memory and ownership.  The library allocates no device memory.  The caller
 * asks lbm_workspace_size() for the size, allocates one device buffer (any
 * allocator, 256-byte aligned), and passes it to lbm_init(); the handle
 * borrows it until lbm_destroy().  The handle itself is a small host
 * allocation plus one page-locked host buffer (cudaHostAlloc) of about
 * 1.8 KB per particle of capacity, through which the particle table goes up
 * and forces and states come back with asynchronous copies.  All GPU work is
 * issued on the caller's CUDA stream given to lbm_init() (NULL = legacy
 * default stream).  Host buffers passed in are read or written during the
 * call only.
 *
 * Errors.  Every function returns LBM_OK (0) or a negative lbm_status.
 * lbm_last_error() gives a one-line message for the last failure on a handle.
 * A function that fails leaves the handle usable unless the status is
 * LBM_ERR_CUDA.  lbm_step() is asynchronous: device-side conditions
 * (particle list overflow, non-finite or supersonic state) are reported by
 * the next call that synchronises (lbm_get_forces, lbm_get_fields,
 * lbm_get_populations, lbm_check).
 */
#ifndef LBM_METABALL_H
#define LBM_METABALL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_MAX_CP 16          /* control points per particle */
#define LBM_MAX_PER_BRICK 16   /* particles whose search boxes meet one 32x4x2 node brick */

enum lbm_status {
    LBM_OK = 0,
    LBM_ERR_BAD_ARG = -1,       /* invalid argument or configuration */
    LBM_ERR_WS_TOO_SMALL = -2,  /* workspace smaller than lbm_workspace_size() */
    LBM_ERR_CAPACITY = -3,      /* more particles than max_particles, a brick list overflowed, a
                                   DEM table overflowed, or a particle moved further in one step
                                   than the DEM's contact planning allowed */
    LBM_ERR_DIVERGED = -4,      /* non-finite populations or |u| > 0.5 seen by lbm_check() */
    LBM_ERR_TIMEOUT = -5,       /* reserved: no kernel of this library waits on a device flag */
    LBM_ERR_CUDA = -6           /* a CUDA call failed; the message names it */
};

enum lbm_storage {
    LBM_STORE_F64 = 0,   /* populations stored and collided in FP64 */
    LBM_STORE_F32 = 1,   /* stored and collided in FP32 */
    LBM_STORE_F16 = 2,   /* stored as FP16 offsets (f_i/w_i - rho0), collided in FP32 */
    LBM_STORE_BF16 = 3   /* stored as BF16 offsets (f_i/w_i - rho0), collided in FP32 */
};

/* Simulation parameters.  Zero-initialise, then set what is needed; the
 * library's defaults are noted where 0 is not meaningful. */
/* DEM arithmetic, lbm_config.dem_mode. */
enum lbm_dem_mode { LBM_DEM_FP64 = 0, LBM_DEM_FP32_COMPENSATED = 1, LBM_DEM_FP64_ALL = 2 };

typedef struct lbm_config {
    int32_t nx, ny, nz;        /* lattice nodes per axis, >= 2 */
    int32_t lattice;           /* 19 (D3Q19) or 15 (D3Q15, §2.2) */
    int32_t storage;           /* enum lbm_storage */
    int32_t periodic[3];       /* 1 = periodic axis, 0 = halfway walls */
    int32_t n_sub;             /* DEM sub-steps per LBM step (§2.3.4); 0 = particles never move */
    int32_t vibb;              /* 1 = VIBB on particle links; 0 = halfway bounce-back on all of them */
    int32_t missing_force;     /* 1 = add the missing-force-point terms of §2.3.5 item 2 */
    int32_t max_particles;     /* capacity reserved in the workspace, >= 1 */
    int32_t dem_mode;          /* arithmetic of the DEM (§2.1, §2.3.4), enum lbm_dem_mode.
                                  0 (LBM_DEM_FP64, the default): the rigid-body state is FP64 and
                                  every sub-step adds to it in FP64.  On FP64 lattices everything
                                  is FP64.  On FP32/FP16/BF16 lattices a particle that cannot touch
                                  a wall or another particle during the step (|v| + |a| + 0.25 lu
                                  of reach) moves in FP64 arithmetic throughout (translation in
                                  closed form, rotation sub-stepped); the others compute their
                                  increments, contact geometry and contact law in FP32 (overlap
                                  error ~1e-6 lu) and add the increments to the FP64 state; up to
                                  256 particles with up to 2048 control points in all (else as
                                  mode 2).
                                  1 (LBM_DEM_FP32_COMPENSATED): lattices below FP64 only (FP64
                                  lattices ignore it): every particle computes in FP32 and keeps
                                  its state as compensated FP32 pairs (about 48 significant bits),
                                  with the same limits; the fastest, below mode 0's accuracy for
                                  particles without contact.
                                  2 (LBM_DEM_FP64_ALL): everything in FP64, contact geometry
                                  included, on any lattice (one CTA; slow for many contacts on
                                  this GPU, whose FP64 rate is a small fraction of its FP32 rate). */
    int32_t q_exact;           /* 0 = link fraction q by Eq. (27); 1 = the root of Eq. (26) by Newton's
                                  method from Eq. (27)'s value (§2.3.1: tolerance 1e-7, at most 100
                                  iterations; a step leaving the bracket [0,1] bisects), in the
                                  storage's working precision (FP64 for FP64, else FP32) */
    double tau;                /* BGK relaxation time, > 1/2 */
    double rho0;               /* reference density (initial fluid, refill, Eq. (31)) */
    double c0;                 /* surface value of M (Eq. (26)); 1 for the metaball of Eq. (4) */
    double u0[3];              /* initial uniform fluid velocity */
    double force[3];           /* body force density on the fluid (Guo forcing) */
    double gravity[3];         /* gravity, applied to particles as (1 - rho0/rho_s) g (§3.1) */
    double kn, eta_n;          /* normal spring and dashpot, Eq. (2) */
    double kt, eta_t, mu_s;    /* tangential spring, dashpot and Coulomb coefficient, Eq. (3) */
    double c_tol;              /* lower bound of M at the closest point, Eq. (5) */
    double mass_spacing;       /* sample spacing of the mass-property integration (0 -> 0.5) */
} lbm_config;

/* One particle: shape, material and rigid-body state.  Control points are in
 * the body frame relative to x; orientation q is a unit quaternion (w,x,y,z)
 * mapping body to world; w is the angular velocity in the world frame.
 * With mass <= 0 lbm_set_particles() computes mass, centroid and inertia by
 * sampling {M >= c0} on a grid of spacing mass_spacing, then shifts the
 * control points so that x is the centroid; otherwise mass and the body-frame
 * inertia tensor (about x) are taken as given. */
typedef struct lbm_particle {
    int32_t n_cp;                 /* 1 .. LBM_MAX_CP */
    int32_t fixed;                /* 1 = never moved by the DEM (its v and w still set u_w) */
    double cp[LBM_MAX_CP][3];     /* control points x_i, body frame (Eq. (4)) */
    double K[LBM_MAX_CP];         /* weights K_i >= 0 (Eq. (4)) */
    double Rs;                    /* sphero radius of the contact skin (§2.1.3) */
    double density;               /* rho_s */
    double mass;
    double inertia[9];            /* body-frame inertia tensor, row major */
    double x[3];
    double q[4];
    double v[3];
    double w[3];
} lbm_particle;

typedef struct lbm_handle lbm_handle;

/* Device bytes lbm_init() needs for this configuration.  Returns
 * LBM_ERR_BAD_ARG for an invalid configuration. */
int lbm_workspace_size(const lbm_config *cfg, size_t *bytes);

/* Create a handle on the current CUDA device.  dev_ws: device buffer of at
 * least lbm_workspace_size() bytes, 256-byte aligned, owned by the caller and
 * borrowed until lbm_destroy().  cuda_stream: a cudaStream_t (NULL = default
 * stream).  Initialises every node to f^eq(rho0, u0) with no particles. */
int lbm_init(const lbm_config *cfg, void *dev_ws, size_t ws_bytes, void *cuda_stream, lbm_handle **out);

/* Replace the particle set (host array of n particles, 0 <= n <=
 * max_particles).  Computes mass properties where mass <= 0, resets the
 * contact history and copies the table to the device (stream ordered; the
 * call does not wait for the stream, only, when the previous upload from the
 * page-locked buffer is still pending, for that copy).  The node flags are
 * recomputed at the start of the next lbm_step(). */
int lbm_set_particles(lbm_handle *h, const lbm_particle *host, int n);

/* Advance nsteps >= 0 LBM steps on the handle's stream (asynchronous).  The
 * work runs on two streams the handle owns (a high-priority one for the
 * particle kernels and the sweep of the bricks particles reach, a
 * low-priority one for the sweep of all other bricks), forked from and joined
 * back into the handle's stream with events inside this call, so the call as
 * a whole is ordered on the handle's stream.  Step numbers and buffer parity
 * are kept on the host and passed to the kernels, so a CUDA graph captured
 * from the handle's stream repeats the captured steps' numbers when replayed:
 * do not replay one.  When every particle is fixed (fixed = 1) the geometry
 * cannot change, and from the fourth step after lbm_set_particles() on the
 * flag pass (§2.3.1, §2.3.3) is left out: its result would be the same. */
int lbm_step(lbm_handle *h, int nsteps);

/* Synchronise and copy out the hydrodynamic force and torque of the last
 * step (F, T: host double[n][3], either may be NULL) and, if state_out is not
 * NULL, the current particle states (host lbm_particle[n]).  One wait on the
 * stream; a device-side error status is returned before any output is
 * written. */
int lbm_get_forces(lbm_handle *h, double *F, double *T, lbm_particle *state_out);

/* Synchronise and copy out the contact force and torque (Eqs. (2)-(3), pair
 * and wall terms summed per particle, world frame, torque about the centre)
 * in the current state, i.e. after the last step, with the tangential springs
 * as they stand: the contact load the next step starts from (F, T: host
 * double[n][3], either may be NULL).  Zero before the first step after
 * lbm_set_particles() and whenever no contact could occur during the last
 * step. */
int lbm_get_contact_forces(lbm_handle *h, double *F, double *T);

/* Synchronise and write the macroscopic fields of the stored populations to
 * caller device buffers (any may be NULL): dev_rho double[nz][ny][nx],
 * dev_u double[3][nz][ny][nx] (u = (sum f e - F/2)/rho, the velocity of the
 * last collision), dev_flags uint16[nz][ny][nx] (0 = fluid, j+1 = solid node
 * owned by particle j).  Solid nodes report rho = 0, u = 0. */
int lbm_get_fields(lbm_handle *h, void *dev_rho, void *dev_u, void *dev_flags);

/* Test hooks: copy the stored (post-collision) populations from / to a
 * caller device buffer double[Q][nz][ny][nx], converting from / to the
 * storage format. */
int lbm_set_populations(lbm_handle *h, const void *dev_f);
int lbm_get_populations(lbm_handle *h, void *dev_f);

/* Synchronise and report the device-side health: LBM_ERR_CAPACITY when a
 * brick list overflowed, LBM_ERR_DIVERGED when populations are non-finite or
 * some fluid node moves faster than 0.5 (checked over the whole lattice). */
int lbm_check(lbm_handle *h);

/* Counters of the last step (any pointer may be NULL): steps taken since
 * lbm_init, new fluid nodes refilled (§2.3.3), particle links (fluid node,
 * direction) updated by VIBB or bounce-back, and 32x4x2-node bricks the sweep
 * treated as near a particle (the rest took the plain path). */
int lbm_get_counters(lbm_handle *h, int64_t *steps, int32_t *nrefill, int32_t *nlinks, int32_t *near_bricks);

/* Launch schedule of the sweep.  plain_ctas_per_sm: CTAs per SM of the
 * persistent plain-brick sweep (1..4; fewer leave CTA slots to the particle
 * kernels that run beside it; 0 = one CTA per brick).  chain_ctas_per_sm:
 * CTAs per SM of the persistent flag and near-brick sweeps (1..4; 0 = the
 * default).  Takes effect from the next lbm_step(); results do not depend on
 * it.  Defaults: 0 and 0 (one plain CTA per brick, 4 flag/near CTAs per SM). */
int lbm_set_schedule(lbm_handle *h, int plain_ctas_per_sm, int chain_ctas_per_sm);

/* Whether the plain sweep issues a brick's 19 pulls before it has read that
 * brick's entry of the near set (the near sweep takes the brick when it is
 * there; its pulls are then wasted).  That removes one dependent load from
 * the start of every plain CTA, at the cost of the reads of the near bricks,
 * and puts more loads in flight, which also slows the latency-bound particle
 * kernels running beside the sweep.  mode 1: always, 0: never, -1 (default):
 * when the particles' search boxes cover under a tenth of the bricks,
 * estimated at lbm_set_particles().  Takes effect from the next lbm_step();
 * results do not depend on it.  LBM_ERR_BAD_ARG for another mode. */
int lbm_set_plain_speculation(lbm_handle *h, int mode);

/* Kernels launched per lbm_step() step (for launch accounting). */
int lbm_kernels_per_step(const lbm_handle *h);

/* Kernel timing.  With enable = 1, every later lbm_step() records a CUDA
 * event pair around each of its kernels on the stream the kernel runs on (up
 * to 65536 launches per kernel; later ones are not recorded).
 * lbm_profile_read() synchronises and returns, for kernel k (0 bin, 1 flags,
 * 2 plain sweep, 3 near sweep, 4 force reduce, 5 DEM, 6 the near set's bricks
 * without particle links), the summed device time
 * in milliseconds and the number of launches recorded since profiling was
 * enabled; enable = 0 stops recording and releases the events.  The events
 * are created on the host side of the CUDA runtime (no device memory is
 * allocated). */
int lbm_profile(lbm_handle *h, int enable);
/* As lbm_profile(), recording only the kernels whose bit is set in mask (bit
 * k: kernel k above), and of those only every every-th launch (every >= 1;
 * lbm_profile_read then counts the recorded launches); mask 0 stops
 * recording.  Event records lengthen a step by microseconds (those on the
 * particle chain's stream most), so a caller timing whole steps records the
 * plain sweep (bit 2, its own stream) alone, on a sample of its launches.
 * LBM_ERR_BAD_ARG for bits beyond kernel 5 or every < 1. */
int lbm_profile_mask(lbm_handle *h, unsigned mask, int every);
int lbm_profile_read(lbm_handle *h, int kernel, double *total_ms, int64_t *launches);

/* Change the stream later work is issued on. */
int lbm_set_stream(lbm_handle *h, void *cuda_stream);

/* Node classification without any device allocation, for callers that
 * cannot call cudaMalloc (a host application that owns the whole device
 * memory pool, or a process that allows no allocation once running).  The
 * paper has no counterpart: this is a deployment variant of the
 * classification step of lbm_step().
 *
 * Writes to dev_flags (device, uint16[nz][ny][nx]) the flags lbm_step()
 * would compute for the n host particles at their given poses: 0 = fluid,
 * j+1 = solid node owned by particle j.  Only cfg's lattice size, periodic
 * axes, lattice and storage fields and c0 are read; particle masses are not
 * needed.  The scratch (particle table, brick lists, counters) lives in one
 * fixed __device__ array of under 6 MB inside the library, reserved on
 * every device that loads the library until the process exits.  Limits: at
 * most 65536 bricks of 32x4x2 nodes (256^3 nodes) and 256 particles; larger
 * inputs return LBM_ERR_CAPACITY before any GPU work, as does a brick met by
 * more than 16 particles (seen on the device, reported after the kernels
 * ran).  Invalid arguments return LBM_ERR_BAD_ARG, CUDA failures, and any
 * other device error bit, LBM_ERR_CUDA.  The call runs on cuda_stream and synchronises it
 * before returning.  The first call on a device looks up the array's device
 * address (make it before any stream capture).  Every call on a device
 * shares the array and clears what must start at zero; calls that overlap on
 * the GPU (concurrent streams or processes sharing the library's context)
 * race on it.  Host calls are serialised by a lock. */
int lbm_flags_noalloc(const lbm_config *cfg, const lbm_particle *host, int n, void *dev_flags, void *cuda_stream);

/* Release the handle (not the workspace).  Synchronises its stream. */
int lbm_destroy(lbm_handle *h);

/* Message of the last failure on h (or of the last failed lbm_init when h is
 * NULL); never NULL. */
const char *lbm_last_error(const lbm_handle *h);

/* ---------------------------------------------------------------------------
 * Batched lattices: many independent drag cases of different box sizes
 * stepped together.  The method per case is that of lbm_step() (§2.2-§2.3;
 * the cases hold fixed particles, so there is no DEM): binning, flags with
 * refilling, the plain and near sweeps with VIBB and momentum exchange.  Each
 * phase is one kernel launch for all cases.  The particles being fixed, the
 * node flags cannot change: the first three steps after particles are set run
 * the flag pass, later steps leave it out (as lbm_step() does for a lattice
 * whose particles are all fixed).  Those static steps run as replays of a
 * CUDA graph of 16 steps captured on first use (the step numbers live in
 * device counters, so the same graph serves every later call); a remainder of
 * fewer than 16 steps is launched directly.  The paper steps one lattice; the
 * batched form has no counterpart there.
 *
 * All cases share the lattice (D3Q19 or D3Q15) and the storage (FP32, FP16
 * or BF16; FP64 is rejected), and have n_sub = 0; sizes, tau, body force and
 * particles may differ.  The workspace (lbm_batch_workspace_size) holds every
 * case's single-lattice layout plus a second per-step region per case and the
 * batch's tables; it is caller-owned, 256-byte aligned and borrowed until
 * lbm_batch_destroy().  Errors as for a single handle; the message of the
 * last failure is lbm_batch_last_error(b) (or of the last failed
 * lbm_batch_init when b is NULL).
 * ------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

int lbm_batch_workspace_size(const lbm_config *cfgs, int ncases, size_t *bytes);

/* cfgs: host array of ncases configurations.  Initialises every case to
 * f^eq(rho0, u0) with no particles, on cuda_stream (NULL = default stream). */
int lbm_batch_init(const lbm_config *cfgs, int ncases, void *dev_ws, size_t ws_bytes, void *cuda_stream,
                   lbm_batch **out);

/* Replace the particles of case c (all with fixed = 1), as lbm_set_particles.
 * Synchronises. */
int lbm_batch_set_particles(lbm_batch *b, int c, const lbm_particle *host, int n);

/* Advance every case by nsteps steps (asynchronous on the batch's stream). */
int lbm_batch_step(lbm_batch *b, int nsteps);

/* Synchronise and copy out the hydrodynamic force and torque of case c's
 * particles after the last step (host double[n][3], either may be NULL). */
int lbm_batch_get_forces(lbm_batch *b, int c, double *F, double *T);

/* The same for every case at once: F and T (host double[N][3], N the sum of
 * the cases' particle counts, either may be NULL) receive the particles of
 * case 0, then case 1, ...  One wait on the batch's stream for all cases
 * (per-case calls wait once each).  LBM_ERR_CAPACITY as lbm_batch_get_forces
 * when a case's brick lists overflowed. */
int lbm_batch_get_all_forces(lbm_batch *b, double *F, double *T);

/* Synchronise and write case c's populations as FP64 f[i][z][y][x] to a
 * caller device buffer (as lbm_get_populations). */
int lbm_batch_get_populations(lbm_batch *b, int c, void *dev_f);

/* Launch schedule: CTAs per case of the flag and near sweeps (1..64) and
 * blocks of 256 consecutive nodes per CTA of the plain sweep (1..64).
 * Results do not depend on it. */
int lbm_batch_set_schedule(lbm_batch *b, int chain_ctas_per_case, int plain_blocks_per_cta);

/* Autotuner: times trial_steps steps (after trial_steps of warm-up) for each
 * schedule of CTAs per case in {4, 8, 16, 32, 64} and 256-node blocks per
 * plain CTA in {1, 2, 4, 8}, keeps the fastest and reports it (any output may
 * be NULL).  The trials are real steps: the batch advances by
 * 40 * trial_steps steps. */
int lbm_batch_tune(lbm_batch *b, int trial_steps, int *chain_ctas_per_case, int *plain_blocks_per_cta,
                   double *best_ms_per_step);

/* Steps taken since lbm_batch_init. */
int64_t lbm_batch_steps(const lbm_batch *b);

/* Release the batch and its cases (not the workspace).  Synchronises. */
int lbm_batch_destroy(lbm_batch *b);

const char *lbm_batch_last_error(const lbm_batch *b);

#ifdef __cplusplus
}
#endif
#endif
