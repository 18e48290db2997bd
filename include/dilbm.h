/*
 * dilbm.h -- C ABI of the GB300 (sm_103a) DI-LBM library.
 *
 * The library advances the diffuse-interface lattice Boltzmann method for
 * fluid-particle interaction of Liu, Huang, Chai & Shi (arXiv:2106.08950) on
 * one GPU: a D2Q9 lattice (Sec. 2.1, Eqs. 3-4) whose every node, once per
 * time step, pulls its streamed populations, evaluates the solid fraction
 * phi of Eq. 14 from the particles, collides with the modified force term
 * (Eqs. 13, 15-17), and hands its share of the hydrodynamic force and torque
 * (Eqs. 18-19) to the particle that owns it; the particles then move by the
 * Newton-Euler equations (Eqs. 22-24) with Wan-Turek repulsion (Eqs. 28-29).
 * Domain edges use non-equilibrium extrapolation (Sec. 3, Guo et al. 2002).
 *
 * Conventions
 *   - Lattice units: dx = dt = 1, cs^2 = 1/3.  Nodes sit at integer
 *     coordinates 0..nx-1, 0..ny-1.  Walls (non-periodic sides) lie on the
 *     first / last node column or row.
 *   - Every call returns DILBM_OK (0) or a negative DILBM_ERR_* code and, on
 *     error, leaves a message for dilbm_last_error() (per host thread).
 *   - All work is issued asynchronously on the CUDA stream given at create;
 *     calls that return data to the host synchronise that stream.
 *   - The caller owns every array it passes; the library copies inputs and
 *     never keeps a caller pointer beyond the call.  The context owns its
 *     device memory and frees it in dilbm_destroy().
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef DILBM_H
#define DILBM_H

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define DILBM_OK               0
#define DILBM_ERR_INVALID_ARG (-1)  /* bad size, parameter or pointer */
#define DILBM_ERR_OOM         (-2)  /* device allocation failed */
#define DILBM_ERR_CUDA        (-3)  /* a CUDA runtime call failed */
#define DILBM_ERR_UNSTABLE    (-4)  /* a node reached rho <= 0 or a non-finite velocity */
#define DILBM_ERR_TIMEOUT     (-5)  /* a bounded device-side wait gave up */
#define DILBM_ERR_OVERFLOW    (-6)  /* more than DILBM_MAX_CANDIDATES particles near one tile */

/* Particles whose (radius + 4 interface widths) disc reaches one lattice tile
 * (128 x 8 nodes); more is reported as DILBM_ERR_OVERFLOW. */
#define DILBM_MAX_CANDIDATES 32

typedef enum { DILBM_D2Q9 = 0 } dilbm_lattice;          /* Eq. 3-4: the only lattice */

typedef enum {
    DILBM_SIDE_PERIODIC = 0,   /* both sides of an axis must be periodic, or neither */
    DILBM_SIDE_VELOCITY = 1,   /* prescribed (ux, uy), density from the inner node (walls, inlets) */
    DILBM_SIDE_PRESSURE = 2    /* prescribed rho, velocity from the inner node (outlets) */
} dilbm_side_kind;

typedef enum {
    DILBM_FP32 = 0,            /* populations stored as FP32 deviations f_i - w_i */
    DILBM_FP16_DEV = 1,        /* stored as FP16 deviations, FP32 arithmetic */
    DILBM_BF16_DEV = 2         /* stored as BF16 deviations, FP32 arithmetic.  Regression
                                  only, not a reduced-precision path held to the drag bound:
                                  its 8-bit mantissa misses a 1e-3 drag error on the cylinder */
} dilbm_storage;

typedef enum {
    DILBM_FORCE_EQ18 = 0,      /* Eq. 18 as printed: -sum_n phi_n sum_i F_i c_i */
    DILBM_FORCE_MOMENTUM = 1   /* the momentum the collision hands the fluid, negated */
} dilbm_force_model;

/*
 * The fluid-particle coupling.  DILBM_METHOD_DI is the paper's method: the
 * smooth solid fraction phi of Eq. 14 and the collision of Eqs. 13, 15-17.
 * DILBM_METHOD_PS is the method the paper compares it with (Sec. 2.2), the
 * partially saturated LBM with the SP collision: B = eps_s (Eq. 8), the exact
 * area of each node's unit cell covered by a particle, the collision of
 * Eq. 12 (f^eq takes the fluid velocity, no correction step) and the force of
 * Eqs. 10-11.  The interface width is unused by PS.  Each step one more
 * kernel tabulates, for every particle, the covered areas of the
 * (2K+1)^2 cells about its centre cell (K = ceil(r_max + 0.7071) + 1, grown
 * when dilbm_set_particles brings a larger radius); the sweep looks them up.
 * PS contexts need particles of radius >= 1, run the sweep in its default
 * shape, and are stepped on their own (batches, servers and
 * dilbm_step_static take DI only).
 */
typedef enum {
    DILBM_METHOD_DI = 0,
    DILBM_METHOD_PS = 1
} dilbm_method;

typedef struct {
    int kind;                  /* dilbm_side_kind */
    double ux, uy;             /* DILBM_SIDE_VELOCITY: boundary velocity */
    double rho;                /* DILBM_SIDE_PRESSURE: boundary density */
} dilbm_side;

typedef struct {
    int nx, ny;                /* lattice nodes, each >= 3 */
    dilbm_side west, east, south, north;
    double gravity[2];         /* acceleration on the particles (physical direction) */
    double rho_f;              /* fluid density in the buoyancy term of Eq. 22 */
    double rho_init;           /* initial density: f = f^eq(rho_init, u0) */
    double u0[2];              /* initial velocity */
    int storage;               /* dilbm_storage */
    int force_model;           /* dilbm_force_model */
    double wan_turek[5];       /* eps_P, eps_P', eps_W, eps_W', xi of Eqs. 28-29 */
    int method;                /* dilbm_method (0: DI) */
} dilbm_grid;

typedef struct {
    double x, y;               /* centre, node units */
    double r;                  /* radius */
    double ux, uy;             /* translational velocity */
    double omega;              /* angular velocity (counter-clockwise) */
    double theta;              /* orientation (integrated omega) */
    double rho_s;              /* particle density; mass rho_s pi r^2 per unit depth */
    int fixed;                 /* non-zero: the particle never moves */
} dilbm_particle;

typedef struct dilbm_ctx dilbm_ctx;

/*
 * Create a simulation (Sec. 2.3, step 1: initialise).
 *   grid            lattice size, sides, gravity, storage and force model.
 *   lattice         DILBM_D2Q9.
 *   tau             relaxation time (Eq. 1), > 0.5; viscosity (tau - 1/2)/3 (Eq. 6).
 *   interface_width epsilon of Eq. 14, > 0.
 *   particles, np   host array of np >= 0 particles, copied; each centre must
 *                   lie inside the lattice.
 *   cuda_stream     cudaStream_t to issue all work on (NULL: the legacy default stream).
 *   out             receives the context.
 * Populations start at f^eq(rho_init, u0) on every node.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int dilbm_create(const dilbm_grid *grid, dilbm_lattice lattice, double tau,
                 double interface_width, const dilbm_particle *particles, int np,
                 void *cuda_stream, dilbm_ctx **out);

/*
 * Advance nsteps >= 0 time steps (Sec. 2.3, steps 2-5; Eqs. 13-19, 22-24,
 * 28-29).  Each step is one fused pull-stream + collide sweep over every node,
 * a per-particle FP64 force/torque reduction and a rigid-body update.
 * Asynchronous: returns once the work is queued; errors raised on the device
 * (UNSTABLE, OVERFLOW) surface at the next dilbm_sync().  Whole pairs of
 * steps replay a CUDA graph captured on the context's stream on first use
 * (not on the legacy default stream, not while timing, and not while the
 * caller is capturing that stream, where the launches are issued directly).
 */
int dilbm_step(dilbm_ctx *ctx, long long nsteps);

/*
 * One lattice split over ranks in horizontal strips (one process per GPU).
 * Each rank holds rows [y0, y1) of the lattice and a copy of every particle;
 * a step is the procedure of Sec. 2.3 on those rows, with two exchanges
 * between ranks that the caller carries out (with NCCL, MPI or host copies):
 *   - pull streaming (Eq. 13, left side) across a cut needs the neighbour's
 *     post-collision row beside it: the three populations crossing each cut,
 *     sent as whole rows of the nine planes;
 *   - the force and torque of Eqs. 18-19 (and the Wan-Turek repulsion of
 *     Eq. 28) are sums over nodes, so each rank adds up the nodes it holds and
 *     the per-particle sums are added over ranks before the rigid-body update
 *     (Eqs. 22-24), which every rank then applies to its copy alike.
 *
 * dilbm_create_strip: as dilbm_create, for rows [y0, y1) of the lattice `grid`
 *   describes: y0 and y1 multiples of 8 (y1 may be ny), at least two rows,
 *   not the whole lattice.  Cuts of a non-periodic y axis at 0 and ny are the
 *   lattice's own sides; every other side (and both on a periodic y axis) is a
 *   cut.  Errors as dilbm_create, and INVALID_ARG for a bad range or a periodic
 *   y axis shorter than the discs' reach plus 8 rows.  dilbm_step,
 *   dilbm_set_moving_frame and batches refuse a strip.
 * dilbm_strip_begin: queue this step's sweep of the strip (its halos are the
 *   rows received in the previous exchange; the initial state at the start),
 *   the per-particle sums over the strip's nodes, and copies of the strip's
 *   first and last rows into the send buffers.  Asynchronous.
 * Exchange (caller, after the stream has reached that point): recv_south <-
 *   the south neighbour's send_north, recv_north <- the north neighbour's
 *   send_south (row_elems stored elements each, the storage type's), and
 *   fpart (np x 5 doubles: Fx, Fy, T, repulsion x, y) <- its sum over all
 *   ranks, identical on every rank.
 * dilbm_strip_end: queue the rigid-body update with the summed fpart and the
 *   binning for the next step.  Asynchronous.
 * dilbm_strip_buffers: device addresses of the exchange buffers (owned by the
 *   context, valid until dilbm_destroy); any pointer may be NULL.
 * Every other call (dilbm_forces, dilbm_fields on the strip's rows,
 * dilbm_get/set_populations of the strip's rows, dilbm_sync) works as on a
 * whole lattice.
 */
int dilbm_create_strip(const dilbm_grid *grid, dilbm_lattice lattice, double tau, double interface_width,
                       const dilbm_particle *particles, int np, int y0, int y1, void *cuda_stream,
                       dilbm_ctx **out);
int dilbm_strip_begin(dilbm_ctx *ctx);
int dilbm_strip_end(dilbm_ctx *ctx);
int dilbm_strip_buffers(dilbm_ctx *ctx, double **fpart, void **send_south, void **send_north, void **recv_south,
                        void **recv_north, long long *row_elems);

/*
 * Hydrodynamic force and torque of the last step (Eqs. 18-19, lattice units,
 * force on the particle), optional Wan-Turek force of the last step, and the
 * current particle state.  force: host, np x 3 (Fx, Fy, T); fcol: host,
 * np x 2 or NULL; state: host, np entries or NULL.  Synchronises the stream.
 * Errors: INVALID_ARG, CUDA, and any sticky device error.
 */
int dilbm_forces(dilbm_ctx *ctx, double *force, double *fcol, dilbm_particle *state);

/*
 * Time mean of the hydrodynamic force and torque (Eqs. 18-19) over the steps
 * since create or the last dilbm_force_mean_reset(): mean host np x 3
 * (Fx, Fy, T); *nsteps receives the number of steps averaged (the mean is 0
 * when it is 0).  Each step adds its force in FP64 on the device.
 * dilbm_force_mean synchronises the stream; the reset is asynchronous.
 */
int dilbm_force_mean(dilbm_ctx *ctx, double *mean, long long *nsteps);
int dilbm_force_mean_reset(dilbm_ctx *ctx);

/*
 * Moving computational domain (Sec. 3.5: the domain moves one lattice unit
 * whenever the particle has moved one, after Wang et al. 2013).  From the
 * next step on, the frame follows particle `particle` (0 <= particle < np;
 * -1 switches the frame off) about the reference x_ref: at the end of each
 * step, with d the particle's x at the start of that step minus x_ref
 * (minimum image on a periodic x axis), the frame moves s = +1 column when
 * d >= 1, s = -1 when d <= -1, else not at all.  Moving by s takes the
 * populations of column x + s to column x (rolled on a periodic x axis;
 * otherwise the entering column repeats its neighbour, a zero-gradient state
 * the edge scheme then overwrites), subtracts s from every particle's x and
 * adds s to the frame offset: lab x = frame x + offset.  The move is plain:
 * in a pressure-driven channel it displaces the linear pressure field by
 * one column against the fixed end densities, which the ends re-absorb.
 * Positions reported by dilbm_forces() are frame positions.  A checkpoint
 * (dilbm_get_populations, dilbm_forces' state) holds frame positions and
 * populations: keep the offset beside it.  One more kernel launch per step
 * while the frame is on.  Requires
 * nx x (bytes per stored population) <= 48 KiB.  Contexts with a moving
 * frame cannot join a batch.
 * Errors: INVALID_ARG (particle out of range, x_ref not finite, lattice too
 * wide), CUDA.
 */
int dilbm_set_moving_frame(dilbm_ctx *ctx, int particle, double x_ref);

/*
 * Failure-detection check, with no fault: one warp waits, with the bounded
 * wait the sweep uses on its staging barriers (1 s limit, timed by the
 * device's global timer), on a shared-memory barrier that nothing ever
 * arrives at.  The wait gives up, the kernel records the timeout in a private
 * error word as the sweep does and returns; the call reads it back.  Returns
 * DILBM_ERR_TIMEOUT (the expected outcome) with *waited_seconds (nullable)
 * the wait measured on the device, DILBM_OK if the wait completed, or
 * DILBM_ERR_CUDA.  Synchronises the stream; allocates 16 bytes for the call.
 * The device stays usable.
 */
int dilbm_wait_probe(void *cuda_stream, double *waited_seconds);

/*
 * Columns the frame has moved since create (0 if it never moved).  offset:
 * host.  Synchronises the stream.  Errors: INVALID_ARG, CUDA.
 */
int dilbm_frame_offset(dilbm_ctx *ctx, long long *offset);

/*
 * Macroscopic fields at the current time level, row-major [ny][nx] FP32:
 * density (Eq. 5), corrected velocity (Eq. 17) and solid fraction (Eq. 14),
 * taken from the populations the next step would collide.  Any pointer may be
 * NULL.  on_device != 0: the pointers are device memory; otherwise host
 * memory and the call synchronises the stream.
 */
int dilbm_fields(dilbm_ctx *ctx, float *rho, float *ux, float *uy, float *phi, int on_device);

/*
 * Checkpoint / resume: the post-collision populations f_i, host FP64 array of
 * 9 x ny x nx (direction-major, rows of x), in the direction order of Eq. 3.
 * dilbm_set_populations also accepts any state written by dilbm_get_populations
 * of a context of the same size.  Both synchronise the stream.
 */
int dilbm_get_populations(dilbm_ctx *ctx, double *f);
int dilbm_set_populations(dilbm_ctx *ctx, const double *f);

/*
 * Replace the particle state: host array of the np given at create, checked
 * as at create (inside the lattice, positive finite radius and density,
 * finite velocities, phi tail within the per-particle tile map).  The state is
 * copied into the context's pinned staging before the call returns, so the
 * caller may reuse the array at once; the upload and the re-binning for the
 * next step are queued on the stream (asynchronous).  Errors: INVALID_ARG
 * (count differs from create, or a particle fails a check; nothing changes),
 * OOM, CUDA.
 */
int dilbm_set_particles(dilbm_ctx *ctx, const dilbm_particle *particles, int np);

/* Wait for queued work; return the first sticky device error, else DILBM_OK. */
int dilbm_sync(dilbm_ctx *ctx);

/* Free the context (synchronises its stream).  NULL is ignored. */
void dilbm_destroy(dilbm_ctx *ctx);

/* Message of the last error on this host thread ("" if none). */
const char *dilbm_last_error(void);

/*
 * Measurement: with timing on, CUDA events bracket every lattice-sweep launch
 * on the context's stream; dilbm_sweep_time() returns their summed duration
 * in milliseconds and the number of launches since timing was (re)enabled.
 * dilbm_launch_count() is the number of kernels this context has launched.
 */
int dilbm_set_timing(dilbm_ctx *ctx, int enable);
int dilbm_sweep_time(dilbm_ctx *ctx, double *ms_total, long long *launches);
long long dilbm_launch_count(const dilbm_ctx *ctx);

/*
 * Batches: many contexts advanced together (the same equations, Eqs. 13-19,
 * 22-24, 28-29, on every member).  One step of a batch is one sweep launch
 * over the concatenated row segments of all members and one particle launch
 * over all their particles, replayed from CUDA graphs captured at create;
 * every member's result is bit for bit the one dilbm_step gives it alone.
 *
 * dilbm_batch_create: members[0..n-1] (1 <= n <= 1024 distinct contexts, all
 *   with the same storage; they stay owned by the caller and must outlive the
 *   batch).  The batch runs on a private stream ordered after, and before,
 *   each member's own stream by events, so member calls (forces, fields,
 *   dilbm_step) may be mixed with batch steps.  cuda_stream is unused.
 * dilbm_batch_step: advance every member nsteps (asynchronous).
 * dilbm_batch_sync: wait; return the first member's sticky device error and
 *   its index in *first_failed (-1 if none; pointer may be NULL).  Every
 *   member's error word is read with one copy.
 * dilbm_batch_errors: wait; codes[k] (host, n ints) receives member k's error
 *   (DILBM_OK, UNSTABLE, TIMEOUT or OVERFLOW).  Returns CUDA on a CUDA error.
 * dilbm_batch_set_timing / dilbm_batch_sweep_time: CUDA events around every
 *   batched sweep launch (timing replaces graph replay by direct launches).
 * dilbm_batch_launch_count: kernels the batch has launched.
 */
typedef struct dilbm_batch dilbm_batch;
int dilbm_batch_create(dilbm_ctx *const *members, int n, void *cuda_stream, dilbm_batch **out);
int dilbm_batch_step(dilbm_batch *batch, long long nsteps);
int dilbm_batch_sync(dilbm_batch *batch, int *first_failed);
int dilbm_batch_errors(dilbm_batch *batch, int *codes);
int dilbm_batch_set_timing(dilbm_batch *batch, int enable);
int dilbm_batch_sweep_time(dilbm_batch *batch, double *ms_total, long long *launches);
long long dilbm_batch_launch_count(const dilbm_batch *batch);
void dilbm_batch_destroy(dilbm_batch *batch);
int dilbm_batch_autotune(dilbm_batch *batch, int reps, int *warps, int *blocks_per_sm);
int dilbm_batch_set_shape(dilbm_batch *batch, int warps, int blocks_per_sm);

/*
 * Launch shape of the lattice sweep, and its autotuner.  A shape is the
 * number of row segments (128 nodes of one row) a block keeps in flight --
 * warps per block, 2, 4 or 8 -- and the persistent blocks per SM
 * (blocks_per_sm, 0: as many as fit).  The tile a row segment belongs to
 * (128 x 8 nodes) is
 * fixed: it orders the force partials.  Every shape runs the same arithmetic
 * on every node, so results are bit for bit the same in every shape.
 *
 * dilbm_autotune / dilbm_batch_autotune time every candidate shape (each
 * warps-per-block value with as many blocks per SM as fit and with half as
 * many) in 3 interleaved rounds of reps
 * sweep launches of the current state
 * (reps <= 0: 10; the launches only write what the next step overwrites),
 * keep the one with the smallest median round time and report it in *warps
 * and *blocks_per_sm (nullable).  The choice is cached
 * per process, keyed by storage, edge handling and lattice size (for a
 * batch: storage, member count and total row segments), so tuning a second
 * context or batch of the same key launches nothing.  Both synchronise.
 * dilbm_set_shape / dilbm_batch_set_shape set a shape by hand.  A PS-LBM
 * context keeps the default shape (8 warps, blocks_per_sm 0): dilbm_autotune
 * reports it without timing and dilbm_set_shape rejects any other.
 * Errors: INVALID_ARG, CUDA.
 */
int dilbm_autotune(dilbm_ctx *ctx, int reps, int *warps, int *blocks_per_sm);
int dilbm_set_shape(dilbm_ctx *ctx, int warps, int blocks_per_sm);

/*
 * Device memory dilbm_create allocates for a lattice of grid->nx x grid->ny
 * with np particles in grid->storage (populations A and B, tile bins, force
 * partials, particle state).  The driver rounds each allocation up, so the
 * memory actually taken is slightly larger.  A PS context adds its covered-area
 * tables, np x (2K+1)^2 x 4 bytes, which depend on the radii and are not
 * counted here.  Host-only arithmetic.
 * Errors: INVALID_ARG (NULL pointer, bad size or storage).
 */
int dilbm_footprint(const dilbm_grid *grid, int np, unsigned long long *bytes);

/*
 * Serving: a request loop that keeps every admitted lattice resident on the
 * device and advances all of them together (continuous batching).  The
 * method is unchanged: each job is the DI-LBM problem of dilbm_create,
 * advanced nsteps steps (Eqs. 13-19, 22-24, 28-29), and its result is bit for
 * bit the one dilbm_step gives it alone.
 *
 * A job is queued at submit (host only).  dilbm_server_progress() runs one
 * macro-step: it launches the next k steps of every running job as one batch
 * (k = min(macro_steps, fewest steps any running job has left, steps until
 * any job's mean-force window opens)), admits
 * queued jobs while the GPU works -- in arrival order, while a job slot is
 * free and the job's dilbm_footprint fits the memory budget -- then waits for
 * the k steps, retires the jobs that reached their step count (their forces
 * and particle state are copied to the host and their device memory freed)
 * and re-forms the batch from the running jobs.  Jobs admitted in one call
 * start their steps in the next.
 *
 * Times are seconds on the server's clock (a monotonic host clock, zero at
 * create; dilbm_server_clock()).  One host thread drives a server.
 */
typedef enum {
    DILBM_ADMIT_FIFO = 0,       /* admit in arrival order; stop at the first job that does not fit */
    DILBM_ADMIT_FIRST_FIT = 1   /* admit every queued job that fits, in arrival order */
} dilbm_admit_policy;

/* dilbm_server_config.storage: each job keeps its own grid.storage; the
 * server steps one batch per storage type, all by the same macro-steps. */
#define DILBM_STORAGE_PER_JOB (-1)
/* dilbm_server_config.storage: FP16 deviation storage for the jobs whose flow
 * 11 stored mantissa bits resolve, FP32 for the others.  A job runs in FP32
 * when its tau exceeds auto_tau_max or its discs cover more than
 * auto_area_max of the lattice: a slow, viscous flow (large tau) or a packed
 * bed of discs needs a pressure gradient whose density deviation is large
 * beside the velocity signal the force of Eqs. 18-19 depends on, and FP16
 * stores the two together.  The server steps one batch per storage type. */
#define DILBM_STORAGE_AUTO (-2)

typedef struct {
    int storage;                /* dilbm_storage of every job (a job's grid.storage is ignored),
                                   or DILBM_STORAGE_PER_JOB */
    int max_jobs;               /* jobs resident at once, 1..1024 */
    long long macro_steps;      /* most steps per macro-step, >= 1 */
    double memory_budget;       /* bytes the resident jobs may take; <= 0: 90% of free device memory at create */
    int policy;                 /* dilbm_admit_policy */
    double auto_tau_max;        /* DILBM_STORAGE_AUTO: largest tau run in FP16 (<= 0: 0.6) */
    double auto_area_max;       /* DILBM_STORAGE_AUTO: largest disc area fraction run in FP16 (<= 0: 0.05) */
} dilbm_server_config;

typedef struct {
    dilbm_grid grid;            /* as for dilbm_create */
    double tau, interface_width;
    const dilbm_particle *particles;   /* host, np entries, copied at submit */
    int np;
    long long nsteps;           /* >= 1 */
    long long mean_window;      /* 0..nsteps: the result also carries the time mean of the force
                                   over the job's last mean_window steps (dilbm_force_mean) */
    double arrival;             /* server-clock time the request arrived; < 0: the submit time */
} dilbm_job;

typedef enum {
    DILBM_JOB_QUEUED = 0,
    DILBM_JOB_RUNNING = 1,
    DILBM_JOB_DONE = 2,
    DILBM_JOB_FAILED = 3
} dilbm_job_state;

typedef struct {
    int state;                  /* dilbm_job_state */
    int error;                  /* DILBM_OK, or the code that failed the job */
    int np;
    long long steps_done;
    double arrival, admitted, finished;   /* server clock; -1 until reached */
    unsigned long long footprint;         /* dilbm_footprint of the job */
    int storage;                          /* the dilbm_storage the job runs in */
} dilbm_job_status;

typedef struct {
    int running, queued;
    long long done, failed;
    long long macro_steps;      /* macro-steps run so far */
    double node_updates;        /* sum over finished steps of the running jobs' nodes */
    double busy_seconds;        /* host time spent inside dilbm_server_progress, of which: */
    double form_seconds;        /*   forming batches and launching macro-steps */
    double admit_seconds;       /*   setting up admitted jobs (mostly while the GPU steps) */
    double wait_seconds;        /*   waiting for macro-steps to finish */
    double retire_seconds;      /*   reading results and freeing finished jobs (the GPU is idle) */
    unsigned long long memory_in_use;     /* sum of the running jobs' footprints */
    long long launches;         /* kernels launched for the jobs so far */
} dilbm_server_stats;

typedef struct dilbm_server dilbm_server;

/* Create a server; cuda_stream (NULL: a private stream) carries the jobs'
 * set-up and read-back.  Errors: INVALID_ARG, CUDA. */
int dilbm_server_create(const dilbm_server_config *cfg, void *cuda_stream, dilbm_server **out);
/* Queue a job; *id receives its handle (>= 0).  A job whose footprint exceeds
 * the budget is rejected here with INVALID_ARG. */
int dilbm_server_submit(dilbm_server *srv, const dilbm_job *job, long long *id);
/* One macro-step (see above); *stats (nullable) receives the counters after it. */
int dilbm_server_progress(dilbm_server *srv, dilbm_server_stats *stats);
/* State and timestamps of a job. */
int dilbm_server_status(const dilbm_server *srv, long long id, dilbm_job_status *st);
/* Result of a DONE job: force (host, np x 3: Fx, Fy, T of its last step,
 * Eqs. 18-19), force_mean (host, np x 3, nullable: their mean over the job's
 * last mean_window steps) and state (host, np entries, nullable); then its
 * record is released.  Errors: INVALID_ARG (unknown id or job not DONE). */
int dilbm_server_result(dilbm_server *srv, long long id, double *force, double *force_mean,
                        dilbm_particle *state);
double dilbm_server_clock(const dilbm_server *srv);
/* Free every job and the server (synchronises). */
void dilbm_server_destroy(dilbm_server *srv);

/*
 * One time step that allocates no device memory.  The paper has no
 * counterpart: this is a calling convention, not part of the method.
 *
 * For callers that cannot call cudaMalloc where they need a step: a solver
 * that owns a fixed device memory pool and allows no further allocations, a
 * stream-ordered pipeline in which an allocation would synchronise the device,
 * or a host that has budgeted every byte of the GPU in advance.  It runs the
 * same kernels as dilbm_step; their scratch memory (tile bins, force
 * partials, particle state in structure-of-arrays form, the error word) lives
 * in one static device array of about 8 MB compiled into the library, which
 * every GPU that loads the library holds until the process exits.
 *
 *   grid, tau, interface_width  as for dilbm_create; storage must be DILBM_FP32.
 *   f_in   device, DILBM_STATIC_POP_FLOATS(nx, ny) floats: the post-collision
 *          populations as deviations f_i - w_i (w_i the D2Q9 weights in FP32),
 *          plane i of ny rows of DILBM_STATIC_PITCH(nx) floats, starting
 *          DILBM_STATIC_POP_OFFSET floats into the buffer; the
 *          DILBM_STATIC_POP_OFFSET floats before and after the planes must be
 *          readable (their values are never used).  Not modified.
 *   f_out  device, same size and layout, receives the next step's
 *          populations; must not alias f_in.
 *   particles, np  device array of np dilbm_particle, read and updated in
 *          place (np <= DILBM_STATIC_MAX_PARTICLES).  They are checked on the
 *          device with dilbm_create's rules (centre inside the lattice, finite
 *          positive radius and density, finite velocities, a phi tail of at
 *          most 128 tiles); a bad particle gives DILBM_ERR_INVALID_ARG before
 *          any other work, with f_out and the particles left unchanged.
 *   force  device, np x 3 doubles: the hydrodynamic force (x, y) and torque
 *          on each particle in this step.
 *   cuda_stream  stream for all work.
 * Limits: ceil(nx/128) * ceil(ny/8) <= DILBM_STATIC_MAX_TILES tiles and
 * np <= DILBM_STATIC_MAX_PARTICLES; larger problems are rejected with
 * DILBM_ERR_INVALID_ARG before any work is queued (use dilbm_create for them).
 * Every call shares the static array: the call clears what must start at zero
 * (bin counts, error word) but calls that overlap on the GPU (other streams,
 * other host threads) race on it and must not be issued.  The first call on a
 * device looks up the array's device address with that device current; make
 * that first call before any stream capture.  The call ends by synchronising
 * the stream to read the error word; it returns DILBM_OK or
 * INVALID_ARG / CUDA / UNSTABLE / TIMEOUT / OVERFLOW, with the message in
 * dilbm_last_error().
 */
#define DILBM_STATIC_MAX_TILES 1024
#define DILBM_STATIC_MAX_PARTICLES 256
#define DILBM_STATIC_PITCH(nx) ((((nx) + 31) / 32) * 32)
#define DILBM_STATIC_POP_OFFSET 256
#define DILBM_STATIC_POP_FLOATS(nx, ny) (9LL * (ny) * DILBM_STATIC_PITCH(nx) + 2 * DILBM_STATIC_POP_OFFSET)
int dilbm_step_static(const dilbm_grid *grid, double tau, double interface_width, const float *f_in,
                      float *f_out, dilbm_particle *particles, int np, double *force, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* DILBM_H */
