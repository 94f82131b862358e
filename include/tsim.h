/*
 * tsim.h -- C ABI of the GB300 IMPM elastomer simulator (libtsim.so).
 *
 * The library advances the gel elastomer of an optical tactile sensor under
 * a moving rigid indenter with the improved Material Point Method of
 * "Simulation of Optical Tactile Sensors Supporting Slip and Rotation using
 * Path Tracing and IMPM" (Sec. III-A, Eqs. 1-9, Algorithm 1).  The calls
 * follow the paper's statement of the problem: initialise the elastomer and
 * its material (Sec. IV-B), set the object and the pose sequence it moves
 * along (Fig. 2 (A)-(B)), step, and read back the deformed surface that the
 * renderer consumes (Sec. IV-B, Fig. 2 (C)).  The object is an analytic SDF
 * with stick/slip contact, or rigid particles taking part in P2G (the
 * paper's own coupling, tsim_set_object_particles).  Context-free calls
 * render the sensor image of a surface (Sec. III-B path tracing,
 * tsim_render) and compare images (Sec. IV, tsim_image_metrics).
 *
 * Conventions
 *   - Every call returns an int status (TSIM_OK or a TSIM_ERR_* code) except
 *     tsim_destroy and tsim_last_error.  On failure tsim_last_error() gives
 *     a human-readable reason for the calling thread.
 *   - Units are SI (metres, seconds, kilograms, pascals).  Arrays are
 *     row-major float32 unless stated otherwise.
 *   - A context holds n_inst independent instances (sensor pads) that
 *     advance in lockstep.  Every instance index argument is 0..n_inst-1.
 *   - The library owns all device state inside the opaque tsim_ctx and
 *     allocates it in tsim_create only; no later call allocates device
 *     memory.  The caller owns every pointer it passes.  Pointers are host
 *     pointers when on_device == 0 and device pointers of the context's
 *     device otherwise.
 *   - Work is enqueued on the CUDA stream given to tsim_create (a
 *     cudaStream_t passed as void*; NULL = legacy default stream).
 *     tsim_step is asynchronous; device-detected errors (non-finite state,
 *     J <= 0, a particle leaving the node box, a full cell block, a device
 *     wait that gave up) are
 *     latched per instance and returned by the next tsim_sync, tsim_stats
 *     or tsim_read_* call, which synchronise the stream.
 *   - Positions live in the gel frame: the block occupies
 *     [0, cx*dx] x [0, cy*dx] x [0, cz*dx] with its base plane at z = 0.
 *     Node (a, b, c) of the node box sits at ((a-ox)dx, (b-oy)dx, (c-oz)dx).
 */
#ifndef TSIM_H
#define TSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define TSIM_OK 0
#define TSIM_ERR_INVALID_ARG 1   /* bad argument; nothing was changed */
#define TSIM_ERR_OOM 2           /* device allocation failed in tsim_create */
#define TSIM_ERR_CUDA 3          /* a CUDA runtime call failed */
#define TSIM_ERR_NUMERIC 4       /* non-finite state or J <= 0 (latched) */
#define TSIM_ERR_DOMAIN 5        /* a particle left the node box (latched) */
#define TSIM_ERR_CAPACITY 6      /* a full cell block found the instance's spill slots full too (latched) */
#define TSIM_ERR_STATE 7         /* calls out of order (e.g. step before particles) */
#define TSIM_ERR_TIMEOUT 8       /* a bounded device wait gave up (latched) */

/* indenter shapes (rigid analytic SDF; Sec. III-A object, Sec. IV-A indenters) */
#define TSIM_NONE (-1)
#define TSIM_SPHERE 0     /* p = [r] */
#define TSIM_CYLINDER 1   /* p = [r, h, edge_round]; axis vertical, flat face down */
#define TSIM_BOX 2        /* p = [hx, hy, hz, edge_round] (half sizes) */
#define TSIM_PRISM 3      /* p = [side, length, edge_round]; equilateral section,
                             apex down, extruded along the local x axis */
#define TSIM_PERLIN 4     /* p = [hx, hy, hz, edge_round, amp, period, persistence,
                             octaves]; rounded plate minus amp * fbm of improved
                             noise (permutation table in perm) */

/* base boundary modes */
#define TSIM_BASE_FIXED 0 /* bottom fixed to the sensor (Sec. III-A, Algorithm 1) */
#define TSIM_BASE_SLIP 1  /* only the normal (z) velocity is held at the base */
#define TSIM_BASE_FREE 2  /* no base (free body; used by tests) */

/* particle tag bits (low 29 bits = particle id) */
#define TSIM_TAG_BOTTOM 0x80000000u  /* bottom cell layer: v_z = 0 after G2P */
#define TSIM_TAG_TOP 0x40000000u     /* surface layer read by tsim_read_surface */
#define TSIM_TAG_MARKER 0x20000000u  /* embedded marker */

typedef struct tsim_ctx tsim_ctx;

/* Elastomer block of cx x cy x cz cells of size dx with ppc (= 8) particles
 * per cell, inside a node box of nx x ny x nz nodes whose node (ox, oy, oz)
 * is the gel origin.  nx, ny, nz must be multiples of 4 (cell blocks), and
 * a node box holds fewer than 2^31 nodes. */
typedef struct {
    int cx, cy, cz;
    int nx, ny, nz;
    int ox, oy, oz;
    int ppc;
    float dx;
} tsim_gel_desc;

/* Compressible Neo-Hookean elastomer (S_p of Eq. 4): Young's modulus E,
 * Poisson ratio nu, density rho; gravity acceleration added to the grid. */
typedef struct {
    float E, nu, rho;
    float gravity[3];
} tsim_material;

/* Rigid indenter.  Its pose is given by the tip (lowest point, the
 * calibration point x_o of Algorithm 1) and a yaw about the vertical axis
 * through the tip; the SDF frame centre sits tip_offset above the tip.
 * mu is the Coulomb friction coefficient of the stick/slip contact: a
 * contact node sticks while |v_t| <= mu |v_n|.  mu_kinetic (<= mu; 0 or
 * negative: mu) sets the slip, which reduces |v_t| by mu_kinetic |v_n| --
 * a reading for the long-distance sliding that Sec. VI names as a
 * limitation of the method. */
typedef struct {
    int kind;
    float p[8];
    float mu;
    float tip_offset;
    int32_t perm[256];
    float mu_kinetic;
} tsim_indenter_desc;

/* Pose keyframe: at substep `substep` the tip is at tip[] with yaw `yaw`
 * (radians); poses between keyframes are linear in the substep index and
 * held constant before the first and after the last keyframe. */
typedef struct {
    int32_t substep;
    float tip[3];
    float yaw;
} tsim_keyframe;

/* Solver: substep dt; relrest_limit = LIMIT of Algorithm 1 (1 gives plain
 * MPM, the paper's "normal" group); relrest_threshold = its threshold;
 * base_mode = TSIM_BASE_*; walls != 0 zeroes the velocity of the 2-node
 * ring of the node box at +-x, +-y, +z (Sec. III-A boundary handling). */
typedef struct {
    float dt;
    int relrest_limit;
    float relrest_threshold;
    int base_mode;
    int walls;
} tsim_solver_desc;

typedef struct {
    int64_t substeps;          /* substeps completed */
    int64_t passes;            /* P2G->grid->G2P passes, summed over instances */
    int64_t particle_updates;  /* particles x passes, summed over instances */
    uint32_t status;           /* OR of latched device error bits of all instances */
    int32_t n_inst;
    int64_t spilled;           /* particles found in spill slots, summed over substeps */
    int32_t spill_max;         /* most particles one instance held in spill slots at once */
    int32_t pad_;
} tsim_stats_t;

/* Create a context of n_inst instances on the current CUDA device.
 * gels, mats: arrays of n_inst descriptors (host).  stream: cudaStream_t or
 * NULL.  Allocates all device state: particle slots, node arrays, staging.
 * *out is NULL on failure.  Paper: Sec. IV-B (elastomer initialisation). */
int tsim_create(int n_inst, const tsim_gel_desc *gels, const tsim_material *mats,
                void *stream, tsim_ctx **out);

/* Solver parameters shared by all instances (Algorithm 1 LIMIT/threshold,
 * boundary handling of Sec. III-A).  Must precede tsim_write_particles. */
int tsim_set_solver(tsim_ctx *ctx, const tsim_solver_desc *solver);

/* Indenter of instance inst (host descriptor). */
int tsim_set_indenter(tsim_ctx *ctx, int inst, const tsim_indenter_desc *ind);

/* Represent the indenter of instance inst by n rigid particles (the paper's
 * own coupling, Sec. III-A and Sec. IV-B: object particles with a
 * prescribed velocity that take part in particle-to-grid): q holds n rows
 * of (x, y, z) in the indenter frame (metres, about the SDF frame centre,
 * before the yaw), each particle of the given mass.  In every pass each
 * object particle adds to the grid at its pose position with the rigid
 * velocity v_lin + omega z x (x - c) and that motion's affine field (Eqs.
 * 1-3, no stress); the SDF contact projection of the grid update is then
 * off for this instance, while the SDF still decides whether x_e is in
 * contact for the relative-rest check.  n = 0 returns to the SDF contact.
 * q: host or device (on_device), copied before the call returns.  n is
 * limited to max(65536, particles / 4) per instance (reserved at create):
 * TSIM_ERR_INVALID_ARG beyond that. */
int tsim_set_object_particles(tsim_ctx *ctx, int inst, const float *q, int n, float mass, int on_device);

/* Pose keyframes of instance inst: n_kf (1..64) rows, increasing substep.
 * Fig. 2 (B): the object moves step by step to its target pose. */
int tsim_set_trajectory(tsim_ctx *ctx, int inst, const tsim_keyframe *kf, int n_kf,
                        int on_device);

/* Set the particle state of instance inst in particle-id order:
 * x[n*3], v[n*3], C[n*9] (affine field, row-major), F[n*9] (deformation
 * gradient, row-major), tag[n] (TSIM_TAG_* | id).  n must equal
 * cx*cy*cz*ppc and ids must be 0..n-1.  Bins the particles into cell
 * blocks and runs the particle-to-grid transfer of this state.
 * Paper: Sec. III-A particle state (x, v, m, C, F). */
int tsim_write_particles(tsim_ctx *ctx, int inst, const float *x, const float *v,
                         const float *C, const float *F, const uint32_t *tag, int n,
                         int on_device);

/* Set the substep index of the next substep (the clock of the pose
 * keyframes), for all instances.  Default 0. */
int tsim_set_substep(tsim_ctx *ctx, int64_t k);

/* Advance every instance by n_substeps IMPM time steps (Algorithm 1):
 * passes of P2G (Eqs. 1-4), grid update with gravity, stick/slip contact,
 * walls and fixed base (Eq. 5), G2P (Eqs. 6-7) until the relative-rest
 * check accepts or LIMIT passes ran, then the F and x move (Eqs. 8-9).
 * Asynchronous on the context stream. */
int tsim_step(tsim_ctx *ctx, int n_substeps);

/* Read the state of instance inst in particle-id order (any of x, v, C, F
 * may be NULL).  v and C are those of the last completed substep.
 * Synchronises; returns latched device errors. */
int tsim_read_particles(tsim_ctx *ctx, int inst, float *x, float *v, float *C, float *F,
                        int n, int on_device);

/* Grid mass and momentum of instance inst after the particle-to-grid
 * transfer of its current state (Eqs. 1-2): out[nx*ny*nz*4] holds
 * (M_i, MG_i.x, MG_i.y, MG_i.z) per node, x fastest.  Synchronises. */
int tsim_read_grid(tsim_ctx *ctx, int inst, float *out, int on_device);

/* Surface of instance inst: height[H*W] (z of the gel surface) and unit
 * normals normal[H*W*3] on a W x H pixel grid with pixel (u, v) centred at
 * ((u+0.5)*pitch, (v+0.5)*pitch).  Heights are the 2-D quadratic B-spline
 * average of the z of TSIM_TAG_TOP particles; pixels with no particle read
 * the gel height; normals come from central differences of the height.
 * W*H <= 1<<20.  Paper: Sec. IV-B, Fig. 2 (C) (depth map of the surface
 * particles).  Synchronises. */
int tsim_read_surface(tsim_ctx *ctx, int inst, float *height, float *normal, int W, int H,
                      float pitch, int on_device);

/* Displacement field of instance inst: u[H*W*3] = the 2-D quadratic
 * B-spline average over TSIM_TAG_TOP particles of x - X, with the weights
 * taken at each particle's reference position X (x_ref[n*3], particle-id
 * order, host or device per on_device) on the pixel grid of
 * tsim_read_surface; pixels with no particle read 0.  W*H <= 1<<19.  This
 * is the surface displacement that the learned surrogate is trained on
 * (Sec. IV-B depth map, taken per component).  Synchronises. */
int tsim_read_displacement(tsim_ctx *ctx, int inst, const float *x_ref, float *u, int W, int H, float pitch,
                           int on_device);

/* Height of the indenter's underside above the gel top, h[H*W], at the pose
 * of the next substep, on the pixel grid of tsim_read_surface: the first
 * crossing of the SDF zero level going up each pixel column from
 * gel top - clip (sphere tracing, at most 128 steps); columns that miss the
 * shape read +clip; values are clamped to [-clip, clip].  This is the
 * indenter heightmap that the surrogate takes as input.  Synchronises. */
int tsim_read_indenter_height(tsim_ctx *ctx, int inst, float *h, int W, int H, float pitch, float clip,
                              int on_device);

/* Positions of m particles given by id (ids[m], host) of instance inst:
 * xyz[m*3].  Used for embedded marker tracks.  Synchronises. */
int tsim_read_markers(tsim_ctx *ctx, int inst, const int32_t *ids, int m, float *xyz,
                      int on_device);

/* Per-substep log of instance inst for the last n substeps (n <= 32768):
 * passes[n] taken by the relative-rest loop and calib[n] the id of the
 * calibration particle x_e.  Either pointer may be NULL.  Synchronises. */
int tsim_read_log(tsim_ctx *ctx, int inst, int32_t *passes, int32_t *calib, int n);

/* Wait for all enqueued work; returns latched device errors. */
int tsim_sync(tsim_ctx *ctx);

/* Counters; synchronises. */
int tsim_stats(tsim_ctx *ctx, tsim_stats_t *out);

/* Execution configuration of the substep schedule.  It changes how the same
 * kernels are launched, never what they compute, so the state evolves as
 * under any other configuration.  Batched contexts of uneven instances are
 * where the choice matters (project addition: the paper has no counterpart). */
typedef struct {
    int grid_threads;      /* threads per CTA of the grid update: 128, 256 or 512 */
    int grid_flat;         /* 0: one launch row per instance, sized by the largest
                              instance; 1: one 1-D launch over the node ranges of
                              all instances packed back to back */
    int graph_chunk;       /* substeps per CUDA graph launch in graph mode (1..200) */
    float us_per_mupdate;  /* set by tsim_autotune: measured microseconds per
                              million particle-updates of the chosen configuration */
} tsim_tuning_t;

/* Set (synchronises; rebuilds graphs) or read the configuration.  Default:
 * 256 threads, per-instance rows, 20 substeps per graph. */
int tsim_set_tuning(tsim_ctx *ctx, const tsim_tuning_t *cfg);
int tsim_get_tuning(tsim_ctx *ctx, tsim_tuning_t *out);

/* Autotuner: advance by n substeps as tsim_step(n) would, timing the
 * candidate configurations on successive equal windows of those substeps
 * (CUDA events; cost per particle-update): the six grid-update shapes
 * {128, 256, 512 threads} x {per-instance, packed} in two interleaved
 * rounds, then in graph mode the chunk lengths {10, 20, 40} with the best
 * shape.  The fastest is kept for later calls and written to *out (may be
 * NULL).  n must allow windows of >= 2 substeps (stream mode; n >= 24) or of
 * a multiple of 40 (graph mode; n >= 600), else TSIM_ERR_INVALID_ARG.
 * Synchronises after every window; latched device errors are returned. */
int tsim_autotune(tsim_ctx *ctx, int n_substeps, tsim_tuning_t *out);

/* Capture the substep sequence in a CUDA graph with a device-driven loop
 * over relative-rest passes (enable != 0) or launch kernels one by one. */
int tsim_use_graph(tsim_ctx *ctx, int enable);

/* Per-kernel timing with CUDA events recorded on the context stream
 * (enable != 0): around every launch of the commit transfer (the accepted
 * pass of Algorithm 1 that moves x and F) and around every substep's loop of
 * repeated passes (transfer, grid update and check of each repeat pass; in
 * graph mode the events bracket the loop node as a whole).
 * tsim_pass_time returns, since the last reset, the commit launches, their
 * total milliseconds and the total milliseconds inside the repeat-pass loops
 * (any output may be NULL), and resets the counters; tsim_kernel_time returns
 * the first two.  Both synchronise. */
int tsim_profile(tsim_ctx *ctx, int enable);
int tsim_pass_time(tsim_ctx *ctx, int64_t *launches, double *commit_ms, double *loop_ms);
int tsim_kernel_time(tsim_ctx *ctx, int64_t *launches, double *total_ms);

/* ---- Allocation-free particle-to-grid transfer --------------------------
 * Not a part of the paper's method: the paper has no counterpart.  It serves
 * callers that cannot allocate device memory -- a plug-in whose host
 * application owns all device memory through its own pool, a real-time loop
 * that must not touch the allocator once running, a process with a memory
 * budget fixed at start-up.  It computes the same transfer as the P2G of a
 * context (mass and momentum of Eqs. 1-4, as tsim_read_grid returns it) for
 * a particle state and a grid the caller owns, using only a fixed scratch
 * array of TSIM_NOALLOC_SCRATCH_BYTES bytes that the library reserves
 * statically on every GPU that loads it (held until the process exits).
 *
 * gel, mat: host descriptors (node box a multiple of 4 in every direction,
 * at most TSIM_NOALLOC_MAX_BLOCKS 4x4x4 cell blocks); dt: substep of the
 * stress impulse of Eq. 4; x[n*3], v[n*3], C[n*9], F[n*9]: device arrays in
 * the layout of tsim_write_particles, 1 <= n <= TSIM_NOALLOC_MAX_PARTICLES,
 * each 4-byte aligned; grid[nx*ny*nz*4]: device output, 16-byte aligned,
 * (M, MG) per node, x fastest (overwritten); stream: cudaStream_t or NULL.
 * All five arrays must be device memory of the current device or managed
 * memory.  Sizes beyond the maxima, misaligned arrays and host pointers
 * return TSIM_ERR_INVALID_ARG before any GPU work.
 * Particles outside the node box give TSIM_ERR_DOMAIN, J <= 0 gives
 * TSIM_ERR_NUMERIC.  The call waits for its work on the stream before it
 * returns.  It never allocates through the caller's allocator: the first
 * call on a device loads the library's device module there (CUDA loads
 * modules lazily by default), which reserves the scratch on that device, and
 * looks up its address -- so that first call may synchronise the device;
 * make it before any stream capture.  Every call shares the scratch and
 * clears what must start at zero, so calls that overlap on the GPU race and
 * must be serialised. */
#define TSIM_NOALLOC_MAX_PARTICLES (1 << 20)
#define TSIM_NOALLOC_MAX_BLOCKS (1 << 15)
#define TSIM_NOALLOC_SCRATCH_BYTES (3 * 4 * TSIM_NOALLOC_MAX_BLOCKS + 4 * TSIM_NOALLOC_MAX_PARTICLES + 256)
int tsim_p2g_noalloc(const tsim_gel_desc *gel, const tsim_material *mat, float dt, const float *x,
                     const float *v, const float *C, const float *F, int n, float *grid, void *stream);

/* ---- sensor image (Sec. III-B path tracing, Sec. IV image metrics) ---- */

#define TSIM_MAX_LEDS 4

/* Path-tracing setup (all lengths in metres, the sensor frame of the
 * readout: pixel (i, j) at ((j + 0.5) pitch, (i + 0.5) pitch)).  LED k is the
 * rectangle c[k] + a u[k] + b v[k], |a|, |b| <= 1, emitting RGB radiance
 * L[k] on the side of u[k] x v[k]; the plane z = z_floor below the surface
 * absorbs (the camera window).  spp samples per pixel (the paper uses 128),
 * at most max_bounces (1..32) reflections per path; seed selects the
 * random numbers (SplitMix64 of a per-sample counter). */
typedef struct {
    float c[TSIM_MAX_LEDS][3];
    float u[TSIM_MAX_LEDS][3];
    float v[TSIM_MAX_LEDS][3];
    float L[TSIM_MAX_LEDS][3];
    int n_lights;
    int spp;
    int max_bounces;
    float z_floor;
    uint64_t seed;
} tsim_render_desc;

/* Sensor image of a membrane height field (Sec. III-B, Sec. IV-B): an
 * orthographic camera below the gel sees the Lambertian membrane (maximum
 * roughness) z = height(x, y) lit by the LEDs; each sample is a reverse
 * path of diffuse reflections (cosine-weighted, attenuated by the albedo at
 * each reflection) that adds what reaches an LED.  height: H x W (e.g. from
 * tsim_read_surface), albedo: H x W x 3 (the base texture), rgb: H x W x 3
 * out, the mean over spp samples.  All three are device arrays (4-byte
 * aligned; TSIM_ERR_INVALID_ARG otherwise).  Asynchronous on stream; calls
 * share a small static device scratch and must not overlap. */
int tsim_render(const float *height, const float *albedo, int W, int H, float pitch,
                const tsim_render_desc *desc, float *rgb, void *stream);

/* Image similarity of two H x W x C device images with values in
 * [0, max_value] (Sec. IV): out[0] = MSE over all values, out[1] = PSNR =
 * 10 log10(max_value^2 / MSE) (infinite for equal images), out[2] = mean
 * SSIM (Wang et al. 2004: 11 x 11 Gaussian window of sigma 1.5 inside the
 * image, K1 = 0.01, K2 = 0.03, averaged over windows and channels).  out is
 * a host array of 3; the call waits for its work on stream.  W, H >= 11. */
int tsim_image_metrics(const float *a, const float *b, int W, int H, int C, float max_value, double *out,
                       void *stream);

/* Reason for the last failure on this thread (never NULL). */
const char *tsim_last_error(void);

/* Particle slots of one 4x4x4-cell block (the library's layout constant):
 * particles beyond it in one block go to their instance's spill slots
 * (TSIM_ERR_CAPACITY only when those are full too).  No GPU work. */
int tsim_block_slots(void);

/* Free the context and all its device memory (NULL is ignored). */
void tsim_destroy(tsim_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* TSIM_H */
