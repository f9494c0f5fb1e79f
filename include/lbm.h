/*
 * lbm.h -- C-ABI of the GB300 D3Q27 central-Hermite-moment MRT lattice Boltzmann library.
 *
 * The library advances the lattice Boltzmann equation (Hosseini et al., Sec. 2.1.1) with the
 * CHM-MRT collision operator Omega = T^-1 S T (f_eq - f) and the fully expanded equilibrium
 * (Sec. 2.1.3), halfway bounce-back walls, Bouzidi interpolated walls (Sec. 2.1.4) and a
 * pulsatile velocity inlet / density outlet (Sec. 2.2), on a voxelised geometry, as
 * hand-written CUDA kernels on one GPU.
 *
 * Conventions used by every entry point:
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3.  Directions i = (cx+1) + 3 (cy+1) + 9 (cz+1),
 *     c in {-1,0,1}^3; the opposite of i is 26 - i.
 *   - Box arrays are dense, x fastest: index = x + nx (y + ny z).  Cell (x,y,z) has its centre
 *     at (x + 1/2, y + 1/2, z + 1/2).
 *   - Time level n: the populations f(x, n) after streaming, wall rules and open-boundary
 *     closures.  lbm_step(dom, k) advances n -> n + k; one step collides with the body force
 *     g(n), streams, and closes the open boundaries with the inflow U(n + 1).  A new domain is
 *     at n = 0 with f = w (rho = 1, u = 0) closed at n = 0.
 *   - Velocities reported at level n are u = (sum_i c_i f_i)/rho + g(n)/2 (half-force shift).
 *   - Ownership: the caller owns every pointer it passes; the library copies what it keeps
 *     during the call.  The library owns the device memory of a domain, obtained through the
 *     allocator callbacks given at creation (cudaMalloc/cudaFree when they are NULL), and
 *     releases it in lbm_destroy.
 *   - Errors: every call returns an lbm_status; no C++ exception crosses this boundary.  On
 *     failure lbm_last_error() returns a message for the calling thread.  Calls that only
 *     enqueue work report launch errors; faults inside a kernel surface at the next call that
 *     synchronises (lbm_get_macroscopic, lbm_get_diagnostics, lbm_sync, lbm_save_state).
 *   - Streams: all device work of a domain is enqueued on the CUDA stream given at creation
 *     (NULL = the legacy default stream).  Calls on one domain must not run concurrently from
 *     several host threads.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_domain lbm_domain;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = 1, /* bad argument; nothing was changed */
    LBM_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
    LBM_ERR_OOM = 3,         /* the allocator returned NULL */
    LBM_ERR_UNSTABLE = 4,    /* a NaN/Inf was found in the populations */
    LBM_ERR_TIMEOUT = 5,     /* a device-side wait gave up (bounded spin) */
    LBM_ERR_STATE = 6,       /* call not valid in the domain's current state */
    LBM_ERR_IO = 7           /* file could not be read or written, or does not match */
} lbm_status;

/* Storage of the populations in HBM.  All arithmetic is FP32 in every mode.
 *   FP32: the deviation f_i - w_i, FP32.
 *   FP16 / BF16: the scaled deviation (f_i - w_i) / w_i in 16 bits. */
typedef enum { LBM_STORE_FP32 = 0, LBM_STORE_FP16 = 1, LBM_STORE_BF16 = 2 } lbm_storage;

/* Streaming scheme; both give bitwise-identical results.
 *   AB: pull from one array into a second (two population arrays).
 *   ESOTERIC: esoteric twist, in place in one array; each cell's update touches only the cells
 *     x + {0,1}^3 (plus a small side buffer at Bouzidi cells). */
typedef enum { LBM_SCHEME_AB = 0, LBM_SCHEME_ESOTERIC = 1 } lbm_scheme;

/* Collision operator.
 *   CHM_MRT: the paper's operator (Sec. 2.1.3): central Hermite moments, full-expansion
 *     equilibrium, second-order rate 1/tau, third- to sixth-order rates omega_hi.
 *   SRT2: the classical single-relaxation-time operator with the second-order equilibrium that
 *     the paper compares against (Sec. 2.1.2), f* = f + (f_eq2 - f)/tau + (1 - 1/(2 tau)) F_i,
 *     F_i the second-order (Guo) force term.
 *   TRT2: the two-relaxation-time operator (Sec. 2.1.2) with the same equilibrium and force
 *     term: even parts relax with 1/tau, odd parts with 1/(trt_magic/(tau - 1/2) + 1/2).
 * The inlet/outlet closures and wall rules are the same for all three. */
typedef enum { LBM_COLLISION_CHM_MRT = 0, LBM_COLLISION_SRT2 = 1, LBM_COLLISION_TRT2 = 2 } lbm_collision;

/* Physical parameters (Sec. 2.1.3: S is diagonal in central Hermite moment space). */
typedef struct {
    double tau;          /* relaxation time of the six second-order moments: rate 1/tau,
                            kinematic viscosity nu = (tau - 1/2)/3; must be > 1/2 */
    double omega_hi[4];  /* rates of the 3rd, 4th, 5th and 6th-order moments (free parameters
                            of the paper), each in (0, 2); default 1 */
    double force[3];     /* constant body acceleration g0 (force density rho g) */
    double force_amp[3]; /* g(n) = force + force_amp cos(force_omega n) */
    double force_omega;  /* angular frequency per step of the body-force modulation */
    double rho_out;      /* density imposed at outlet cells; default 1 */
    int32_t periodic[3]; /* nonzero: the axis wraps (its extent must be a multiple of the brick's
                            extent along it: 4 in the default build) */
    int32_t storage;     /* lbm_storage */
    int32_t scheme;      /* lbm_scheme; default ESOTERIC */
    int32_t collision;   /* lbm_collision; default CHM_MRT */
    double trt_magic;    /* TRT2 only: Lambda = (tau - 1/2)(1/w- - 1/2) > 0; default 3/16 (halfway
                            bounce-back then places a plane wall exactly half-way, any tau) */
} lbm_params;

/* Device memory callbacks: return a device pointer aligned to 256 bytes, or NULL. */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* ctx);
typedef void (*lbm_free_fn)(void* ptr, void* ctx);

typedef struct {
    int32_t nx, ny, nz;
    int64_t n_fluid;         /* cells updated per step (mask 1, 2 or 3) */
    int64_t n_bricks;        /* bricks (64 cells) holding at least one fluid or halo cell */
    int64_t n_slots;         /* 64 * n_bricks: population slots per direction */
    int64_t n_wall_cells;    /* fluid cells with at least one wall link */
    int64_t n_bouzidi_cells; /* fluid cells with at least one Bouzidi link */
    int64_t n_open_cells;    /* inlet + outlet cells */
    int64_t time;            /* current time level n */
    int32_t storage;
    int32_t bytes_per_value; /* 4 (FP32) or 2 (FP16/BF16) */
    int64_t device_bytes;    /* device memory held by the domain */
    int32_t launch_config;   /* launch configuration of the step kernel in use */
    int32_t scheme;          /* lbm_scheme */
    int64_t n_store_bricks;  /* bricks with population storage (active + twist halo) */
    int64_t n_halo;          /* halo cells (mask value 4) of a sub-domain of a slab decomposition */
} lbm_info;

typedef struct {
    double mass;     /* sum of rho over fluid cells (FP64 accumulation) */
    double flux_in;  /* sum over inlet cells of rho u . n_in (n_in the inward normal) */
    double flux_out; /* sum over outlet cells of -rho u . n_in (outflow positive) */
    double max_u;    /* max |u| over fluid cells */
    int64_t n_nonfinite; /* fluid cells whose rho or u is NaN or Inf */
    int64_t time;
} lbm_diagnostics;

/* Fills *p with the defaults: tau 0.6, omega_hi 1, no force, rho_out 1, not periodic, FP32,
 * esoteric twist. */
void lbm_default_params(lbm_params* p);

/*
 * Builds a domain from a voxel mask (Sec. 2.2: voxelised vessel geometry).
 *   mask[nx*ny*nz]: 0 solid, 1 fluid, 2 velocity inlet, 3 density outlet, 4 halo (a cell of a
 *     neighbouring sub-domain, see lbm_halo_pack).  Inlet and outlet cells must lie on exactly
 *     one non-periodic box face; the face's inward normal is theirs.  Neighbours outside a
 *     non-periodic face count as solid.
 *   Wall links (Sec. 2.1.4, q = |x_f - x_s| / |c|), n_links entries, may be 0 / NULL:
 *     link_cell[l]  box index of a cell with mask 1,
 *     link_dir[l]   direction beta with x_f + c_beta not fluid,
 *     link_q[l]     q in (0, 1]: the wall cuts the segment x_f -> x_f + c_beta at q.
 *     Wall links without an entry use halfway bounce-back.  Duplicates are rejected.
 *   inlet_center[3], inlet_radius: the inflow profile u = U(n) 2 (1 - r^2/R^2) n_in, r the
 *     distance from the cell centre to inlet_center in the inlet plane (0 beyond R).  May be
 *     NULL / ignored when the mask has no inlet cells.
 *   tau_cell[nx*ny*nz]: optional relaxation time per cell (a viscosity field, e.g. an absorbing
 *     layer before an outlet; > 1/2 at fluid cells); the second-order rate of a cell is then
 *     1/tau_cell.  NULL: params->tau everywhere.
 *   params: see lbm_params; NULL means lbm_default_params.
 *   alloc/release/alloc_ctx: device allocator (both NULL: cudaMalloc / cudaFree).
 *   cuda_stream: cudaStream_t for all work of the domain (NULL: legacy default stream).
 *   *out receives the domain, or NULL on failure.
 * Errors: INVALID_ARG (sizes, mask values, links, parameters), OOM, CUDA.
 */
lbm_status lbm_create_domain(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz,
                             const int64_t* link_cell, const uint8_t* link_dir,
                             const double* link_q, int64_t n_links, const double* inlet_center,
                             double inlet_radius, const double* tau_cell, const lbm_params* params,
                             lbm_alloc_fn alloc, lbm_free_fn release, void* alloc_ctx,
                             void* cuda_stream, lbm_domain** out);

/*
 * Sets the inflow waveform (Sec. 2.2: inflow curve over one cycle):
 *   s(t) = a[0] + sum_{k=1..n_harm} a[k] cos(2 pi k t / P) + b[k-1] sin(2 pi k t / P),
 *   U(t) = u_peak s(t) / max_{t = 0..P-1} s(t),   P = period_steps (an integer >= 1).
 * The domain's inlet cells are re-closed at the current level.  Until this is called U = 0.
 * Errors: INVALID_ARG (n_harm outside 0..15, P not a positive integer <= 2^24, max s <= 0).
 */
lbm_status lbm_set_inlet_waveform(lbm_domain* dom, const double* a, const double* b,
                                  int32_t n_harm, double period_steps, double u_peak);

/*
 * Initial condition from macroscopic fields (dense box arrays; rho[nx*ny*nz], u = three planes
 * ux, uy, uz of nx*ny*nz each): the post-collision populations of level n - 1 are set to
 * f_eq(rho, u) (full expansion) at every fluid cell, so that level n is their stream with the
 * wall rules and closures.  device_ptrs != 0: rho and u are device pointers.
 */
lbm_status lbm_init_equilibrium(lbm_domain* dom, const float* rho, const float* u,
                                int32_t device_ptrs);

/* Enqueues n >= 0 fused stream-collide steps (Sec. 2.1.1, 2.1.3, 2.1.4) on the domain's
 * stream; returns without waiting.  Errors: INVALID_ARG (n < 0), CUDA (launch failure). */
lbm_status lbm_step(lbm_domain* dom, int64_t n);

/*
 * rho and u = (sum c f)/rho + g(n)/2 at the current level n (Sec. 2.1.1 moments).
 *   dense != 0: rho[nx*ny*nz] and u[3][nx*ny*nz] on the box, solid cells 0.
 *   dense == 0: rho[n_fluid], u[3][n_fluid], fluid cells in increasing box index.
 *   device_ptrs != 0: rho and u are device pointers (written on the domain's stream);
 *   otherwise host pointers (the call stages through device memory and waits).
 */
lbm_status lbm_get_macroscopic(lbm_domain* dom, float* rho, float* u, int32_t dense,
                               int32_t device_ptrs);

/* FP64 reductions over the current level (mass, inlet/outlet flux, max |u|, non-finite
 * count); waits for the stream.  Returns UNSTABLE (after filling *out) if any fluid cell is
 * non-finite.  The reduction order is fixed, so results are reproducible run to run. */
lbm_status lbm_get_diagnostics(lbm_domain* dom, lbm_diagnostics* out);

/*
 * The same reduction as lbm_get_diagnostics, for callers that must not allocate device memory
 * at the time of the call: a monitoring loop with latency bounds (cudaMalloc may block and
 * synchronise the device), or an application whose device memory is already reserved in full
 * by another framework's pool.  It allocates nothing: its scratch is a fixed array of about
 * 320 KiB inside this library, present on every device that loads the library until the
 * process exits.  The paper has no counterpart; this is a library service.
 *   Limit: domains of at most 2,097,152 fluid cells (INVALID_ARG beyond, nothing launched).
 *   The first call on a device looks up the array's device address with that device current.
 *   The call waits for the domain's stream and copies the result to the host, so it must not
 *   be made while that stream is being captured.
 *   All calls share the array; calls whose work overlaps on the GPU (domains on different
 *   streams or host threads) race on it, so serialise them.  Nothing in it needs clearing
 *   between calls: each call overwrites every word it reads.
 *   Waits for the domain's stream.  Returns UNSTABLE (after filling *out) on non-finite
 *   populations, like lbm_get_diagnostics.
 */
lbm_status lbm_get_diagnostics_noalloc(lbm_domain* dom, lbm_diagnostics* out);

lbm_status lbm_get_info(const lbm_domain* dom, lbm_info* out);

/* Number of launch configurations of the fused step kernel. */
#define LBM_N_LAUNCH_CONFIGS 8

/* Selects the step kernel's launch configuration: 0 = 256 threads (four 4^3 bricks) per CTA
 * with a register budget for 3 resident CTAs per SM; 1, 2, 3, 4 = 128 threads with 7, 6, 8 or
 * 10; 5 = a persistent, software-pipelined variant (128 threads, 6 CTAs per SM; the next cell's
 * populations are copied into shared memory asynchronously while the current one is computed;
 * FP32 esoteric twist only, other domains use 3); 6, 7 = two cells per thread (128 threads = four
 * bricks per CTA, 4 or 3 CTAs per SM; the two cells' collisions as packed FP32x2 arithmetic;
 * esoteric twist with CHM-MRT at unit higher-order rates only, other domains use 2).  Results
 * do not depend on it.  Default 2.
 * Errors: INVALID_ARG. */
lbm_status lbm_set_launch_config(lbm_domain* dom, int32_t config);

/* Times every launch configuration on this domain (trial_steps steps each, CUDA events on the
 * domain's stream) and selects the fastest.  The domain's populations and time level are left
 * as they were.  ms_per_step (may be NULL) receives LBM_N_LAUNCH_CONFIGS times (-1 for a
 * configuration that has no kernel of its own for this domain and is not timed); *best_config
 * (may be NULL) the choice.  Waits for the stream.  Allocates one population array while it
 * runs.  Errors: INVALID_ARG, OOM, CUDA. */
lbm_status lbm_autotune(lbm_domain* dom, int32_t trial_steps, int32_t* best_config, float* ms_per_step);

/*
 * Batches: several domains advanced together, one kernel launch per step over all of them
 * (a concatenated brick work list), with chunks of graph_steps steps captured once into a CUDA
 * graph and replayed (the per-step force and inflow of every domain are uploaded by the graph's
 * first node).  Results are bit-identical to stepping each domain alone.
 *   lbm_batch_create: doms[n] (1..4096 distinct domains, esoteric twist, one storage precision,
 *     one collision operator, and for CHM-MRT all or none with unit higher-order rates) stay
 *     owned by the caller and must outlive the batch; graph_steps in 1..4096.  The batch runs (and captures) its work on a private
 *     non-blocking stream, ordered by events after the work already enqueued on cuda_stream
 *     (NULL: legacy default) and on each domain's stream, and before anything enqueued there
 *     later.  Small tables are allocated through doms[0]'s allocator.  Errors: INVALID_ARG, OOM,
 *     CUDA.
 *   lbm_batch_step: n >= 0 steps of every domain (each domain's time advances by n); waits for
 *     the previous chunk before refilling its host argument table.  When all domains share
 *     one time parity the captured kernels are specialised for it; the graph is captured again
 *     whenever a chunk starts with another parity pattern than the captured one (an odd
 *     graph_steps does this every chunk: prefer an even one).
 *   lbm_batch_set_launch_config / lbm_batch_autotune: as for single domains (the batched kernel
 *     has configurations 0-4; the others run as 4, and autotune does not time them); autotune
 *     keeps every domain's state (it copies and restores the populations) and needs trial_steps
 *     <= graph_steps.
 */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(lbm_domain* const* doms, int32_t n, int32_t graph_steps, void* cuda_stream,
                            lbm_batch** out);
lbm_status lbm_batch_step(lbm_batch* batch, int64_t n);
lbm_status lbm_batch_set_launch_config(lbm_batch* batch, int32_t config);
lbm_status lbm_batch_autotune(lbm_batch* batch, int32_t trial_steps, int32_t* best_config, float* ms_per_step);
void lbm_batch_destroy(lbm_batch* batch);

/*
 * Persistent mode of a batch (enable != 0): each chunk of graph_steps steps becomes one
 * cooperative kernel launch, captured in the chunk's CUDA graph, whose CTAs stay resident for
 * the whole chunk and advance every member step after step, meeting at a grid-wide barrier
 * between steps (a member's next step reads what neighbouring CTAs wrote).  Results are the same
 * bit for bit as one launch per step.  Every wait at a barrier gives up after barrier_timeout_s
 * seconds (in (0, 3600]; 1.0 is a sensible value): the CTA that gives up flags the chunk, every
 * CTA leaves at its next barrier, and the next lbm_batch_step or lbm_batch_sync returns
 * LBM_ERR_TIMEOUT -- the members' populations are then undefined (reload a checkpoint).
 * enable = 0 returns to one launch per step.  lbm_batch_autotune always times the one-launch
 * configurations.  Waits for the batch's stream.  Errors: INVALID_ARG, CUDA.
 * lbm_batch_sync: waits for the batch's work; TIMEOUT if a persistent chunk gave up.
 */
lbm_status lbm_batch_set_persistent(lbm_batch* batch, int32_t enable, double barrier_timeout_s);
lbm_status lbm_batch_sync(lbm_batch* batch);

/*
 * Learned coarse-grid corrector (not part of the paper: its Sec. 3.4 shows that a 2x coarser
 * grid keeps useful accuracy at ~14x less cost; the corrector nudges the coarse velocity toward
 * the fine solution restricted onto the coarse grid).  A 3-layer 3-D convolutional network,
 * 16 channels, 3x3x3 kernels, zero padding, ReLU, BF16 weights and activations with FP32
 * accumulation on the tensor cores, evaluated on the 4^3 tiles near fluid:
 *   X0 = [u/u_scale (3), (rho-1)/rho_scale, fluid mask, 0 (11)]  (zero at solid cells)
 *   O  = conv3(relu(conv2(relu(conv1(X0)))));  du = du_scale * clamp(O[0:3], -2, 2) at fluid
 *   cells (the clamp bounds a correction to twice du_scale per component).
 * Parameters (FP32, lbm_corrector_num_params() of them): W1[27][16][16], b1[16], W2, b2, W3, b3
 * with W[o][out][in], offset o = (dx+1) + 3(dy+1) + 9(dz+1).
 *   lbm_corrector_create: mask[nx*ny*nz] (host; nonzero = fluid) of the coarse box (extents
 *     multiples of 4): the network is evaluated on the tiles near its fluid (for training over
 *     several geometries give the union of their masks); the scales; initial params (copied).
 *     Memory through the allocator callbacks.
 *   The calls below take a dense device cell mask (nonzero = fluid, inside the creation mask;
 *   NULL: the creation mask) for the input features, and an output mask (nonzero = cells the
 *   correction and the loss act on, within the cell mask; NULL: the cell mask).
 *   lbm_corrector_forward: rho[n], u[3][n] dense device fields -> du[3][n] device.
 *   lbm_corrector_gradients: loss L = mean over fluid cells and components of
 *     (O[0:3] - (u_target - u)/du_scale)^2 and dL/dparams (host, FP32); waits.
 *   lbm_corrector_train_step: the same, then one Adam step (b1 0.9, b2 0.999, eps 1e-8) with
 *     learning rate lr; *loss (may be NULL) gets L before the update.
 *   lbm_corrector_apply: rho, u of the domain's current level -> gain * du (features on mask,
 *     correction on out_mask; device, may be NULL; gain in (0, 1] nudges instead of replacing)
 *     -> lbm_apply_velocity_correction.
 *   lbm_apply_velocity_correction: the post-collision populations of the previous level gain
 *     f_eq(rho, u + du) - f_eq(rho, u) at every fluid cell except inlet and outlet cells (whose
 *     unknowns the closures rebuild each step; rho, u of the current level); du are
 *     three planes on the dense box (host or device pointers); waits for host pointers, and
 *     with device pointers is enqueued on the domain's stream (du must stay valid until that
 *     work has run).  The first call allocates a staging buffer of 7 planes that the domain
 *     keeps.
 *   lbm_restrict: coarse rho, u (dense, device) = mean over the fluid children of each coarse
 *     cell of the fine dense fields (fine extents even; fine_mask nonzero = fluid, device).
 * All device pointers belong to the caller.  Errors: INVALID_ARG, OOM, CUDA.
 */
typedef struct lbm_corrector lbm_corrector;
int64_t lbm_corrector_num_params(void);
lbm_status lbm_corrector_create(const uint8_t* mask, int32_t nx, int32_t ny, int32_t nz, double u_scale,
                                double rho_scale, double du_scale, const float* params, lbm_alloc_fn alloc,
                                lbm_free_fn release, void* alloc_ctx, void* cuda_stream, lbm_corrector** out);
lbm_status lbm_corrector_get_params(lbm_corrector* c, float* params);
lbm_status lbm_corrector_set_params(lbm_corrector* c, const float* params);
lbm_status lbm_corrector_forward(lbm_corrector* c, const uint8_t* mask, const uint8_t* out_mask, const float* rho,
                                 const float* u, float* du);
lbm_status lbm_corrector_gradients(lbm_corrector* c, const uint8_t* mask, const uint8_t* out_mask, const float* rho,
                                   const float* u, const float* u_target, float* grad, double* loss);
lbm_status lbm_corrector_train_step(lbm_corrector* c, const uint8_t* mask, const uint8_t* out_mask, const float* rho,
                                    const float* u, const float* u_target, double lr, double* loss);
lbm_status lbm_corrector_apply(lbm_corrector* c, lbm_domain* dom, const uint8_t* mask, const uint8_t* out_mask,
                               double gain);
void lbm_corrector_destroy(lbm_corrector* c);
lbm_status lbm_apply_velocity_correction(lbm_domain* dom, const float* du, int32_t device_ptrs);
lbm_status lbm_restrict(const float* fine_rho, const float* fine_u, const uint8_t* fine_mask, int32_t fnx,
                        int32_t fny, int32_t fnz, float* coarse_rho, float* coarse_u, void* cuda_stream);

/*
 * Flow metrics of the paper's comparisons, on the device.
 *   lbm_mean_reset / lbm_mean_sample / lbm_mean_get: running means of rho and u (the time
 *     averaging of Sec. 3.3).  reset allocates (once, through the domain's allocator: 32 bytes per
 *     fluid cell) and zeroes FP64 sums; sample adds the current level's rho, u of every fluid
 *     cell (asynchronous, one kernel; call it between lbm_step calls at the sampling interval);
 *     get writes the means (as lbm_get_macroscopic: dense box or compact fluid list, host or
 *     device pointers; host pointers wait) and *n_samples (may be NULL).  Errors: INVALID_ARG,
 *     STATE (sample or get before reset, get without samples), OOM, CUDA.
 *   lbm_probe: rho, ux, uy, uz of n fluid cells at the current level (monitoring points,
 *     Sec. 2.2.2), out[p][4]; fluid_index[p] is the position of the cell in the compact fluid
 *     list (fluid cells in box order, x fastest).  Host pointers: indices are checked
 *     (INVALID_ARG outside [0, n_fluid)) and the call waits; device pointers: asynchronous, an
 *     index outside the range yields NaNs.
 *   lbm_similarity_index: the similarity index of Sec. 3.4 between two velocity fields u_a, u_b
 *     (device pointers, three planes [3][n] each) over the points with mask[p] != 0 (device
 *     pointer; NULL: all n points), read with the factor 1/2 that bounds it by 1:
 *     SI = mean_p 1/2 (1 + cos theta_p) (1 - | |u_a,p|/max|u_a| - |u_b,p|/max|u_b| |), the maxima
 *     over the same points, cos theta = 0 where either vector is zero, 0 for an empty set.
 *     FP64 terms and fixed-order reductions (reproducible); a fixed scratch inside the library,
 *     no allocation; calls are serialised; waits for cuda_stream (NULL: legacy default).
 *     Errors: INVALID_ARG, CUDA.
 */
lbm_status lbm_mean_reset(lbm_domain* dom);
lbm_status lbm_mean_sample(lbm_domain* dom);
lbm_status lbm_mean_get(lbm_domain* dom, float* rho, float* u, int32_t dense, int32_t device_ptrs, int64_t* n_samples);
lbm_status lbm_probe(lbm_domain* dom, const int64_t* fluid_index, int32_t n, float* out, int32_t device_ptrs);
lbm_status lbm_similarity_index(const float* u_a, const float* u_b, const uint8_t* mask, int64_t n, double* si,
                                void* cuda_stream);

/*
 * Slab decomposition: one domain split along one axis into sub-domains, each advanced by its own
 * lbm_domain (several on one GPU, or one per GPU), with one exchange of face populations per
 * step.  The method's cost is lattice points times steps (Sec. 3.4, Sec. 5: "per processor"),
 * which the split shares out among processing units.
 *   A sub-domain's mask marks the cells it receives from its neighbour with the value 4 (halo):
 *   a one-cell layer on a non-periodic face of its box, holding the neighbour's layer of cells
 *   next to the cut (4 where that cell is fluid, 0 where it is solid).  Halo cells need the A-B
 *   scheme (INVALID_ARG otherwise) and must lie on a non-periodic face; they are stored but never
 *   updated, they are not fluid cells (n_fluid, exports, diagnostics, means and probes leave them
 *   out: lbm_info.n_halo counts them), and they count as fluid for their neighbours' wall links.
 *   lbm_halo_size: *values = 9 x (area of the face) values per exchange buffer of `face`
 *     (0 low x, 1 high x, 2 low y, 3 high y, 4 low z, 5 high z), 0 if that face has no halo
 *     layer.  Positions on a face run over the other two axes, the lower axis fastest.
 *   lbm_halo_pack: writes into buf[9][area] the populations of the current level's
 *     post-collision state that leave the box through `face` (c . n_out = +1, in increasing
 *     direction index) from the cells of the layer just inside the face's halo layer (0 where
 *     that cell is not fluid).  buf is a device pointer; values keep the storage precision (4
 *     bytes for FP32, 2 for FP16/BF16) and are copied bit for bit.
 *   lbm_halo_unpack: writes buf, as packed by the neighbour on its face across the cut (the
 *     same 9 directions, in the same order), into this face's halo layer, where the next
 *     lbm_step pulls them.
 *   Both enqueue on the domain's stream and return without waiting (buf must stay valid until
 *   the work has run).  Exchanged after every lbm_step (and once after lbm_init_equilibrium or
 *   lbm_apply_velocity_correction), the sub-domains reproduce the undivided domain's fields at
 *   their fluid cells bit for bit.  Errors: INVALID_ARG (NULL, face outside 0..5, a face without
 *   a halo layer), CUDA.
 */
lbm_status lbm_halo_size(const lbm_domain* dom, int32_t face, int64_t* values);
lbm_status lbm_halo_pack(lbm_domain* dom, int32_t face, void* buf);
lbm_status lbm_halo_unpack(lbm_domain* dom, int32_t face, const void* buf);

/* Waits for all work enqueued on the domain. */
lbm_status lbm_sync(lbm_domain* dom);

/* Checkpoint: the stored populations (in storage precision), the time level, the waveform and
 * the parameters, to a binary file.  lbm_load_state restores them into a domain built from the
 * same mask and links (IO on a mismatch).  Both wait for the stream. */
lbm_status lbm_save_state(lbm_domain* dom, const char* path);
lbm_status lbm_load_state(lbm_domain* dom, const char* path);

/* Releases the domain and its device memory (after waiting for its stream). NULL is a no-op. */
void lbm_destroy(lbm_domain* dom);

/* Message of the last failed call on this thread ("" if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */
