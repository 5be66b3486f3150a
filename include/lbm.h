/*
 * lbm.h -- C ABI of liblbm, a GB300 (sm_103a) implementation of the time step
 * of the improved two-component pseudopotential lattice Boltzmann method of
 * Sedahmed et al., Phys. Fluids (2022), arXiv 2207.01534, on a D3Q19 lattice
 * over the fluid voxels of a porous geometry.
 *
 * Conventions for every call:
 *   - Errors are returned as lbm_status codes; nothing throws across the ABI.
 *     After a failure, lbm_last_error(ctx) returns a human-readable reason
 *     (for lbm_create, lbm_last_error(NULL) holds the reason).
 *   - Dense host arrays are indexed v = x + nx*(y + ny*z) (x fastest), and all
 *     host arrays are owned by the caller; the library copies what it needs and
 *     keeps no host pointer after a call returns.
 *   - Device work is issued on the context's CUDA stream (default: the legacy
 *     default stream; see lbm_set_stream).  lbm_step only enqueues work.
 *     Calls that return host data (read_fields, saturation, get_populations,
 *     synchronize) synchronise that stream.
 *   - A context belongs to the device that was current at lbm_create; call it
 *     with that device current.  Contexts are not thread-safe.
 *
 * Component 1 is the droplet / injected fluid ("oil"), component 2 the
 * surrounding / initially saturating fluid ("water") (Section 2, Section 4.1).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,       /* invalid argument or geometry */
    LBM_ERR_ALLOC = -2,     /* device or host allocation failed */
    LBM_ERR_CUDA = -3,      /* a CUDA call failed (message in lbm_last_error) */
    LBM_ERR_NONFINITE = -4, /* the periodic check found a NaN/Inf density (sticky) */
    LBM_ERR_DRIFT = -5,     /* mass drift above the limit on a closed domain (sticky) */
    LBM_ERR_TIMEOUT = -6,   /* a bounded device wait gave up (sticky) */
    LBM_ERR_UNSUPPORTED = -7
} lbm_status;

/* Population storage precision.  Arithmetic is FP32 for the 32- and 16-bit
 * forms and FP64 for LBM_STORE_FP64. */
enum {
    LBM_STORE_FP32 = 0,
    LBM_STORE_FP64 = 1,
    LBM_STORE_FP16DEV = 2, /* moving populations as FP16 deviations from w_i*rho_ref */
    LBM_STORE_BF16DEV = 3  /* same with BF16 */
};

/* Kernel schedule of the step.  AUTO selects LBM_KERNEL_SPLIT (the fastest
 * measured on the workloads of Section 4); the others are opt-in. */
enum {
    LBM_KERNEL_AUTO = 0,
    LBM_KERNEL_SPLIT = 1, /* density, wall and fused collide-stream passes */
    LBM_KERNEL_FUSED = 2, /* single persistent pass per step (see lbm_step) */
    LBM_KERNEL_WAVE = 3,  /* the split passes per z slab, as a dependency graph (see lbm_step) */
    LBM_KERNEL_PUSH = 4,  /* collide-stream pass that also accumulates the next densities (FP32; see lbm_step) */
    LBM_KERNEL_BRICK = 5, /* one pass per step over 8^3 bricks, halo densities in shared memory (see lbm_step) */
    LBM_KERNEL_FLOW = 6,  /* one launch per step: collide-stream, then next densities from L2 (see lbm_step) */
    LBM_KERNEL_PERSISTENT = 7 /* batches: many steps of all samples in one cooperative launch (see lbm_step) */
};

/* Open-plane rule for the prescribed component (Section 2, boundary rule 1):
 * non-equilibrium extrapolation from the first interior node, or the Zou-He
 * method (entering populations from the node's own density, zero tangential
 * velocity and normal non-equilibrium bounce-back). */
enum { LBM_BC_NEEM = 0, LBM_BC_ZOU_HE = 1 };

/* Field selection bits for lbm_read_fields. */
enum {
    LBM_FIELD_RHO1 = 1u,
    LBM_FIELD_RHO2 = 2u,
    LBM_FIELD_UX = 4u,
    LBM_FIELD_UY = 8u,
    LBM_FIELD_UZ = 16u,
    LBM_FIELD_P = 32u
};

/* Geometry of one domain.  solid: nx*ny*nz bytes, nonzero = solid (phi = 1 of
 * Eq. 14).  periodic[a] != 0 makes axis a periodic.  open_axis = -1: no open
 * boundary; open_axis = 2: the z = 0 plane is the inlet and z = nz-1 the outlet
 * (Section 2 inlet/outlet rules; only the z axis is supported).  A fluid voxel
 * may touch a non-periodic face only across the open planes: closed faces must
 * be solid voxels.  sample_lo <= z < sample_hi selects the slab that
 * lbm_saturation counts (hi <= lo: the whole domain).  xi_field (optional,
 * nx*ny*nz floats) gives the wettability parameter xi per solid voxel (Eq. 15
 * chi); NULL uses params.xi everywhere. */
typedef struct {
    int32_t nx, ny, nz;
    const uint8_t *solid;
    int32_t periodic[3];
    int32_t open_axis;
    int32_t sample_lo, sample_hi;
    const float *xi_field;
} lbm_geometry;

/* Model parameters (Section 2).  tau: relaxation times tau^(1), tau^(2)
 * (Eq. 7, read as nu = c_s^2 (tau - 1/2)).  G: cohesion strength G_coh (Eq.
 * 11; the paper uses 3.5).  xi: wettability, chi^(1) = 1 + xi, chi^(2) = 1 - xi
 * (Eq. 15).  rho_in1 / rho_out2: prescribed component densities at the inlet
 * and outlet planes.  bc: LBM_BC_* (the rule that imposes them).  body_force: acceleration
 * g, F^b = rho^sigma g (Eq. 10).  velocity_shift: 1 adds F^sigma/2 to the
 * component momenta in Eq. 8 (the explicit-forcing reading, default); 0 uses
 * the printed Eq. 4 momenta.  storage: LBM_STORE_*.  rho_ref: per-component
 * reference density for the 16-bit deviation storage.  reduce_every: n > 0
 * runs the FP64 finiteness / mass check every n steps inside lbm_step.
 * kernel: LBM_KERNEL_*. */
typedef struct {
    double tau[2];
    double G;
    double xi;
    double rho_in1, rho_out2;
    double body_force[3];
    int32_t bc;
    int32_t storage;
    int32_t velocity_shift;
    int32_t reduce_every;
    double rho_ref[2];
    int32_t kernel;
    double drift_limit; /* relative mass drift that raises LBM_ERR_DRIFT (closed domains) */
} lbm_params;

/* Sizes and counters of a context. */
typedef struct {
    int64_t n_fluid;        /* fluid nodes N_f */
    int64_t n_wall;         /* solid voxels with at least one fluid neighbour */
    int64_t n_voxels;       /* nx*ny*nz */
    int64_t step;           /* time steps taken since the last initialisation */
    int64_t device_bytes;   /* device memory held by the context */
    int64_t launches;       /* kernels launched by this context so far */
    int32_t storage;
    int32_t kernel;         /* schedule actually used */
} lbm_info;

/* Fill *p with the defaults: tau = (1, 1), G = 3.5, xi = 0, rho_in1 = rho_out2
 * = 1, no body force, NEEM, FP32, velocity_shift = 1, reduce_every = 0,
 * rho_ref = (0, 0), kernel AUTO, drift_limit = 1e-6. */
lbm_status lbm_default_params(lbm_params *p);

/* Create a context: validates the geometry, builds the compact fluid index,
 * neighbour data and wall list on the host, allocates device memory (through
 * the allocator set by lbm_set_allocator, else cudaMalloc) and uploads it.
 * Populations start at zero: call lbm_init_densities or lbm_set_populations. */
lbm_status lbm_create(const lbm_geometry *geom, const lbm_params *params, lbm_ctx **out);
void lbm_destroy(lbm_ctx *ctx);

/* Device allocator used by later lbm_create calls in this process (for
 * example a framework's caching allocator).  alloc(bytes, user) returns a
 * device pointer or NULL; free(ptr, user) releases it.  Pass NULL, NULL to
 * restore cudaMalloc / cudaFree. */
lbm_status lbm_set_allocator(void *(*alloc)(size_t, void *), void (*free_fn)(void *, void *), void *user);

/* Rest-equilibrium initial state f_i = w_i rho^sigma (Eq. 2 with u = 0) from
 * dense host densities (doubles, nx*ny*nz each; solid voxels ignored).  Resets
 * the step counter and captures the frozen open-boundary populations (Section
 * 2 open boundary rule 2: missing populations keep their initial values). */
lbm_status lbm_init_densities(lbm_ctx *ctx, const double *rho1, const double *rho2);

/* Set / get the post-stream populations f_i^sigma of every fluid voxel.
 * Host layout [sigma][i][v], 2*19*nx*ny*nz doubles, D3Q19 order of Section 2;
 * solid entries are ignored on set and written as 0 on get.  set resets the
 * step counter and the frozen boundary populations like lbm_init_densities. */
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f);
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f);

/* Enqueue n time steps (Eqs. 1-15 with the inlet/outlet rules of Section 2).
 * Returns the sticky status observed so far (a failed periodic check from an
 * earlier step, a CUDA launch error), without synchronising. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t n);

/* Same as lbm_step, and also accumulates the device time of each kernel of
 * the split schedule into kernel_ms[0..nk) (density, wall, fused, plane,
 * pipeline), measured with CUDA events on the context stream. */
lbm_status lbm_step_timed(lbm_ctx *ctx, int64_t n, double *kernel_ms, int32_t nk);

/* Fields of the current state into dense host arrays of n_per_field doubles
 * (>= nx*ny*nz) each, in bit order RHO1, RHO2, UX, UY, UZ, P, packed
 * consecutively for the bits set in mask.  u = u^eq (Eq. 8, Section 2), P by
 * Eq. 12 over ordered pairs: c_s^2 (rho1 + rho2) + c_s^2 G rho1 rho2.  Solid
 * voxels read 0.  Synchronises. */
lbm_status lbm_read_fields(lbm_ctx *ctx, uint32_t mask, double *out, size_t n_per_field);

/* FP64 reductions of the current state (Section 4.1): out[0] = S_w, fraction
 * of sample fluid nodes with rho2 > rho1; out[1] = smooth non-wetting
 * saturation, mean of rho1 / (rho1 + rho2) over the sample; out[2], out[3] =
 * mass of components 1 and 2 over all fluid nodes.  Synchronises. */
lbm_status lbm_saturation(lbm_ctx *ctx, double out[4]);

/* Change the prescribed inlet density of component 1 (capillary-pressure
 * ramp of Section 4.1); takes effect from the next lbm_step. */
lbm_status lbm_set_inlet(lbm_ctx *ctx, double rho_in1);

/* Use this CUDA stream (a cudaStream_t) for all later device work. */
lbm_status lbm_set_stream(lbm_ctx *ctx, void *cuda_stream);

/* Wait for all enqueued work; returns the sticky device status. */
lbm_status lbm_synchronize(lbm_ctx *ctx);

lbm_status lbm_get_info(const lbm_ctx *ctx, lbm_info *info);
const char *lbm_last_error(const lbm_ctx *ctx);

/* ---- Batches: many independent samples stepped together ------------------
 * The drainage study of Section 4 runs one lattice per rock sample, contact
 * angle and viscosity ratio; those lattices are independent, so a batch steps
 * all of them with three launches per step (the density, wall and
 * collide-and-stream passes of every sample), each block working on one
 * sample.  Each sample's arithmetic is that of its solo run, node for node, so
 * its results are bitwise those of the same lattice stepped alone.
 *
 * lbm_create_batch creates n sample lattices from geoms[k], params[k] (as
 * lbm_create; kernel is forced to SPLIT, and every sample must use the same
 * storage type) and the batch that owns them.  The samples are reached with
 * lbm_batch_get and are initialised, read and retargeted (lbm_set_inlet) one
 * by one; they are stepped only through the batch (lbm_step on a sample
 * returns LBM_ERR_ARG), and all samples must be at the same step.  The batch
 * itself accepts lbm_step, lbm_set_stream (the samples follow), lbm_synchronize
 * (the first failing sample's status), lbm_get_info (sums over the samples),
 * lbm_autotune and lbm_destroy (which destroys the samples; lbm_destroy on a
 * sample does nothing).  On failure nothing is created and lbm_last_error(NULL)
 * names the sample. */
lbm_status lbm_create_batch(int32_t n, const lbm_geometry *geoms, const lbm_params *params, lbm_ctx **out);
int32_t lbm_batch_size(const lbm_ctx *batch);
lbm_status lbm_batch_get(lbm_ctx *batch, int32_t k, lbm_ctx **sample);

/* LBM_KERNEL_PERSISTENT (batches of up to 96 samples; params[0].kernel of
 * lbm_create_batch; LBM_ERR_UNSUPPORTED for a single lattice or a larger
 * batch): lbm_step runs up to 256 steps of every sample in one cooperative
 * launch whose blocks are all resident.  Each step is the split schedule's
 * three passes over all samples (densities with the open-plane rule, virtual
 * wall densities, force + collision + streaming), separated by grid-wide
 * barriers; the blocks deal the batch's node and wall blocks among themselves
 * with the same per-node arithmetic as the batched passes, so every sample's
 * results are bitwise those of its solo run.  Each barrier wait is bounded
 * (lbm_set_wait_limit, default 1 s); see Failure handling.  reduce_every > 0
 * on any sample steps the batch with the three-launch passes instead. */

/* lbm_step on a single lattice or a batch with the split schedule (or a
 * single lattice with the flow schedule), reduce_every = 0 and n >= 4 replays
 * steps from two CUDA graphs, captured
 * once on a private stream at the first even step after step 0 and
 * recaptured after any change of the lattice's parameters: 32 steps at a time
 * while at least 32 remain, then two at a time.  Setting the environment
 * variable LBM_NO_GRAPH disables them.
 *
 * LBM_KERNEL_WAVE (single lattices): the same three passes, launched per slab
 * of whole z planes (at least two per slab) from a graph of G steps (G = 4, or
 * the environment variable LBM_WAVE_STEPS, even) in which each pass of a slab
 * waits only for the passes of the slabs it reads: density(t, k) after
 * collide-stream(t-1, k-1..k+1), wall(t, k) after density(t, k-1..k+1),
 * collide-stream(t, k) after density and wall of (t, k-1..k+1).  Slabs of one
 * step and consecutive steps overlap, and a slab's populations are read twice
 * while they are still in L2.  The slab count is chosen from the node count
 * (LBM_WAVE_SLABS overrides it).  Results are those of the split schedule,
 * bit for bit; steps outside a graph run the split passes.
 *
 * LBM_KERNEL_FLOW (single lattices with fluid nodes, every storage type):
 * one launch per step.  Its blocks take slots in order from a ticket counter;
 * slot k collides and streams fluid chunk k, then computes the next step's
 * densities of an earlier chunk once every chunk writing its cells has
 * published a completion flag (the populations are then a few microseconds
 * old, mostly still in L2), then the virtual densities of an earlier wall
 * chunk; every wait targets a lower slot and gives up after the time limit of
 * lbm_set_wait_limit (LBM_ERR_TIMEOUT).  The per-node arithmetic is that of
 * the split passes, so results are bitwise those of LBM_KERNEL_SPLIT.
 * Environment variables LBM_FLOW_CHUNK (nodes per chunk, default 512),
 * LBM_FLOW_LAG_D and LBM_FLOW_LAG_W (slots, default 8) tune the plan at
 * lbm_create.  A density and wall pass runs first whenever the densities of
 * the current state are not already complete (after initialisation or a
 * parameter change).
 *
 * LBM_KERNEL_PUSH (FP32 storage, single lattices): no density pass.  The
 * collide-stream pass adds every post-collision population into the density
 * accumulator of the node it streams into (integer fixed point with a
 * resolution of 2^-26, so the sums are independent of the order of the
 * atomic adds and the results are bitwise reproducible); a plane pass then
 * applies the open-plane rule and sets the plane nodes' densities, and the
 * wall pass follows.  The force stencil reads these densities, which differ
 * from FP32 sums by at most a few units of 2^-26.  Graphs replay 30 steps
 * while at least 30 remain, then six.
 *
 * LBM_KERNEL_BRICK (FP32, FP16 and BF16 storage, single lattices): one launch
 * per step.  Fluid nodes are numbered brick by brick (8^3 voxels); one block
 * per brick stages the densities of the brick and a two-voxel halo in shared
 * memory, computes the virtual densities of the walls of the brick and a
 * one-voxel halo there (Eq. 15), collides and streams the brick's nodes with
 * the force stencil read from shared memory, and adds every stored
 * post-collision population into a shared-memory fixed-point accumulator of
 * the node it streams into (same encoding as LBM_KERNEL_PUSH).  Cells inside
 * the brick are then stored and the brick's faces and halo added atomically
 * into the next step's densities; a plane pass applies the open-plane rule.
 * No density or wall pass re-reads the populations.  Results agree with the
 * split schedule to the fixed-point rounding of the densities and are bitwise
 * reproducible; graphs replay as for LBM_KERNEL_PUSH.  lbm_record steps with this
 * schedule; the reverse pass recomputes its segments with the split passes. */

/* Autotuner: times a few steps of the context's own lattice (or batch) at
 * each candidate block size of the split schedule (64, 128, 256 threads;
 * 128 until the autotuner chooses),
 * keeps the fastest, and caches it in the JSON file cache_path (a flat object
 * of "key": block pairs; the key names the GPU, compute capability, storage
 * type, batch size and node counts).  A cached key is applied without timing.
 * The state, step counter and status word are saved before the trial steps
 * and put back afterwards (this needs a temporary copy of the populations).
 * cache_path may be NULL (no cache); *block_out (may be NULL) receives the
 * block size in use.  The single-pass schedule has a fixed block (its chunk)
 * and is returned as is.  Synchronises. */
lbm_status lbm_autotune(lbm_ctx *ctx, const char *cache_path, int32_t *block_out);

/* ---- Reverse pass (gradients) -------------------------------------------
 * Gradients of J = the smooth non-wetting saturation of the sample slab
 * (out[1] of lbm_saturation) after n steps, with respect to the per-voxel
 * wettability xi (chi^(1,2) = 1 +/- xi in the virtual wall density, Eq. 15)
 * and the inlet density rho_in1 of the open-boundary extrapolation (Section
 * 2).  The paper has no adjoint; this is the exact discrete adjoint of the
 * step as implemented (FP32 or FP64 storage, split schedule, single lattice,
 * LBM_BC_NEEM open planes; LBM_ERR_UNSUPPORTED otherwise).
 *
 * lbm_set_xi_field sets xi on every wall voxel from a dense nx*ny*nz float
 * array (host pointer when on_device = 0, device pointer otherwise); values
 * at non-wall voxels are ignored.
 *
 * lbm_record takes nsteps steps like lbm_step and keeps a copy of the state
 * every `every` steps (checkpoints: ceil(nsteps/every) + 1 copies of the
 * populations).  lbm_adjoint then computes the loss J of the final state and
 * runs the reverse pass: each segment of `every` steps is recomputed from its
 * checkpoint (keeping its every - 1 intermediate states), then reversed.
 * With the split or wave schedule and reduce_every = 0, lbm_record also keeps the densities and
 * virtual wall densities of every step (nsteps dense pairs over the voxels)
 * when they take at most a quarter of the free device memory: its steps then
 * each write their densities into their own slot (the whole recording is
 * captured as one CUDA graph the first time and replayed while its length,
 * buffers, starting parity and parameters stay the same; LBM_NO_GRAPH turns
 * that off), and the reverse pass recomputes only the collide-stream
 * pass of each state (and the open-plane rule), not its density and wall
 * passes.  The gradient is the same bit for bit; the environment variable
 * LBM_RECORD_DENSITIES=0 turns the kept densities off.  With kept densities,
 * lbm_adjoint recomputes segment k - 1 on a private stream, into a second set
 * of segment buffers, while it reverses segment k (LBM_ADJ_OVERLAP=0: one
 * segment after the other); the gradient is again the same bit for bit.
 * Outputs: grad_xi (device pointer to nx*ny*nz floats, or NULL) receives
 * dloss * dJ/dxi on wall voxels and 0 elsewhere; *grad_rho_in1 (host, or
 * NULL) receives dloss * dJ/drho_in1 (0 without open planes); *loss (host, or
 * NULL) receives J.  The context is left at the recorded final state, and the
 * recording stays usable until the state or a parameter changes (lbm_step,
 * initialisation, lbm_set_inlet, lbm_set_xi_field).  Synchronises. */
lbm_status lbm_set_xi_field(lbm_ctx *ctx, const float *xi, int32_t on_device);
lbm_status lbm_record(lbm_ctx *ctx, int64_t nsteps, int32_t every);
lbm_status lbm_adjoint(lbm_ctx *ctx, double dloss, float *grad_xi, double *grad_rho_in1, double *loss);

/* ---- Failure handling ----------------------------------------------------
 * The single-pass and flow schedules (LBM_KERNEL_FUSED, LBM_KERNEL_FLOW) and
 * the persistent batch launch (LBM_KERNEL_PERSISTENT) order their blocks with
 * device waits; each wait gives up after a time limit (default 1 s, measured with the
 * GPU's global timer), sets an abort word that stops every block, and raises
 * LBM_ERR_TIMEOUT from the next lbm_step / lbm_synchronize.  The kernel then
 * returns normally: the context stays usable, the populations of the
 * abandoned step are undefined, and the next initialisation (or
 * lbm_set_populations) starts over; the schedule's counters are cleared
 * before its next launch.
 *
 * lbm_set_wait_limit sets the limit (0 < seconds <= 60).  lbm_inject_stall
 * makes the next single-pass step wait for a round that never completes (the
 * next flow step: one density item waits for a flag value that is never
 * written; the next persistent launch: one block never reaches its first
 * grid barrier), so that the timeout path can be tested without faulting or
 * hanging the GPU (LBM_ERR_UNSUPPORTED for other schedules).  For a batch,
 * re-initialising a sample (lbm_init_densities, lbm_set_populations) clears
 * the batch's timeout record. */
lbm_status lbm_set_wait_limit(lbm_ctx *ctx, double seconds);
lbm_status lbm_inject_stall(lbm_ctx *ctx);

/* ---- Checkpoint / resume (the paper has none) ----------------------------
 * lbm_save writes the lattice's state to a file: every population cell (in
 * the storage type, as stored), the open-plane boundary cells, the frozen
 * missing populations of the open planes, the step count, the deviation
 * reference densities of 16-bit storage and the initial masses of the drift
 * check, behind a header that names the storage type, the grid and a hash of
 * the solid mask.  lbm_load reads such a file into a lattice created with
 * the same geometry and storage type (LBM_ERR_ARG for any other file, or one
 * that is truncated) and sets its step count; stepping on from there gives
 * bitwise the results of the uninterrupted run.  Both synchronise; a sample
 * of a batch can be saved and loaded, a batch itself cannot (LBM_ERR_ARG). */
lbm_status lbm_save(lbm_ctx *ctx, const char *path);
lbm_status lbm_load(lbm_ctx *ctx, const char *path);

/* Largest n accepted by lbm_saturation_static. */
#define LBM_SATURATION_STATIC_MAX_N 16777216

/* The reduction of lbm_saturation, for callers that cannot allocate device
 * memory (their device memory belongs to another allocator that has reserved
 * it, or they must not pay for an allocation or the device-wide
 * synchronisation that cudaMalloc / cudaFree can cause).  The paper has no
 * counterpart: this is a library convenience, not part of the method.
 *
 * Inputs (device pointers, caller-owned): rho1[n], rho2[n] component
 * densities of the fluid nodes (FP32); sample[n] optional (NULL = all nodes),
 * nonzero marks the nodes counted by the saturation.  Output (device pointer,
 * caller-owned): out[4] = S_w (fraction of sample nodes with rho2 > rho1),
 * smooth S_nw (mean of rho1 / (rho1 + rho2) over the sample), mass1, mass2
 * (FP64 sums over all n nodes).  stream: a cudaStream_t or NULL.
 *
 * Allocates nothing.  Scratch is a 256 KB FP64 array in the library's static
 * device memory, held by every GPU that loads the library until exit; it is
 * shared by all calls and keeps the last call's partial sums (each call
 * overwrites every entry it reads, so nothing needs clearing).  Calls that
 * overlap on the GPU (different streams, or different host threads on one
 * device) race on that array.  The first call on each device looks up the
 * array's device address with that device current, and so does the first
 * call in a new context of that device (after cudaDeviceReset the array is
 * loaded again at another address); make such a first call before any stream
 * capture.  Returns LBM_ERR_ARG for n < 0, NULL pointers or
 * n > LBM_SATURATION_STATIC_MAX_N, LBM_ERR_CUDA if the lookup or a launch
 * fails; the work is enqueued on stream, not waited for. */
lbm_status lbm_saturation_static(const float *rho1, const float *rho2, const uint8_t *sample, int64_t n, double *out,
                                 void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
