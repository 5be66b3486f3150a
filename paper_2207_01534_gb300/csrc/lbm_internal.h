// lbm_internal.h -- device state shared by the host API and the kernel
// translation units of liblbm.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Node flag bits (uint8 per fluid node; bits 24..29 of a wall's mask word use
// the same face bits shifted by 24).  A periodic-face bit means the neighbour
// across that face wraps to the opposite face.  INLET / OUTLET mark the nodes
// of the z = 0 and z = nz-1 open planes.
enum : uint32_t {
    F_XLO = 1u, F_XHI = 2u, F_YLO = 4u, F_YHI = 8u, F_ZLO = 16u, F_ZHI = 32u,
    F_INLET = 64u, F_OUTLET = 128u
};
constexpr uint32_t kFaceMask = 63u;
constexpr int kWallFaceShift = 24;

// Everything a kernel needs, passed by value.
struct DevState {
    // populations: moving pairs M[18][npad] (storage type) and rest pairs
    // R[npad] (compute precision); see lbm_kernels.cuh
    void *f;
    void *rest;
    int64_t npad;            // stride between direction rows (multiple of 64)
    int32_t n_fluid;
    const uint32_t *pvox;    // [n_fluid] voxel index v = x + nx*(y + ny*z)
    const uint8_t *nflags;   // [n_fluid]
    const int32_t *cidx;     // [nv] compact index of a fluid voxel, -1 solid
    void *psi;               // [nv] pairs (psi1, psi2) in the compute type
    int32_t nx, ny, nz;
    int32_t sx, sxy;         // strides nx, nx*ny
    int64_t nv;
    // walls (solid voxels with at least one fluid neighbour)
    int32_t n_wall;
    const uint32_t *wpvox;   // [n_wall]
    const uint32_t *wmask;   // [n_wall] bit i: direction i leads to an in-domain fluid voxel; face bits << 24
    const void *winv;        // [n_wall] 1 / sum of w_i over those directions (Eq. 15 denominator), compute type
    const void *wxi;         // [n_wall] xi at the wall voxel, compute type
    // open planes (z): bc cells hold the missing population pairs of the
    // odd-parity layout, [plane][k][nxy] in the storage type; frozen holds the
    // initial values of the non-prescribed component's missing populations,
    // [plane][k][nxy] (double).
    int32_t open_z;
    int32_t zou_he;          // plane rule for the prescribed component: 0 extrapolation, 1 Zou-He
    void *bc;
    const double *frozen;
    int32_t nxy;
    // sample slab for saturation
    int32_t sample_lo, sample_hi;
    // model parameters
    double tau1, tau2, G, gx, gy, gz, rho_in1, rho_out2;
    double rref1, rref2;
    int32_t velocity_shift;
    // the same parameters rounded to FP32 once on the host (set_float_params),
    // for the kernels that compute in FP32: converting a double in every
    // thread would run on the FP64 pipe, which GB300 provides at a small
    // fraction of the FP32 rate
    float ftau1, ftau2, fG, fgx, fgy, fgz, frho_in1, frho_out2, frref1, frref2;
};

// Round the double parameters of s into its FP32 copies (round to nearest,
// as a conversion in a kernel would).
inline void set_float_params(DevState &s)
{
    s.ftau1 = (float)s.tau1;
    s.ftau2 = (float)s.tau2;
    s.fG = (float)s.G;
    s.fgx = (float)s.gx;
    s.fgy = (float)s.gy;
    s.fgz = (float)s.gz;
    s.frho_in1 = (float)s.rho_in1;
    s.frho_out2 = (float)s.rho_out2;
    s.frref1 = (float)s.rref1;
    s.frref2 = (float)s.rref2;
}

// Single-pass schedule: one cooperative launch per step (all blocks
// co-resident).  Chunks are dealt round-robin: in round r block b collides and
// streams chunk r*G + b (F), computes the next-step densities of chunk
// (r - lag_d)*G + b (D, with the open-plane extrapolation), and the wall
// densities of wall chunk (r - lag_w)*G + b (W).  D waits for F of every chunk
// up to need_f[c]; W for D up to need_d[c].  F never waits, and the lags make
// every wait target a phase that is already done or running without waiting,
// so the launch always finishes; waits are bounded anyway (wait_ns of the
// global timer, and kPipeMaxPolls polls as a backstop).
// Completion frontiers are tagged with the launch epoch, so nothing is reset
// between launches.
constexpr int kChunk = 256;             // fluid nodes per chunk = threads per block
constexpr int kPipeMaxPolls = 1 << 22;  // polls of a frontier before a block gives up

struct PipeState {
    // Completion counters per chunk round R (chunks R*G .. R*G+G-1), one per
    // warp slot: warp w of every block adds 1 when its nodes of that round are
    // done (or it has none), so in launch `epoch` a round is complete once all
    // its counters reach epoch * G.  They only grow: nothing is reset between
    // launches.
    unsigned long long *round_f; // [n_rounds][8 warp slots] for F, at stride 16 (128-byte lines)
    unsigned long long *round_d; // [n_rounds][8 warp slots] for D, at stride 16
    const int *need_f;           // [n_chunks] last F chunk that D of the chunk reads
    const int *need_d;           // [n_chunks] last D chunk that W of the wall chunk reads (-1: none)
    const int *wstart;           // [n_chunks + 1] wall index range of each wall chunk
    int *abort;                  // set when a block gives up: every block stops
    int *status;                 // host-mapped status word (bit 4: timeout)
    void *psi_next;              // densities of the next step (the other psi buffer)
    int epoch;                   // 1 + launches of this schedule so far
    int n_chunks, n_rounds, lag_d, lag_w, rounds;
    unsigned long long wait_ns;  // a wait gives up after this long (global timer)
};

// Flow schedule: one launch per time step.  The launch has n_slots blocks of
// kFlowThreads threads; a block takes the next ticket of a counter that only
// grows (slot k = ticket mod n_slots, launch stamp = ticket / n_slots + 1), so
// slots are handed out in order and a block only ever waits for items of
// lower slots, which are already running.  Fluid chunks are runs of `chunk`
// consecutive nodes (a multiple of kFlowThreads).  Slot k runs, in this order:
//   F(k)   collide and stream fluid chunk k when k < n_chunks; it reads only
//          data of earlier launches;
//   D(d)   d = items[k].x >= 0: the next step's densities of chunk d (open-
//          plane rule first), after F of every chunk in dep_f[d] is done;
//   W(w)   w = items[k].y >= 0: the next step's virtual wall densities of wall
//          chunk w (walls between the first voxels of fluid chunks w and
//          w+1), after D of every chunk in dep_d[w] is done;
// and publishes the stamp in fdone[k] / ddone[d] as soon as F / D is done.
// D and W lag F by a few slots, so the populations D reads were written a
// few microseconds earlier and are still in L2.  Waits are bounded by time
// (global timer).
constexpr int kFlowThreads = 128;
struct FlowState {
    unsigned long long *ticket;  // slot tickets of every launch so far
    int *fdone;                  // [n_chunks] stamp of the launch whose F(c) is done
    int *ddone;                  // [n_chunks] same for D(c)
    int *abort;                  // stamp of a launch that gave up
    int *status;                 // host-mapped status word (bit 4: timeout)
    const int2 *dep_f;           // [n_chunks] F chunk range that D(c) reads
    const int2 *dep_d;           // [n_chunks] D chunk range that W(c) reads (y < x: none)
    const int *wstart;           // [n_chunks + 1] wall index range of wall chunk c
    const int2 *items;           // [n_slots] (D chunk, W chunk) run by slot k, -1: none
    void *psi_next;              // densities of the next step (the other psi buffer)
    int chunk;                   // fluid nodes per chunk
    int n_chunks, n_slots;
    int stall_slot;              // >= 0: that slot's D waits for a stamp that never comes (failure test)
    unsigned long long wait_ns;  // a wait gives up after this long
};

// Batches of up to kParamStates samples pass every sample's DevState and the
// first launch block of every sample in the kernel's parameter space (32 KB):
// a block finds its sample by a binary search over the block offsets, with no
// table in global memory and no copy to shared memory.
constexpr int kParamStates = 96;
struct BatchTable {
    DevState s[kParamStates];
    int start_n[kParamStates + 1];  // first block of each sample in the node passes; [count] = total
    int start_w[kParamStates + 1];  // same for the wall pass
    int count;
};

// Persistent batch launch (lbm_persist.cuh): `steps` time steps of every
// sample of a batch table in one cooperative launch, the passes separated by
// grid barriers on a counter that only grows during the launch.
struct PersistArgs {
    unsigned long long *bar;     // grid barrier counter (cleared before the launch)
    int *abort;                  // set by a block that gave up
    int *status;                 // host-mapped status word (bit value 4: timeout)
    unsigned long long base;     // counter value when the launch starts (0)
    unsigned long long wait_ns;  // a barrier wait gives up after this long
    long long step0;             // step of the batch when the launch starts
    int steps;                   // time steps of this launch
    int stall;                   // failure test: block 0 never arrives at the first barrier
};
static_assert(sizeof(BatchTable) + sizeof(PersistArgs) <= 32764, "kernel parameters of the persistent launch");

// Per-storage-type kernel launchers, explicitly instantiated in one
// translation unit per storage type.
template <typename TS>
struct Ops {
    // densities into psi; neem != 0 first applies the open-plane extrapolation.
    // [n0, n1) / [w0, w1): node / wall ranges (n1, w1 < 0: to the end)
    static void dens(const DevState &s, int parity, int neem, cudaStream_t st, int block = 256, int n0 = 0,
                     int n1 = -1);
    static void wall(const DevState &s, cudaStream_t st, int block = 256, int w0 = 0, int w1 = -1);
    static void fused(const DevState &s, int parity, cudaStream_t st, int block = 256, int n0 = 0, int n1 = -1);
    // the same three passes over many samples in one launch each: states[k] is
    // sample k; map[b] = (sample, block within the sample) for launch block b
    static void dens_batch(const DevState *states, const int2 *map, int nblocks, int parity, int neem,
                           cudaStream_t st, int block);
    static void wall_batch(const DevState *states, const int2 *map, int nblocks, cudaStream_t st, int block);
    static void fused_batch(const DevState *states, const int2 *map, int nblocks, int parity, cudaStream_t st,
                            int block);
    // the same passes with the batch table in parameter space
    static void dens_table(const BatchTable &t, int parity, int neem, cudaStream_t st, int block);
    static void wall_table(const BatchTable &t, cudaStream_t st, int block);
    static void fused_table(const BatchTable &t, int parity, cudaStream_t st, int block);
    // pa.steps steps of the whole table in one cooperative launch of `grid`
    // blocks of `block` threads (block = the table's block size)
    static cudaError_t persist(const BatchTable &t, const PersistArgs &pa, int grid, int block, cudaStream_t st);
    // resident blocks of `block` threads on the current device for persist()
    static int persist_grid(int block);
    static void plane(const DevState &s, int parity_next, cudaStream_t st);
    // rest equilibrium from device densities rho[2][nv] (double); parity-0 layout
    static void init_eq(const DevState &s, const double *rho, cudaStream_t st);
    // populations [2][19][nv] (double, device) -> parity-0 layout
    static void scatter(const DevState &s, const double *f, cudaStream_t st);
    // current layout -> populations [2][19][nv] (double, device); solids untouched
    static void gather(const DevState &s, int parity, double *f, cudaStream_t st);
    // capture the frozen missing populations from the parity-0 layout
    static void capture_frozen(const DevState &s, double *frozen, cudaStream_t st);
    // fields (rho1, rho2, ux, uy, uz, P) selected by mask, packed [k][nv]
    // (double, device; solids 0); needs dens+wall first
    static void fields(const DevState &s, int parity, double *out, uint32_t mask, cudaStream_t st);
    // FP64 reduction over psi (needs dens first): partials[nblocks][8] then out[8]
    static void reduce(const DevState &s, double *partials, int nblocks, double *out, cudaStream_t st);
    // one step of the single-pass schedule at parity `parity` on `grid` blocks
    static void pipe(const DevState &s, const PipeState &ps, int parity, int grid, cudaStream_t st);
    // resident blocks per SM of the single-pass kernel
    static int pipe_blocks_per_sm();
    // one step of the flow schedule at parity `parity` (fs.n_slots blocks)
    static void flow(const DevState &s, const FlowState &fs, int parity, cudaStream_t st);
};

// Push schedule (FP32 storage only, lbm_push.cu): the collide-stream pass
// adds every post-collision population into the fixed-point density
// accumulator of the node it streams into.
struct PushBufs {
    const unsigned long long *rd;  // densities of this step (dense, fluid and wall voxels)
    unsigned long long *acc;       // next step's accumulators (cleared, fluid voxels)
    unsigned long long *clr;       // the buffer to clear for the step after (by the finish pass)
    const uint32_t *nmask;         // [n_fluid] bit j: x + e_j is an in-domain fluid voxel
};
void push_fused(const DevState &s, const PushBufs &pb, int parity, cudaStream_t st);
// After the pass: plane nodes (open-plane rule at the next parity, exact
// density), the walls [w_lo, w_hi) and the clearing of clr in one launch,
// then the other walls (those within two planes of an open plane).  Returns
// the launch count.
int push_finish(const DevState &s, unsigned long long *acc, unsigned long long *clr, int parity_next, int w_lo,
                int w_hi, cudaStream_t st);
// densities from the float psi of a density + wall pass (fluid and wall voxels)
// (walls = false: fluid voxels only, as the brick schedule keeps them)
void push_prime(const DevState &s, unsigned long long *acc, cudaStream_t st, bool walls = true);

// Brick schedule (all but FP64 storage, lbm_brick.cu): one block per brick
// of 8^3 voxels collides and streams the brick's nodes, with the densities of
// the brick and its halo, the virtual densities of its walls and the next
// step's density accumulators in shared memory.  Fluid nodes are numbered
// brick by brick.
constexpr int kBrick = 8;        // brick edge (voxels)
constexpr int kR1 = kBrick + 2;  // brick plus a one-voxel halo
constexpr int kR2 = kBrick + 4;  // brick plus a two-voxel halo
constexpr int kR1Cells = kR1 * kR1 * kR1;
constexpr int kR2Cells = kR2 * kR2 * kR2;
constexpr int kBrickThreads = 128;
constexpr int kBrickBlocks = 768 / kBrickThreads;  // resident blocks per SM (80 registers a thread)
struct BrickInfo {
    int x0, y0, z0;  // origin (voxels)
    int ext;         // extents bx | by << 8 | bz << 16 (clipped at the domain's end)
    int n0, n1;      // its fluid nodes
    int w0, w1;      // its wall entries: the walls of the brick and its one-voxel halo
};
struct BrickBufs {
    const BrickInfo *info;          // [bricks with fluid nodes]
    const uint16_t *nloc;           // [n_fluid] lx + 8 ly + 64 lz inside the node's brick
    const uint32_t *wcell;          // [entries] fluid-direction mask (bits 1..18) | halo-region cell << 20
    const float2 *wcoef;            // [entries] ((1 + xi) / W, (1 - xi) / W), W the Eq. 15 denominator
    const unsigned long long *rd;   // densities of this step (fluid voxels)
    unsigned long long *acc;        // next step's accumulators (face and halo voxels cleared)
    unsigned long long *clr;        // the buffer whose face voxels this step clears
    int per;                        // periodic axes: bit 0 x, bit 1 y, bit 2 z
};
template <typename TS>
void brick_step(const DevState &s, const BrickBufs &bb, int nbricks, int parity, cudaStream_t st);
// plane nodes after the brick launch: open-plane rule at the next parity, density totals
template <typename TS>
void brick_plane(const DevState &s, unsigned long long *acc, int parity_next, cudaStream_t st);
// wall coefficients of the brick entries from the wall arrays (after a new xi field)
void brick_coef(const DevState &s, const int32_t *wid, int n, float2 *coef, bool fp64, cudaStream_t st);

// Geometry preprocessing on the device (lbm_geom.cu): the compact index,
// flag bytes, wall list and plane prefixes of lbm_create from the solid mask
// in device memory, entry for entry those of the host preprocessing.
struct GeomPlan {
    int nx, ny, nz, per[3], open_z;
    int bpp, nblocks;          // 1024-voxel blocks per z plane, in all
    const uint8_t *d_solid;    // nx*ny*nz mask on the device
};
GeomPlan geom_plan(const uint8_t *d_solid, int nx, int ny, int nz, const int per[3], int open_z);
// pass 1: block counts (d_cnt[nblocks]), offsets (d_off[nblocks]), error bits
// (*d_err, or-ed: 1 closed face, 2 solid behind an open plane) and d_out =
// [N, NW, first node of z planes 0..nz, first wall of z planes 0..nz]
void geom_count(const GeomPlan &g, int2 *d_cnt, int2 *d_off, int *d_err, int *d_out, cudaStream_t st);
// pass 2: the arrays (winv / wxi in FP64 when fp64, else FP32); d_xi (nx*ny*nz
// floats) or, when null, xi0 for every wall
void geom_fill(const GeomPlan &g, const float *d_xi, double xi0, const int2 *d_off, int32_t *cidx, uint32_t *pvox,
               uint8_t *nflags, uint32_t *wpvox, uint32_t *wmask, void *winv, void *wxi, bool fp64, cudaStream_t st);

constexpr int kReduceBlocks = 1024;
constexpr int kReduceThreads = 256;
constexpr int kReduceSlots = 8;  // m1, m2, count, nw, smooth, nonfinite, unused, unused

}  // namespace lbm
