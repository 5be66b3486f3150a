// lbm_capi.cu -- host side of liblbm: geometry preprocessing (compact fluid
// index, neighbour flags, wall list, open planes), device memory, the C ABI
// declared in include/lbm.h, and the schedule of kernels per time step.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_kernels.cuh"
#include "lbm_adjoint.cuh"

namespace lbm {
// instantiated in lbm_adj32.cu / lbm_adj64.cu
extern template struct Adj<float>;
extern template struct Adj<double>;
}

using namespace lbm;

namespace {

// NVTX range over one ABI call (shows in Nsight Systems / ncu range filters;
// without a tool attached the calls do nothing)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

std::string g_create_err;
void *(*g_alloc)(size_t, void *) = nullptr;
void (*g_free)(void *, void *) = nullptr;
void *g_alloc_user = nullptr;

constexpr int kNumTimed = 5;  // dens, wall, fused, plane, pipeline

}  // namespace

struct lbm_ctx {
    int device = 0;
    cudaStream_t stream = 0;
    int nx = 0, ny = 0, nz = 0;
    int64_t nv = 0;
    int periodic[3] = {0, 0, 0};
    int open_axis = -1;
    lbm_params p{};
    int storage = LBM_STORE_FP32;
    int kernel = LBM_KERNEL_SPLIT;
    DevState s{};
    void *(*alloc_fn)(size_t, void *) = nullptr;
    void (*free_fn)(void *, void *) = nullptr;
    void *alloc_user = nullptr;
    std::vector<std::pair<void *, size_t>> allocs;  // live device allocations and their sizes
    int64_t step = 0, launches = 0, bytes = 0;
    lbm_status sticky = LBM_OK;
    std::string err;
    double *d_partials = nullptr;
    double *d_red = nullptr;
    double *d_frozen = nullptr;
    int *h_flag = nullptr;  // pinned, device-mapped status word
    int *d_flag = nullptr;
    // push and brick schedules: rotating density accumulators (two for push,
    // three for brick), fluid-neighbour masks, and the step whose densities
    // acc[step % ring] holds (-1: none)
    unsigned long long *acc[3] = {nullptr, nullptr, nullptr};
    uint32_t *d_nmask = nullptr;
    int64_t push_step = -1;
    // brick schedule: per-brick tables (lbm_brick.cuh) and the wall ids of
    // its wall entries (for new coefficients after a change of xi)
    BrickBufs bb{};
    int n_bricks = 0, n_bentries = 0;
    int32_t *d_bwid = nullptr;
    double mass0[2] = {0, 0};
    cudaEvent_t ev[kNumTimed + 1];
    bool have_ev = false;
    // single-pass schedule
    PipeState ps{};
    // threads per block of the split-schedule passes: 128 by default (on the 128^3 pack
    // 0.0839 vs 0.0864 ms per step at 256, FP16 0.0666 vs 0.0703), lbm_autotune may change it
    int block = 128;
    // batch contexts: samples stepped together by batched launches
    std::vector<lbm_ctx *> subs;
    lbm_ctx *parent = nullptr;
    DevState *d_states = nullptr;
    int2 *d_map_n = nullptr, *d_map_w = nullptr;
    int n_map_n = 0, n_map_w = 0, map_block = 0;
    BatchTable *table = nullptr;  // batches of up to kParamStates samples: states and block offsets
    bool states_dirty = true;
    // persistent batch launch (LBM_KERNEL_PERSISTENT): grid-barrier counter
    // and abort word, both cleared before every launch
    unsigned long long *d_bar = nullptr;
    int *d_abort = nullptr;
    // CUDA graph of two split-schedule steps, captured on a private stream
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool graph_dirty = true;
    int64_t graph_launches = 0;  // kernels per replay
    // a short graph for the steps left over after the long one's replays
    cudaGraphExec_t graph_short = nullptr;
    int64_t graph_short_launches = 0;
    int graph_short_steps = 0;
    int graph_steps = 2;         // steps per replay
    // wavefront schedule: per-plane prefix counts of fluid nodes and walls,
    // slab boundaries (z planes), and the capture streams / events
    std::vector<int> plane_n, plane_w, slab_z;
    bool per_z = false;  // z periodic: the first and last slabs are neighbours
    std::vector<cudaStream_t> wave_streams;
    std::vector<cudaEvent_t> wave_events;
    size_t f_bytes = 0, rest_bytes = 0, bc_bytes = 0;  // the state a step reads and writes
    std::vector<uint8_t> solid_host;  // the mask, for host-side statistics
    // recording for the reverse pass (lbm_record / lbm_adjoint)
    struct Record {
        bool valid = false;
        int64_t step0 = 0, n = 0, every = 0, step_end = 0;
        std::vector<void *> ckpt;  // state at step0 + k*every
        void *final_state = nullptr;
        std::vector<void *> seg;   // states inside one segment
        std::vector<void *> psis;  // densities (psi) of each state of a segment
        // densities of every recorded step, written by the recording steps
        // themselves when they fit (then the reverse pass recomputes only the
        // collide-stream pass of each state, not its density and wall passes)
        void *dens_all = nullptr;
        size_t dens_all_bytes = 0;
        bool dens_stored = false;
        // a second set of segment states, a side stream and its events: the
        // recompute of one segment overlaps the reverse of the next
        std::vector<void *> seg2;
        cudaStream_t side = nullptr;
        cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        // the recording steps with kept densities as one CUDA graph, replayed
        // while the recording's shape, buffers, parity and parameters stay
        cudaGraphExec_t graph = nullptr;
        std::vector<void *> graph_key;  // buffers it writes
        int64_t graph_n = 0, graph_every = 0, graph_launches = 0;
        int graph_par = -1, graph_block = 0;
        DevState graph_state{};  // the kernel arguments it holds (every parameter and pointer)
        void *lam[2] = {nullptr, nullptr}, *rb[2] = {nullptr, nullptr};
        void *abar = nullptr, *wbar = nullptr, *psi = nullptr;
        double *gxi = nullptr, *grin = nullptr;
        int64_t count = 0;  // fluid nodes of the sample slab
    } rec;
    void *psi_alt = nullptr;
    // flow schedule: its plan and counters (FlowState), the two density
    // buffers (the densities of step t live in flow_psi[t & 1]), and the step
    // whose densities flow_psi holds complete (-1: none; the next flow step
    // first runs a density and wall pass)
    FlowState fs{};
    void *flow_psi[2] = {nullptr, nullptr};
    int64_t flow_ok_step = -1;
    int flow_lag[2] = {0, 0};
    int flow_stall_slot = -1;  // a slot with a D item (lbm_inject_stall)
    void *fields_buf = nullptr;  // lbm_read_fields output on the device
    size_t fields_bytes = 0;
    int pipe_grid = 0;
    int64_t pipe_launches = 0;
    bool pipe_reset = false;  // a single-pass launch gave up: clear its counters before the next
    bool stall_next = false;  // lbm_inject_stall: the next single-pass launch waits for nothing
};

namespace lbm {

__global__ void __launch_bounds__(kReduceThreads) k_reduce_final(const double *partials, int nblocks, double *out)
{
    __shared__ double sm[kReduceThreads / 32];
    for (int k = 0; k < 6; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(long long)b * kReduceSlots + k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            double w = threadIdx.x < kReduceThreads / 32 ? sm[threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
            if (threadIdx.x == 0) out[k] = w;
        }
        __syncthreads();
    }
}

// Sets status bits from a finished reduction: 1 = non-finite density,
// 2 = relative mass drift above the limit (closed domains only).
__global__ void k_check(const double *red, double m01, double m02, double limit, int closed, int *flag)
{
    int bits = 0;
    if (red[5] > 0.0) bits |= 1;
    if (closed) {
        if (fabs(red[0] - m01) > limit * fabs(m01) || fabs(red[1] - m02) > limit * fabs(m02)) bits |= 2;
    }
    if (bits) atomicOr(flag, bits);
}

}  // namespace lbm

namespace {

// Run fn(z) for every z plane in [0, nz) on the host's cores (planes handed
// out in order through a shared counter; fn must only write what plane z
// owns).
template <class Fn>
void parallel_planes(int nz, Fn &&fn)
{
    unsigned t = std::thread::hardware_concurrency();
    t = std::max(1u, std::min(t, 64u));
    t = std::min<unsigned>(t, (unsigned)std::max(1, nz / 2));
    if (t <= 1) {
        for (int z = 0; z < nz; ++z) fn(z);
        return;
    }
    std::atomic<int> next(0);
    auto work = [&]() {
        for (int z = next++; z < nz; z = next++) fn(z);
    };
    std::vector<std::thread> th;
    for (unsigned k = 1; k < t; ++k) th.emplace_back(work);
    work();
    for (std::thread &x : th) x.join();
}

lbm_status fail(lbm_ctx *c, lbm_status st, const std::string &msg)
{
    if (c)
        c->err = msg;
    else
        g_create_err = msg;
    return st;
}

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Device path of the geometry preprocessing: one temporary device block for
// the uploaded mask (and xi field), the block counts and offsets, and the
// small result record; released after the fill pass has run.
struct DevPrep {
    void *buf = nullptr;
    uint8_t *mask = nullptr;
    float *xi = nullptr;
    int2 *cnt = nullptr, *off = nullptr;
    int *small = nullptr;  // [err, N, NW, plane_n[0..nz], plane_w[0..nz]]
    GeomPlan plan{};
    void release()
    {
        if (!buf) return;
        if (g_free) {
            cudaStreamSynchronize(0);  // the fill pass reads the mask
            g_free(buf, g_alloc_user);
        } else {
            cudaFreeAsync(buf, 0);  // stream-ordered after the fill pass
        }
        buf = nullptr;
    }
    ~DevPrep() { release(); }
};

// Upload the mask, count fluid voxels and walls per block on the device and
// read back the totals, plane prefixes and geometry checks.
lbm_status dev_prep_count(DevPrep &dp, const lbm_geometry *g, int nx, int ny, int nz, const int per[3], bool open_z,
                          int64_t *N, int64_t *NW, std::vector<int> &plane_n, std::vector<int> &plane_w,
                          bool *closed_face, bool *plane_solid)
{
    const int64_t nv = (int64_t)nx * ny * nz;
    dp.plan = geom_plan(nullptr, nx, ny, nz, per, open_z ? 1 : 0);
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t nb = (size_t)dp.plan.nblocks, nsmall = 3 + 2 * ((size_t)nz + 1);
    const size_t b_mask = al((size_t)nv), b_xi = g->xi_field ? al((size_t)nv * 4) : 0, b_cnt = al(nb * 8);
    const size_t total = b_mask + b_xi + 2 * b_cnt + al(nsmall * 4);
    if (g_alloc) {
        dp.buf = g_alloc(total, g_alloc_user);
    } else if (cudaMallocAsync(&dp.buf, total, 0) != cudaSuccess) {
        cudaGetLastError();
        dp.buf = nullptr;
    }
    if (!dp.buf) return fail(nullptr, LBM_ERR_ALLOC, "device allocation failed (geometry preprocessing)");
    char *q = (char *)dp.buf;
    dp.mask = (uint8_t *)q;
    q += b_mask;
    if (b_xi) {
        dp.xi = (float *)q;
        q += b_xi;
    }
    dp.cnt = (int2 *)q;
    q += b_cnt;
    dp.off = (int2 *)q;
    q += b_cnt;
    dp.small = (int *)q;
    dp.plan.d_solid = dp.mask;
    cudaError_t e = cudaMemcpy(dp.mask, g->solid, (size_t)nv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && dp.xi) e = cudaMemcpy(dp.xi, g->xi_field, (size_t)nv * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(dp.small, 0, 4, 0);
    if (e == cudaSuccess) {
        geom_count(dp.plan, dp.cnt, dp.off, dp.small, dp.small + 1, 0);
        e = cudaGetLastError();
    }
    std::vector<int> h(nsmall);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), dp.small, nsmall * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, std::string("geometry preprocessing: ") + cudaGetErrorString(e));
    *closed_face = (h[0] & 1) != 0;
    *plane_solid = (h[0] & 2) != 0;
    *N = h[1];
    *NW = h[2];
    for (int z = 0; z <= nz; ++z) {
        plane_n[(size_t)z] = h[3 + (size_t)z];
        plane_w[(size_t)z] = h[3 + ((size_t)nz + 1) + (size_t)z];
    }
    return LBM_OK;
}


void *dalloc(lbm_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    void *ptr = nullptr;
    if (c->alloc_fn) {
        ptr = c->alloc_fn(bytes, c->alloc_user);
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) {
        c->allocs.push_back({ptr, bytes});
        c->bytes += (int64_t)bytes;
    }
    return ptr;
}

void dfree(lbm_ctx *c, void *ptr)
{
    if (!ptr) return;
    for (size_t k = 0; k < c->allocs.size(); ++k)
        if (c->allocs[k].first == ptr) {
            c->bytes -= (int64_t)c->allocs[k].second;
            c->allocs.erase(c->allocs.begin() + (long)k);
            break;
        }
    if (c->free_fn)
        c->free_fn(ptr, c->alloc_user);
    else
        cudaFree(ptr);
}

// Short-lived device buffers of one call (uploads, read-backs): stream-ordered
// on the context's stream when the library allocates with the CUDA runtime,
// so freeing one does not wait for the device; through the user's allocator
// otherwise (then after a synchronisation of the stream).
void *talloc(lbm_ctx *c, size_t bytes)
{
    if (c->alloc_fn) return dalloc(c, bytes);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes ? bytes : 256, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void tfree(lbm_ctx *c, void *p)
{
    if (!p) return;
    if (c->alloc_fn) {
        cudaStreamSynchronize(c->stream);
        dfree(c, p);
    } else {
        cudaFreeAsync(p, c->stream);
    }
}

// Run fn with the storage type of the context as a template tag.
template <class Fn>
void dispatch(const lbm_ctx *c, Fn &&fn)
{
    switch (c->storage) {
    case LBM_STORE_FP64: fn(double{}); break;
    case LBM_STORE_FP16DEV: fn(__half{}); break;
    case LBM_STORE_BF16DEV: fn(__nv_bfloat16{}); break;
    default: fn(float{}); break;
    }
}

bool is16(int storage) { return storage == LBM_STORE_FP16DEV || storage == LBM_STORE_BF16DEV; }

// Reference densities of the 16-bit deviation storage: the parameters when
// given, else the mean of each component over the fluid voxels of the state
// being loaded.
void choose_rho_ref(lbm_ctx *c, const double *r1, const double *r2, int64_t stride)
{
    if (!is16(c->storage) || c->p.rho_ref[0] != 0.0 || c->p.rho_ref[1] != 0.0) return;
    double m[2] = {0, 0};
    int64_t cnt = 0;
    for (int64_t v = 0; v < c->nv; ++v) {
        if (c->solid_host[(size_t)v]) continue;
        double a = 0, b = 0;
        for (int i = 0; i < (stride ? 19 : 1); ++i) {
            a += r1[v + i * stride];
            b += r2[v + i * stride];
        }
        m[0] += a;
        m[1] += b;
        ++cnt;
    }
    c->s.rref1 = cnt ? m[0] / (double)cnt : 0.0;
    c->s.rref2 = cnt ? m[1] / (double)cnt : 0.0;
    set_float_params(c->s);
}

constexpr int kEx[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
constexpr int kEy[19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
constexpr int kEz[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};

double weight(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

lbm_status check_launch(lbm_ctx *c, const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->sticky = LBM_ERR_CUDA;
        return cuda_fail(c, e, where);
    }
    return LBM_OK;
}

lbm_status device_status(lbm_ctx *c)
{
    if (c->sticky != LBM_OK) return c->sticky;
    for (lbm_ctx *q : c->subs) {
        lbm_status st = device_status(q);
        if (st != LBM_OK) return fail(c, st, "a sample of the batch: " + q->err);
    }
    const int f = c->h_flag ? *(volatile int *)c->h_flag : 0;
    if (f & 1) return fail(c, LBM_ERR_NONFINITE, "non-finite density found by the periodic check");
    if (f & 2) return fail(c, LBM_ERR_DRIFT, "mass drift above drift_limit");
    if (f & 4) {
        c->pipe_reset = true;
        return fail(c, LBM_ERR_TIMEOUT, "a bounded device wait gave up (populations undefined: reinitialise)");
    }
    return LBM_OK;
}

// Host-side change of a lattice's parameters: a captured graph holds the old
// kernel arguments, and a batch holds a device copy of every sample's state.
void touch(lbm_ctx *c)
{
    c->graph_dirty = true;
    c->rec.valid = false;
    c->push_step = -1;
    c->flow_ok_step = -1;
    if (c->parent) {
        c->parent->states_dirty = true;
        c->parent->graph_dirty = true;
    }
}

// A batch has no lattice of its own: its samples are read and written through
// lbm_batch_get.
lbm_status no_batch(lbm_ctx *c, const char *what)
{
    return fail(c, LBM_ERR_ARG, std::string(what) + " takes a lattice; use lbm_batch_get for a sample of a batch");
}

void run_reduce(lbm_ctx *c)
{
    dispatch(c, [&](auto tag) {
        using TS = decltype(tag);
        Ops<TS>::dens(c->s, (int)(c->step & 1), c->step > 0, c->stream);
        Ops<TS>::wall(c->s, c->stream);
        Ops<TS>::reduce(c->s, c->d_partials, kReduceBlocks, c->d_red, c->stream);
    });
    c->launches += 3 + (c->s.n_wall > 0 ? 1 : 0);
}

lbm_status capture_initial_mass(lbm_ctx *c)
{
    run_reduce(c);
    double red[kReduceSlots];
    cudaError_t e = cudaMemcpyAsync(red, c->d_red, sizeof(red), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "initial mass");
    c->mass0[0] = red[0];
    c->mass0[1] = red[1];
    if (c->h_flag) *c->h_flag = 0;
    // a new state of a sample also clears its batch's record of an abandoned
    // persistent launch (the sample's batch starts over from here)
    if (c->parent && c->parent->h_flag) *c->parent->h_flag = 0;
    return LBM_OK;
}

bool acc_schedule(const lbm_ctx *c) { return c->kernel == LBM_KERNEL_PUSH || c->kernel == LBM_KERNEL_BRICK; }

// Accumulator k steps ahead of the current one.  The push schedule rotates
// two buffers (its finish pass clears the one the collide-stream pass has
// just read); the brick schedule three (each brick clears its own voxels of
// the buffer after next while others may still read the current one).
unsigned long long *acc_at(const lbm_ctx *c, int k)
{
    const int ring = c->kernel == LBM_KERNEL_PUSH ? 2 : 3;
    return c->acc[(c->step + k) % ring];
}

// Push and brick schedules: the accumulator of the current step from a
// density and wall pass (any state), and a cleared accumulator for the next
// step.  The brick schedule keeps fluid voxels only (it recomputes walls).
void push_prime_ctx(lbm_ctx *c)
{
    if (c->push_step == c->step) return;
    const int par = (int)(c->step & 1);
    dispatch(c, [&](auto tag) {
        using TS = decltype(tag);
        Ops<TS>::dens(c->s, par, c->step > 0, c->stream, c->block);
        Ops<TS>::wall(c->s, c->stream, c->block);
    });
    push_prime(c->s, acc_at(c, 0), c->stream, c->kernel != LBM_KERNEL_BRICK);
    cudaMemsetAsync(acc_at(c, 1), 0, (size_t)c->nv * 8, c->stream);
    c->launches += 3;
    c->push_step = c->step;
}

// Flow schedule: the densities of the current step in flow_psi[step & 1]
// (ordinary density and wall passes, with the pending open-plane rule after
// step 0), unless the last flow step left them there.
void flow_prime(lbm_ctx *c)
{
    c->s.psi = c->flow_psi[c->step & 1];
    if (c->flow_ok_step == c->step) return;
    dispatch(c, [&](auto tag) {
        using TS = decltype(tag);
        Ops<TS>::dens(c->s, (int)(c->step & 1), c->step > 0, c->stream, c->block);
        Ops<TS>::wall(c->s, c->stream, c->block);
    });
    c->launches += (c->s.n_fluid > 0 ? 1 : 0) + (c->s.n_wall > 0 ? 1 : 0);
    c->flow_ok_step = c->step;
}

// One time step of the split schedule.  ev != nullptr records events around
// the kernels for lbm_step_timed.
void enqueue_step(lbm_ctx *c, cudaEvent_t *ev)
{
    const int par = (int)(c->step & 1);
    cudaStream_t st = c->stream;
    if (c->kernel == LBM_KERNEL_PUSH) {
        push_prime_ctx(c);
        PushBufs pb;
        pb.rd = acc_at(c, 0);
        pb.acc = acc_at(c, 1);
        pb.clr = acc_at(c, 2);  // = rd: read by this collide-stream pass, cleared by its finish pass
        pb.nmask = c->d_nmask;
        if (ev) cudaEventRecord(ev[0], st);
        push_fused(c->s, pb, par, st);
        if (ev) cudaEventRecord(ev[1], st);
        // walls at least two planes from an open plane go with the plane nodes
        const int nz = c->s.nz;
        const int w_lo = c->plane_w[(size_t)std::min(2, nz)];
        const int w_hi = std::max(w_lo, c->plane_w[(size_t)std::max(0, nz - 2)]);
        const int nl = push_finish(c->s, pb.acc, pb.clr, 1 - par, w_lo, w_hi, st);
        if (ev) cudaEventRecord(ev[2], st);
        if (ev) cudaEventRecord(ev[3], st);
        c->launches += (c->s.n_fluid > 0 ? 1 : 0) + nl;
        c->step++;
        c->push_step = c->step;
        if (c->p.reduce_every > 0 && c->step % c->p.reduce_every == 0) {
            run_reduce(c);
            k_check<<<1, 1, 0, st>>>(c->d_red, c->mass0[0], c->mass0[1], c->p.drift_limit, c->s.open_z ? 0 : 1,
                                     c->d_flag);
            c->launches += 1;
        }
        return;
    }
    if (c->kernel == LBM_KERNEL_BRICK) {
        push_prime_ctx(c);
        BrickBufs bb = c->bb;
        bb.rd = acc_at(c, 0);
        bb.acc = acc_at(c, 1);
        bb.clr = acc_at(c, 2);
        dispatch(c, [&](auto tag) {
            using TS = decltype(tag);
            if constexpr (!std::is_same<TS, double>::value) {
                if (ev) cudaEventRecord(ev[0], st);
                brick_step<TS>(c->s, bb, c->n_bricks, par, st);
                if (ev) cudaEventRecord(ev[1], st);
                brick_plane<TS>(c->s, bb.acc, 1 - par, st);
                if (ev) cudaEventRecord(ev[2], st);
            }
        });
        c->launches += (c->n_bricks > 0 ? 1 : 0) + (c->s.open_z ? 1 : 0);
        c->step++;
        c->push_step = c->step;
        if (c->p.reduce_every > 0 && c->step % c->p.reduce_every == 0) {
            run_reduce(c);
            k_check<<<1, 1, 0, st>>>(c->d_red, c->mass0[0], c->mass0[1], c->p.drift_limit, c->s.open_z ? 0 : 1,
                                     c->d_flag);
            c->launches += 1;
        }
        return;
    }
    if (c->kernel == LBM_KERNEL_FLOW) {
        flow_prime(c);
        FlowState fs = c->fs;
        fs.psi_next = c->flow_psi[(c->step + 1) & 1];
        if (c->stall_next) fs.stall_slot = c->flow_stall_slot;
        c->stall_next = false;
        dispatch(c, [&](auto tag) {
            using TS = decltype(tag);
            if (ev) cudaEventRecord(ev[0], st);
            Ops<TS>::flow(c->s, fs, par, st);
            if (ev) cudaEventRecord(ev[1], st);
        });
        c->launches += fs.n_slots > 0 ? 1 : 0;
    } else if (c->kernel == LBM_KERNEL_FUSED) {
        PipeState &ps = c->ps;
        if (c->pipe_reset) {  // counters of an abandoned launch: start over
            cudaMemsetAsync(ps.round_f, 0, (size_t)ps.n_chunks * 8 * 16 * 8, st);
            cudaMemsetAsync(ps.round_d, 0, (size_t)ps.n_chunks * 8 * 16 * 8, st);
            cudaMemsetAsync(ps.abort, 0, 4, st);
            c->pipe_launches = 0;
            c->pipe_reset = false;
        }
        ps.epoch = (int)(c->pipe_launches + 1) + (c->stall_next ? (1 << 20) : 0);
        c->stall_next = false;
        ps.psi_next = c->psi_alt;
        dispatch(c, [&](auto tag) {
            using TS = decltype(tag);
            if (ev) cudaEventRecord(ev[0], st);
            Ops<TS>::pipe(c->s, ps, par, c->pipe_grid, st);
            if (ev) cudaEventRecord(ev[1], st);
        });
        void *t = c->s.psi;
        c->s.psi = c->psi_alt;
        c->psi_alt = t;
        c->pipe_launches++;
        c->launches += c->s.n_fluid > 0 ? 1 : 0;
    } else {
    dispatch(c, [&](auto tag) {
        using TS = decltype(tag);
        if (ev) cudaEventRecord(ev[0], st);
        Ops<TS>::dens(c->s, par, c->step > 0, st, c->block);
        if (ev) cudaEventRecord(ev[1], st);
        Ops<TS>::wall(c->s, st, c->block);
        if (ev) cudaEventRecord(ev[2], st);
        Ops<TS>::fused(c->s, par, st, c->block);
        if (ev) cudaEventRecord(ev[3], st);
        if (ev) cudaEventRecord(ev[4], st);
    });
    c->launches += 2 + (c->s.n_wall > 0 ? 1 : 0);
    }
    c->step++;
    if (c->kernel == LBM_KERNEL_FLOW) {
        c->s.psi = c->flow_psi[c->step & 1];
        c->flow_ok_step = c->step;
    }
    if (c->p.reduce_every > 0 && c->step % c->p.reduce_every == 0) {
        run_reduce(c);
        k_check<<<1, 1, 0, st>>>(c->d_red, c->mass0[0], c->mass0[1], c->p.drift_limit, c->s.open_z ? 0 : 1,
                                 c->d_flag);
        c->launches += 1;
    }
}

// Sample states and block maps of a batch.  map entry b = (sample, block
// within the sample) for the node passes and for the wall pass.
lbm_status upload_states(lbm_ctx *c);

lbm_status build_maps(lbm_ctx *c, int block)
{
    std::vector<int2> mn, mw;
    for (size_t k = 0; k < c->subs.size(); ++k) {
        const DevState &s = c->subs[k]->s;
        for (int j = 0; j < (s.n_fluid + block - 1) / block; ++j) mn.push_back(make_int2((int)k, j));
        for (int j = 0; j < (s.n_wall + block - 1) / block; ++j) mw.push_back(make_int2((int)k, j));
    }
    if (c->d_map_n) dfree(c, c->d_map_n);
    if (c->d_map_w) dfree(c, c->d_map_w);
    c->d_map_n = (int2 *)dalloc(c, std::max<size_t>(1, mn.size()) * sizeof(int2));
    c->d_map_w = (int2 *)dalloc(c, std::max<size_t>(1, mw.size()) * sizeof(int2));
    if (!c->d_map_n || !c->d_map_w) return fail(c, LBM_ERR_ALLOC, "batch block maps");
    cudaError_t e = cudaSuccess;
    if (!mn.empty()) e = cudaMemcpy(c->d_map_n, mn.data(), mn.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !mw.empty())
        e = cudaMemcpy(c->d_map_w, mw.data(), mw.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "batch block maps");
    c->n_map_n = (int)mn.size();
    c->n_map_w = (int)mw.size();
    c->map_block = block;
    c->graph_dirty = true;
    c->states_dirty = true;
    // the parameter-space table holds block offsets of this block size
    if (c->subs.size() <= (size_t)kParamStates) return upload_states(c);
    return LBM_OK;
}

lbm_status upload_states(lbm_ctx *c)
{
    if (c->subs.size() <= (size_t)kParamStates) {
        // the batch table travels with every launch (parameter space)
        if (!c->table) c->table = new BatchTable();
        BatchTable &t = *c->table;
        std::memset(&t, 0, sizeof(t));
        t.count = (int)c->subs.size();
        const int b = c->map_block;
        for (int k = 0; k < t.count; ++k) {
            const DevState &q = c->subs[(size_t)k]->s;
            t.s[k] = q;
            t.start_n[k + 1] = t.start_n[k] + (q.n_fluid + b - 1) / b;
            t.start_w[k + 1] = t.start_w[k] + (q.n_wall + b - 1) / b;
        }
        c->states_dirty = false;
        return LBM_OK;
    }
    std::vector<DevState> h(c->subs.size());
    for (size_t k = 0; k < c->subs.size(); ++k) h[k] = c->subs[k]->s;
    cudaError_t e = cudaMemcpyAsync(c->d_states, h.data(), h.size() * sizeof(DevState), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // h is released below
    if (e != cudaSuccess) return cuda_fail(c, e, "batch states");
    c->states_dirty = false;
    return LBM_OK;
}

// One step of a batch: the three split-schedule passes of every sample in
// three launches.
void enqueue_batch_step(lbm_ctx *c)
{
    lbm_ctx *s0 = c->subs[0];
    const int par = (int)(s0->step & 1);
    cudaStream_t st = c->stream;
    dispatch(c, [&](auto tag) {
        using TS = decltype(tag);
        if (c->table) {
            Ops<TS>::dens_table(*c->table, par, s0->step > 0, st, c->map_block);
            Ops<TS>::wall_table(*c->table, st, c->map_block);
            Ops<TS>::fused_table(*c->table, par, st, c->map_block);
        } else {
            Ops<TS>::dens_batch(c->d_states, c->d_map_n, c->n_map_n, par, s0->step > 0, st, c->map_block);
            Ops<TS>::wall_batch(c->d_states, c->d_map_w, c->n_map_w, st, c->map_block);
            Ops<TS>::fused_batch(c->d_states, c->d_map_n, c->n_map_n, par, st, c->map_block);
        }
    });
    c->launches += 3;
    for (lbm_ctx *q : c->subs) {
        q->step++;
        if (q->p.reduce_every > 0 && q->step % q->p.reduce_every == 0) {
            run_reduce(q);
            k_check<<<1, 1, 0, st>>>(q->d_red, q->mass0[0], q->mass0[1], q->p.drift_limit, q->s.open_z ? 0 : 1,
                                     q->d_flag);
            c->launches += q->launches;  // counted on the batch
            q->launches = 0;
            c->launches += 1;
        }
    }
    c->step++;
}

bool any_reduce(const lbm_ctx *c)
{
    if (c->p.reduce_every > 0) return true;
    for (const lbm_ctx *q : c->subs)
        if (q->p.reduce_every > 0) return true;
    return false;
}

int64_t cur_step(const lbm_ctx *c) { return c->subs.empty() ? c->step : c->subs[0]->step; }

void step_once(lbm_ctx *c)
{
    if (c->subs.empty())
        enqueue_step(c, nullptr);
    else
        enqueue_batch_step(c);
}

// Capture two steps (even parity, after the first step) into a CUDA graph on a
// private stream; the graph is then launched on the context's stream.
// Slab boundaries (z planes) for the wavefront schedule: contiguous groups of
// at least two planes with about equal fluid-node counts.  Fewer than three
// slabs: no wavefront (empty).
std::vector<int> plan_slabs(const lbm_ctx *c)
{
    const int nz = c->nz;
    const int64_t N = c->s.n_fluid;
    int K = std::max(1, (int)std::min<int64_t>(16, (N + 65535) / 65536));
    if (const char *e = std::getenv("LBM_WAVE_SLABS")) K = std::max(1, std::atoi(e));
    K = std::min(K, nz / 2);
    std::vector<int> z{0};
    if (K < 3) return {};
    for (int k = 1; k < K; ++k) {
        const int64_t target = N * k / K;
        int zz = z.back() + 2;
        while (zz < nz - 2 && c->plane_n[(size_t)zz] < target) ++zz;
        if (zz > nz - 2) break;
        z.push_back(zz);
    }
    z.push_back(nz);
    if ((int)z.size() - 1 < 3) return {};
    return z;
}

lbm_status capture_wave(lbm_ctx *c);

// Capture `steps` steps on the private stream into *out; the step counters
// and the launch count are put back afterwards (*launches: kernels per replay).
lbm_status capture_steps(lbm_ctx *c, int steps, cudaGraphExec_t *out, int64_t *launches)
{
    const cudaStream_t user = c->stream;
    const int64_t step0 = c->step, launches0 = c->launches;
    std::vector<int64_t> sub_steps;
    for (lbm_ctx *q : c->subs) sub_steps.push_back(q->step);
    c->stream = c->cap_stream;
    const int64_t push0 = c->push_step;
    const int64_t flow0 = c->flow_ok_step;
    void *psi0 = c->s.psi;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess)
        for (int q = 0; q < steps; ++q) step_once(c);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(c->cap_stream, &g) : e;
    c->stream = user;
    c->step = step0;
    c->push_step = push0;
    c->flow_ok_step = flow0;
    c->s.psi = psi0;
    for (size_t k = 0; k < c->subs.size(); ++k) c->subs[k]->step = sub_steps[k];
    *launches = c->launches - launches0;
    c->launches = launches0;
    if (e2 == cudaSuccess) e2 = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        *out = nullptr;
        return cuda_fail(c, e2, "graph capture");
    }
    return LBM_OK;
}

lbm_status ensure_graph(lbm_ctx *c)
{
    if (c->graph && !c->graph_dirty) return LBM_OK;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    if (c->graph_short) {
        cudaGraphExecDestroy(c->graph_short);
        c->graph_short = nullptr;
        c->graph_short_steps = 0;
    }
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "graph stream");
    if (c->kernel == LBM_KERNEL_WAVE && c->subs.empty()) {
        c->slab_z = plan_slabs(c);
        if (!c->slab_z.empty()) return capture_wave(c);
    }
    // long graph: 32 steps (30 for the accumulator schedules, whose buffers
    // rotate every three steps and parity every two); short graph: one period
    const int period = acc_schedule(c) ? 6 : 2;
    lbm_status st = capture_steps(c, acc_schedule(c) ? 30 : 32, &c->graph, &c->graph_launches);
    if (st != LBM_OK) return st;
    c->graph_steps = acc_schedule(c) ? 30 : 32;
    st = capture_steps(c, period, &c->graph_short, &c->graph_short_launches);
    if (st != LBM_OK) return st;
    c->graph_short_steps = period;
    c->graph_dirty = false;
    return LBM_OK;
}

// The wavefront graph: G steps of density / wall / collide-stream passes per
// slab, each launched on its own capture stream after the events of the
// passes it reads (one stream per pass kind and slab, so stream order adds no
// dependency that the data does not have).
lbm_status capture_wave(lbm_ctx *c)
{
    const int K = (int)c->slab_z.size() - 1;
    int G = 4;
    if (const char *e = std::getenv("LBM_WAVE_STEPS")) G = std::max(2, std::atoi(e) & ~1);
    // lag: density(t, k) also waits for collide-stream(t, k - L), which keeps
    // about L slabs in flight so that a slab's populations are still in L2
    // when its collide-stream pass reads them again (0: no such edge)
    int L = 3;
    if (const char *e = std::getenv("LBM_WAVE_LAG")) L = std::max(0, std::atoi(e));
    const bool per_z = c->per_z;
    auto nb = [&](int k, int d) {  // neighbour slab k + d, or -1
        int q = k + d;
        if (q < 0 || q >= K) {
            if (!per_z) return -1;
            q = (q + K) % K;
        }
        return q;
    };
    while ((int)c->wave_streams.size() < 3 * K) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "wave streams");
        c->wave_streams.push_back(st);
    }
    while ((int)c->wave_events.size() < 3 * K * G + 1) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "wave events");
        c->wave_events.push_back(ev);
    }
    auto EV = [&](int t, int kind, int k) { return c->wave_events[(size_t)1 + ((size_t)t * 3 + kind) * K + k]; };
    auto ST = [&](int kind, int k) { return c->wave_streams[(size_t)kind * K + k]; };
    const cudaStream_t cap = c->cap_stream;
    const int64_t launches0 = c->launches;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaEventRecord(c->wave_events[0], cap);
        for (int i = 0; i < 3 * K; ++i) cudaStreamWaitEvent(c->wave_streams[(size_t)i], c->wave_events[0], 0);
        for (int t = 0; t < G; ++t) {
            const int64_t step = c->step + t;
            const int par = (int)(step & 1);
            dispatch(c, [&](auto tag) {
                using TS = decltype(tag);
                auto dens = [&](int k) {
                    cudaStream_t st = ST(0, k);
                    if (t > 0)
                        for (int d = -1; d <= 1; ++d)
                            if (nb(k, d) >= 0) cudaStreamWaitEvent(st, EV(t - 1, 2, nb(k, d)), 0);
                    if (!per_z && L >= 3 && k >= L) cudaStreamWaitEvent(st, EV(t, 2, k - L), 0);
                    const int n0 = c->plane_n[(size_t)c->slab_z[(size_t)k]];
                    const int n1 = c->plane_n[(size_t)c->slab_z[(size_t)k + 1]];
                    Ops<TS>::dens(c->s, par, step > 0, st, c->block, n0, n1);
                    c->launches += n1 > n0;
                    cudaEventRecord(EV(t, 0, k), st);
                };
                auto wall = [&](int k) {
                    cudaStream_t st = ST(1, k);
                    for (int d = -1; d <= 1; ++d)
                        if (nb(k, d) >= 0) cudaStreamWaitEvent(st, EV(t, 0, nb(k, d)), 0);
                    const int w0 = c->plane_w[(size_t)c->slab_z[(size_t)k]];
                    const int w1 = c->plane_w[(size_t)c->slab_z[(size_t)k + 1]];
                    Ops<TS>::wall(c->s, st, c->block, w0, w1);
                    c->launches += w1 > w0;
                    cudaEventRecord(EV(t, 1, k), st);
                };
                auto fused = [&](int k) {
                    cudaStream_t st = ST(2, k);
                    for (int d = -1; d <= 1; ++d)
                        if (nb(k, d) >= 0) {
                            cudaStreamWaitEvent(st, EV(t, 0, nb(k, d)), 0);
                            cudaStreamWaitEvent(st, EV(t, 1, nb(k, d)), 0);
                        }
                    const int n0 = c->plane_n[(size_t)c->slab_z[(size_t)k]];
                    const int n1 = c->plane_n[(size_t)c->slab_z[(size_t)k + 1]];
                    Ops<TS>::fused(c->s, par, st, c->block, n0, n1);
                    c->launches += n1 > n0;
                    cudaEventRecord(EV(t, 2, k), st);
                };
                // emission order must be a topological order of the edges.
                // Open z: density k, wall k-1, collide-stream k-2 (wall k-1
                // needs densities up to k; collide-stream k-2 needs walls up to
                // k-1), so collide-stream k-L exists before density k for L >= 3.
                // Periodic z: the first and last slabs depend on each other;
                // all densities, then all walls, then all collide-streams.
                if (!per_z) {
                    for (int k = 0; k < K; ++k) {
                        dens(k);
                        if (k >= 1) wall(k - 1);
                        if (k >= 2) fused(k - 2);
                    }
                    wall(K - 1);
                    fused(K - 2);
                    fused(K - 1);
                } else {
                    for (int k = 0; k < K; ++k) dens(k);
                    for (int k = 0; k < K; ++k) wall(k);
                    for (int k = 0; k < K; ++k) fused(k);
                }
            });
        }
        // join every capture stream back into the origin stream
        for (int i = 0; i < 3 * K; ++i) {
            cudaEventRecord(EV(G - 1, i / K, i % K), c->wave_streams[(size_t)i]);
            cudaStreamWaitEvent(cap, EV(G - 1, i / K, i % K), 0);
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(cap, &g) : e;
    c->graph_launches = c->launches - launches0;
    c->launches = launches0;
    if (e2 == cudaSuccess) e2 = cudaGraphInstantiate(&c->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        c->graph = nullptr;
        cudaGetLastError();
        return cuda_fail(c, e2, "wave graph capture");
    }
    c->graph_steps = G;
    c->graph_dirty = false;
    return LBM_OK;
}

void free_record(lbm_ctx *c);

void destroy_ctx(lbm_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (lbm_ctx *q : c->subs) destroy_ctx(q);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph_short) cudaGraphExecDestroy(c->graph_short);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaStream_t st : c->wave_streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : c->wave_events) cudaEventDestroy(ev);
    free_record(c);
    if (c->rec.side) cudaStreamDestroy(c->rec.side);
    if (c->rec.graph) cudaGraphExecDestroy(c->rec.graph);
    for (cudaEvent_t ev : c->rec.ev)
        if (ev) cudaEventDestroy(ev);
    std::vector<std::pair<void *, size_t>> a = c->allocs;
    for (auto &q : a) dfree(c, q.first);
    if (c->h_flag) cudaFreeHost(c->h_flag);
    if (c->have_ev)
        for (auto &ev : c->ev) cudaEventDestroy(ev);
    delete c->table;
    delete c;
}

// ---- autotuner ------------------------------------------------------------
// Sweeps the threads per block of the split schedule's three passes over a
// few timed steps of the context's own lattice(s), keeps the fastest and
// caches it in a JSON object {"key": block, ...} keyed by GPU, storage type,
// batch size and node counts.
constexpr int kTuneBlocks[] = {64, 128, 256};
constexpr int kTuneWarm = 2, kTuneSteps = 8;

std::string tune_key(const lbm_ctx *c)
{
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, c->device);
    std::string name = prop.name;
    for (char &ch : name)
        if (ch == '"' || ch == '\\' || ch < 32) ch = '_';
    static const char *kStore[] = {"fp32", "fp64", "fp16dev", "bf16dev"};
    int64_t nf = c->s.n_fluid, nw = c->s.n_wall;
    for (const lbm_ctx *q : c->subs) {
        nf += q->s.n_fluid;
        nw += q->s.n_wall;
    }
    char buf[256];
    std::snprintf(buf, sizeof(buf), "|sm_%d%d|%s|samples=%d|fluid=%lld|walls=%lld", prop.major, prop.minor,
                  kStore[c->storage & 3], c->subs.empty() ? 1 : (int)c->subs.size(), (long long)nf, (long long)nw);
    return name + buf;
}

// Minimal reader of the cache: "string": integer pairs of one flat object.
std::vector<std::pair<std::string, int>> read_cache(const char *path)
{
    std::vector<std::pair<std::string, int>> kv;
    FILE *fp = path ? std::fopen(path, "rb") : nullptr;
    if (!fp) return kv;
    std::string txt;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), fp)) > 0) txt.append(buf, n);
    std::fclose(fp);
    size_t i = 0;
    while (true) {
        size_t a = txt.find('"', i);
        if (a == std::string::npos) break;
        size_t b = txt.find('"', a + 1);
        if (b == std::string::npos) break;
        size_t colon = txt.find(':', b);
        if (colon == std::string::npos) break;
        char *end = nullptr;
        long v = std::strtol(txt.c_str() + colon + 1, &end, 10);
        if (end == txt.c_str() + colon + 1) break;
        kv.push_back({txt.substr(a + 1, b - a - 1), (int)v});
        i = (size_t)(end - txt.c_str());
    }
    return kv;
}

bool write_cache(const char *path, const std::vector<std::pair<std::string, int>> &kv)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE *fp = std::fopen(tmp.c_str(), "wb");
    if (!fp) return false;
    std::fputs("{\n", fp);
    for (size_t k = 0; k < kv.size(); ++k)
        std::fprintf(fp, "  \"%s\": %d%s\n", kv[k].first.c_str(), kv[k].second, k + 1 < kv.size() ? "," : "");
    std::fputs("}\n", fp);
    const bool ok = std::fclose(fp) == 0;
    return ok && std::rename(tmp.c_str(), path) == 0;
}

lbm_status apply_block(lbm_ctx *c, int block)
{
    if (!c->subs.empty()) return build_maps(c, block);
    c->block = block;
    c->graph_dirty = true;
    return LBM_OK;
}

// Time kTuneSteps steps at each candidate, from a saved copy of the state
// that is put back afterwards (with the step counters and status words).
lbm_status tune(lbm_ctx *c, int *best)
{
    std::vector<lbm_ctx *> lat = c->subs.empty() ? std::vector<lbm_ctx *>{c} : c->subs;
    struct Saved {
        void *buf;
        int64_t step;
        int flag;
    };
    std::vector<Saved> saved;
    lbm_status st = LBM_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_autotune");
    for (lbm_ctx *q : lat) {
        const size_t tot = q->f_bytes + q->rest_bytes + q->bc_bytes;
        char *b = (char *)dalloc(q, tot);
        if (!b) {
            st = fail(c, LBM_ERR_ALLOC, "lbm_autotune: state copy");
            break;
        }
        saved.push_back({b, q->step, q->h_flag ? *q->h_flag : 0});
        e = cudaMemcpyAsync(b, q->s.f, q->f_bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b + q->f_bytes, q->s.rest, q->rest_bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess && q->bc_bytes)
            e = cudaMemcpyAsync(b + q->f_bytes + q->rest_bytes, q->s.bc, q->bc_bytes, cudaMemcpyDeviceToDevice,
                                c->stream);
        if (e != cudaSuccess) {
            st = cuda_fail(c, e, "lbm_autotune: state copy");
            break;
        }
    }
    const int64_t step0 = c->step;
    const int block0 = c->subs.empty() ? c->block : c->map_block;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    float best_ms = 0.f;
    *best = block0;
    if (st == LBM_OK && (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess))
        st = cuda_fail(c, cudaGetLastError(), "lbm_autotune: events");
    for (int cand : kTuneBlocks) {
        if (st != LBM_OK) break;
        st = apply_block(c, cand);
        if (st != LBM_OK) break;
        for (int k = 0; k < kTuneWarm; ++k) step_once(c);
        cudaEventRecord(ev[0], c->stream);
        for (int k = 0; k < kTuneSteps; ++k) step_once(c);
        cudaEventRecord(ev[1], c->stream);
        e = cudaEventSynchronize(ev[1]);
        if (e != cudaSuccess) {
            st = cuda_fail(c, e, "lbm_autotune: timed steps");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (best_ms == 0.f || ms < best_ms) {
            best_ms = ms;
            *best = cand;
        }
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    // put the state back
    for (size_t k = 0; k < saved.size(); ++k) {
        lbm_ctx *q = lat[k];
        char *b = (char *)saved[k].buf;
        cudaMemcpyAsync(q->s.f, b, q->f_bytes, cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(q->s.rest, b + q->f_bytes, q->rest_bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (q->bc_bytes)
            cudaMemcpyAsync(q->s.bc, b + q->f_bytes + q->rest_bytes, q->bc_bytes, cudaMemcpyDeviceToDevice,
                            c->stream);
    }
    e = cudaStreamSynchronize(c->stream);
    for (size_t k = 0; k < saved.size(); ++k) {
        lbm_ctx *q = lat[k];
        dfree(q, saved[k].buf);
        q->step = saved[k].step;
        q->push_step = -1;
        q->flow_ok_step = -1;
        if (q->h_flag) *q->h_flag = saved[k].flag;
    }
    c->step = step0;
    if (st == LBM_OK && e != cudaSuccess) st = cuda_fail(c, e, "lbm_autotune: restore");
    if (st != LBM_OK) apply_block(c, block0);
    return st;
}

// ---- recording and reverse pass ------------------------------------------
size_t state_bytes(const lbm_ctx *c) { return c->f_bytes + c->rest_bytes + c->bc_bytes; }

// Copy the live state (post-stream, with the pending open-plane extrapolation
// applied: it is idempotent) into buf.
void snap_save(lbm_ctx *c, void *buf)
{
    if (c->step > 0)
        dispatch(c, [&](auto tag) { Ops<decltype(tag)>::plane(c->s, (int)(c->step & 1), c->stream); });
    char *b = (char *)buf;
    cudaMemcpyAsync(b, c->s.f, c->f_bytes, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(b + c->f_bytes, c->s.rest, c->rest_bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (c->bc_bytes)
        cudaMemcpyAsync(b + c->f_bytes + c->rest_bytes, c->s.bc, c->bc_bytes, cudaMemcpyDeviceToDevice, c->stream);
}

// The lattice with its populations read from a saved state and psi in psi_buf.
DevState snap_state(const lbm_ctx *c, void *buf, void *psi_buf)
{
    DevState s = c->s;
    char *b = (char *)buf;
    s.f = b;
    s.rest = b + c->f_bytes;
    if (c->bc_bytes) s.bc = b + c->f_bytes + c->rest_bytes;
    s.psi = psi_buf;
    return s;
}

void free_record(lbm_ctx *c)
{
    auto &r = c->rec;
    for (void *q : r.ckpt) dfree(c, q);
    for (void *q : r.seg) dfree(c, q);
    for (void *q : r.psis) dfree(c, q);
    r.ckpt.clear();
    r.seg.clear();
    r.psis.clear();
    for (void **q : {&r.final_state, &r.lam[0], &r.lam[1], &r.rb[0], &r.rb[1], &r.abar, &r.wbar, &r.psi})
        if (*q) {
            dfree(c, *q);
            *q = nullptr;
        }
    for (void *q : r.seg2) dfree(c, q);
    r.seg2.clear();
    if (r.dens_all) dfree(c, r.dens_all);
    r.dens_all = nullptr;
    r.dens_all_bytes = 0;
    r.dens_stored = false;
    if (r.gxi) dfree(c, r.gxi);
    if (r.grin) dfree(c, r.grin);
    r.gxi = r.grin = nullptr;
    r.valid = false;
}

bool adjoint_supported(const lbm_ctx *c)
{
    return c->subs.empty() && !c->parent && c->kernel != LBM_KERNEL_FUSED &&
           (c->storage == LBM_STORE_FP32 || c->storage == LBM_STORE_FP64) && !(c->s.open_z && c->s.zou_he);
}

template <class Fn>
void dispatch_adj(const lbm_ctx *c, Fn &&fn)
{
    if (c->storage == LBM_STORE_FP64) fn(double{});
    else fn(float{});
}

// Slot plan of the flow schedule (see FlowState).  Dependency ranges are
// voxel windows turned into chunk ranges: the cells D(c) reads are written by
// F of its nodes' D3Q19 neighbours, which lie within `reach` voxels of the
// chunk's voxel range (a plane node also reads its interior node, one z plane
// further, and that node's cells); W(c) reads the densities of its walls'
// fluid neighbours.  With a periodic z axis, chunks that touch the first or
// last z plane depend on every chunk.  D(c) is placed lag_d slots after the
// last F it reads, W(c) lag_w slots after the last D it reads (at least one
// slot each, so every wait targets a lower slot), one item of each kind per
// slot in order of those positions.
struct FlowPlan {
    std::vector<int2> dep_f, dep_d, items;
    std::vector<int> wstart;
    int n_chunks = 0, n_slots = 0, stall_slot = -1;
};

FlowPlan build_flow_plan(const std::vector<uint32_t> &pvox, const std::vector<uint8_t> &nflags,
                         const std::vector<uint32_t> &wpvox, int nx, int ny, int nz, const int per[3], int chunk,
                         int lag_d, int lag_w)
{
    FlowPlan fp;
    const int64_t N = (int64_t)pvox.size(), NW = (int64_t)wpvox.size();
    const int64_t K = chunk, NC = (N + K - 1) / K;
    const int64_t nv = (int64_t)nx * ny * nz, sxy = (int64_t)nx * ny;
    fp.n_chunks = (int)NC;
    const int64_t rx = per[0] ? nx - 1 : 1, ry = per[1] ? (int64_t)(ny - 1) * nx : nx;
    const int64_t reach = sxy + std::max(rx, ry);
    // chunk of the first node at voxel >= v / of the last node at voxel <= v
    auto first_chunk = [&](int64_t v) {
        const int64_t n = std::lower_bound(pvox.begin(), pvox.end(), (uint32_t)std::max<int64_t>(0, v)) - pvox.begin();
        return (int)std::min(NC - 1, n / K);
    };
    auto last_chunk = [&](int64_t v) {
        if (v >= nv) return (int)(NC - 1);
        const int64_t n = std::upper_bound(pvox.begin(), pvox.end(), (uint32_t)v) - pvox.begin() - 1;
        return (int)std::max<int64_t>(0, n / K);
    };
    auto window = [&](int64_t vlo, int64_t vhi, int64_t r) {
        const bool wrap = per[2] && (vlo < sxy || vhi >= nv - sxy);
        if (wrap) return make_int2(0, (int)NC - 1);
        return make_int2(first_chunk(vlo - r), last_chunk(vhi + r));
    };
    fp.dep_f.resize((size_t)NC);
    for (int64_t c = 0; c < NC; ++c) {
        const int64_t n0 = c * K, n1 = std::min(N, n0 + K) - 1;
        bool plane = false;
        for (int64_t n = n0; n <= n1 && !plane; ++n) plane = (nflags[(size_t)n] & (F_INLET | F_OUTLET)) != 0;
        fp.dep_f[(size_t)c] = window(pvox[(size_t)n0], pvox[(size_t)n1], reach + (plane ? sxy : 0));
    }
    // wall chunk c: walls with voxel in [first voxel of chunk c, first voxel of chunk c + 1)
    fp.wstart.assign((size_t)NC + 1, 0);
    for (int64_t c = 1; c < NC; ++c)
        fp.wstart[(size_t)c] = (int)(std::lower_bound(wpvox.begin(), wpvox.end(), pvox[(size_t)(c * K)]) - wpvox.begin());
    fp.wstart[(size_t)NC] = (int)NW;
    fp.dep_d.resize((size_t)NC);
    for (int64_t c = 0; c < NC; ++c) {
        const int w0 = fp.wstart[(size_t)c], w1 = fp.wstart[(size_t)c + 1];
        fp.dep_d[(size_t)c] = w1 > w0 ? window(wpvox[(size_t)w0], wpvox[(size_t)w1 - 1], reach) : make_int2(0, -1);
    }
    // positions, then one item of each kind per slot in position order
    auto place = [](std::vector<std::pair<int64_t, int>> &pos, std::vector<int> &slot) {
        std::stable_sort(pos.begin(), pos.end());
        int64_t next = 0;
        for (auto &q : pos) {
            const int64_t k = std::max(q.first, next);
            slot[(size_t)q.second] = (int)k;
            next = k + 1;
        }
    };
    std::vector<int> slot_d((size_t)NC, -1), slot_w((size_t)NC, -1);
    std::vector<std::pair<int64_t, int>> pos;
    for (int64_t c = 0; c < NC; ++c) pos.push_back({std::max<int64_t>(c, fp.dep_f[(size_t)c].y) + lag_d, (int)c});
    place(pos, slot_d);
    bool mono = true;
    for (int64_t c = 1; c < NC; ++c) mono = mono && slot_d[(size_t)c] > slot_d[(size_t)c - 1];
    pos.clear();
    for (int64_t c = 0; c < NC; ++c) {
        const int2 r = fp.dep_d[(size_t)c];
        if (r.y < r.x) continue;
        int64_t m = 0;
        if (mono) {
            m = slot_d[(size_t)r.y];
        } else {
            for (int q = r.x; q <= r.y; ++q) m = std::max<int64_t>(m, slot_d[(size_t)q]);
        }
        pos.push_back({m + lag_w, (int)c});
    }
    place(pos, slot_w);
    int64_t n_slots = NC;
    for (int64_t c = 0; c < NC; ++c) n_slots = std::max<int64_t>(n_slots, std::max(slot_d[(size_t)c], slot_w[(size_t)c]) + 1);
    fp.n_slots = (int)n_slots;
    fp.items.assign((size_t)n_slots, make_int2(-1, -1));
    for (int64_t c = 0; c < NC; ++c) {
        fp.items[(size_t)slot_d[(size_t)c]].x = (int)c;
        if (slot_w[(size_t)c] >= 0) fp.items[(size_t)slot_w[(size_t)c]].y = (int)c;
    }
    fp.stall_slot = NC > 0 ? slot_d[0] : -1;
    return fp;
}

// Every wait of the plan targets items of lower slots (no block can wait for
// a block that has not started).
bool flow_plan_ordered(const FlowPlan &fp)
{
    std::vector<int> slot_d((size_t)fp.n_chunks, -1);
    for (int k = 0; k < fp.n_slots; ++k)
        if (fp.items[(size_t)k].x >= 0) slot_d[(size_t)fp.items[(size_t)k].x] = k;
    for (int k = 0; k < fp.n_slots; ++k) {
        const int2 it = fp.items[(size_t)k];
        if (it.x >= 0 && fp.dep_f[(size_t)it.x].y >= k) return false;
        if (it.y >= 0) {
            const int2 r = fp.dep_d[(size_t)it.y];
            for (int q = r.x; q <= r.y; ++q)
                if (slot_d[(size_t)q] < 0 || slot_d[(size_t)q] >= k) return false;
        }
    }
    for (int c = 0; c < fp.n_chunks; ++c)
        if (slot_d[(size_t)c] < 0) return false;
    return true;
}

template <typename C>
__global__ void k_set_wxi(const uint32_t *wpvox, int n_wall, const float *xi, C *wxi)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < n_wall) wxi[w] = (C)xi[wpvox[w]];
}

}  // namespace

extern "C" {

lbm_status lbm_default_params(lbm_params *p)
{
    if (!p) return LBM_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->tau[0] = p->tau[1] = 1.0;
    p->G = 3.5;
    p->xi = 0.0;
    p->rho_in1 = p->rho_out2 = 1.0;
    p->bc = LBM_BC_NEEM;
    p->storage = LBM_STORE_FP32;
    p->velocity_shift = 1;
    p->reduce_every = 0;
    p->kernel = LBM_KERNEL_AUTO;
    p->drift_limit = 1e-6;
    return LBM_OK;
}

lbm_status lbm_set_allocator(void *(*alloc)(size_t, void *), void (*free_fn)(void *, void *), void *user)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return LBM_ERR_ARG;
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_user = user;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_geometry *g, const lbm_params *p, lbm_ctx **out)
{
    NvtxRange nvtx_range("lbm_create");
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!g || !p || !g->solid) return fail(nullptr, LBM_ERR_ARG, "geometry, params and solid must be non-NULL");
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_ERR_ARG, "dimensions must be positive");
    const int64_t nv = (int64_t)nx * ny * nz;
    if (nv >= (int64_t)1 << 31) return fail(nullptr, LBM_ERR_ARG, "at most 2^31 - 1 voxels per domain");
    if (g->open_axis != -1 && g->open_axis != 2)
        return fail(nullptr, LBM_ERR_UNSUPPORTED, "open_axis must be -1 or 2 (z)");
    const bool open_z = g->open_axis == 2;
    if (open_z && (g->periodic[2] || nz < 3))
        return fail(nullptr, LBM_ERR_ARG, "the open axis must be non-periodic and at least 3 voxels long");
    if (p->storage < LBM_STORE_FP32 || p->storage > LBM_STORE_BF16DEV)
        return fail(nullptr, LBM_ERR_UNSUPPORTED, "unknown storage type");
    if (!(p->tau[0] > 0.5) || !(p->tau[1] > 0.5)) return fail(nullptr, LBM_ERR_ARG, "tau must exceed 1/2");
    if (p->bc != LBM_BC_NEEM && p->bc != LBM_BC_ZOU_HE) return fail(nullptr, LBM_ERR_UNSUPPORTED, "unknown open-plane rule");
    if (p->reduce_every < 0) return fail(nullptr, LBM_ERR_ARG, "reduce_every must be >= 0");
    if (p->kernel == LBM_KERNEL_PERSISTENT)
        return fail(nullptr, LBM_ERR_UNSUPPORTED, "the persistent launch steps batches (lbm_create_batch)");

    const int per[3] = {g->periodic[0] ? 1 : 0, g->periodic[1] ? 1 : 0, g->periodic[2] ? 1 : 0};
    const int dims[3] = {nx, ny, nz};
    const uint8_t *solid = g->solid;

    // compact fluid index in voxel order (x fastest): streaming partners of a
    // warp's nodes are then mostly contiguous too.  The brick schedule numbers
    // the nodes brick by brick instead (voxel order inside a brick).
    const bool brick = p->kernel == LBM_KERNEL_BRICK;
    const int nbx = (nx + kBrick - 1) / kBrick, nby = (ny + kBrick - 1) / kBrick, nbz = (nz + kBrick - 1) / kBrick;
    auto face_bits = [&](const int c[3]) {
        uint32_t f = 0;
        if (per[0] && c[0] == 0) f |= F_XLO;
        if (per[0] && c[0] == nx - 1) f |= F_XHI;
        if (per[1] && c[1] == 0) f |= F_YLO;
        if (per[1] && c[1] == ny - 1) f |= F_YHI;
        if (per[2] && c[2] == 0) f |= F_ZLO;
        if (per[2] && c[2] == nz - 1) f |= F_ZHI;
        return f;
    };
    // The split and wave schedules read the geometry only on the device:
    // it is built there from the uploaded mask (lbm_geom.cu).  The other
    // schedules also plan on the host and take the host path below (so does
    // every schedule with the environment variable LBM_HOST_PREP set).
    const bool dev_prep = !brick &&
                          (p->kernel == LBM_KERNEL_AUTO || p->kernel == LBM_KERNEL_SPLIT ||
                           p->kernel == LBM_KERNEL_WAVE) &&
                          std::getenv("LBM_HOST_PREP") == nullptr;
    std::vector<int32_t> cidx;
    std::vector<uint32_t> pvox;
    std::vector<uint8_t> nflags;
    std::vector<uint32_t> wpvox, wmask;
    std::vector<double> winv, wxi;
    std::vector<int> plane_n((size_t)nz + 1, 0), plane_w((size_t)nz + 1, 0);
    int64_t N = 0, NW = 0;
    bool closed_face = false, plane_solid = false;
    DevPrep dp;
    if (dev_prep) {
        // the geometry checks concern voxels on the faces of the box only and
        // are made here, before any device work (the device pass repeats
        // them): a fluid voxel on a face of a closed axis (neither periodic
        // nor the open axis) has a neighbour outside the domain; an
        // open-plane fluid voxel needs a fluid interior neighbour
        const int64_t sxy = (int64_t)nx * ny;
        auto fluid_on_face = [&](int a, int k) {
            for (int u = 0; u < (a == 0 ? ny : nx); ++u)
                for (int w = 0; w < (a == 2 ? ny : nz); ++w) {
                    const int64_t v = a == 0 ? k + (int64_t)nx * (u + (int64_t)ny * w)
                                    : a == 1 ? u + (int64_t)nx * (k + (int64_t)ny * w)
                                             : u + (int64_t)nx * (w + (int64_t)ny * k);
                    if (!solid[v]) return true;
                }
            return false;
        };
        for (int a = 0; a < 3 && !closed_face; ++a)
            if (!per[a] && !(open_z && a == 2))
                closed_face = fluid_on_face(a, 0) || fluid_on_face(a, dims[a] - 1);
        if (open_z)
            for (int64_t q = 0; q < sxy && !plane_solid; ++q)
                plane_solid = (!solid[q] && solid[q + sxy]) ||
                              (!solid[(nz - 1) * sxy + q] && solid[(nz - 2) * sxy + q]);
        if (closed_face)
            return fail(nullptr, LBM_ERR_ARG, "a fluid voxel touches a closed (non-periodic, non-open) face");
        if (plane_solid) return fail(nullptr, LBM_ERR_ARG, "an open-plane fluid voxel has a solid interior neighbour");
        lbm_status st = dev_prep_count(dp, g, nx, ny, nz, per, open_z, &N, &NW, plane_n, plane_w, &closed_face,
                                       &plane_solid);
        if (st != LBM_OK) return st;
        if (closed_face)
            return fail(nullptr, LBM_ERR_ARG, "a fluid voxel touches a closed (non-periodic, non-open) face");
        if (plane_solid) return fail(nullptr, LBM_ERR_ARG, "an open-plane fluid voxel has a solid interior neighbour");
    } else {
    // each fluid voxel: its index, its flag byte, and the geometry checks
    cidx.assign((size_t)nv, -1);
    auto add_node = [&](int x, int y, int z) {
        const int64_t v = x + (int64_t)nx * (y + (int64_t)ny * z);
        if (solid[v]) return;
        cidx[(size_t)v] = (int32_t)pvox.size();
        pvox.push_back((uint32_t)v);
        const int c[3] = {x, y, z};
        uint32_t f = face_bits(c);
        if (open_z && z == 0) f |= F_INLET;
        if (open_z && z == nz - 1) f |= F_OUTLET;
        nflags.push_back((uint8_t)f);
        // only a node on a face of the box can have a neighbour outside it
        const bool face = x == 0 || x == nx - 1 || y == 0 || y == ny - 1 || z == 0 || z == nz - 1;
        for (int j = 1; j < 19 && face; ++j) {
            const int e[3] = {kEx[j], kEy[j], kEz[j]};
            for (int a = 0; a < 3; ++a) {
                const int m = c[a] + e[a];
                if ((m < 0 || m >= dims[a]) && !per[a] && !(open_z && a == 2)) closed_face = true;
            }
        }
        if (open_z && (z == 0 || z == nz - 1) && solid[v + (z == 0 ? 1 : -1) * (int64_t)nx * ny]) plane_solid = true;
    };
    if (brick) {
        for (int bz = 0; bz < nbz; ++bz)
            for (int by = 0; by < nby; ++by)
                for (int bx = 0; bx < nbx; ++bx)
                    for (int z = bz * kBrick; z < std::min(nz, (bz + 1) * kBrick); ++z)
                        for (int y = by * kBrick; y < std::min(ny, (by + 1) * kBrick); ++y)
                            for (int x = bx * kBrick; x < std::min(nx, (bx + 1) * kBrick); ++x) add_node(x, y, z);
    } else {
        // voxel order, numbered plane by plane on host threads: the fluid
        // count of every z plane, then each plane's nodes at its prefix offset
        std::vector<int64_t> first((size_t)nz + 1, 0);
        std::vector<uint8_t> bad((size_t)nz, 0);  // bit 0 closed face, bit 1 solid behind a plane
        parallel_planes(nz, [&](int z) {
            const uint8_t *sp = solid + (int64_t)nx * ny * z;
            int64_t n = 0;
            for (int64_t q = 0; q < (int64_t)nx * ny; ++q) n += sp[q] ? 0 : 1;
            first[(size_t)z + 1] = n;
        });
        for (int z = 0; z < nz; ++z) first[(size_t)z + 1] += first[(size_t)z];
        pvox.resize((size_t)first[(size_t)nz]);
        nflags.resize((size_t)first[(size_t)nz]);
        parallel_planes(nz, [&](int z) {
            int64_t n = first[(size_t)z];
            uint8_t b = 0;
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const int64_t v = x + (int64_t)nx * (y + (int64_t)ny * z);
                    if (solid[v]) continue;
                    cidx[(size_t)v] = (int32_t)n;
                    pvox[(size_t)n] = (uint32_t)v;
                    const int c[3] = {x, y, z};
                    uint32_t f = face_bits(c);
                    if (open_z && z == 0) f |= F_INLET;
                    if (open_z && z == nz - 1) f |= F_OUTLET;
                    nflags[(size_t)n] = (uint8_t)f;
                    ++n;
                    const bool face = x == 0 || x == nx - 1 || y == 0 || y == ny - 1 || z == 0 || z == nz - 1;
                    for (int j = 1; j < 19 && face; ++j) {
                        const int e[3] = {kEx[j], kEy[j], kEz[j]};
                        for (int a = 0; a < 3; ++a) {
                            const int m = c[a] + e[a];
                            if ((m < 0 || m >= dims[a]) && !per[a] && !(open_z && a == 2)) b |= 1;
                        }
                    }
                    if (open_z && (z == 0 || z == nz - 1) && solid[v + (z == 0 ? 1 : -1) * (int64_t)nx * ny]) b |= 2;
                }
            bad[(size_t)z] = b;
        });
        for (int z = 0; z < nz; ++z) {
            closed_face = closed_face || (bad[(size_t)z] & 1);
            plane_solid = plane_solid || (bad[(size_t)z] & 2);
        }
    }
    if (closed_face)
        return fail(nullptr, LBM_ERR_ARG, "a fluid voxel touches a closed (non-periodic, non-open) face");
    if (plane_solid) return fail(nullptr, LBM_ERR_ARG, "an open-plane fluid voxel has a solid interior neighbour");
    N = (int64_t)pvox.size();

    // walls: solid voxels with at least one in-domain fluid neighbour (Eq. 15)
    // (voxels away from the box's faces find their neighbours at fixed
    // offsets; the others wrap or leave the domain), found plane by plane on
    // host threads and concatenated in voxel order
    int64_t noff[19];
    for (int j = 0; j < 19; ++j) noff[j] = kEx[j] + (int64_t)nx * (kEy[j] + (int64_t)ny * kEz[j]);
    struct PlaneWalls {
        std::vector<uint32_t> pv, mask;
        std::vector<double> inv;
    };
    std::vector<PlaneWalls> pw((size_t)nz);
    parallel_planes(nz, [&](int z) {
        PlaneWalls &out = pw[(size_t)z];
        for (int y = 0; y < ny; ++y) {
            const int64_t row = (int64_t)nx * (y + (int64_t)ny * z);
            const bool inner_yz = y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2;
            for (int x = 0; x < nx; ++x) {
                const int64_t v = row + x;
                if (!solid[v]) continue;
                const int c[3] = {x, y, z};
                uint32_t mask = 0;
                double den = 0;
                if (inner_yz && x >= 1 && x <= nx - 2) {
                    for (int j = 1; j < 19; ++j)
                        if (!solid[v + noff[j]]) {
                            mask |= 1u << j;
                            den += weight(j);
                        }
                } else {
                    for (int j = 1; j < 19; ++j) {
                        int m[3] = {c[0] + kEx[j], c[1] + kEy[j], c[2] + kEz[j]};
                        bool in = true;
                        for (int a = 0; a < 3; ++a) {
                            if (m[a] < 0 || m[a] >= dims[a]) {
                                if (!per[a]) in = false;
                                m[a] = (m[a] + dims[a]) % dims[a];
                            }
                        }
                        if (!in) continue;
                        const int64_t u = m[0] + (int64_t)nx * (m[1] + (int64_t)ny * m[2]);
                        if (!solid[u]) {
                            mask |= 1u << j;
                            den += weight(j);
                        }
                    }
                }
                if (!mask) continue;
                out.pv.push_back((uint32_t)v);
                out.mask.push_back(mask | (face_bits(c) << kWallFaceShift));
                out.inv.push_back(1.0 / den);
            }
        }
    });
    {
        size_t tot = 0;
        for (const PlaneWalls &q : pw) tot += q.pv.size();
        wpvox.reserve(tot);
        wmask.reserve(tot);
        winv.reserve(tot);
        wxi.reserve(tot);
        for (const PlaneWalls &q : pw) {
            wpvox.insert(wpvox.end(), q.pv.begin(), q.pv.end());
            wmask.insert(wmask.end(), q.mask.begin(), q.mask.end());
            winv.insert(winv.end(), q.inv.begin(), q.inv.end());
            for (uint32_t v : q.pv) wxi.push_back(g->xi_field ? (double)g->xi_field[v] : p->xi);
        }
    }
    NW = (int64_t)wpvox.size();
    // first node / wall of every z plane (both lists are in voxel order)
    for (int z = 0; z <= nz; ++z) {
        const uint32_t v0 = (uint32_t)std::min<int64_t>((int64_t)z * nx * ny, UINT32_MAX);
        plane_n[(size_t)z] = (int)(std::lower_bound(pvox.begin(), pvox.end(), v0) - pvox.begin());
        plane_w[(size_t)z] = (int)(std::lower_bound(wpvox.begin(), wpvox.end(), v0) - wpvox.begin());
    }
    }  // host path
    // brick tables: per brick with fluid nodes its node range and the wall
    // voxels of the brick and its one-voxel halo (one entry per halo-region
    // cell, so a wall seen twice through a short periodic axis has two)
    std::vector<BrickInfo> binfo;
    std::vector<uint16_t> nloc;
    std::vector<uint32_t> wcell;
    std::vector<int32_t> bwid;
    std::vector<float> wcoef;
    if (brick) {
        std::vector<int32_t> wid_of((size_t)nv, -1);
        for (int64_t w = 0; w < NW; ++w) wid_of[(size_t)wpvox[(size_t)w]] = (int32_t)w;
        nloc.assign((size_t)N, 0);
        int64_t n = 0;
        for (int bz = 0; bz < nbz; ++bz)
            for (int by = 0; by < nby; ++by)
                for (int bx = 0; bx < nbx; ++bx) {
                    BrickInfo b{};
                    b.x0 = bx * kBrick;
                    b.y0 = by * kBrick;
                    b.z0 = bz * kBrick;
                    const int ex = std::min(kBrick, nx - b.x0), ey = std::min(kBrick, ny - b.y0),
                              ez = std::min(kBrick, nz - b.z0);
                    b.ext = ex | (ey << 8) | (ez << 16);
                    b.n0 = (int)n;
                    for (int lz = 0; lz < ez; ++lz)
                        for (int ly = 0; ly < ey; ++ly)
                            for (int lx = 0; lx < ex; ++lx)
                                if (!solid[(b.x0 + lx) + (int64_t)nx * ((b.y0 + ly) + (int64_t)ny * (b.z0 + lz))])
                                    nloc[(size_t)n++] = (uint16_t)(lx + kBrick * ly + kBrick * kBrick * lz);
                    b.n1 = (int)n;
                    if (b.n1 == b.n0) continue;
                    b.w0 = (int)wcell.size();
                    for (int lz = -1; lz <= ez; ++lz)
                        for (int ly = -1; ly <= ey; ++ly)
                            for (int lx = -1; lx <= ex; ++lx) {
                                int g[3] = {b.x0 + lx, b.y0 + ly, b.z0 + lz};
                                bool in = true;
                                for (int a = 0; a < 3; ++a)
                                    if (g[a] < 0 || g[a] >= dims[a]) {
                                        if (!per[a]) in = false;
                                        g[a] = ((g[a] % dims[a]) + dims[a]) % dims[a];
                                    }
                                if (!in) continue;
                                const int32_t w = wid_of[(size_t)(g[0] + (int64_t)nx * (g[1] + (int64_t)ny * g[2]))];
                                if (w < 0) continue;
                                const uint32_t cell = (uint32_t)((lz + 1) * kR1 * kR1 + (ly + 1) * kR1 + (lx + 1));
                                wcell.push_back((wmask[(size_t)w] & 0x7fffeu) | (cell << 20));
                                bwid.push_back(w);
                                const float inv = (float)winv[(size_t)w], xi = (float)wxi[(size_t)w];
                                wcoef.push_back((1.f + xi) * inv);
                                wcoef.push_back((1.f - xi) * inv);
                            }
                    b.w1 = (int)wcell.size();
                    binfo.push_back(b);
                }
    }
    if (18 * (((N + 63) / 64) * 64 + 64) >= ((int64_t)1 << 31))
        return fail(nullptr, LBM_ERR_UNSUPPORTED, "more than 113 million fluid nodes in one context");

    lbm_ctx *c = new lbm_ctx();
    cudaGetDevice(&c->device);
    c->alloc_fn = g_alloc;
    c->free_fn = g_free;
    c->alloc_user = g_alloc_user;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->nv = nv;
    for (int a = 0; a < 3; ++a) c->periodic[a] = per[a];
    c->open_axis = g->open_axis;
    c->p = *p;
    c->storage = p->storage;
    c->kernel = p->kernel == LBM_KERNEL_FUSED ? LBM_KERNEL_FUSED
                : p->kernel == LBM_KERNEL_WAVE    ? LBM_KERNEL_WAVE
                : p->kernel == LBM_KERNEL_PUSH    ? LBM_KERNEL_PUSH
                : p->kernel == LBM_KERNEL_BRICK   ? LBM_KERNEL_BRICK
                : p->kernel == LBM_KERNEL_FLOW    ? LBM_KERNEL_FLOW
                                                  : LBM_KERNEL_SPLIT;  // AUTO and SPLIT
    if (c->kernel == LBM_KERNEL_FLOW && N == 0) c->kernel = LBM_KERNEL_SPLIT;
    if (c->kernel == LBM_KERNEL_PUSH && c->storage != LBM_STORE_FP32) {
        delete c;
        return fail(nullptr, LBM_ERR_UNSUPPORTED, "the push schedule needs FP32 storage");
    }
    if (c->kernel == LBM_KERNEL_BRICK && c->storage == LBM_STORE_FP64) {
        delete c;
        return fail(nullptr, LBM_ERR_UNSUPPORTED, "the brick schedule needs FP32, FP16 or BF16 storage");
    }

    const size_t sz = p->storage == LBM_STORE_FP64 ? 8 : (is16(p->storage) ? 2 : 4);  // stored element bytes
    const size_t szc = p->storage == LBM_STORE_FP64 ? 8 : 4;                            // compute-type bytes
    const int64_t npad = ((N + 63) / 64) * 64 + 64;
    const int nxy = nx * ny;
    DevState &s = c->s;
    s.npad = npad;
    s.n_fluid = (int32_t)N;
    s.nx = nx;
    s.ny = ny;
    s.nz = nz;
    s.sx = nx;
    s.sxy = nxy;
    s.nv = nv;
    s.n_wall = (int32_t)NW;
    s.open_z = open_z ? 1 : 0;
    s.zou_he = p->bc == LBM_BC_ZOU_HE ? 1 : 0;
    s.nxy = nxy;
    s.sample_lo = g->sample_lo;
    s.sample_hi = g->sample_hi;
    s.tau1 = p->tau[0];
    s.tau2 = p->tau[1];
    s.G = p->G;
    s.gx = p->body_force[0];
    s.gy = p->body_force[1];
    s.gz = p->body_force[2];
    s.rho_in1 = p->rho_in1;
    s.rho_out2 = p->rho_out2;
    s.rref1 = p->rho_ref[0];
    s.rref2 = p->rho_ref[1];
    set_float_params(s);
    c->solid_host.assign(solid, solid + nv);
    c->per_z = per[2] != 0;
    c->plane_n = std::move(plane_n);
    c->plane_w = std::move(plane_w);
    s.velocity_shift = p->velocity_shift ? 1 : 0;

    bool ok = true;
    auto A = [&](size_t bytes) {
        void *q = dalloc(c, bytes);
        if (!q) ok = false;
        return q;
    };
    s.f = A((size_t)18 * npad * 2 * sz);    // moving pairs M[18][npad]
    s.rest = A((size_t)npad * 2 * szc);      // rest pairs R[npad]
    void *d_pvox = A((size_t)N * 4);
    void *d_nflags = A((size_t)N);
    void *d_cidx = A((size_t)nv * 4);
    s.psi = A((size_t)nv * 2 * szc);
    void *d_wpvox = A((size_t)NW * 4);
    void *d_wmask = A((size_t)NW * 4);
    void *d_winv = A((size_t)NW * szc);
    void *d_wxi = A((size_t)NW * szc);
    c->f_bytes = (size_t)18 * npad * 2 * sz;
    c->rest_bytes = (size_t)npad * 2 * szc;
    c->bc_bytes = open_z ? (size_t)2 * 2 * 5 * nxy * sz : 0;
    if (open_z) {
        s.bc = A((size_t)2 * 2 * 5 * nxy * sz);
        c->d_frozen = (double *)A((size_t)2 * 5 * nxy * 8);
    }
    c->d_partials = (double *)A((size_t)kReduceBlocks * kReduceSlots * 8);
    c->d_red = (double *)A((size_t)kReduceSlots * 8);
    std::vector<uint32_t> nmask;
    if (brick) {
        for (int q = 0; q < 3; ++q) c->acc[q] = (unsigned long long *)A((size_t)nv * 8);
        c->n_bricks = (int)binfo.size();
        c->n_bentries = (int)wcell.size();
        c->bb.info = (const BrickInfo *)A(std::max<size_t>(1, binfo.size()) * sizeof(BrickInfo));
        c->bb.nloc = (const uint16_t *)A(std::max<size_t>(1, nloc.size()) * 2);
        c->bb.wcell = (const uint32_t *)A(std::max<size_t>(1, wcell.size()) * 4);
        c->bb.wcoef = (const float2 *)A(std::max<size_t>(1, wcell.size()) * 8);
        c->d_bwid = (int32_t *)A(std::max<size_t>(1, bwid.size()) * 4);
        c->bb.per = per[0] | (per[1] << 1) | (per[2] << 2);
    }
    if (c->kernel == LBM_KERNEL_PUSH) {
        for (int q = 0; q < 2; ++q) c->acc[q] = (unsigned long long *)A((size_t)nv * 8);
        c->d_nmask = (uint32_t *)A((size_t)N * 4);
        nmask.assign((size_t)N, 0u);
        for (int64_t n = 0; n < N; ++n) {
            const int64_t v = pvox[(size_t)n];
            const int cc[3] = {(int)(v % nx), (int)((v / nx) % ny), (int)(v / ((int64_t)nx * ny))};
            for (int j = 1; j < 19; ++j) {
                int m[3] = {cc[0] + kEx[j], cc[1] + kEy[j], cc[2] + kEz[j]};
                bool in = true;
                for (int a = 0; a < 3; ++a)
                    if (m[a] < 0 || m[a] >= dims[a]) {
                        if (!per[a]) in = false;
                        m[a] = (m[a] + dims[a]) % dims[a];
                    }
                if (in && !solid[m[0] + (int64_t)nx * (m[1] + (int64_t)ny * m[2])]) nmask[(size_t)n] |= 1u << j;
            }
        }
    }

    // Single-pass schedule: chunk dependencies.  D of chunk c reads the
    // post-stream populations of its nodes, written by F of their fluid
    // neighbours; at an open plane it also reads the interior node's, written
    // by F of that node's neighbours.  W of wall chunk c (the walls whose voxel
    // lies between the first voxels of fluid chunks c and c+1) reads D of the
    // chunks of its fluid neighbours.
    std::vector<int2> dep_f, dep_d;
    std::vector<int> wst;
    if (c->kernel == LBM_KERNEL_FUSED && N > 0) {
        const int64_t NC = (N + kChunk - 1) / kChunk;
        dep_f.assign((size_t)NC, make_int2(0, -1));
        dep_d.assign((size_t)NC, make_int2(0, -1));
        wst.assign((size_t)NC + 1, 0);
        auto nb_voxel = [&](int64_t v, int j, int64_t *out) {
            int m[3] = {(int)(v % nx) + kEx[j], (int)((v / nx) % ny) + kEy[j], (int)(v / ((int64_t)nx * ny)) + kEz[j]};
            for (int a = 0; a < 3; ++a) {
                if (m[a] < 0 || m[a] >= dims[a]) {
                    if (!per[a]) return false;
                    m[a] = (m[a] + dims[a]) % dims[a];
                }
            }
            *out = m[0] + (int64_t)nx * (m[1] + (int64_t)ny * m[2]);
            return true;
        };
        auto widen = [&](int2 &r, int ch) {
            if (r.y < r.x) r = make_int2(ch, ch);
            r.x = std::min(r.x, ch);
            r.y = std::max(r.y, ch);
        };
        auto add_writers = [&](int2 &r, int64_t v) {  // F chunks writing the post-stream cells of voxel v
            widen(r, cidx[(size_t)v] / kChunk);
            for (int j = 1; j < 19; ++j) {
                int64_t u;
                if (nb_voxel(v, j, &u) && cidx[(size_t)u] >= 0) widen(r, cidx[(size_t)u] / kChunk);
            }
        };
        for (int64_t n = 0; n < N; ++n) {
            int2 &r = dep_f[(size_t)(n / kChunk)];
            const int64_t v = pvox[(size_t)n];
            add_writers(r, v);
            if (nflags[(size_t)n] & (F_INLET | F_OUTLET))
                add_writers(r, v + ((nflags[(size_t)n] & F_INLET) ? 1 : -1) * (int64_t)nx * ny);
        }
        size_t w = 0;
        for (int64_t ch = 0; ch < NC; ++ch) {
            const int64_t v_hi = ch + 1 < NC ? (int64_t)pvox[(size_t)((ch + 1) * kChunk)] : nv;
            wst[(size_t)ch] = (int)w;
            for (; w < wpvox.size() && (int64_t)wpvox[w] < v_hi; ++w) {
                for (int j = 1; j < 19; ++j) {
                    int64_t u;
                    if ((wmask[w] & (1u << j)) && nb_voxel(wpvox[w], j, &u)) widen(dep_d[(size_t)ch], cidx[(size_t)u] / kChunk);
                }
            }
        }
        wst[(size_t)NC] = (int)wpvox.size();
        PipeState &ps = c->ps;
        ps.n_chunks = (int)NC;
        ps.need_f = (const int *)A((size_t)NC * 4);
        ps.need_d = (const int *)A((size_t)NC * 4);
        ps.wstart = (const int *)A((size_t)(NC + 1) * 4);
        // round counters: at most NC rounds (grid >= 1), 128 bytes apart
        ps.round_f = (unsigned long long *)A((size_t)NC * 8 * 16 * 8);
        ps.round_d = (unsigned long long *)A((size_t)NC * 8 * 16 * 8);
        ps.abort = (int *)A(4);
        ps.wait_ns = 1000000000ull;  // one second
        c->psi_alt = A((size_t)nv * 2 * szc);
    }
    // Flow schedule: the slot plan and its counters, and the second density
    // buffer.  LBM_FLOW_LAG_D / LBM_FLOW_LAG_W (slots, >= 1) override the
    // lags, LBM_FLOW_CHUNK the nodes per chunk (rounded to kFlowThreads).
    FlowPlan flow;
    if (c->kernel == LBM_KERNEL_FLOW) {
        int lag_d = 8, lag_w = 8, chunk = 4 * kFlowThreads;
        if (const char *ev = std::getenv("LBM_FLOW_LAG_D")) lag_d = std::max(1, std::atoi(ev));
        if (const char *ev = std::getenv("LBM_FLOW_LAG_W")) lag_w = std::max(1, std::atoi(ev));
        if (const char *ev = std::getenv("LBM_FLOW_CHUNK"))
            chunk = std::max(1, std::min(64, std::atoi(ev) / kFlowThreads)) * kFlowThreads;
        c->flow_lag[0] = lag_d;
        c->flow_lag[1] = lag_w;
        flow = build_flow_plan(pvox, nflags, wpvox, nx, ny, nz, per, chunk, lag_d, lag_w);
        c->fs.chunk = chunk;
        if (!flow_plan_ordered(flow)) {
            lbm_destroy(c);
            return fail(nullptr, LBM_ERR_ARG, "internal: flow plan has a wait on a later slot");
        }
        FlowState &fs = c->fs;
        const size_t NC = (size_t)flow.n_chunks;
        fs.ticket = (unsigned long long *)A(8);
        fs.fdone = (int *)A(NC * 4);
        fs.ddone = (int *)A(NC * 4);
        fs.abort = (int *)A(4);
        fs.dep_f = (const int2 *)A(NC * 8);
        fs.dep_d = (const int2 *)A(NC * 8);
        fs.wstart = (const int *)A((NC + 1) * 4);
        fs.items = (const int2 *)A((size_t)flow.n_slots * 8);
        fs.n_chunks = flow.n_chunks;
        fs.n_slots = flow.n_slots;
        fs.stall_slot = -1;
        fs.wait_ns = 1000000000ull;  // one second
        c->flow_stall_slot = flow.stall_slot;
        c->flow_psi[0] = s.psi;
        c->flow_psi[1] = A((size_t)nv * 2 * szc);
    }
    if (!ok) {
        lbm_destroy(c);
        return fail(nullptr, LBM_ERR_ALLOC, "device allocation failed");
    }
    s.pvox = (const uint32_t *)d_pvox;
    s.nflags = (const uint8_t *)d_nflags;
    s.cidx = (const int32_t *)d_cidx;
    s.wpvox = (const uint32_t *)d_wpvox;
    s.wmask = (const uint32_t *)d_wmask;
    s.winv = d_winv;
    s.wxi = d_wxi;
    s.frozen = c->d_frozen;

    std::vector<float> winv32, wxi32;
    const void *winv_h = winv.data(), *wxi_h = wxi.data();
    if (szc == 4) {
        winv32.assign(winv.begin(), winv.end());
        wxi32.assign(wxi.begin(), wxi.end());
        winv_h = winv32.data();
        wxi_h = wxi32.data();
    }
    cudaError_t e = cudaSuccess;
    auto H2D = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    if (dev_prep) {
        geom_fill(dp.plan, dp.xi, p->xi, dp.off, (int32_t *)d_cidx, (uint32_t *)d_pvox, (uint8_t *)d_nflags,
                  (uint32_t *)d_wpvox, (uint32_t *)d_wmask, d_winv, d_wxi, szc == 8, 0);
        e = cudaGetLastError();
    } else {
        H2D(d_pvox, pvox.data(), (size_t)N * 4);
        H2D(d_nflags, nflags.data(), (size_t)N);
        H2D(d_cidx, cidx.data(), (size_t)nv * 4);
    }
    if (c->d_nmask) H2D(c->d_nmask, nmask.data(), (size_t)N * 4);
    if (brick) {
        H2D((void *)c->bb.info, binfo.data(), binfo.size() * sizeof(BrickInfo));
        H2D((void *)c->bb.nloc, nloc.data(), nloc.size() * 2);
        H2D((void *)c->bb.wcell, wcell.data(), wcell.size() * 4);
        H2D((void *)c->bb.wcoef, wcoef.data(), wcoef.size() * 4);
        H2D(c->d_bwid, bwid.data(), bwid.size() * 4);
        for (int q = 0; q < 3; ++q)
            if (e == cudaSuccess) e = cudaMemset(c->acc[q], 0, (size_t)nv * 8);
    }
    if (!dev_prep) {
        H2D(d_wpvox, wpvox.data(), (size_t)NW * 4);
        H2D(d_wmask, wmask.data(), (size_t)NW * 4);
        H2D(d_winv, winv_h, (size_t)NW * szc);
        H2D(d_wxi, wxi_h, (size_t)NW * szc);
    }
    if (e == cudaSuccess) e = cudaMemset(s.f, 0, (size_t)18 * npad * 2 * sz);
    if (e == cudaSuccess) e = cudaMemset(s.rest, 0, (size_t)npad * 2 * szc);
    if (e == cudaSuccess) e = cudaMemset(s.psi, 0, (size_t)nv * 2 * szc);
    if (e == cudaSuccess && open_z) e = cudaMemset(s.bc, 0, (size_t)2 * 2 * 5 * nxy * sz);
    if (e == cudaSuccess && open_z) e = cudaMemset(c->d_frozen, 0, (size_t)2 * 5 * nxy * 8);
    if (e == cudaSuccess && c->ps.n_chunks > 0) {
        PipeState &ps = c->ps;
        const int64_t NC = ps.n_chunks;
        e = cudaMemset(ps.round_f, 0, (size_t)NC * 8 * 16 * 8);
        if (e == cudaSuccess) e = cudaMemset(ps.round_d, 0, (size_t)NC * 8 * 16 * 8);
        if (e == cudaSuccess) e = cudaMemset(ps.abort, 0, 4);
        if (e == cudaSuccess) e = cudaMemset(c->psi_alt, 0, (size_t)nv * 2 * szc);
        std::vector<int> nf((size_t)NC), nd((size_t)NC);
        for (int64_t ch = 0; ch < NC; ++ch) {
            nf[(size_t)ch] = dep_f[(size_t)ch].y;
            nd[(size_t)ch] = dep_d[(size_t)ch].y >= dep_d[(size_t)ch].x ? dep_d[(size_t)ch].y : -1;
        }
        H2D((void *)ps.need_f, nf.data(), (size_t)NC * 4);
        H2D((void *)ps.need_d, nd.data(), (size_t)NC * 4);
        H2D((void *)ps.wstart, wst.data(), (size_t)(NC + 1) * 4);
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        int per_sm = 0;
        dispatch(c, [&](auto tag) { per_sm = Ops<decltype(tag)>::pipe_blocks_per_sm(); });
        // every block must be resident (cooperative launch); lags in rounds
        // cover the dependency reach so that waits target earlier rounds
        c->pipe_grid = std::max(1, std::min(ps.n_chunks, std::max(1, per_sm) * std::max(1, sms)));
        const int G = c->pipe_grid;
        int reach_f = 0, reach_d = 0;
        for (int64_t ch = 0; ch < NC; ++ch) {
            reach_f = std::max(reach_f, nf[(size_t)ch] - (int)ch);
            if (nd[(size_t)ch] >= 0) reach_d = std::max(reach_d, nd[(size_t)ch] - (int)ch);
        }
        int lag = 1 + (reach_f + G - 1) / G;
        if (const char *ev = std::getenv("LBM_PIPE_LAG")) lag = std::max(1, std::atoi(ev));
        ps.lag_d = lag;
        ps.lag_w = ps.lag_d + 1 + (reach_d + G - 1) / G;
        ps.n_rounds = (ps.n_chunks + G - 1) / G;
        ps.rounds = ps.n_rounds + ps.lag_w;
    }
    if (e == cudaSuccess && c->kernel == LBM_KERNEL_FLOW) {
        FlowState &fs = c->fs;
        const size_t NC = (size_t)flow.n_chunks;
        e = cudaMemset(fs.ticket, 0, 8);
        if (e == cudaSuccess) e = cudaMemset(fs.fdone, 0, NC * 4);
        if (e == cudaSuccess) e = cudaMemset(fs.ddone, 0, NC * 4);
        if (e == cudaSuccess) e = cudaMemset(fs.abort, 0, 4);
        if (e == cudaSuccess) e = cudaMemset(c->flow_psi[1], 0, (size_t)nv * 2 * szc);
        H2D((void *)fs.dep_f, flow.dep_f.data(), NC * 8);
        H2D((void *)fs.dep_d, flow.dep_d.data(), NC * 8);
        H2D((void *)fs.wstart, flow.wstart.data(), (NC + 1) * 4);
        H2D((void *)fs.items, flow.items.data(), (size_t)flow.n_slots * 8);
    }
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c->h_flag, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *c->h_flag = 0;
        e = cudaHostGetDevicePointer((void **)&c->d_flag, c->h_flag, 0);
        c->ps.status = c->d_flag;
        c->fs.status = c->d_flag;
    }
    if (e != cudaSuccess) {
        lbm_destroy(c);
        return fail(nullptr, LBM_ERR_CUDA, std::string("lbm_create: ") + cudaGetErrorString(e));
    }
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *c)
{
    if (!c || c->parent) return;  // sample contexts belong to their batch
    destroy_ctx(c);
}

lbm_status lbm_init_densities(lbm_ctx *c, const double *rho1, const double *rho2)
{
    if (!c || !rho1 || !rho2) return LBM_ERR_ARG;
    if (!c->subs.empty()) return no_batch(c, "lbm_init_densities");
    choose_rho_ref(c, rho1, rho2, 0);
    touch(c);
    const size_t bytes = (size_t)c->nv * 8;
    double *d = (double *)talloc(c, 2 * bytes);
    if (!d) return fail(c, LBM_ERR_ALLOC, "temporary density buffer");
    cudaError_t e = cudaMemcpyAsync(d, rho1, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + c->nv, rho2, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(c->stream);
        tfree(c, d);
        return cuda_fail(c, e, "lbm_init_densities");
    }
    dispatch(c, [&](auto tag) {
        using TS = decltype(tag);
        Ops<TS>::init_eq(c->s, d, c->stream);
        Ops<TS>::capture_frozen(c->s, c->d_frozen, c->stream);
    });
    c->launches += 2;
    c->step = 0;
    lbm_status st = check_launch(c, "lbm_init_densities");
    tfree(c, d);
    if (st != LBM_OK) return st;
    return capture_initial_mass(c);
}

lbm_status lbm_set_populations(lbm_ctx *c, const double *f)
{
    if (!c || !f) return LBM_ERR_ARG;
    if (!c->subs.empty()) return no_batch(c, "lbm_set_populations");
    choose_rho_ref(c, f, f + 19 * c->nv, c->nv);
    touch(c);
    const size_t bytes = (size_t)38 * c->nv * 8;
    double *d = (double *)talloc(c, bytes);
    if (!d) return fail(c, LBM_ERR_ALLOC, "temporary population buffer");
    cudaError_t e = cudaMemcpyAsync(d, f, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(c->stream);
        tfree(c, d);
        return cuda_fail(c, e, "lbm_set_populations");
    }
    dispatch(c, [&](auto tag) {
        using TS = decltype(tag);
        Ops<TS>::scatter(c->s, d, c->stream);
        Ops<TS>::capture_frozen(c->s, c->d_frozen, c->stream);
    });
    c->launches += 2;
    c->step = 0;
    lbm_status st = check_launch(c, "lbm_set_populations");
    tfree(c, d);
    if (st != LBM_OK) return st;
    return capture_initial_mass(c);
}

lbm_status lbm_get_populations(lbm_ctx *c, double *f)
{
    if (!c || !f) return LBM_ERR_ARG;
    if (!c->subs.empty()) return no_batch(c, "lbm_get_populations");
    const size_t bytes = (size_t)38 * c->nv * 8;
    double *d = (double *)talloc(c, bytes);
    if (!d) return fail(c, LBM_ERR_ALLOC, "temporary population buffer");
    cudaError_t e = cudaMemsetAsync(d, 0, bytes, c->stream);
    dispatch(c, [&](auto tag) {
        using TS = decltype(tag);
        // the open-plane extrapolation of the last step is applied lazily by
        // the next density pass; apply it now (idempotent) so the returned
        // state is the post-step state
        if (c->step > 0) Ops<TS>::plane(c->s, (int)(c->step & 1), c->stream);
        Ops<TS>::gather(c->s, (int)(c->step & 1), d, c->stream);
    });
    c->launches += 1;
    lbm_status st = check_launch(c, "lbm_get_populations");
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, bytes, cudaMemcpyDeviceToHost, c->stream);
    tfree(c, d);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_get_populations");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "lbm_get_populations");
    return st != LBM_OK ? st : device_status(c);
}

// A batch's steps in persistent cooperative launches of up to kPersistSteps
// steps each (lbm_persist.cuh).
constexpr int kPersistSteps = 256;

lbm_status step_persistent(lbm_ctx *c, int64_t n)
{
    cudaStream_t st = c->stream;
    c->pipe_reset = false;
    const int nbn = c->table->start_n[c->table->count], nbw = c->table->start_w[c->table->count];
    int grid = 0;
    dispatch(c, [&](auto tag) { grid = Ops<decltype(tag)>::persist_grid(c->map_block); });
    grid = std::min(grid, std::max(1, std::max(nbn, nbw)));
    if (grid <= 0) return fail(c, LBM_ERR_CUDA, "the persistent launch does not fit on this device");
    for (int64_t k = 0; k < n;) {
        const int steps = (int)std::min<int64_t>(kPersistSteps, n - k);
        // every launch starts its barrier count and abort word from zero (a
        // launch that gave up leaves its count short)
        cudaMemsetAsync(c->d_bar, 0, sizeof(unsigned long long), st);
        cudaMemsetAsync(c->d_abort, 0, sizeof(int), st);
        PersistArgs pa{};
        pa.bar = c->d_bar;
        pa.abort = c->d_abort;
        pa.status = c->d_flag;
        pa.base = 0;
        pa.wait_ns = c->ps.wait_ns;
        pa.step0 = cur_step(c);
        pa.steps = steps;
        pa.stall = c->stall_next ? 1 : 0;
        c->stall_next = false;
        cudaError_t e = cudaSuccess;
        dispatch(c, [&](auto tag) { e = Ops<decltype(tag)>::persist(*c->table, pa, grid, c->map_block, st); });
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(c, e, "persistent launch");
        }
        for (lbm_ctx *q : c->subs) q->step += steps;
        c->step += steps;
        c->launches += 1;
        k += steps;
    }
    lbm_status stt = check_launch(c, "lbm_step");
    return stt != LBM_OK ? stt : device_status(c);
}

lbm_status lbm_step(lbm_ctx *c, int64_t n)
{
    NvtxRange nvtx_range("lbm_step");
    if (!c || n < 0) return LBM_ERR_ARG;
    if (n > 0) c->rec.valid = false;
    if (c->parent) return fail(c, LBM_ERR_ARG, "a sample of a batch is stepped through its batch");
    if (!c->subs.empty()) {
        for (lbm_ctx *q : c->subs)
            if (q->step != c->subs[0]->step) return fail(c, LBM_ERR_ARG, "the samples of a batch are at different steps");
        if (c->states_dirty) {
            lbm_status st = upload_states(c);
            if (st != LBM_OK) return st;
        }
    }
    if (c->kernel == LBM_KERNEL_PERSISTENT && !any_reduce(c) && n > 0) return step_persistent(c, n);
    int64_t k = 0;
    if (acc_schedule(c) && n > 0) push_prime_ctx(c);
    const int align = acc_schedule(c) ? 6 : 2;
    const bool graphs = c->kernel != LBM_KERNEL_FUSED && !any_reduce(c) && n >= 2 * align && !c->stall_next &&
                        std::getenv("LBM_NO_GRAPH") == nullptr;
    if (graphs) {
        // the first step (no plane extrapolation yet) and steps off the
        // graph's period (parity; accumulator rotation) run plain
        while (k < n && (cur_step(c) == 0 || cur_step(c) % align != 0)) {
            step_once(c);
            ++k;
        }
        // the flow schedule's graphs start from complete densities of the
        // current step: compute them outside the graph if needed
        if (n - k >= 2 && c->kernel == LBM_KERNEL_FLOW) flow_prime(c);
        if (n - k >= 2 && ensure_graph(c) == LBM_OK) {
            // the long graph while it fits, then the short one
            const cudaGraphExec_t gx[2] = {c->graph, c->graph_short};
            const int gn[2] = {c->graph_steps, c->graph_short_steps};
            const int64_t gl[2] = {c->graph_launches, c->graph_short_launches};
            for (int q = 0; q < 2; ++q) {
                if (!gx[q] || gn[q] <= 0) continue;
                for (; n - k >= gn[q]; k += gn[q]) {
                    cudaGraphLaunch(gx[q], c->stream);
                    c->step += gn[q];
                    if (acc_schedule(c)) c->push_step = c->step;
                    if (c->kernel == LBM_KERNEL_FLOW) {
                        c->s.psi = c->flow_psi[c->step & 1];
                        c->flow_ok_step = c->step;
                    }
                    for (lbm_ctx *qq : c->subs) qq->step += gn[q];
                    c->launches += gl[q];
                }
            }
        }
    }
    for (; k < n; ++k) step_once(c);
    lbm_status st = check_launch(c, "lbm_step");
    return st != LBM_OK ? st : device_status(c);
}

lbm_status lbm_create_batch(int32_t n, const lbm_geometry *geoms, const lbm_params *params, lbm_ctx **out)
{
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n <= 0 || !geoms || !params) return fail(nullptr, LBM_ERR_ARG, "need n > 0 geometries and parameter sets");
    std::vector<lbm_ctx *> subs;
    for (int32_t k = 0; k < n; ++k) {
        lbm_params pk = params[k];
        if (pk.kernel == LBM_KERNEL_FUSED || pk.kernel == LBM_KERNEL_BRICK || pk.kernel == LBM_KERNEL_FLOW ||
            pk.kernel == LBM_KERNEL_AUTO || pk.kernel == LBM_KERNEL_PERSISTENT)
            pk.kernel = LBM_KERNEL_SPLIT;
        lbm_ctx *q = nullptr;
        lbm_status st = lbm_create(&geoms[k], &pk, &q);
        if (st == LBM_OK && q->storage != (subs.empty() ? q->storage : subs[0]->storage)) {
            lbm_destroy(q);
            st = fail(nullptr, LBM_ERR_ARG, "all samples of a batch need the same storage type");
        }
        if (st != LBM_OK) {
            g_create_err = "sample " + std::to_string(k) + ": " + g_create_err;
            for (lbm_ctx *r : subs) destroy_ctx(r);
            return st;
        }
        subs.push_back(q);
    }
    lbm_ctx *c = new lbm_ctx();
    cudaGetDevice(&c->device);
    c->alloc_fn = g_alloc;
    c->free_fn = g_free;
    c->alloc_user = g_alloc_user;
    c->storage = subs[0]->storage;
    c->kernel = LBM_KERNEL_SPLIT;
    lbm_default_params(&c->p);
    c->subs = subs;
    for (lbm_ctx *q : subs) q->parent = c;
    c->d_states = (DevState *)dalloc(c, (size_t)n * sizeof(DevState));
    if (!c->d_states) {
        destroy_ctx(c);
        return fail(nullptr, LBM_ERR_ALLOC, "batch states");
    }
    if (build_maps(c, 128) != LBM_OK) {
        g_create_err = c->err;
        destroy_ctx(c);
        return LBM_ERR_ALLOC;
    }
    if (params[0].kernel == LBM_KERNEL_PERSISTENT) {
        if (n > kParamStates) {
            destroy_ctx(c);
            return fail(nullptr, LBM_ERR_UNSUPPORTED,
                        "the persistent launch takes at most " + std::to_string(kParamStates) + " samples");
        }
        c->kernel = LBM_KERNEL_PERSISTENT;
        c->ps.wait_ns = 1000000000ull;  // one second
        c->d_bar = (unsigned long long *)dalloc(c, sizeof(unsigned long long));
        c->d_abort = (int *)dalloc(c, sizeof(int));
        cudaError_t e = c->d_bar && c->d_abort ? cudaSuccess : cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaMemset(c->d_bar, 0, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(c->d_abort, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&c->h_flag, sizeof(int), cudaHostAllocMapped);
        if (e == cudaSuccess) {
            *c->h_flag = 0;
            e = cudaHostGetDevicePointer((void **)&c->d_flag, c->h_flag, 0);
        }
        if (e != cudaSuccess) {
            destroy_ctx(c);
            return fail(nullptr, LBM_ERR_ALLOC, "persistent launch counters");
        }
    }
    *out = c;
    return LBM_OK;
}

int32_t lbm_batch_size(const lbm_ctx *c) { return c ? (int32_t)c->subs.size() : 0; }

lbm_status lbm_batch_get(lbm_ctx *c, int32_t k, lbm_ctx **sample)
{
    if (!c || !sample || k < 0 || k >= (int32_t)c->subs.size()) return LBM_ERR_ARG;
    *sample = c->subs[(size_t)k];
    return LBM_OK;
}

lbm_status lbm_step_timed(lbm_ctx *c, int64_t n, double *kernel_ms, int32_t nk)
{
    if (!c || n < 0 || (nk > 0 && !kernel_ms)) return LBM_ERR_ARG;
    if (!c->subs.empty()) return no_batch(c, "lbm_step_timed");
    if (c->parent) return fail(c, LBM_ERR_ARG, "a sample of a batch is stepped through its batch");
    if (!c->have_ev) {
        for (auto &ev : c->ev) cudaEventCreate(&ev);
        c->have_ev = true;
    }
    if (acc_schedule(c)) push_prime_ctx(c);
    for (int64_t k = 0; k < n; ++k) {
        enqueue_step(c, c->ev);
        if (c->kernel == LBM_KERNEL_BRICK) {  // brick launch, plane pass
            cudaError_t e = cudaEventSynchronize(c->ev[2]);
            if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step_timed");
            const int slot[2] = {2, 3};
            for (int q = 0; q < 2; ++q) {
                float ms = 0;
                cudaEventElapsedTime(&ms, c->ev[q], c->ev[q + 1]);
                if (slot[q] < nk) kernel_ms[slot[q]] += ms;
            }
            continue;
        }
        if (c->kernel == LBM_KERNEL_PUSH) {  // collide-stream; plane nodes with the walls
            cudaError_t e = cudaEventSynchronize(c->ev[3]);
            if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step_timed");
            const int slot[2] = {2, 3};
            for (int q = 0; q < 2; ++q) {
                float ms = 0;
                cudaEventElapsedTime(&ms, c->ev[q], c->ev[q + 1]);
                if (slot[q] < nk) kernel_ms[slot[q]] += ms;
            }
            continue;
        }
        const bool fused = c->kernel == LBM_KERNEL_FUSED || c->kernel == LBM_KERNEL_FLOW;
        cudaError_t e = cudaEventSynchronize(c->ev[fused ? 1 : 4]);
        if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step_timed");
        if (fused) {
            float ms = 0;
            cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
            if (nk > 4) kernel_ms[4] += ms;
            continue;
        }
        for (int q = 0; q < 4 && q < nk; ++q) {
            float ms = 0;
            cudaEventElapsedTime(&ms, c->ev[q], c->ev[q + 1]);
            kernel_ms[q] += ms;
        }
    }
    lbm_status st = check_launch(c, "lbm_step_timed");
    return st != LBM_OK ? st : device_status(c);
}

lbm_status lbm_read_fields(lbm_ctx *c, uint32_t mask, double *out, size_t n_per_field)
{
    if (!c || !out) return LBM_ERR_ARG;
    if (!c->subs.empty()) return no_batch(c, "lbm_read_fields");
    if (n_per_field < (size_t)c->nv) return fail(c, LBM_ERR_ARG, "n_per_field is smaller than nx*ny*nz");
    mask &= 63u;
    const int nfield = __builtin_popcount(mask);
    if (nfield == 0) return LBM_OK;
    // a buffer kept by the context for the requested fields (grown when more
    // are asked for), so repeated reads neither allocate nor free
    const size_t bytes = (size_t)nfield * c->nv * 8;
    if (c->fields_bytes < bytes) {
        if (c->fields_buf) dfree(c, c->fields_buf);
        c->fields_buf = dalloc(c, bytes);
        c->fields_bytes = c->fields_buf ? bytes : 0;
        if (!c->fields_buf) return fail(c, LBM_ERR_ALLOC, "field buffer");
    }
    double *d = (double *)c->fields_buf;
    const int par = (int)(c->step & 1);
    dispatch(c, [&](auto tag) {
        using TS = decltype(tag);
        Ops<TS>::dens(c->s, par, c->step > 0, c->stream);
        Ops<TS>::wall(c->s, c->stream);
        Ops<TS>::fields(c->s, par, d, mask, c->stream);
    });
    c->launches += 3;
    lbm_status st = check_launch(c, "lbm_read_fields");
    cudaError_t e = cudaSuccess;
    if (n_per_field == (size_t)c->nv) {
        e = cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, c->stream);
    } else {
        for (int k = 0; k < nfield && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(out + (size_t)k * n_per_field, d + (size_t)k * c->nv, (size_t)c->nv * 8,
                                cudaMemcpyDeviceToHost, c->stream);
    }
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_read_fields");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "lbm_read_fields");
    return st != LBM_OK ? st : device_status(c);
}

lbm_status lbm_saturation(lbm_ctx *c, double out[4])
{
    if (!c || !out) return LBM_ERR_ARG;
    if (!c->subs.empty()) return no_batch(c, "lbm_saturation");
    run_reduce(c);
    lbm_status st = check_launch(c, "lbm_saturation");
    double red[kReduceSlots];
    cudaError_t e = cudaMemcpyAsync(red, c->d_red, sizeof(red), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_saturation");
    out[0] = red[2] > 0 ? red[3] / red[2] : 0.0;
    out[1] = red[2] > 0 ? red[4] / red[2] : 0.0;
    out[2] = red[0];
    out[3] = red[1];
    return st != LBM_OK ? st : device_status(c);
}

lbm_status lbm_set_inlet(lbm_ctx *c, double rho_in1)
{
    if (!c) return LBM_ERR_ARG;
    if (!c->subs.empty()) return no_batch(c, "lbm_set_inlet");
    c->p.rho_in1 = rho_in1;
    c->s.rho_in1 = rho_in1;
    set_float_params(c->s);
    touch(c);
    return LBM_OK;
}

lbm_status lbm_set_stream(lbm_ctx *c, void *stream)
{
    if (!c) return LBM_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    for (lbm_ctx *q : c->subs) q->stream = (cudaStream_t)stream;
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_ctx *c)
{
    if (!c) return LBM_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->sticky = LBM_ERR_CUDA;
        return cuda_fail(c, e, "lbm_synchronize");
    }
    return device_status(c);
}

lbm_status lbm_get_info(const lbm_ctx *c, lbm_info *info)
{
    if (!c || !info) return LBM_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n_fluid = c->s.n_fluid;
    info->n_wall = c->s.n_wall;
    info->n_voxels = c->nv;
    info->step = c->step;
    info->device_bytes = c->bytes;
    for (const lbm_ctx *q : c->subs) {  // a batch reports the sum over its samples
        info->n_fluid += q->s.n_fluid;
        info->n_wall += q->s.n_wall;
        info->n_voxels += q->nv;
        info->device_bytes += q->bytes;
        info->step = q->step;
    }
    info->launches = c->launches;
    info->storage = c->storage;
    info->kernel = c->kernel;
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_ctx *c, const char *cache_path, int32_t *block_out)
{
    NvtxRange nvtx_range("lbm_autotune");
    if (!c) return LBM_ERR_ARG;
    if (c->parent) return fail(c, LBM_ERR_ARG, "a sample of a batch is tuned through its batch");
    if (c->kernel == LBM_KERNEL_FUSED) {  // the single-pass schedule's block is its chunk
        if (block_out) *block_out = kChunk;
        return LBM_OK;
    }
    const std::string key = tune_key(c);
    std::vector<std::pair<std::string, int>> kv = read_cache(cache_path);
    for (auto &e : kv)
        if (e.first == key) {
            for (int cand : kTuneBlocks)
                if (cand == e.second) {
                    lbm_status st = apply_block(c, cand);
                    if (st == LBM_OK && block_out) *block_out = cand;
                    return st;
                }
        }
    int best = 0;
    lbm_status st = tune(c, &best);
    if (st != LBM_OK) return st;
    st = apply_block(c, best);
    if (st != LBM_OK) return st;
    if (block_out) *block_out = best;
    if (cache_path && *cache_path) {
        bool found = false;
        for (auto &e : kv)
            if (e.first == key) {
                e.second = best;
                found = true;
            }
        if (!found) kv.push_back({key, best});
        if (!write_cache(cache_path, kv)) return fail(c, LBM_ERR_ARG, "lbm_autotune: cannot write the cache file");
    }
    return LBM_OK;
}

lbm_status lbm_set_xi_field(lbm_ctx *c, const float *xi, int32_t on_device)
{
    if (!c || !xi) return LBM_ERR_ARG;
    if (!c->subs.empty()) return no_batch(c, "lbm_set_xi_field");
    if (c->s.n_wall == 0) return LBM_OK;
    const float *src = xi;
    float *tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        tmp = (float *)dalloc(c, (size_t)c->nv * 4);
        if (!tmp) return fail(c, LBM_ERR_ALLOC, "temporary xi buffer");
        e = cudaMemcpyAsync(tmp, xi, (size_t)c->nv * 4, cudaMemcpyHostToDevice, c->stream);
        src = tmp;
    }
    const int g = (c->s.n_wall + 255) / 256;
    if (e == cudaSuccess) {
        if (c->storage == LBM_STORE_FP64)
            k_set_wxi<double><<<g, 256, 0, c->stream>>>(c->s.wpvox, c->s.n_wall, src, (double *)c->s.wxi);
        else
            k_set_wxi<float><<<g, 256, 0, c->stream>>>(c->s.wpvox, c->s.n_wall, src, (float *)c->s.wxi);
        c->launches += 1;
        if (c->kernel == LBM_KERNEL_BRICK && c->n_bentries > 0) {
            brick_coef(c->s, c->d_bwid, c->n_bentries, const_cast<float2 *>(c->bb.wcoef),
                       c->storage == LBM_STORE_FP64, c->stream);
            c->launches += 1;
        }
    }
    if (tmp) {
        cudaStreamSynchronize(c->stream);
        dfree(c, tmp);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_set_xi_field");
    touch(c);
    return check_launch(c, "lbm_set_xi_field");
}

lbm_status lbm_record(lbm_ctx *c, int64_t nsteps, int32_t every)
{
    NvtxRange nvtx_range("lbm_record");
    if (!c || nsteps < 1 || every < 1) return LBM_ERR_ARG;
    if (!adjoint_supported(c))
        return fail(c, LBM_ERR_UNSUPPORTED, "the reverse pass needs a single lattice with FP32 or FP64 storage, "
                                            "the split schedule and the extrapolation open-plane rule");
    auto &r = c->rec;
    const int64_t nck = (nsteps + every - 1) / every;
    const size_t sb = state_bytes(c);
    if ((int64_t)r.ckpt.size() != nck || r.every != every) {
        free_record(c);
        for (int64_t k = 0; k < nck; ++k) {
            void *q = dalloc(c, sb);
            if (!q) {
                free_record(c);
                return fail(c, LBM_ERR_ALLOC, "lbm_record: checkpoints");
            }
            r.ckpt.push_back(q);
        }
        r.final_state = dalloc(c, sb);
        if (!r.final_state) {
            free_record(c);
            return fail(c, LBM_ERR_ALLOC, "lbm_record: final state");
        }
    }
    r.step0 = c->step;
    r.n = nsteps;
    r.every = every;
    // the densities of every step, if they take at most a quarter of the free
    // device memory (LBM_RECORD_DENSITIES=0: never)
    const size_t pb = (size_t)c->nv * (c->storage == LBM_STORE_FP64 ? 16 : 8);
    const size_t dens_need = pb * (size_t)nsteps;
    // (the split passes write them into c->s.psi; the other schedules keep
    // their densities elsewhere, and a periodic check runs a density pass of
    // the next state after its step, so those recompute them)
    bool store = !(std::getenv("LBM_RECORD_DENSITIES") && std::atoi(std::getenv("LBM_RECORD_DENSITIES")) == 0) &&
                 (c->kernel == LBM_KERNEL_SPLIT || c->kernel == LBM_KERNEL_WAVE) && c->p.reduce_every == 0;
    if (store && r.dens_all_bytes < dens_need) {
        if (r.dens_all) dfree(c, r.dens_all);
        r.dens_all = nullptr;
        r.dens_all_bytes = 0;
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && dens_need <= fr / 4) r.dens_all = dalloc(c, dens_need);
        if (r.dens_all) r.dens_all_bytes = dens_need;
    }
    store = store && r.dens_all && r.dens_all_bytes >= dens_need;
    r.dens_stored = store;
    // with kept densities, the whole recording as one graph: captured the
    // first time, replayed while nothing it holds has changed
    const bool use_graph = store && std::getenv("LBM_NO_GRAPH") == nullptr;
    if (use_graph) {
        std::vector<void *> key = r.ckpt;
        key.push_back(r.final_state);
        key.push_back(r.dens_all);
        key.push_back(c->s.psi);
        key.push_back(c->s.f);
        const int par0 = (int)(c->step & 1) + (c->step > 0 ? 2 : 0);
        if (r.graph && (r.graph_key != key || r.graph_n != nsteps || r.graph_every != every ||
                        r.graph_par != par0 || r.graph_block != c->block ||
                        std::memcmp(&r.graph_state, &c->s, sizeof(DevState)) != 0)) {
            cudaGraphExecDestroy(r.graph);
            r.graph = nullptr;
        }
        if (r.graph) {
            cudaError_t e = cudaGraphLaunch(r.graph, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "lbm_record: graph");
            c->step += nsteps;
            c->launches += r.graph_launches;
        } else {
            if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
                return cuda_fail(c, cudaGetLastError(), "lbm_record: capture stream");
            // the capture stream starts after the work already on the context's stream
            cudaEvent_t ev0 = nullptr;
            cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming);
            cudaEventRecord(ev0, c->stream);
            cudaStreamWaitEvent(c->cap_stream, ev0, 0);
            const cudaStream_t user = c->stream;
            const int64_t step0 = c->step, l0 = c->launches;
            void *psi0 = c->s.psi;
            c->stream = c->cap_stream;
            cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
            lbm_status sst = LBM_OK;
            for (int64_t k = 0; e == cudaSuccess && sst == LBM_OK && k < nck; ++k) {
                snap_save(c, r.ckpt[(size_t)k]);
                const int64_t len = std::min<int64_t>(every, nsteps - k * every);
                for (int64_t q = 0; q < len && sst == LBM_OK; ++q) {
                    c->s.psi = (char *)r.dens_all + (size_t)(k * every + q) * pb;
                    step_once(c);
                }
            }
            c->s.psi = psi0;
            cudaGraph_t g = nullptr;
            cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(c->cap_stream, &g) : e;
            c->stream = user;
            if (e2 == cudaSuccess) e2 = cudaGraphInstantiate(&r.graph, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaEventDestroy(ev0);
            if (e2 != cudaSuccess) {
                r.graph = nullptr;
                cudaGetLastError();
                return cuda_fail(c, e2, "lbm_record: graph capture");
            }
            r.graph_key = key;
            r.graph_n = nsteps;
            r.graph_every = every;
            r.graph_par = par0;
            r.graph_block = c->block;
            std::memcpy(&r.graph_state, &c->s, sizeof(DevState));
            r.graph_launches = c->launches - l0;
            (void)step0;
            e = cudaGraphLaunch(r.graph, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "lbm_record: graph");
        }
    }
    for (int64_t k = 0; !use_graph && k < nck; ++k) {
        snap_save(c, r.ckpt[(size_t)k]);
        const int64_t len = std::min<int64_t>(every, nsteps - k * every);
        if (store) {
            // one step at a time, each writing its densities (and wall
            // densities) into its own slot of dens_all
            void *psi0 = c->s.psi;
            for (int64_t q = 0; q < len; ++q) {
                c->s.psi = (char *)r.dens_all + (size_t)(k * every + q) * pb;
                lbm_status st = lbm_step(c, 1);
                if (st != LBM_OK) {
                    c->s.psi = psi0;
                    return st;
                }
            }
            c->s.psi = psi0;
        } else {
            lbm_status st = lbm_step(c, len);
            if (st != LBM_OK) return st;
        }
    }
    snap_save(c, r.final_state);
    r.step_end = c->step;
    lbm_status st = check_launch(c, "lbm_record");
    if (st != LBM_OK) return st;
    r.valid = true;
    return device_status(c);
}

lbm_status lbm_adjoint(lbm_ctx *c, double dloss, float *grad_xi, double *grad_rho_in1, double *loss)
{
    NvtxRange nvtx_range("lbm_adjoint");
    if (!c) return LBM_ERR_ARG;
    auto &r = c->rec;
    if (!r.valid || c->step != r.step_end)
        return fail(c, LBM_ERR_ARG, "lbm_adjoint needs a recording (lbm_record) that is still current");
    const size_t sb = state_bytes(c);
    const size_t csz = c->storage == LBM_STORE_FP64 ? 16 : 8;  // compute-type pair
    const int64_t npad = c->s.npad, nv = c->nv;
    // reverse-pass buffers (kept for later calls)
    while ((int64_t)r.seg.size() < r.every - 1) {
        void *q = dalloc(c, sb);
        if (!q) return fail(c, LBM_ERR_ALLOC, "lbm_adjoint: segment states");
        r.seg.push_back(q);
    }
    while (!r.dens_stored && (int64_t)r.psis.size() < r.every) {
        void *q = dalloc(c, (size_t)c->nv * (c->storage == LBM_STORE_FP64 ? 16 : 8));
        if (!q) return fail(c, LBM_ERR_ALLOC, "lbm_adjoint: segment densities");
        r.psis.push_back(q);
    }
    auto need = [&](void *&q, size_t bytes) {
        if (!q) q = dalloc(c, bytes);
        return q != nullptr;
    };
    if (!need(r.lam[0], (size_t)19 * npad * csz) || !need(r.lam[1], (size_t)19 * npad * csz) ||
        !need(r.rb[0], (size_t)nv * csz) || !need(r.rb[1], (size_t)nv * csz) || !need(r.abar, (size_t)3 * nv * csz) ||
        !need(r.wbar, (size_t)nv * csz) || !need(r.psi, (size_t)nv * csz))
        return fail(c, LBM_ERR_ALLOC, "lbm_adjoint: adjoint buffers");
    if (!r.gxi) r.gxi = (double *)dalloc(c, (size_t)std::max(1, c->s.n_wall) * 8);
    if (!r.grin) r.grin = (double *)dalloc(c, (size_t)std::max(1, c->s.nxy) * 8);
    if (!r.gxi || !r.grin) return fail(c, LBM_ERR_ALLOC, "lbm_adjoint: gradient accumulators");
    cudaStream_t st = c->stream;

    // loss of the final state (its densities land in the live psi)
    run_reduce(c);
    double red[kReduceSlots];
    cudaError_t e = cudaMemcpyAsync(red, c->d_red, sizeof(red), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_adjoint: loss");
    const double count = red[2];
    const double J = count > 0 ? red[4] / count : 0.0;

    AdjState a{};
    a.lam_in = r.lam[0];
    a.lam_out = r.lam[1];
    a.rb_in = r.rb[0];
    a.rb_out = r.rb[1];
    a.abar = r.abar;
    a.wbar = r.wbar;
    a.gxi = r.gxi;
    a.grin = r.grin;
    cudaMemsetAsync(a.lam_in, 0, (size_t)19 * npad * csz, st);
    cudaMemsetAsync(a.rb_in, 0, (size_t)nv * csz, st);
    cudaMemsetAsync(a.abar, 0, (size_t)3 * nv * csz, st);
    cudaMemsetAsync(a.wbar, 0, (size_t)nv * csz, st);
    cudaMemsetAsync(a.gxi, 0, (size_t)std::max(1, c->s.n_wall) * 8, st);
    cudaMemsetAsync(a.grin, 0, (size_t)std::max(1, c->s.nxy) * 8, st);
    dispatch_adj(c, [&](auto tag) {
        using TS = decltype(tag);
        Adj<TS>::seed(c->s, a, count > 0 ? 1.0 / count : 0.0, st);
    });
    c->launches += 1;

    const int64_t nck = (int64_t)r.ckpt.size();
    const size_t pb = (size_t)c->nv * csz;
    // The states of segment k: its checkpoint, the every - 1 recomputed states
    // in buffer set `set`, and the next checkpoint (or the final state).
    auto states = [&](int64_t k, int set) {
        const int64_t len = std::min<int64_t>(r.every, r.n - k * r.every);
        std::vector<void *> S((size_t)len + 1);
        S[0] = r.ckpt[(size_t)k];
        for (int64_t q = 1; q < len; ++q) S[(size_t)q] = (set ? r.seg2 : r.seg)[(size_t)q - 1];
        S[(size_t)len] = k + 1 < nck ? r.ckpt[(size_t)k + 1] : r.final_state;
        return S;
    };
    // densities of state q of segment k: recorded, or recomputed into psis[q]
    auto psi_of = [&](int64_t k, int64_t q) -> void * {
        return r.dens_stored ? (void *)((char *)r.dens_all + (size_t)(k * r.every + q) * pb) : r.psis[(size_t)q];
    };
    // Recompute segment k from its checkpoint, out of place, on stream s: with
    // recorded densities, the open-plane rule on each recomputed state and the
    // collide-stream pass; otherwise the density pass of state q (in its own
    // buffer), which applies the pending open-plane rule and writes the
    // densities of state q into psis[q], then the wall and collide-stream
    // passes.  The live state is not touched.
    auto recompute = [&](int64_t k, int set, cudaStream_t s) {
        const std::vector<void *> S = states(k, set);
        const int64_t len = (int64_t)S.size() - 1;
        for (int64_t q = 0; q < len; ++q) {
            const int64_t step = r.step0 + k * r.every + q;
            const int par = (int)(step & 1);
            const DevState s_q = snap_state(c, S[(size_t)q], psi_of(k, q));
            const DevState s_n = snap_state(c, S[(size_t)q + 1], psi_of(k, q));
            dispatch_adj(c, [&](auto tag) {
                using TS = decltype(tag);
                if (r.dens_stored) {
                    // the checkpoint already holds its open-plane rule; a
                    // recomputed state gets it here, as the density pass
                    // would apply it
                    if (q > 0 && step > 0) {
                        Ops<TS>::plane(s_q, par, s);
                        c->launches += s_q.open_z && s_q.nxy > 0 ? 1 : 0;
                    }
                } else {
                    Ops<TS>::dens(s_q, par, step > 0, s, c->block);
                    Ops<TS>::wall(s_q, s, c->block);
                    c->launches += 2;
                }
                if (q + 1 < len) {
                    Adj<TS>::fused_to(s_q, par, s_n.f, s_n.rest, s);
                    c->launches += 1;
                }
            });
        }
    };
    // Reverse the steps of segment k on the context's stream.
    auto reverse = [&](int64_t k, int set) {
        const std::vector<void *> S = states(k, set);
        const int64_t len = (int64_t)S.size() - 1;
        for (int64_t q = len - 1; q >= 0; --q) {
            const int par = (int)((r.step0 + k * r.every + q) & 1);
            const DevState s_t = snap_state(c, S[(size_t)q], psi_of(k, q));
            const DevState s_n = snap_state(c, S[(size_t)q + 1], psi_of(k, q));
            dispatch_adj(c, [&](auto tag) {
                using TS = decltype(tag);
                if (c->nz > 3) {
                    Adj<TS>::plane(s_n, a, 1 - par, 2, st);
                } else {
                    Adj<TS>::plane(s_n, a, 1 - par, 1, st);  // outlet (extrapolated last)
                    Adj<TS>::plane(s_n, a, 1 - par, 0, st);  // inlet
                }
                Adj<TS>::node(s_t, a, par, st);
                Adj<TS>::wall(s_t, a, st);
                Adj<TS>::dens(s_t, a, st);
            });
            c->launches += 5;
            std::swap(a.lam_in, a.lam_out);
            std::swap(a.rb_in, a.rb_out);
        }
    };
    // With recorded densities and a second set of segment buffers, segment
    // k - 1 is recomputed on a side stream while segment k is reversed: the
    // two touch disjoint buffers (the recompute writes only its own set and
    // reads checkpoints and densities), and the reverse kernels leave most of
    // the memory bandwidth free.  Otherwise segment by segment on one stream.
    bool overlap = r.dens_stored && nck > 1 && r.every > 1 &&
                   !(std::getenv("LBM_ADJ_OVERLAP") && std::atoi(std::getenv("LBM_ADJ_OVERLAP")) == 0);
    if (overlap) {
        while ((int64_t)r.seg2.size() < r.every - 1) {
            void *q = dalloc(c, sb);
            if (!q) break;
            r.seg2.push_back(q);
        }
        overlap = (int64_t)r.seg2.size() >= r.every - 1;
        if (overlap && !r.side) {
            overlap = cudaStreamCreateWithFlags(&r.side, cudaStreamNonBlocking) == cudaSuccess;
            for (int q = 0; overlap && q < 5; ++q)
                overlap = cudaEventCreateWithFlags(&r.ev[q], cudaEventDisableTiming) == cudaSuccess;
            if (!overlap) cudaGetLastError();
        }
    }
    if (overlap) {
        cudaStream_t side = r.side;
        cudaEvent_t *rec_done = &r.ev[0], *rev_done = &r.ev[2];
        cudaEventRecord(r.ev[4], st);  // everything enqueued so far (the seed) before the side stream starts
        cudaStreamWaitEvent(side, r.ev[4], 0);
        recompute(nck - 1, (int)((nck - 1) & 1), side);
        cudaEventRecord(rec_done[(nck - 1) & 1], side);
        for (int64_t k = nck - 1; k >= 0; --k) {
            const int set = (int)(k & 1);
            if (k >= 1) {
                const int oset = (int)((k - 1) & 1);
                if (k + 1 < nck) cudaStreamWaitEvent(side, rev_done[oset], 0);  // segment k + 1 used that set
                recompute(k - 1, oset, side);
                cudaEventRecord(rec_done[oset], side);
            }
            cudaStreamWaitEvent(st, rec_done[set], 0);
            reverse(k, set);
            cudaEventRecord(rev_done[set], st);
        }
    } else {
        for (int64_t k = nck - 1; k >= 0; --k) {
            recompute(k, 0, st);
            reverse(k, 0);
        }
    }
    // the recompute never touched the live state: it is still the final one
    lbm_status stt = check_launch(c, "lbm_adjoint");
    if (stt != LBM_OK) return stt;
    if (grad_xi) {
        cudaMemsetAsync(grad_xi, 0, (size_t)nv * 4, st);
        dispatch_adj(c, [&](auto tag) { Adj<decltype(tag)>::xi_out(c->s, a, dloss, grad_xi, st); });
        c->launches += 1;
    }
    std::vector<double> gr((size_t)std::max(1, c->s.nxy), 0.0);
    e = cudaMemcpyAsync(gr.data(), a.grin, gr.size() * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_adjoint");
    double g = 0.0;
    for (double v : gr) g += v;  // fixed order
    if (grad_rho_in1) *grad_rho_in1 = c->s.open_z ? g * dloss : 0.0;
    if (loss) *loss = J;
    stt = check_launch(c, "lbm_adjoint");
    return stt != LBM_OK ? stt : device_status(c);
}

lbm_status lbm_set_wait_limit(lbm_ctx *c, double seconds)
{
    if (!c || !(seconds > 0.0) || seconds > 60.0) return LBM_ERR_ARG;
    c->ps.wait_ns = (unsigned long long)(seconds * 1e9);
    c->fs.wait_ns = c->ps.wait_ns;
    return LBM_OK;
}

lbm_status lbm_inject_stall(lbm_ctx *c)
{
    if (!c) return LBM_ERR_ARG;
    if (c->kernel != LBM_KERNEL_FUSED && c->kernel != LBM_KERNEL_PERSISTENT &&
        !(c->kernel == LBM_KERNEL_FLOW && c->flow_stall_slot >= 0))
        return fail(c, LBM_ERR_UNSUPPORTED, "only the single-pass, flow and persistent schedules have device waits");
    c->stall_next = true;
    return LBM_OK;
}

// ---- checkpoint / resume --------------------------------------------------
// File layout (host byte order): a fixed header, then the raw device state
// (moving population cells, rest pairs, open-plane boundary cells) and the
// frozen missing populations of the open planes.
struct StateFileHeader {
    char magic[8];               // "LBMSTAT1"
    int32_t version, storage, nx, ny, nz, n_fluid, open_axis, periodic;
    int64_t npad, nv, step;
    uint64_t geometry_hash;      // FNV-1a of the solid mask
    double rref[2], mass0[2];
    uint64_t f_bytes, rest_bytes, bc_bytes, frozen_bytes;
};

static uint64_t mask_hash(const std::vector<uint8_t> &m)
{
    uint64_t h = 1469598103934665603ull;
    for (uint8_t b : m) {
        h ^= b;
        h *= 1099511628211ull;
    }
    return h;
}

static StateFileHeader state_header(const lbm_ctx *c)
{
    StateFileHeader h{};
    std::memcpy(h.magic, "LBMSTAT1", 8);
    h.version = 1;
    h.storage = c->storage;
    h.nx = c->nx;
    h.ny = c->ny;
    h.nz = c->nz;
    h.n_fluid = c->s.n_fluid;
    h.open_axis = c->open_axis;
    h.periodic = c->periodic[0] | (c->periodic[1] << 1) | (c->periodic[2] << 2);
    h.npad = c->s.npad;
    h.nv = c->nv;
    h.step = c->step;
    h.geometry_hash = mask_hash(c->solid_host);
    h.rref[0] = c->s.rref1;
    h.rref[1] = c->s.rref2;
    h.mass0[0] = c->mass0[0];
    h.mass0[1] = c->mass0[1];
    h.f_bytes = c->f_bytes;
    h.rest_bytes = c->rest_bytes;
    h.bc_bytes = c->bc_bytes;
    h.frozen_bytes = c->s.open_z ? (uint64_t)2 * 5 * c->s.nxy * 8 : 0;
    return h;
}

lbm_status lbm_save(lbm_ctx *c, const char *path)
{
    NvtxRange nvtx_range("lbm_save");
    if (!c || !path) return LBM_ERR_ARG;
    if (!c->subs.empty()) return no_batch(c, "lbm_save");
    const StateFileHeader h = state_header(c);
    const size_t n = h.f_bytes + h.rest_bytes + h.bc_bytes + h.frozen_bytes;
    std::vector<char> buf(n);
    size_t off = 0;
    cudaError_t e = cudaSuccess;
    const std::pair<const void *, size_t> parts[4] = {
        {c->s.f, h.f_bytes}, {c->s.rest, h.rest_bytes}, {c->s.bc, h.bc_bytes}, {c->d_frozen, h.frozen_bytes}};
    for (const auto &q : parts) {
        if (q.second && e == cudaSuccess)
            e = cudaMemcpyAsync(buf.data() + off, q.first, q.second, cudaMemcpyDeviceToHost, c->stream);
        off += q.second;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_save");
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(c, LBM_ERR_ARG, std::string("lbm_save: cannot open ") + path);
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && (n == 0 || std::fwrite(buf.data(), 1, n, fp) == n);
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return fail(c, LBM_ERR_ARG, std::string("lbm_save: cannot write ") + path);
    return device_status(c);
}

lbm_status lbm_load(lbm_ctx *c, const char *path)
{
    NvtxRange nvtx_range("lbm_load");
    if (!c || !path) return LBM_ERR_ARG;
    if (!c->subs.empty()) return no_batch(c, "lbm_load");
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(c, LBM_ERR_ARG, std::string("lbm_load: cannot open ") + path);
    StateFileHeader h{};
    const StateFileHeader mine = state_header(c);
    bool ok = std::fread(&h, sizeof(h), 1, fp) == 1;
    if (!ok || std::memcmp(h.magic, "LBMSTAT1", 8) != 0 || h.version != 1) {
        std::fclose(fp);
        return fail(c, LBM_ERR_ARG, "lbm_load: not a state file of this library");
    }
    if (h.storage != mine.storage || h.nx != mine.nx || h.ny != mine.ny || h.nz != mine.nz ||
        h.n_fluid != mine.n_fluid || h.open_axis != mine.open_axis || h.periodic != mine.periodic ||
        h.npad != mine.npad || h.geometry_hash != mine.geometry_hash || h.f_bytes != mine.f_bytes ||
        h.rest_bytes != mine.rest_bytes || h.bc_bytes != mine.bc_bytes || h.frozen_bytes != mine.frozen_bytes) {
        std::fclose(fp);
        return fail(c, LBM_ERR_ARG, "lbm_load: the file holds another lattice (geometry or storage differ)");
    }
    const size_t n = h.f_bytes + h.rest_bytes + h.bc_bytes + h.frozen_bytes;
    std::vector<char> buf(n);
    ok = n == 0 || std::fread(buf.data(), 1, n, fp) == n;
    std::fclose(fp);
    if (!ok) return fail(c, LBM_ERR_ARG, "lbm_load: the file is truncated");
    size_t off = 0;
    cudaError_t e = cudaSuccess;
    const std::pair<void *, size_t> parts[4] = {
        {c->s.f, h.f_bytes}, {c->s.rest, h.rest_bytes}, {c->s.bc, h.bc_bytes}, {c->d_frozen, h.frozen_bytes}};
    for (const auto &q : parts) {
        if (q.second && e == cudaSuccess)
            e = cudaMemcpyAsync(q.first, buf.data() + off, q.second, cudaMemcpyHostToDevice, c->stream);
        off += q.second;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // buf is released below
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_load");
    c->s.rref1 = h.rref[0];
    c->s.rref2 = h.rref[1];
    set_float_params(c->s);
    c->mass0[0] = h.mass0[0];
    c->mass0[1] = h.mass0[1];
    c->step = h.step;
    touch(c);
    if (c->h_flag) *c->h_flag = 0;
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
