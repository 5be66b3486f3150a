// lbm_flow.cuh -- the flow schedule: one launch per time step that collides
// and streams every fluid chunk (F), computes the next step's densities of
// each chunk (D, Eq. 3 after the open-plane rule of Section 2) a few dozen
// slots later, while the populations F wrote are still in L2, and then the
// next step's virtual wall densities (W, Eqs. 14-15).  The arithmetic of each
// item is that of the split passes (fused_node, dens_node, wall_node), so the
// results are bitwise those of the split schedule; only the order of the work
// and where its operands come from differ.  See FlowState for the slot plan.
//
// Ordering.  A block publishes each item as soon as it is done, with a
// release store after a block barrier and a device-scope fence (no item's
// flag waits for the block's later items); a waiting block reads the
// flags of the whole dependency range with acquire loads and a block-wide
// vote, then reads the data other blocks wrote with L2-only loads.  F reads
// only data written before the launch began (populations of the previous
// step, densities in the other psi buffer).
#pragma once

#include "lbm_pipe.cuh"

namespace lbm {

// Resident blocks per SM the register budget is sized for (kFlowThreads
// threads a block): 85 registers a thread for FP32 / 16-bit storage, 128 for
// FP64.
template <typename TS>
struct FlowOcc {
    static constexpr int blocks = 6;
};
template <>
struct FlowOcc<double> {
    static constexpr int blocks = 4;
};

constexpr int kFlowMaxPolls = 1 << 22;  // polls of a range before a block gives up

__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// A flag read.  Relaxed, not acquire: what a waiter then reads of other
// blocks' output it reads with L2-only loads issued after the block-wide vote
// on the flags, and the producer's fence put that output in L2 before the
// flag.  (An acquire load would also discard the SM's L1 lines, which the
// co-resident blocks' density stencils live on.)
__device__ __forceinline__ int ld_flag(const int *p)
{
#ifdef LBM_FLOW_ACQUIRE
    return ld_acquire(p);
#else
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
#endif
}

// Wait until flags[r.x .. r.y] all equal `want` (every thread of the block
// calls this).  Returns false if the launch `stamp` was abandoned, by this
// block (time limit or poll backstop: sets the abort word and the timeout
// status bit) or by another.
__device__ __forceinline__ bool flow_wait(const int *flags, int2 r, int want, int stamp, const FlowState &fs)
{
    unsigned long long t0 = 0;
    int backoff = 32;
    for (int it = 0; it < kFlowMaxPolls; ++it) {
        int ok = 1;
        for (int c = r.x + (int)threadIdx.x; c <= r.y; c += blockDim.x) ok &= ld_flag(flags + c) == want;
        if (__syncthreads_and(ok)) return true;
        int stop = 0;
        if (threadIdx.x == 0) {
            const unsigned long long t = global_ns();
            if (it == 0) t0 = t;
            if (*(volatile int *)fs.abort == stamp) {
                stop = 1;
            } else if (t - t0 > fs.wait_ns) {
                atomicExch(fs.abort, stamp);
                atomicOr(fs.status, 4);
                stop = 1;
            }
        }
        if (__syncthreads_or(stop)) return false;
        __nanosleep(backoff);
        backoff = min(backoff * 2, 1024);
    }
    if (threadIdx.x == 0) {
        atomicExch(fs.abort, stamp);
        atomicOr(fs.status, 4);
    }
    __syncthreads();
    return false;
}

// Publish an item: every thread's stores of it precede the barrier, and the
// release store (after a device-scope fence) makes them visible with the flag.
__device__ __forceinline__ void flow_publish(int *flag, int stamp)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release_gpu(flag, stamp);
    }
}

template <typename TS, int P>
__global__ void __launch_bounds__(kFlowThreads, FlowOcc<TS>::blocks) k_flow(DevState s, FlowState fs)
{
    __shared__ unsigned long long sh_ticket;
    pdl_trigger();
    pdl_wait();
    if (threadIdx.x == 0) sh_ticket = atomicAdd(fs.ticket, 1ull);
    __syncthreads();
    const unsigned long long t = sh_ticket;
    const int k = (int)(t % (unsigned long long)fs.n_slots);
    const int stamp = (int)(t / (unsigned long long)fs.n_slots) + 1;
    const int2 it = fs.items[k];

    // F: collide and stream chunk k (inputs from earlier launches only); its
    // flag is published at once, so no F ever waits, directly or through the
    // flag of its block's later items
    if (k < fs.n_chunks) {
        const int n1 = min(s.n_fluid, (k + 1) * fs.chunk);
        for (int n = k * fs.chunk + (int)threadIdx.x; n < n1; n += kFlowThreads) fused_node<TS, P>(n, s);
        flow_publish(fs.fdone + k, stamp);
    }
    // D: next-step densities of chunk it.x once every writer of its cells is done
    if (it.x >= 0) {
        const int want = stamp + (k == fs.stall_slot ? (1 << 20) : 0);
        if (!flow_wait(fs.fdone, fs.dep_f[it.x], want, stamp, fs)) return;
        const int n1 = min(s.n_fluid, (it.x + 1) * fs.chunk);
        for (int n = it.x * fs.chunk + (int)threadIdx.x; n < n1; n += kFlowThreads)
            dens_node<TS, 1 - P>(n, s, fs.psi_next);
        flow_publish(fs.ddone + it.x, stamp);
    }
    // W: next-step virtual densities of wall chunk it.y once its fluid
    // neighbours' densities are done
    if (it.y >= 0) {
        if (!flow_wait(fs.ddone, fs.dep_d[it.y], stamp, stamp, fs)) return;
        const int w1 = fs.wstart[it.y + 1];
        for (int w = fs.wstart[it.y] + (int)threadIdx.x; w < w1; w += kFlowThreads) wall_node<TS, LD_CG>(w, s, fs.psi_next);
    }
}

}  // namespace lbm
