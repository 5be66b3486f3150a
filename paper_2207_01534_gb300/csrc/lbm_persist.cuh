// lbm_persist.cuh -- a batch of independent lattices stepped by one
// persistent cooperative launch for many time steps.  Every block of the
// launch is resident (cooperative launch); for each step the launch runs the
// three passes of the split schedule over all samples of the batch table --
// densities with the open-plane rule (Eqs. 3, 11; Section 2), virtual wall
// densities (Eq. 15), then force, collision and A-A streaming (Eqs. 1-2, 6-11,
// 13) -- separated by grid-wide barriers.  The blocks deal the batch's node
// and wall blocks among themselves (virtual block vb = blockIdx.x,
// blockIdx.x + gridDim.x, ...), with the node and sample of a virtual block
// found in the parameter-space table exactly as the table passes find them,
// so every node gets the arithmetic of its solo run and each sample's results
// are bitwise those of the same lattice stepped alone.
//
// Data written earlier in the same launch is read with coherent loads (never
// through the read-only path).  Each barrier wait is bounded by the global
// timer; a block that gives up sets the timeout bit of the status word and
// the abort word and returns, and every other block then gives up at its
// next wait, so the launch always ends.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_pipe.cuh"

namespace lbm {

// Barrier of all gridDim.x blocks: thread 0 of each block publishes its
// block's writes (device-scope fence), counts the block in, and waits with
// acquire loads for the count of this barrier.  Returns false (block-uniform)
// when the wait gave up or another block did.
__device__ __forceinline__ bool grid_barrier(const PersistArgs &pa, unsigned long long &target, bool arrive = true)
{
    __shared__ int ok_sh;
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        int ok = 1;
        if (arrive) {
            __threadfence();
            atomicAdd(pa.bar, 1ull);
        }
        const unsigned long long t0 = global_ns();
        int backoff = 32;
        for (int it = 0;; ++it) {
            if (ld_acquire64(pa.bar) >= target) break;
            if (*(volatile int *)pa.abort || global_ns() - t0 > pa.wait_ns || it >= kPipeMaxPolls) {
                atomicExch(pa.abort, 1);
                atomicOr(pa.status, 4);
                ok = 0;
                break;
            }
            __nanosleep(backoff);
            backoff = min(backoff * 2, 256);
        }
        __threadfence();  // the other blocks' writes before any load of this block's threads
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

template <typename TS, int P>
__device__ __forceinline__ void persist_dens(const BatchTable &t, int neem)
{
    const int nbn = t.start_n[t.count];
    for (int vb = blockIdx.x; vb < nbn; vb += gridDim.x) {
        // last node of the last sample first, as k_dens_table
        const int rb = nbn - 1 - vb;
        const int k = table_sample(t.start_n, t.count, rb);
        const DevState &s = t.s[k];
        const int n = (rb - t.start_n[k]) * (int)blockDim.x + (int)threadIdx.x;
        if (n < s.n_fluid) dens_node_geo<TS, P, LD_CA>(n, s.pvox[n], s.nflags[n], s, neem && s.open_z);
    }
}

template <typename TS>
__device__ __forceinline__ void persist_wall(const BatchTable &t)
{
    const int nbw = t.start_w[t.count];
    for (int vb = blockIdx.x; vb < nbw; vb += gridDim.x) {
        const int k = table_sample(t.start_w, t.count, vb);
        const DevState &s = t.s[k];
        const int w = (vb - t.start_w[k]) * (int)blockDim.x + (int)threadIdx.x;
        if (w < s.n_wall) wall_node<TS, LD_CG>(w, s, s.psi);
    }
}

template <typename TS, int P>
__device__ __forceinline__ void persist_fused(const BatchTable &t, unsigned *rec)
{
    const int nbn = t.start_n[t.count];
    for (int vb = blockIdx.x; vb < nbn; vb += gridDim.x) {
        const int k = table_sample(t.start_n, t.count, vb);
        const DevState &s = t.s[k];
        const int n = (vb - t.start_n[k]) * (int)blockDim.x + (int)threadIdx.x;
        if (n < s.n_fluid)
            fused_node_geo<TS, P, true, LD_CA>(n, s.pvox[n], s.nflags[n], s, rec + threadIdx.x, (int)blockDim.x);
    }
}

template <typename TS>
__global__ void __launch_bounds__(256, PipeOcc<TS>::blocks) k_persist(const __grid_constant__ BatchTable t,
                                                                       PersistArgs pa)
{
    extern __shared__ unsigned slot_rec[];  // slot_rec_bytes(1, blockDim.x)
    unsigned long long target = pa.base;
    for (int q = 0; q < pa.steps; ++q) {
        const long long step = pa.step0 + q;
        const int neem = step > 0;
        if (step & 1) persist_dens<TS, 1>(t, neem);
        else persist_dens<TS, 0>(t, neem);
        if (!grid_barrier(pa, target, !(pa.stall && q == 0 && blockIdx.x == 0))) return;
        persist_wall<TS>(t);
        if (!grid_barrier(pa, target)) return;
        if (step & 1) persist_fused<TS, 1>(t, slot_rec);
        else persist_fused<TS, 0>(t, slot_rec);
        if (!grid_barrier(pa, target)) return;
    }
}

}  // namespace lbm
