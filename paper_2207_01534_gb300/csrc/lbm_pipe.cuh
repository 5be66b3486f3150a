// lbm_pipe.cuh -- the single-pass schedule: one cooperative launch per time
// step.  Blocks work through chunks of three kinds of work, dealt round-robin:
//   F(c)  collide and stream the fluid nodes of chunk c,
//   D(c)  next-step densities of chunk c (open-plane extrapolation first for
//         plane nodes), read back while F's output is still in L2,
//   W(c)  virtual densities of the walls between fluid chunks c and c+1.
// D(c) may start once F is done for every chunk <= need_f[c]; W(c) once D is
// done for every chunk <= need_d[c] (see PipeState for the round structure).
//
// Ordering.  Each warp counts itself into a round's completion counters after
// its own stores and a device-scope fence; waiting warps read the counters
// with acquire loads; data written in this launch is read
// with L2-only loads.  Waits are bounded: after ps.wait_ns (global timer) a
// block sets the abort word and the timeout status bit, and every block stops.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Round counters are split into kWarps sub-counters (one per warp slot of a
// block, 128 bytes apart): warp w of every block adds 1 to sub-counter w of
// the round when its 32 nodes are done.  A round is complete in launch e when
// every sub-counter has reached e * G.
constexpr int kWarps = kChunk / 32;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (one warp) until round `r` of counter array `ctr` is complete.
// Returns false after a timeout (ps.wait_ns of the global timer, or
// kPipeMaxPolls polls) or an abort by another block (warp-uniform).
__device__ __forceinline__ bool wait_round(const unsigned long long *ctr, int r, unsigned long long target,
                                           const PipeState &ps)
{
    const int lane = threadIdx.x & 31;
    int backoff = 32;
    const unsigned long long t0 = __shfl_sync(0xffffffffu, global_ns(), 0);
    for (int it = 0; it < kPipeMaxPolls; ++it) {
        const bool mine = lane >= kWarps || ld_acquire64(ctr + 16 * (r * kWarps + lane)) >= target;
        if (__all_sync(0xffffffffu, mine)) return true;
        if (*(volatile int *)ps.abort) break;
        const unsigned long long t = __shfl_sync(0xffffffffu, global_ns(), 0);
        if (t - t0 > ps.wait_ns) break;
        __nanosleep(backoff);
        backoff = min(backoff * 2, 512);
    }
    if (lane == 0) {
        atomicExch(ps.abort, 1);
        atomicOr(ps.status, 4);
    }
    return false;
}

// Count this warp into round r once its lanes' stores are done.
__device__ __forceinline__ void finish_round(unsigned long long *ctr, int r)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        __threadfence();
        atomicAdd(ctr + 16 * (r * kWarps + (threadIdx.x >> 5)), 1ULL);
    }
}

// D: open-plane extrapolation (plane nodes) then the density pair of one node
// at the parity PN of the next step, into psi_next.
template <typename TS, int PN>
__device__ __forceinline__ void dens_node(int n, const DevState &s, void *psi_next)
{
    using C2 = typename Traits<TS>::C2;
    const uint32_t pv = s.pvox[n];
    const uint32_t fl = s.nflags[n];
    if (fl & (F_INLET | F_OUTLET)) {
        const int plane = (fl & F_INLET) ? 0 : 1;
        const int p = plane == 0 ? (int)pv : (int)pv - (s.nz - 1) * s.sxy;
        neem_node<TS, PN, LD_CG>(plane, p, n, pv, fl, s);
    }
    const Nbr b = make_nbr(fl, s);
    C2 f[19], dm;
    load_pops<TS, PN, LD_CG>(f, dm, n, pv, fl, b, s);
    reinterpret_cast<C2 *>(psi_next)[pv] = density_of<TS>(dm, s);
}

template <typename TS, int P>
__global__ void __launch_bounds__(kChunk, PipeOcc<TS>::blocks) k_pipe(DevState s, PipeState ps)
{
    const int G = gridDim.x;
    const unsigned long long full = (unsigned long long)ps.epoch * (unsigned long long)G;
    for (int r = 0; r < ps.rounds; ++r) {
        if (r < ps.n_rounds) {
            const int cf = r * G + blockIdx.x;
            const int n = cf * kChunk + threadIdx.x;
            if (cf < ps.n_chunks && n < s.n_fluid) fused_node<TS, P>(n, s);
            finish_round(ps.round_f, r);
        }
        const int rd = r - ps.lag_d;
        if (rd >= 0 && rd < ps.n_rounds) {
            const int cd = rd * G + blockIdx.x;
            if (cd < ps.n_chunks) {
                if (!wait_round(ps.round_f, ps.need_f[cd] / G, full, ps)) return;
                const int n = cd * kChunk + threadIdx.x;
                if (n < s.n_fluid) dens_node<TS, 1 - P>(n, s, ps.psi_next);
            }
            finish_round(ps.round_d, rd);
        }
        const int rw = r - ps.lag_w;
        if (rw >= 0 && rw < ps.n_rounds) {
            const int cw = rw * G + blockIdx.x;
            if (cw < ps.n_chunks) {
                const int need = ps.need_d[cw];
                if (need >= 0 && !wait_round(ps.round_d, need / G, full, ps)) return;
                // this warp's share of the wall chunk
                for (int w = ps.wstart[cw] + threadIdx.x; w < ps.wstart[cw + 1]; w += kChunk)
                    wall_node<TS, LD_CG>(w, s, ps.psi_next);
            }
        }
    }
}

}  // namespace lbm
