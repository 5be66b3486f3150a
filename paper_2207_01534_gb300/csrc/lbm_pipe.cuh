// lbm_pipe.cuh -- the single-pass schedule: one persistent launch per time
// step.  Blocks claim chunks of three kinds of work:
//   F(c)  collide and stream the fluid nodes of chunk c,
//   D(c)  next-step densities of chunk c (open-plane extrapolation first for
//         plane nodes), read back while F's output is still in L2,
//   W(c)  virtual densities of the walls between fluid chunks c and c+1.
// D(c) may start once F is done for every chunk <= need_f[c]; W(c) once D is
// done for every chunk <= need_d[c].  A block prefers a ready W, then a ready
// D, then the next F; it never waits inside a phase.
//
// Ordering.  A phase publishes its chunk flag after a block barrier and a
// device-scope fence (release).  Completion frontiers ("every chunk below f
// is done") advance in order through the flags, with a fence before each
// update, and are read with acquire loads; data written in this launch is read
// with L2-only loads.  Idle polling is bounded: after kPipeMaxIdle polls
// without work a block sets the abort word and the timeout status bit, and
// every block stops.
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

constexpr unsigned long long kLo = 0xffffffffULL;

// Count part of an epoch-tagged word (0 when the word belongs to an older launch).
__device__ __forceinline__ int tagged_count(unsigned long long v, unsigned long long tag)
{
    return (v & ~kLo) == tag ? (int)(v & kLo) : 0;
}

// Move a completion frontier forward over consecutive finished chunks.
// Called by a whole warp: each round the 32 lanes check 32 flags at once and
// lane 0 jumps the frontier over the finished prefix with one fenced CAS.
__device__ __forceinline__ void advance_front(unsigned long long *front, const int *flags, unsigned long long tag,
                                              int epoch, int n_chunks)
{
    const int lane = threadIdx.x & 31;
    for (int round = 0; round < 16; ++round) {
        const unsigned long long v = ld_acquire64(front);
        const int f = tagged_count(v, tag);
        if (f >= n_chunks) return;
        const int m = f + lane;
        const bool done = m >= n_chunks || ld_acquire(flags + m) >= epoch;
        const unsigned ballot = __ballot_sync(0xffffffffu, done);
        const int run = ballot == 0xffffffffu ? 32 : __ffs(~ballot) - 1;  // finished prefix length
        if (run == 0) return;
        int ok = 0;
        if (lane == 0) {
            __threadfence();
            const int nf = min(f + run, n_chunks);
            ok = atomicCAS(front, v, tag | (unsigned long long)nf) == v;
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok && run < 32) return;  // stopped at an unfinished chunk
    }
}

// Claim the next chunk of a queue if it exists and is ready (ready_upto >=
// the chunk's need).  Returns the chunk or -1; *more says whether the queue
// still has unclaimed chunks.
__device__ __forceinline__ int try_claim(unsigned long long *ctr, unsigned long long tag, int n_chunks, const int *need,
                                         int ready_upto, bool *more)
{
    *more = true;
    for (int r = 0; r < 32; ++r) {  // retry when another block claimed first
        const unsigned long long v = ld_acquire64(ctr);
        const int k = tagged_count(v, tag);
        if (k >= n_chunks) {
            *more = false;
            return -1;
        }
        if (need && need[k] > ready_upto) return -1;
        if (atomicCAS(ctr, v, tag | (unsigned long long)(k + 1)) == v) return k;
    }
    return -1;
}

// Publish a phase of this block for chunk c.
__device__ __forceinline__ void publish(int *flags, int c, int epoch)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release(flags + c, epoch);
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
        neem_node<TS, PN, true>(plane, p, n, pv, fl, s);
    }
    const Nbr b = make_nbr(fl, s);
    C2 f[19];
    load_pops<TS, PN, true>(f, n, pv, fl, b, s);
    reinterpret_cast<C2 *>(psi_next)[pv] = sum19(f);
}

// Resident blocks per SM the register budget is sized for.
template <typename TS>
struct PipeOcc {
    static constexpr int blocks = 3;
};
template <>
struct PipeOcc<double> {
    static constexpr int blocks = 2;
};

enum : int { kJobNone = 0, kJobF = 1, kJobD = 2, kJobW = 3, kJobExit = 4 };

template <typename TS, int P>
__global__ void __launch_bounds__(kChunk, PipeOcc<TS>::blocks) k_pipe(DevState s, PipeState ps)
{
    __shared__ int sh_job, sh_idx;
    const unsigned long long tag = (unsigned long long)(unsigned)ps.epoch << 32;
    unsigned long long *ctr_f = ps.ctr, *ctr_d = ps.ctr + 16, *ctr_w = ps.ctr + 32;  // separate 128-byte lines
    unsigned long long *front_f = ps.front, *front_d = ps.front + 16;
    int idle = 0, backoff = 64;
    for (;;) {
        if (threadIdx.x == 0) {
            int job = kJobNone, idx = -1;
            if (*(volatile int *)ps.abort) {
                job = kJobExit;
            } else {
                const int fd = tagged_count(ld_acquire64(front_d), tag);  // D done below fd
                const int ff = tagged_count(ld_acquire64(front_f), tag);  // F done below ff
                bool more_w, more_d, more_f;
                idx = try_claim(ctr_w, tag, ps.n_chunks, ps.need_d, fd - 1, &more_w);
                if (idx >= 0) {
                    job = kJobW;
                } else {
                    idx = try_claim(ctr_d, tag, ps.n_chunks, ps.need_f, ff - 1, &more_d);
                    if (idx >= 0) {
                        job = kJobD;
                    } else {
                        idx = try_claim(ctr_f, tag, ps.n_chunks, nullptr, 0, &more_f);
                        if (idx >= 0) job = kJobF;
                        else if (!more_w && !more_d && !more_f) job = kJobExit;
                    }
                }
            }
            sh_job = job;
            sh_idx = idx;
        }
        __syncthreads();
        const int job = sh_job, idx = sh_idx;
        __syncthreads();
        if (job == kJobExit) return;
        if (job == kJobNone) {
            // nothing ready yet: help the frontiers along, then back off
            if (threadIdx.x < 32) {
                advance_front(front_f, ps.flag_f, tag, ps.epoch, ps.n_chunks);
                advance_front(front_d, ps.flag_d, tag, ps.epoch, ps.n_chunks);
            }
            if (threadIdx.x == 0 && ++idle > kPipeMaxIdle) {
                atomicExch(ps.abort, 1);
                atomicOr(ps.status, 4);
            }
            __nanosleep(backoff);
            backoff = min(backoff * 2, 2048);
            continue;
        }
        backoff = 64;
        idle = 0;
        if (job == kJobF) {
            const int n = idx * kChunk + threadIdx.x;
            if (n < s.n_fluid) fused_node<TS, P>(n, s);
            publish(ps.flag_f, idx, ps.epoch);
            if (threadIdx.x < 32) advance_front(front_f, ps.flag_f, tag, ps.epoch, ps.n_chunks);
        } else if (job == kJobD) {
            const int n = idx * kChunk + threadIdx.x;
            if (n < s.n_fluid) dens_node<TS, 1 - P>(n, s, ps.psi_next);
            publish(ps.flag_d, idx, ps.epoch);
            if (threadIdx.x < 32) advance_front(front_d, ps.flag_d, tag, ps.epoch, ps.n_chunks);
        } else {
            for (int w = ps.wstart[idx] + threadIdx.x; w < ps.wstart[idx + 1]; w += kChunk)
                wall_node<TS, true>(w, s, ps.psi_next);
        }
    }
}

}  // namespace lbm
