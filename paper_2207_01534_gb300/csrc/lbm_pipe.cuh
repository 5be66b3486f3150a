// lbm_pipe.cuh -- the single-pass schedule: one persistent launch per time
// step that collides and streams every fluid node (F), computes the densities
// of the next step (D, including the open-plane extrapolation) right behind
// it while the freshly written populations are still in L2, and then the wall
// virtual densities (W).  Populations are read from DRAM once per step.
//
// Ordering.  F(k) reads only data written by earlier launches.  D(c) reads
// populations that F of neighbouring chunks wrote in this launch, so it waits
// for their chunk flags (acquire) and reads with L2-only loads; F publishes its
// flag after a block barrier and a device fence (release).  W(c) waits for D
// the same way.  Every wait is bounded: after kPipeMaxPolls polls it sets the
// abort word and a timeout bit in the host-mapped status word, and all blocks
// stop at their next ticket.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Publish a phase of this block for chunk c: every thread's stores are
// ordered before the flag by the barrier and the device-scope fence.
__device__ __forceinline__ void publish(int *flags, int c, int epoch)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release(flags + c, epoch);
    }
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Wait until every chunk <= hi of a phase has published `epoch` in flags.
// front holds (epoch << 32) | f, meaning all chunks below f are known done in
// that epoch; the fast path is one load of it.  Otherwise the whole block
// scans flags[f .. hi] with independent acquire loads, advances front to the
// first chunk not done (atomicMax: front only grows), and retries after a
// short sleep.  Returns false after a timeout or an abort (block-uniform).
__device__ __forceinline__ bool wait_upto(const int *flags, unsigned long long *front, int hi, int epoch,
                                          const PipeState &ps, int *sh)
{
    const unsigned long long tag = (unsigned long long)(unsigned)epoch << 32;
    for (int it = 0; it < kPipeMaxPolls; ++it) {
        if (threadIdx.x == 0) {
            const unsigned long long f = ld_acquire64(front);
            sh[0] = (f & 0xffffffff00000000ULL) == tag ? (int)(f & 0xffffffffULL) : 0;
            sh[1] = 0x7fffffff;
            sh[2] = *(volatile int *)ps.abort;
        }
        __syncthreads();
        const int lo = sh[0];
        if (lo > hi) return true;
        if (sh[2]) break;
        int bad = 0x7fffffff;
        for (int m = lo + threadIdx.x; m <= hi; m += blockDim.x)
            if (ld_acquire(flags + m) < epoch) bad = min(bad, m);
        if (bad != 0x7fffffff) atomicMin(&sh[1], bad);
        __syncthreads();
        const int first_bad = sh[1];
        if (threadIdx.x == 0) atomicMax(front, tag | (unsigned)(first_bad == 0x7fffffff ? hi + 1 : first_bad));
        if (first_bad == 0x7fffffff) {
            __syncthreads();  // sh is rewritten by the next call
            return true;
        }
        __nanosleep(128);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicExch(ps.abort, 1);
        atomicOr(ps.status, 4);
    }
    __syncthreads();
    return false;
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

template <typename TS, int P>
__global__ void __launch_bounds__(kChunk, PipeOcc<TS>::blocks) k_pipe(DevState s, PipeState ps)
{
    __shared__ int sh_k;
    __shared__ int sh_w[3];
    for (;;) {
        if (threadIdx.x == 0)
            sh_k = *(volatile int *)ps.abort ? ps.tickets : (int)(atomicAdd(ps.counter, 1ULL) - ps.base);
        __syncthreads();
        const int k = sh_k;
        if (k >= ps.tickets) return;  // the same value in every thread of the block
        if (k < ps.n_chunks) {
            const int n = k * kChunk + threadIdx.x;
            if (n < s.n_fluid) fused_node<TS, P>(n, s);
            publish(ps.flag_f, k, ps.epoch);
        }
        const int c = k - ps.lag_d;
        if (c >= 0 && c < ps.n_chunks) {
            if (!wait_upto(ps.flag_f, ps.front, ps.dep_f[c].y, ps.epoch, ps, sh_w)) return;
            const int n = c * kChunk + threadIdx.x;
            if (n < s.n_fluid) dens_node<TS, 1 - P>(n, s, ps.psi_next);
            publish(ps.flag_d, c, ps.epoch);
        }
        const int cw = k - ps.lag_w;
        if (cw >= 0 && cw < ps.n_chunks) {
            if (!wait_upto(ps.flag_d, ps.front + 1, ps.dep_d[cw].y, ps.epoch, ps, sh_w)) return;
            for (int w = ps.wstart[cw] + threadIdx.x; w < ps.wstart[cw + 1]; w += kChunk)
                wall_node<TS, true>(w, s, ps.psi_next);
        }
        __syncthreads();  // sh_k is rewritten at the top
    }
}

}  // namespace lbm
