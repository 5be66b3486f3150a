// lbm_brick.cuh -- the brick schedule: one launch per time step does the
// whole update of Section 2 (densities, Eqs. 3, 11; wall densities, Eqs.
// 14-15; forces, Eqs. 10-13; collision, Eqs. 1-2, 6-9; A-A streaming with
// bounce-back), plus a small pass over the open planes.
//
// The lattice is cut into bricks of 8 x 8 x 8 voxels and the fluid nodes are
// numbered brick by brick (voxel order inside a brick), so the nodes of a
// brick are one contiguous range.  One block works on one brick:
//
//   1. It stages the densities of this step over the brick and a two-voxel
//      halo (12^3 cells) from the fixed-point accumulator of the step into
//      shared memory, and marks the fluid cells of the one-voxel halo region
//      (10^3 cells).
//   2. It computes the virtual density of every wall voxel of the one-voxel
//      region (Eq. 15) from the staged densities of its fluid neighbours, in
//      shared memory: no separate wall pass.
//   3. Every fluid node of the brick is collided and streamed exactly as in
//      the split schedule (same per-node functions), its force stencil read
//      from shared memory.  Each post-collision population is then added into
//      a shared-memory fixed-point accumulator of the cell it streams into
//      (x + e_j when that is fluid, x itself when solid: half-way
//      bounce-back; none when it leaves through an open plane).
//   4. The accumulator goes out once per cell: cells at least one voxel
//      inside the brick receive nothing from other bricks and are stored;
//      the others (brick faces and the halo) are added atomically into the
//      next step's accumulator.
//
// After the launch the plane pass applies the open-plane rule to the plane
// nodes and stores their densities as totals.  The next step's densities are
// thus formed while the populations are in registers; nothing re-reads them.
//
// Accumulators (lbm_fixed.cuh) rotate over three dense buffers as in the push
// schedule: step t stages buffer t % 3, adds into (t + 1) % 3, and clears
// its face nodes' voxels of (t + 2) % 3.  Only fluid voxels are ever written,
// so solid voxels hold zero, and a fluid voxel's total (19 biased
// contributions) is never zero: a staged cell is fluid exactly when its word
// is non-zero.
#pragma once

#include "lbm_fixed.cuh"
#include "lbm_kernels.cuh"

namespace lbm {

// cell offsets of direction i in the two staged regions
__host__ __device__ constexpr int d1(int i) { return ez(i) * kR1 * kR1 + ey(i) * kR1 + ex(i); }
__host__ __device__ constexpr int d2(int i) { return ez(i) * kR2 * kR2 + ey(i) * kR2 + ex(i); }

// Global coordinate along one axis of length n of a brick-local position g
// (-1: outside a non-periodic axis).  Positions are at most two voxels
// outside the domain, so one period fixes them unless the axis is shorter
// than that.
__device__ __forceinline__ int wrap_axis(int g, int n, bool periodic)
{
    if (g >= 0 && g < n) return g;
    if (!periodic) return -1;
    g += g < 0 ? n : -n;
    if (g >= 0 && g < n) return g;
    g %= n;
    return g < 0 ? g + n : g;
}

// Asynchronous 8-byte global -> shared copy (completes at cp_async_wait).
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename TS, int P>
__global__ void __launch_bounds__(kBrickThreads, kBrickBlocks) k_brick(DevState s, BrickBufs bb)
{
    using C = float;
    using C2 = float2;
    __shared__ float2 ps[kR2Cells];     // densities (walls: virtual densities), brick + 2
    __shared__ uint32_t a1[kR1Cells];   // next-step accumulators, component 1
    __shared__ uint32_t a2[kR1Cells];   // component 2
    __shared__ uint8_t fluid[kR1Cells];
    pdl_trigger();
    const BrickInfo bi = bb.info[blockIdx.x];
    const int bx = bi.ext & 255, by = (bi.ext >> 8) & 255, bz = bi.ext >> 16;
    for (int k = threadIdx.x; k < kR1Cells; k += kBrickThreads) {
        a1[k] = 0u;
        a2[k] = 0u;
    }
    pdl_wait();
    // 1. stage the accumulator words of brick + 2 with asynchronous copies
    //    (zero outside the domain), then decode each in place
    unsigned long long *raw = reinterpret_cast<unsigned long long *>(ps);
    for (int k = threadIdx.x; k < kR2Cells; k += kBrickThreads) {
        const int lx = k % kR2 - 2, ly = (k / kR2) % kR2 - 2, lz = k / (kR2 * kR2) - 2;
        const bool in2 = lx < bx + 2 && ly < by + 2 && lz < bz + 2;
        const int gx = in2 ? wrap_axis(bi.x0 + lx, s.nx, bb.per & 1) : -1;
        const int gy = in2 ? wrap_axis(bi.y0 + ly, s.ny, bb.per & 2) : -1;
        const int gz = in2 ? wrap_axis(bi.z0 + lz, s.nz, bb.per & 4) : -1;
        if (gx >= 0 && gy >= 0 && gz >= 0)
            cp_async8(raw + k, bb.rd + (gx + s.sx * gy + (long long)s.sxy * gz));
        else
            raw[k] = 0ull;
    }
    // this thread's wall entry of step 2, loaded while the copies run
    const int e0 = bi.w0 + (int)threadIdx.x;
    uint32_t wc0 = 0u;
    float2 co0 = make_float2(0.f, 0.f);
    if (e0 < bi.w1) {
        wc0 = __ldg(bb.wcell + e0);
        co0 = __ldg(bb.wcoef + e0);
    }
    cp_async_wait();
    for (int k = threadIdx.x; k < kR2Cells; k += kBrickThreads) {
        const unsigned long long w = raw[k];
        ps[k] = w ? fix_dec2(w) : make_float2(0.f, 0.f);
        // every cell of the one-voxel region gets a mark; cells past a
        // clipped brick's extent are never targets and are marked solid
        const int lx = k % kR2 - 2, ly = (k / kR2) % kR2 - 2, lz = k / (kR2 * kR2) - 2;
        if (lx >= -1 && ly >= -1 && lz >= -1 && lx <= kBrick && ly <= kBrick && lz <= kBrick)
            fluid[(lz + 1) * kR1 * kR1 + (ly + 1) * kR1 + (lx + 1)] =
                (w && lx <= bx && ly <= by && lz <= bz) ? 1 : 0;
    }
    __syncthreads();
    // 2. wall voxels of brick + 1 (Eq. 15); they read fluid cells only
    for (int e = e0; e < bi.w1; e += kBrickThreads) {
        const uint32_t wc = e == e0 ? wc0 : __ldg(bb.wcell + e);
        const float2 co = e == e0 ? co0 : __ldg(bb.wcoef + e);
        const int c1 = (int)(wc >> 20);
        const int c2 = (c1 / (kR1 * kR1) + 1) * kR2 * kR2 + ((c1 / kR1) % kR1 + 1) * kR2 + (c1 % kR1 + 1);
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 1; j < 19; ++j)
            if (wc & (1u << j)) a = fma2(bc2<float2>(wgt<float>(j)), ps[c2 + d2(j)], a);
        ps[c2] = mul2(a, co);
    }
    __syncthreads();
    // 3. collide and stream the brick's nodes; accumulate the next densities
    for (int n = bi.n0 + (int)threadIdx.x; n < bi.n1; n += kBrickThreads) {
        const uint32_t pv = s.pvox[n];
        const uint32_t fl = s.nflags[n];
        const int loc = __ldg(bb.nloc + n);
        const int lx = loc & 7, ly = (loc >> 3) & 7, lz = loc >> 6;
        const int c1 = (lz + 1) * kR1 * kR1 + (ly + 1) * kR1 + (lx + 1);
        const int c2 = (lz + 2) * kR2 * kR2 + (ly + 2) * kR2 + (lx + 2);
        const Nbr b = make_nbr(fl, s);
        C2 f[19], dm;
        load_pops<TS, P>(f, dm, n, pv, fl, b, s);
        const C2 rho = density_of<TS>(dm, s);
        C2 F[3];
        {
            C2 a[3] = {mk2(C(0), C(0)), mk2(C(0), C(0)), mk2(C(0), C(0))};
#pragma unroll
            for (int j = 1; j < 19; ++j) {
                const int off = (ez(j) != 0 && outside(j, fl)) ? d2(mirz(j)) : d2(j);
                const C2 d = sub2(ps[c2 + off], rho);
                const C w = wgt<C>(j);
                if (ex(j)) a[0] = fma2(bc2<C2>(w * ex(j)), d, a[0]);
                if (ey(j)) a[1] = fma2(bc2<C2>(w * ey(j)), d, a[1]);
                if (ez(j)) a[2] = fma2(bc2<C2>(w * ez(j)), d, a[2]);
            }
            const C mG = -pick<C>(s.G, s.fG);
            const C g[3] = {pick<C>(s.gx, s.fgx), pick<C>(s.gy, s.fgy), pick<C>(s.gz, s.fgz)};
#pragma unroll
            for (int k = 0; k < 3; ++k) F[k] = mul2(rho, fma2(bc2<C2>(mG), mk2(a[k].y, a[k].x), bc2<C2>(g[k])));
        }
        C u[3], inv_rho;
        mix_velocity<C, C2>(f, rho, F, s, inv_rho, u);
        collide<C, C2>(f, rho, inv_rho, u, F, s);
        store_pops<TS, P, true>(f, dm, n, pv, fl, b, s);  // f: the stored values
        uint32_t s1 = fix_enc(f[0].x), s2 = fix_enc(f[0].y);
#pragma unroll
        for (int j = 1; j < 19; ++j) {
            if (ez(j) != 0 && outside(j, fl)) continue;  // leaves the domain
            const uint32_t e1 = fix_enc(f[j].x), e2 = fix_enc(f[j].y);
            const int t = c1 + d1(j);
            if (fluid[t]) {
                atomicAdd(&a1[t], e1);
                atomicAdd(&a2[t], e2);
            } else {  // bounced back into x
                s1 += e1;
                s2 += e2;
            }
        }
        atomicAdd(&a1[c1], s1);
        atomicAdd(&a2[c1], s2);
        const bool inner = lx >= 1 && ly >= 1 && lz >= 1 && lx <= bx - 2 && ly <= by - 2 && lz <= bz - 2;
        if (!inner) bb.clr[pv] = 0ull;
    }
    __syncthreads();
    // 4. write out: inner cells whole, face and halo cells atomically
    for (int k = threadIdx.x; k < kR1Cells; k += kBrickThreads) {
        if (!fluid[k]) continue;
        const unsigned long long w = (unsigned long long)a1[k] | ((unsigned long long)a2[k] << 32);
        const int lx = k % kR1 - 1, ly = (k / kR1) % kR1 - 1, lz = k / (kR1 * kR1) - 1;
        const int gx = wrap_axis(bi.x0 + lx, s.nx, bb.per & 1);
        const int gy = wrap_axis(bi.y0 + ly, s.ny, bb.per & 2);
        const int gz = wrap_axis(bi.z0 + lz, s.nz, bb.per & 4);
        unsigned long long *q = bb.acc + (gx + s.sx * gy + (long long)s.sxy * gz);
        const bool inner = lx >= 1 && ly >= 1 && lz >= 1 && lx <= bx - 2 && ly <= by - 2 && lz <= bz - 2;
        if (inner) *q = w;
        else if (w) atomicAdd(q, w);
    }
}

// Plane nodes after the brick launch: the open-plane rule at the parity PN of
// the next step, then the node's density from its populations as a total.
template <typename TS, int PN>
__global__ void __launch_bounds__(128) k_plane_acc(DevState s, unsigned long long *acc)
{
    using C2 = typename Traits<TS>::C2;
    pdl_trigger();
    pdl_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * s.nxy) return;
    const int plane = t >= s.nxy ? 1 : 0;
    const int p = t - plane * s.nxy;
    const uint32_t pvb = plane == 0 ? (uint32_t)p : (uint32_t)(p + (s.nz - 1) * s.sxy);
    const int nb = s.cidx[pvb];
    if (nb < 0) return;
    const uint32_t flb = s.nflags[nb];
    neem_node<TS, PN, LD_NC>(plane, p, nb, pvb, flb, s);
    const Nbr b = make_nbr(flb, s);
    C2 f[19], dm;
    // coherent loads: this thread has just written these cells
    load_pops<TS, PN, LD_CA>(f, dm, nb, pvb, flb, b, s);
    acc[pvb] = fix_total2(density_of<TS>(dm, s));
}

// New wall coefficients ((1 + xi) / W, (1 - xi) / W) of the brick wall
// entries after a change of the xi field.
template <typename CW>
__global__ void k_brick_coef(const int32_t *wid, int n, const CW *winv, const CW *wxi, float2 *coef)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float inv = (float)winv[wid[e]], xi = (float)wxi[wid[e]];
    coef[e] = make_float2((1.f + xi) * inv, (1.f - xi) * inv);
}

}  // namespace lbm
