// lbm_push.cuh -- the push schedule (FP32 storage): the collide-stream pass
// also accumulates the densities of the next step, so no separate density
// pass re-reads the populations.
//
// After the collision at node x, every post-collision population f*_j(x)
// becomes a post-stream population of exactly one node: x + e_j when that is
// an in-domain fluid voxel, x itself when it is solid (half-way bounce-back),
// and none when it leaves through an open plane; the rest population stays
// at x.  Adding each one into the density accumulator of its destination
// gives every interior node its next density (Eq. 3) as the sum of its 19
// incoming populations.  Plane nodes are finished afterwards by the finish
// pass (the open-plane rule rewrites populations there), and so are the
// walls (Eq. 15).
//
// Accumulators are integer fixed point (lbm_fixed.cuh): the sums do not
// depend on the order of the atomic adds, so results are bitwise reproducible.
//
// Three accumulator buffers rotate: the collide-stream pass of step t reads
// buffer t % 3 in its force stencil and adds into (t + 1) % 3; the finish
// pass of step t completes (t + 1) % 3 and clears (t + 2) % 3, which the
// pass of step t - 1 has finished reading and the pass of step t + 1 adds
// into.
#pragma once

#include "lbm_fixed.cuh"
#include "lbm_kernels.cuh"

namespace lbm {

__device__ __forceinline__ unsigned long long ld_pol(const unsigned long long *q, unsigned long long pol)
{
    unsigned long long v;
    asm("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(q), "l"(pol));
    return v;
}

// The stencil sum_i w_i psi(x + e_i) e_i of Eqs. 10 and 13 for both
// components, from the accumulator densities, in integer arithmetic: with
// the weights scaled by 36 (2 on faces, 1 on edges) every term is an integer
// multiple of the encoded word, the per-voxel offsets of the encoding cancel
// because sum_i w_i e_i = 0 (which also makes the mirrored reads beyond an
// open plane harmless), and wrap-around in 32 bits cannot change the result
// because the exact sum is below 2^31 in magnitude (at most 6 * 2^26 times
// the largest density, and the encoding itself holds densities below 4.5).
// The sum is exact; one conversion per axis and component follows, where
// decoding every neighbour would take 36.
__device__ __forceinline__ void stencil_acc(uint32_t pv, uint32_t fl, const Nbr &b, const unsigned long long *rd,
                                            float2 a[3])
{
    const unsigned long long *q = rd + pv;
    const unsigned long long pol = l2_policy();
    uint32_t sx[3] = {0u, 0u, 0u}, sy[3] = {0u, 0u, 0u};
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        const int off = (ez(j) != 0 && outside(j, fl)) ? nb_off(mirz(j), b) : nb_off(j, b);
        const unsigned long long w = ld_pol(q + off, pol);
        const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
        const uint32_t m = (ex(j) != 0) + (ey(j) != 0) + (ez(j) != 0) == 1 ? 2u : 1u;
        const int e[3] = {ex(j), ey(j), ez(j)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (e[k] > 0) { sx[k] += m * lo; sy[k] += m * hi; }
            if (e[k] < 0) { sx[k] -= m * lo; sy[k] -= m * hi; }
        }
    }
    const float sc = 1.0f / (36.0f * (float)(1 << kFixShift));
#pragma unroll
    for (int k = 0; k < 3; ++k) a[k] = make_float2((float)(int)sx[k] * sc, (float)(int)sy[k] * sc);
}

__device__ __forceinline__ float2 shfl_up2(float2 v)
{
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float2 shfl_down2(float2 v)
{
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}

// D3Q19 direction with velocity (x, y, z)
// Atomic add into an accumulator under an evict-last L2 policy: the lines
// are read again by the next step's force stencil and wall pass, while the
// populations stream through L2 in between.
__device__ __forceinline__ void red_acc(unsigned long long *p, unsigned long long v, unsigned long long pol)
{
    asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}

__host__ __device__ constexpr int dir_of(int x, int y, int z)
{
    int d = -1;
    for (int i = 0; i < 19; ++i)
        if (ex(i) == x && ey(i) == y && ez(i) == z) d = i;
    return d;
}

// Pushes of the row group (Y, Z): the directions (0, Y, Z), (1, Y, Z) and
// (-1, Y, Z) of one node land in one x row of destinations.  When the
// previous lane of the warp holds the node's -x neighbour (left) its
// (1, Y, Z) population lands where this node's (0, Y, Z) one does, and the
// next lane's (-1, Y, Z) one likewise when it holds the +x neighbour (right):
// the three are added here into one atomic.  A population whose destination
// is solid was bounced into the node's own total (self) beforehand; one that
// leaves through an open plane is dropped.  The sum of k populations carries
// k encoding biases, so every voxel still receives exactly 19.
template <int Y, int Z>
__device__ __forceinline__ void push_row(const float2 f[19], uint32_t nm, bool live, bool left, bool right,
                                         uint32_t pv, const Nbr &b, unsigned long long *acc, unsigned long long pol)
{
    constexpr int j0 = dir_of(0, Y, Z), jp = dir_of(1, Y, Z), jm = dir_of(-1, Y, Z);
    const float2 up = shfl_up2(f[jp]);
    const float2 dn = shfl_down2(f[jm]);
    if (!live) return;
    if (nm & (1u << j0)) {
        float2 t = f[j0];
        uint32_t k = 1;
        if (left) { t = add2(t, up); ++k; }
        if (right) { t = add2(t, dn); ++k; }
        red_acc(acc + ((int)pv + nb_off(j0, b)), fix_enc2n(t, k), pol);
    }
    if ((nm & (1u << jp)) && !right) red_acc(acc + ((int)pv + nb_off(jp, b)), fix_enc2n(f[jp], 1), pol);
    if ((nm & (1u << jm)) && !left) red_acc(acc + ((int)pv + nb_off(jm, b)), fix_enc2n(f[jm], 1), pol);
}

// directions that leave through the inlet (e_z < 0) and the outlet (e_z > 0)
constexpr uint32_t dir_mask_z(int sign)
{
    uint32_t m = 0;
    for (int j = 1; j < 19; ++j)
        if (ez(j) * sign > 0) m |= 1u << j;
    return m;
}
constexpr uint32_t kLeaveIn = dir_mask_z(-1), kLeaveOut = dir_mask_z(1);

// Collide-stream pass of the push schedule.  The force stencil reads the
// accumulator densities of this step first (stencil_acc); the node's own
// density for the collision is the sum of its loaded populations (so the
// collision conserves the stored mass as in the split passes).  After the
// stores, every post-collision population goes into the accumulator of the
// node it becomes a post-stream population of, combined across the lanes of
// a warp that hold x-neighbours (push_row): one atomic per destination row
// instead of one per population where the fluid runs along x.
template <int P>
__global__ void __launch_bounds__(256, 3) k_fused_push(DevState s, PushBufs pb)
{
    using TS = float;
    pdl_trigger();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = n < s.n_fluid;
    // a lane past the last node gets a voxel no node's -x neighbour can have
    const uint32_t pv = live ? s.pvox[n] : 0xfffffffeu;
    const uint32_t fl = live ? s.nflags[n] : 0u;
    const uint32_t nm = live ? pb.nmask[n] : 0u;
    pdl_wait();
    float2 f[19];
    if (live) {
        const Nbr b = make_nbr(fl, s);
        float2 a[3];
        stencil_acc(pv, fl, b, pb.rd, a);
        float2 dm;
        load_pops<TS, P>(f, dm, n, pv, fl, b, s);
        const float2 rho = dm;
        const float mG = -s.fG;
        const float g[3] = {s.fgx, s.fgy, s.fgz};
        float2 F[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) F[k] = mul2(rho, fma2(bc2<float2>(mG), make_float2(a[k].y, a[k].x), bc2<float2>(g[k])));
        float u[3], inv_rho;
        mix_velocity<float, float2>(f, rho, F, s, inv_rho, u);
        collide<float, float2>(f, rho, inv_rho, u, F, s);
        store_pops<TS, P>(f, dm, n, pv, fl, b, s);
    } else {
#pragma unroll
        for (int j = 0; j < 19; ++j) f[j] = make_float2(0.f, 0.f);
    }
    const int lane = (int)(threadIdx.x & 31u);
    const uint32_t pv_prev = __shfl_up_sync(0xffffffffu, pv, 1);
    // the previous lane holds this node's -x neighbour in the same row (at
    // x = 0 of a periodic row the -x neighbour wraps to the row's end)
    const bool left = live && lane > 0 && pv_prev + 1u == pv && !(fl & F_XLO);
    const uint32_t lm = __ballot_sync(0xffffffffu, left);
    const bool right = lane < 31 && ((lm >> (lane + 1)) & 1u);
    const Nbr b = make_nbr(fl, s);
    const unsigned long long pol = l2_policy();
    // the rest population and every bounced one stay at x: the bounced
    // directions are those whose destination is neither fluid nor beyond an
    // open plane
    const uint32_t leave = ((fl & F_INLET) ? kLeaveIn : 0u) | ((fl & F_OUTLET) ? kLeaveOut : 0u);
    const uint32_t bounce = ~(nm | leave) & 0x7fffeu;
    float2 self = f[0];
#pragma unroll
    for (int j = 1; j < 19; ++j)
        if (bounce & (1u << j)) self = add2(self, f[j]);
    uint32_t kself = 1u + (uint32_t)__popc(bounce);
    // row (0, 0): the node itself with the +x population of the left lane and
    // the -x one of the right lane
    {
        constexpr int jp = dir_of(1, 0, 0), jm = dir_of(-1, 0, 0);
        const float2 up = shfl_up2(f[jp]);
        const float2 dn = shfl_down2(f[jm]);
        if (live) {
            if (left) { self = add2(self, up); ++kself; }
            if (right) { self = add2(self, dn); ++kself; }
            red_acc(pb.acc + pv, fix_enc2n(self, kself), pol);
            if ((nm & (1u << jp)) && !right) red_acc(pb.acc + ((int)pv + nb_off(jp, b)), fix_enc2n(f[jp], 1), pol);
            if ((nm & (1u << jm)) && !left) red_acc(pb.acc + ((int)pv + nb_off(jm, b)), fix_enc2n(f[jm], 1), pol);
        }
    }
    push_row<1, 0>(f, nm, live, left, right, pv, b, pb.acc, pol);
    push_row<-1, 0>(f, nm, live, left, right, pv, b, pb.acc, pol);
    push_row<0, 1>(f, nm, live, left, right, pv, b, pb.acc, pol);
    push_row<0, -1>(f, nm, live, left, right, pv, b, pb.acc, pol);
    if (!live) return;
    // rows with a single direction each: (0, +-1, +-1)
#pragma unroll
    for (int j = 15; j < 19; ++j)
        if (nm & (1u << j)) red_acc(pb.acc + ((int)pv + nb_off(j, b)), fix_enc2n(f[j], 1), pol);
}

// Plane node t (inlet nodes first, then outlet) after the collide-stream
// pass: the open-plane rule (at the parity PN of the next step), then the
// node's exact density as a total.
template <int PN>
__device__ __forceinline__ void plane_push_node(int t, int nb, uint32_t flb, const DevState &s,
                                                unsigned long long *acc)
{
    using TS = float;
    const int plane = t >= s.nxy ? 1 : 0;
    const int p = t - plane * s.nxy;
    const uint32_t pvb = plane == 0 ? (uint32_t)p : (uint32_t)(p + (s.nz - 1) * s.sxy);
    neem_node<TS, PN, LD_NC>(plane, p, nb, pvb, flb, s);
    const Nbr bb = make_nbr(flb, s);
    float2 f[19], dm;
    // read back through L2: the cells were just written by this thread, and
    // the read-only cache is not coherent with those writes
    load_pops<TS, PN, LD_CA>(f, dm, nb, pvb, flb, bb, s);
    acc[pvb] = fix_total2(dm);
}

__device__ __forceinline__ int plane_voxel(int t, const DevState &s)
{
    return t < s.nxy ? t : t - s.nxy + (s.nz - 1) * s.sxy;
}

// Wall w (Eq. 15) from the accumulator densities of its fluid neighbours.
// The weighted sum runs in integer arithmetic on the encoded words, in three
// partial sums (the faces, weight 1/18, and two groups of six edges, weight
// 1/36) of at most six terms each, so that each stays below 2^31 in magnitude
// once the offsets of its terms are taken off (densities below 5.3; the
// encoding holds below 4.5): three conversions per component instead of one
// per neighbour.
__device__ __forceinline__ void wall_push_node(int w, uint32_t pv, uint32_t mask, float inv, const DevState &s,
                                               unsigned long long *acc)
{
    const Nbr b = make_nbr(mask >> kWallFaceShift, s);
    uint32_t sx[3] = {0u, 0u, 0u}, sy[3] = {0u, 0u, 0u};
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        if (mask & (1u << j)) {
            const unsigned long long v = __ldcg(acc + ((int)pv + nb_off(j, b)));
            const int g = j <= 6 ? 0 : j <= 12 ? 1 : 2;
            sx[g] += (uint32_t)v;
            sy[g] += (uint32_t)(v >> 32);
        }
    }
    const uint32_t cnt[3] = {(uint32_t)__popc(mask & 0x7eu), (uint32_t)__popc(mask & (0x3fu << 7)),
                             (uint32_t)__popc(mask & (0x3fu << 13))};
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        const float wg = g == 0 ? 2.f : 1.f;
        ax = fmaf(wg, (float)(int)(sx[g] - cnt[g] * kFixOffset), ax);
        ay = fmaf(wg, (float)(int)(sy[g] - cnt[g] * kFixOffset), ay);
    }
    const float sc = 1.0f / (36.0f * (float)(1 << kFixShift));
    const float xi = reinterpret_cast<const float *>(s.wxi)[w];
    acc[pv] = fix_total2(make_float2(ax * sc * (1.f + xi) * inv, ay * sc * (1.f - xi) * inv));
}

// After the collide-stream pass, one launch: the first nbp blocks finish the
// open-plane nodes, the next nbw blocks the walls [w0, w1), which lie at
// least two planes away from an open plane and so read no plane node's
// density, and the rest clear the buffer the step after next adds into
// (clr, nv words).  Every block waits for the collide-stream pass: with
// programmatic launches a small grid can start while the pass before it is
// still running, and that pass may be the one that read clr.  The node's or
// wall's geometry never changes and is read before the wait; xi after it
// (lbm_set_xi_field may have changed it).
template <int PN>
__global__ void __launch_bounds__(256) k_pw_push(DevState s, unsigned long long *acc, unsigned long long *clr,
                                                 int nbp, int nbw, int w0, int w1)
{
    pdl_trigger();
    const int bx = (int)blockIdx.x;
    if (bx >= nbp + nbw) {
        const long long i = (long long)(bx - nbp - nbw) * blockDim.x + threadIdx.x;  // a pair of words
        pdl_wait();
        if (2 * i + 1 < s.nv && ((uintptr_t)clr & 15u) == 0) {
            reinterpret_cast<ulonglong2 *>(clr)[i] = make_ulonglong2(0ull, 0ull);
        } else {
            if (2 * i < s.nv) clr[2 * i] = 0ull;
            if (2 * i + 1 < s.nv) clr[2 * i + 1] = 0ull;
        }
        return;
    }
    if (bx < nbp) {
        const int t = bx * (int)blockDim.x + (int)threadIdx.x;
        const int nb = t < 2 * s.nxy ? s.cidx[plane_voxel(t, s)] : -1;
        const uint32_t flb = nb >= 0 ? s.nflags[nb] : 0u;
        pdl_wait();
        if (nb >= 0) plane_push_node<PN>(t, nb, flb, s, acc);
        return;
    }
    const int w = w0 + (bx - nbp) * (int)blockDim.x + (int)threadIdx.x;
    const bool live = w < w1;
    const uint32_t pv = live ? s.wpvox[w] : 0u;
    const uint32_t mask = live ? s.wmask[w] : 0u;
    const float inv = live ? reinterpret_cast<const float *>(s.winv)[w] : 0.f;
    pdl_wait();
    if (live) wall_push_node(w, pv, mask, inv, s, acc);
}

// The remaining walls, [w0, w1) and [w2, w3), after the plane nodes: those
// within two planes of an open plane (all walls when no plane is open).
__global__ void __launch_bounds__(256) k_wall_push(DevState s, unsigned long long *acc, int w0, int w1, int w2, int w3)
{
    pdl_trigger();
    const int t = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int w = t < w1 - w0 ? w0 + t : w2 + (t - (w1 - w0));
    const bool live = t < (w1 - w0) + (w3 - w2);
    const uint32_t pv = live ? s.wpvox[w] : 0u;
    const uint32_t mask = live ? s.wmask[w] : 0u;
    const float inv = live ? reinterpret_cast<const float *>(s.winv)[w] : 0.f;
    pdl_wait();
    if (live) wall_push_node(w, pv, mask, inv, s, acc);
}

// Float densities (psi, after a density and wall pass) into an accumulator
// buffer as totals: starts the schedule from any state.
__global__ void k_psi_to_acc(const float2 *psi, const int32_t *cidx, const uint32_t *wpvox, int n_wall, long long nv,
                             unsigned long long *acc)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv && cidx[v] >= 0) acc[v] = fix_total2(psi[v]);
    if (v < n_wall) acc[wpvox[v]] = fix_total2(psi[wpvox[v]]);
}

}  // namespace lbm
