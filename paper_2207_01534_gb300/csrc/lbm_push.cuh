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
// incoming populations.  Plane nodes are finished afterwards by the plane
// pass (the open-plane rule rewrites populations there), then walls (Eq. 15).
//
// Accumulators are integer fixed point (lbm_fixed.cuh): the sums do not
// depend on the order of the atomic adds, so results are bitwise reproducible.
//
// Three accumulator buffers rotate: the pass of step t reads buffer t % 3 in
// its force stencil, adds into (t + 1) % 3, and clears its own voxel of
// (t + 2) % 3, which the pass of step t - 1 has finished reading and the pass
// of step t + 1 adds into.
#pragma once

#include "lbm_fixed.cuh"
#include "lbm_kernels.cuh"

namespace lbm {

// Force of Eqs. 10, 11, 13 from the accumulator densities (as forces()).
__device__ __forceinline__ void forces_acc(float2 rho, uint32_t pv, uint32_t fl, const Nbr &b, const DevState &s,
                                           const unsigned long long *rd, float2 F[3])
{
    const unsigned long long *q = rd + pv;
    float2 a[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        const int off = (ez(j) != 0 && outside(j, fl)) ? nb_off(mirz(j), b) : nb_off(j, b);
        const float2 d = sub2(fix_dec2(__ldg(q + off)), rho);
        const float w = wgt<float>(j);
        if (ex(j)) a[0] = fma2(bc2<float2>(w * ex(j)), d, a[0]);
        if (ey(j)) a[1] = fma2(bc2<float2>(w * ey(j)), d, a[1]);
        if (ez(j)) a[2] = fma2(bc2<float2>(w * ez(j)), d, a[2]);
    }
    const float mG = -s.fG;
    const float g[3] = {s.fgx, s.fgy, s.fgz};
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k] = mul2(rho, fma2(bc2<float2>(mG), make_float2(a[k].y, a[k].x), bc2<float2>(g[k])));
}

template <int P>
__global__ void __launch_bounds__(256, 3) k_fused_push(DevState s, PushBufs pb)
{
    using TS = float;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n_fluid) return;
    const uint32_t pv = s.pvox[n];
    const uint32_t fl = s.nflags[n];
    const Nbr b = make_nbr(fl, s);
    float2 f[19], dm;
    load_pops<TS, P>(f, dm, n, pv, fl, b, s);
    const float2 rho = dm;
    float2 F[3];
    float u[3], inv_rho;
    forces_acc(rho, pv, fl, b, s, pb.rd, F);
    mix_velocity<float, float2>(f, rho, F, s, inv_rho, u);
    collide<float, float2>(f, rho, inv_rho, u, F, s);
    store_pops<TS, P>(f, dm, n, pv, fl, b, s);
    // next-step densities: every post-collision population into the
    // accumulator of the node it becomes a post-stream population of
    const uint32_t nm = pb.nmask[n];
    unsigned long long self = fix_enc2(f[0]);
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        if (ez(j) != 0 && outside(j, fl)) continue;  // leaves the domain
        const unsigned long long e = fix_enc2(f[j]);
        if (nm & (1u << j))
            atomicAdd(pb.acc + ((int)pv + nb_off(j, b)), e);
        else
            self += e;  // bounced back into x
    }
    atomicAdd(pb.acc + pv, self);
    pb.clr[pv] = 0ull;
}

// Plane nodes after the collide-stream pass: the open-plane rule (at the
// parity PN of the next step), then the node's exact density as a total.
template <int PN>
__global__ void __launch_bounds__(128) k_plane_push(DevState s, unsigned long long *acc)
{
    using TS = float;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * s.nxy) return;
    const int plane = t >= s.nxy ? 1 : 0;
    const int p = t - plane * s.nxy;
    const uint32_t pvb = plane == 0 ? (uint32_t)p : (uint32_t)(p + (s.nz - 1) * s.sxy);
    const int nb = s.cidx[pvb];
    if (nb < 0) return;
    const uint32_t flb = s.nflags[nb];
    neem_node<TS, PN, LD_NC>(plane, p, nb, pvb, flb, s);
    const Nbr bb = make_nbr(flb, s);
    float2 f[19], dm;
    // read back through L2: the cells were just written by this thread, and
    // the read-only cache is not coherent with those writes
    load_pops<TS, PN, LD_CA>(f, dm, nb, pvb, flb, bb, s);
    acc[pvb] = fix_total2(dm);
}

// Walls (Eq. 15) from the accumulator densities of their fluid neighbours.
__global__ void __launch_bounds__(256) k_wall_push(DevState s, unsigned long long *acc)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= s.n_wall) return;
    const uint32_t pv = s.wpvox[w];
    const uint32_t mask = s.wmask[w];
    const Nbr b = make_nbr(mask >> kWallFaceShift, s);
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 1; j < 19; ++j)
        if (mask & (1u << j)) a = fma2(bc2<float2>(wgt<float>(j)), fix_dec2(acc[(int)pv + nb_off(j, b)]), a);
    const float inv = reinterpret_cast<const float *>(s.winv)[w];
    const float xi = reinterpret_cast<const float *>(s.wxi)[w];
    acc[pv] = fix_total2(mul2(a, make_float2((1.f + xi) * inv, (1.f - xi) * inv)));
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
