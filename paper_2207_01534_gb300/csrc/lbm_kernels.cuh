// lbm_kernels.cuh -- sm_103a kernels of the two-component pseudopotential
// D3Q19 step (Sedahmed et al. 2022, Section 2).  Included by one translation
// unit per population storage type.
//
// Data layout (all in device memory):
//   populations  A[sigma][i][npad]  SoA over the compact fluid index n, stored
//                in place with the A-A pattern: one copy of every population.
//   psi          dense (psi1, psi2) pairs over all nx*ny*nz voxels: rho^sigma
//                on fluid voxels (Eq. 3 / 11), rho-tilde^sigma on wall voxels
//                (Eqs. 14-15), so the force stencil needs no neighbour table.
//   cidx         dense compact index (-1 on solids) for the streaming partner.
//
// A-A slots.  Define slot_j(x), j = 1..18, as the storage cell that holds the
// post-stream population f_opp(j)(x) when a step starts and that receives the
// post-collision f*_j(x) when the step ends.  On even steps slot_j(x) =
// A[opp(j)][x] (everything local); on odd steps slot_j(x) = A[j][x + e_j] when
// x + e_j is fluid, A[opp(j)][x] when it is solid (half-way bounce-back), and a
// boundary cell bc[...] when x + e_j lies beyond an open plane.  The rest
// population always lives in A[0][x].  Every cell belongs to exactly one
// (node, direction) on a given parity, so a node's reads and writes never race
// with another node's.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------------------
// D3Q19 (Section 2 ordering).  Written as constexpr functions so that fully
// unrolled direction loops fold every velocity component and weight.
__host__ __device__ constexpr int ex(int i)
{
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int ey(int i)
{
    return (i == 3 || i == 7 || i == 8 || i == 15 || i == 17) ? 1
           : (i == 4 || i == 9 || i == 10 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int ez(int i)
{
    return (i == 5 || i == 11 || i == 12 || i == 15 || i == 16) ? 1
           : (i == 6 || i == 13 || i == 14 || i == 17 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i)
{
    return i == 0 ? 0 : (i <= 6 ? ((i & 1) ? i + 1 : i - 1) : (7 + 4 * ((i - 7) / 4) + 3 - (i - 7) % 4));
}
// direction with the z component reflected (mirror across an open z plane)
__host__ __device__ constexpr int mirz(int i)
{
    return i == 5 ? 6 : i == 6 ? 5 : i == 11 ? 13 : i == 13 ? 11 : i == 12 ? 14 : i == 14 ? 12
         : i == 15 ? 17 : i == 17 ? 15 : i == 16 ? 18 : i == 18 ? 16 : i;
}
// position of a missing incoming direction in its plane's list:
// inlet {5, 11, 12, 15, 16}, outlet {6, 13, 14, 17, 18}
__host__ __device__ constexpr int miss_k(int i)
{
    return (i == 5 || i == 6) ? 0 : (i == 11 || i == 13) ? 1 : (i == 12 || i == 14) ? 2
         : (i == 15 || i == 17) ? 3 : 4;
}
__host__ __device__ constexpr int miss_dir(int plane, int k)
{
    return plane == 0 ? (k == 0 ? 5 : k == 1 ? 11 : k == 2 ? 12 : k == 3 ? 15 : 16)
                      : (k == 0 ? 6 : k == 1 ? 13 : k == 2 ? 14 : k == 3 ? 17 : 18);
}
template <typename C>
__host__ __device__ constexpr C wgt(int i)
{
    return i == 0 ? C(1) / C(3) : (i <= 6 ? C(1) / C(18) : C(1) / C(36));
}

// ---------------------------------------------------------------------------
// Storage traits: how a population is kept in memory.
template <typename TS>
struct Traits;

template <>
struct Traits<float> {
    using C = float;
    using C2 = float2;
    __device__ static __forceinline__ float load(const float *p, float) { return __ldg(p); }
    __device__ static __forceinline__ float load_cg(const float *p, float) { return __ldcg(p); }
    __device__ static __forceinline__ void store(float *p, float v, float) { *p = v; }
};

template <>
struct Traits<double> {
    using C = double;
    using C2 = double2;
    __device__ static __forceinline__ double load(const double *p, double) { return __ldg(p); }
    __device__ static __forceinline__ double load_cg(const double *p, double) { return __ldcg(p); }
    __device__ static __forceinline__ void store(double *p, double v, double) { *p = v; }
};

// ---------------------------------------------------------------------------
// Geometry helpers

// Offsets from a node to its neighbours one step down / up each axis,
// including the wrap across the periodic faces that the node touches (fl
// holds its face bits).  Computed once per node; the offset of direction i
// is then one or two integer adds.
struct Nbr {
    int dx[2], dy[2], dz[2];  // [0]: -1 move, [1]: +1 move
};

__device__ __forceinline__ Nbr make_nbr(uint32_t fl, const DevState &s)
{
    Nbr b;
    b.dx[0] = -1 + ((fl & F_XLO) ? s.nx : 0);
    b.dx[1] = 1 - ((fl & F_XHI) ? s.nx : 0);
    b.dy[0] = -s.sx + ((fl & F_YLO) ? s.ny * s.sx : 0);
    b.dy[1] = s.sx - ((fl & F_YHI) ? s.ny * s.sx : 0);
    b.dz[0] = -s.sxy + ((fl & F_ZLO) ? s.nz * s.sxy : 0);
    b.dz[1] = s.sxy - ((fl & F_ZHI) ? s.nz * s.sxy : 0);
    return b;
}

__device__ __forceinline__ int nb_off(int i, const Nbr &b)
{
    int o = 0;
    if (ex(i)) o += b.dx[ex(i) > 0];
    if (ey(i)) o += b.dy[ey(i) > 0];
    if (ez(i)) o += b.dz[ez(i) > 0];
    return o;
}

// Does direction j leave the domain through an open plane?
__device__ __forceinline__ bool outside(int j, uint32_t fl)
{
    return (ez(j) < 0 && (fl & F_INLET)) || (ez(j) > 0 && (fl & F_OUTLET));
}

// slot_j(x) as an offset into one component's population block (>= 0;
// 19 * npad < 2^31 is checked at creation) or as -1 - (offset into one
// component's boundary block).
template <int P>
__device__ __forceinline__ int slot_of(int j, int n, uint32_t pv, uint32_t fl, const Nbr &b, const DevState &s)
{
    if (P == 0) return opp(j) * (int)s.npad + n;
    if (outside(j, fl)) {
        const int plane = (fl & F_INLET) ? 0 : 1;
        const int p = plane == 0 ? (int)pv : (int)pv - (s.nz - 1) * s.sxy;
        return -1 - ((plane * 10 + miss_k(opp(j))) * s.nxy + p);
    }
    const int c = __ldg(s.cidx + ((int)pv + nb_off(j, b)));
    return c >= 0 ? j * (int)s.npad + c : opp(j) * (int)s.npad + n;
}

template <typename TS>
__device__ __forceinline__ TS *cell(const DevState &s, int sigma, int slot)
{
    return slot >= 0 ? reinterpret_cast<TS *>(s.f) + (long long)sigma * 19 * s.npad + slot
                     : reinterpret_cast<TS *>(s.bc) + (long long)sigma * 5 * s.nxy + (-1 - slot);
}

template <typename TS>
__device__ __forceinline__ typename Traits<TS>::C ref_of(const DevState &s, int sigma, int i)
{
    using C = typename Traits<TS>::C;
    return wgt<C>(i) * (C)(sigma == 0 ? s.rref1 : s.rref2);
}

// Offset of slot_j(x) inside one component's population block when x + e_j
// is not beyond an open plane (the caller handles that case).
template <int P>
__device__ __forceinline__ unsigned slot_in_block(int j, int n, uint32_t pv, const Nbr &b, const DevState &s)
{
    const unsigned np = (unsigned)s.npad;
    if (P == 0) return (unsigned)opp(j) * np + (unsigned)n;
    const int c = __ldg(s.cidx + ((int)pv + nb_off(j, b)));
    return c >= 0 ? (unsigned)j * np + (unsigned)c : (unsigned)opp(j) * np + (unsigned)n;
}

// Offset of the boundary cell that replaces slot_j(x) for a direction j
// leaving through an open plane, inside one component's boundary block.
__device__ __forceinline__ unsigned bc_cell(int j, uint32_t pv, uint32_t fl, const DevState &s)
{
    const int plane = (fl & F_INLET) ? 0 : 1;
    const int p = plane == 0 ? (int)pv : (int)pv - (s.nz - 1) * s.sxy;
    return (unsigned)((plane * 10 + miss_k(opp(j))) * s.nxy + p);
}

template <typename TS, bool L2ONLY>
__device__ __forceinline__ typename Traits<TS>::C ld_pop(const TS *p, typename Traits<TS>::C ref)
{
    return L2ONLY ? Traits<TS>::load_cg(p, ref) : Traits<TS>::load(p, ref);
}

// Post-stream populations f[sigma][i] of node n at parity P.  L2ONLY loads
// bypass L1 (for data written earlier in the same launch).
template <typename TS, int P, bool L2ONLY = false>
__device__ __forceinline__ void load_pops(typename Traits<TS>::C f[2][19], int n, uint32_t pv, uint32_t fl,
                                          const Nbr &b, const DevState &s)
{
    const TS *A0 = reinterpret_cast<const TS *>(s.f);
    const TS *A1 = A0 + 19 * s.npad;
    const bool plane = P == 1 && (fl & (F_INLET | F_OUTLET));
    f[0][0] = ld_pop<TS, L2ONLY>(A0 + n, ref_of<TS>(s, 0, 0));
    f[1][0] = ld_pop<TS, L2ONLY>(A1 + n, ref_of<TS>(s, 1, 0));
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        if (ez(j) != 0 && plane && outside(j, fl)) {
            const TS *B0 = reinterpret_cast<const TS *>(s.bc);
            const unsigned q = bc_cell(j, pv, fl, s);
            f[0][opp(j)] = ld_pop<TS, L2ONLY>(B0 + q, ref_of<TS>(s, 0, j));
            f[1][opp(j)] = ld_pop<TS, L2ONLY>(B0 + 5 * s.nxy + q, ref_of<TS>(s, 1, j));
        } else {
            const unsigned q = slot_in_block<P>(j, n, pv, b, s);
            f[0][opp(j)] = ld_pop<TS, L2ONLY>(A0 + q, ref_of<TS>(s, 0, j));
            f[1][opp(j)] = ld_pop<TS, L2ONLY>(A1 + q, ref_of<TS>(s, 1, j));
        }
    }
}

// Post-collision populations f[sigma][i] of node n into their slots.
template <typename TS, int P>
__device__ __forceinline__ void store_pops(const typename Traits<TS>::C f[2][19], int n, uint32_t pv, uint32_t fl,
                                           const Nbr &b, const DevState &s)
{
    TS *A0 = reinterpret_cast<TS *>(s.f);
    TS *A1 = A0 + 19 * s.npad;
    const bool plane = P == 1 && (fl & (F_INLET | F_OUTLET));
    Traits<TS>::store(A0 + n, f[0][0], ref_of<TS>(s, 0, 0));
    Traits<TS>::store(A1 + n, f[1][0], ref_of<TS>(s, 1, 0));
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        if (ez(j) != 0 && plane && outside(j, fl)) continue;  // leaves the domain
        const unsigned q = slot_in_block<P>(j, n, pv, b, s);
        Traits<TS>::store(A0 + q, f[0][j], ref_of<TS>(s, 0, j));
        Traits<TS>::store(A1 + q, f[1][j], ref_of<TS>(s, 1, j));
    }
}

template <typename C>
__device__ __forceinline__ C sum19(const C f[19])
{
    C r = f[0];
#pragma unroll
    for (int i = 1; i < 19; ++i) r += f[i];
    return r;
}

// Force of Eqs. 10, 11, 13: F^sigma = -G psi^sigma(x) sum_i w_i psi^sigma-bar(x+e_i) e_i
// (+ rho^sigma g), psi being rho on fluid and rho-tilde on wall voxels; beyond
// an open plane the mirrored direction's neighbour is used (Section 2).
template <typename TS>
__device__ __forceinline__ void forces(typename Traits<TS>::C rho1, typename Traits<TS>::C rho2, uint32_t pv,
                                       uint32_t fl, const Nbr &b, const DevState &s, typename Traits<TS>::C F1[3],
                                       typename Traits<TS>::C F2[3])
{
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    const C2 *psi = reinterpret_cast<const C2 *>(s.psi);
    C a1[3] = {0, 0, 0}, a2[3] = {0, 0, 0};
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        const int off = outside(j, fl) ? nb_off(mirz(j), b) : nb_off(j, b);
        // neighbour minus own value: the same sum, since sum_j w_j e_j = 0,
        // with far less cancellation error in FP32 near uniform regions
        const C2 q = psi[(int)pv + off];
        const C d1 = q.x - rho1, d2 = q.y - rho2;
        const C w = wgt<C>(j);
        if (ex(j)) { a1[0] += (w * ex(j)) * d1; a2[0] += (w * ex(j)) * d2; }
        if (ey(j)) { a1[1] += (w * ey(j)) * d1; a2[1] += (w * ey(j)) * d2; }
        if (ez(j)) { a1[2] += (w * ez(j)) * d1; a2[2] += (w * ez(j)) * d2; }
    }
    const C G = (C)s.G;
    const C g[3] = {(C)s.gx, (C)s.gy, (C)s.gz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        F1[a] = -G * rho1 * a2[a] + rho1 * g[a];
        F2[a] = -G * rho2 * a1[a] + rho2 * g[a];
    }
}

// Eqs. 6-8: tau_s = sum rho^sigma tau^sigma / rho (nu = c_s^2 (tau - 1/2));
// u = (sum_sigma sum_i e_i f_i^sigma [+ F^sigma / 2]) / rho.
template <typename C>
__device__ __forceinline__ void mix_velocity(const C f[2][19], C rho1, C rho2, const C F1[3], const C F2[3],
                                             const DevState &s, C &inv_rho, C u[3])
{
    C m[3] = {0, 0, 0};
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const C t = f[0][i] + f[1][i];
        if (ex(i)) m[0] += ex(i) * t;
        if (ey(i)) m[1] += ey(i) * t;
        if (ez(i)) m[2] += ez(i) * t;
    }
    inv_rho = C(1) / (rho1 + rho2);
    const C h = s.velocity_shift ? C(0.5) : C(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = (m[a] + h * (F1[a] + F2[a])) * inv_rho;
}

// Eq. 1 with Eq. 2 equilibrium and Eq. 9 forcing, in place on f[sigma][i]:
// f* = (1 - 1/tau_s) f + f^eq / tau_s + (1 - 1/(2 tau_s)) S.  Directions are
// taken in opposite pairs (i, opp(i)): with eu = e_i.u and eF = e_i.F, the
// pair shares sym = 1 + 4.5 eu^2 - 1.5 u^2 and 9 eu eF - 3 u.F, and differs
// only in the sign of 3 eu and 3 eF, so each pair is computed once.
template <typename C>
__device__ __forceinline__ void collide(C f[2][19], C rho1, C rho2, C inv_rho, const C u[3], const C F1[3],
                                        const C F2[3], const DevState &s)
{
    const C tau_s = (rho1 * (C)s.tau1 + rho2 * (C)s.tau2) * inv_rho;
    const C om = C(1) / tau_s;
    const C keep = C(1) - om;
    const C cf = C(1) - C(0.5) * om;
    const C usq = C(1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const C cuF1 = C(-3) * (u[0] * F1[0] + u[1] * F1[1] + u[2] * F1[2]);
    const C cuF2 = C(-3) * (u[0] * F2[0] + u[1] * F2[1] + u[2] * F2[2]);
    const C r1o = om * rho1, r2o = om * rho2;
    // The rest population is written last as rho^sigma minus the 18 moving
    // post-collision populations.  In exact arithmetic this equals Eq. 1 for
    // i = 0 (sum_i f^eq_i = rho, sum_i S_i = 0); in FP32 it removes the mass
    // bias of the rounded weights (their FP32 sum exceeds 1 by ~1.5e-8, which
    // would otherwise create mass at every collision).
    C sum1 = 0, sum2 = 0;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        if (opp(i) < i) continue;  // each pair once, from its first member
        const int o = opp(i);
        const C w = wgt<C>(i);
        const C eu = ex(i) * u[0] + ey(i) * u[1] + ez(i) * u[2];
        const C eF1 = ex(i) * F1[0] + ey(i) * F1[1] + ez(i) * F1[2];
        const C eF2 = ex(i) * F2[0] + ey(i) * F2[1] + ez(i) * F2[2];
        const C sym = C(1) + C(4.5) * eu * eu - usq;
        const C ant = C(3) * eu;
        const C A1 = w * (r1o * sym + cf * (C(9) * eu * eF1 + cuF1));
        const C B1 = w * (r1o * ant + cf * C(3) * eF1);
        const C A2 = w * (r2o * sym + cf * (C(9) * eu * eF2 + cuF2));
        const C B2 = w * (r2o * ant + cf * C(3) * eF2);
        f[0][i] = keep * f[0][i] + (A1 + B1);
        f[0][o] = keep * f[0][o] + (A1 - B1);
        f[1][i] = keep * f[1][i] + (A2 + B2);
        f[1][o] = keep * f[1][o] + (A2 - B2);
    }
    // accumulated one direction at a time, in direction order: summing each
    // pair first biases the FP32 rounding and drifts the mass measurably
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        sum1 += f[0][i];
        sum2 += f[1][i];
    }
    f[0][0] = rho1 - sum1;
    f[1][0] = rho2 - sum2;
}

// ---------------------------------------------------------------------------
// Kernels of the split schedule

template <typename TS, int P>
__global__ void __launch_bounds__(256) k_dens(DevState s)
{
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n_fluid) return;
    const uint32_t pv = s.pvox[n];
    const uint32_t fl = s.nflags[n];
    C f[2][19];
    const Nbr b = make_nbr(fl, s);
    load_pops<TS, P>(f, n, pv, fl, b, s);
    C2 q;
    q.x = sum19<C>(f[0]);
    q.y = sum19<C>(f[1]);
    reinterpret_cast<C2 *>(s.psi)[pv] = q;
}

// Eq. 15 at every wall voxel: rho-tilde^sigma = chi^sigma * (sum of w_i rho^sigma
// over in-domain fluid neighbours) / (sum of those w_i), chi = 1 +/- xi.
template <typename TS>
__global__ void __launch_bounds__(256) k_wall(DevState s)
{
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= s.n_wall) return;
    const uint32_t pv = s.wpvox[w];
    const uint32_t mask = s.wmask[w];
    const uint32_t fl = mask >> kWallFaceShift;
    C2 *psi = reinterpret_cast<C2 *>(s.psi);
    const Nbr b = make_nbr(fl, s);
    C s1 = 0, s2 = 0;
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        if (mask & (1u << j)) {
            const C2 q = psi[(int)pv + nb_off(j, b)];
            s1 += wgt<C>(j) * q.x;
            s2 += wgt<C>(j) * q.y;
        }
    }
    const C inv = reinterpret_cast<const C *>(s.winv)[w];
    const C xi = reinterpret_cast<const C *>(s.wxi)[w];
    C2 q;
    q.x = (C(1) + xi) * s1 * inv;
    q.y = (C(1) - xi) * s2 * inv;
    psi[pv] = q;
}

template <typename TS, int P>
__global__ void __launch_bounds__(256, 3) k_fused(DevState s)
{
    using C = typename Traits<TS>::C;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n_fluid) return;
    const uint32_t pv = s.pvox[n];
    const uint32_t fl = s.nflags[n];
    C f[2][19];
    const Nbr b = make_nbr(fl, s);
    load_pops<TS, P>(f, n, pv, fl, b, s);
    const C rho1 = sum19<C>(f[0]);
    const C rho2 = sum19<C>(f[1]);
    C F1[3], F2[3], u[3], inv_rho;
    forces<TS>(rho1, rho2, pv, fl, b, s, F1, F2);
    mix_velocity<C>(f, rho1, rho2, F1, F2, s, inv_rho, u);
    collide<C>(f, rho1, rho2, inv_rho, u, F1, F2, s);
    store_pops<TS, P>(f, n, pv, fl, b, s);
}

// Open planes, run after a step for the parity PN of the step that reads next:
// the prescribed component (1 at the inlet, 2 at the outlet) gets all 19
// populations by non-equilibrium extrapolation from the first interior node,
// f_i(xb) = f^eq_i(rho_b, u) + f_i(xi) - f^eq_i(rho(xi), u) with u the
// barycentric velocity of xi; the other component's missing populations get
// their initial values back (Section 2).
template <typename TS, int PN, bool L2ONLY>
__device__ __forceinline__ void neem_node(int plane, int p, int nb, uint32_t pvb, uint32_t flb, const DevState &s)
{
    using C = typename Traits<TS>::C;
    const uint32_t pvi = plane == 0 ? pvb + s.sxy : pvb - s.sxy;
    const int ni = s.cidx[pvi];
    const uint32_t fli = s.nflags[ni];
    const Nbr bi = make_nbr(fli, s);
    const Nbr bb = make_nbr(flb, s);
    C fi[2][19];
    load_pops<TS, PN, L2ONLY>(fi, ni, pvi, fli, bi, s);
    const C r1 = sum19<C>(fi[0]);
    const C r2 = sum19<C>(fi[1]);
    C m[3] = {0, 0, 0};
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const C tt = fi[0][i] + fi[1][i];
        if (ex(i)) m[0] += ex(i) * tt;
        if (ey(i)) m[1] += ey(i) * tt;
        if (ez(i)) m[2] += ez(i) * tt;
    }
    const C ir = C(1) / (r1 + r2);
    const C u[3] = {m[0] * ir, m[1] * ir, m[2] * ir};
    const C usq = C(1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const C rb = (C)(plane == 0 ? s.rho_in1 : s.rho_out2);
    const C rin = plane == 0 ? r1 : r2;
    TS *A = reinterpret_cast<TS *>(s.f);
    const int pc = plane;  // prescribed component index
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const C eu = ex(i) * u[0] + ey(i) * u[1] + ez(i) * u[2];
        const C base = C(1) + C(3) * eu + C(4.5) * eu * eu - usq;
        const C fin = plane == 0 ? fi[0][i] : fi[1][i];
        const C v = wgt<C>(i) * rb * base + fin - wgt<C>(i) * rin * base;
        if (i == 0)
            Traits<TS>::store(A + (long long)pc * 19 * s.npad + nb, v, ref_of<TS>(s, pc, 0));
        else
            Traits<TS>::store(cell<TS>(s, pc, slot_of<PN>(opp(i), nb, pvb, flb, bb, s)), v, ref_of<TS>(s, pc, i));
    }
    const int qc = 1 - pc;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int i = miss_dir(plane, k);
        const C v = (C)s.frozen[(long long)(plane * 5 + k) * s.nxy + p];
        Traits<TS>::store(cell<TS>(s, qc, slot_of<PN>(opp(i), nb, pvb, flb, bb, s)), v, ref_of<TS>(s, qc, i));
    }
}

template <typename TS, int PN>
__global__ void __launch_bounds__(128) k_plane(DevState s)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * s.nxy) return;
    const int plane = t >= s.nxy ? 1 : 0;
    const int p = t - plane * s.nxy;
    const uint32_t pvb = plane == 0 ? (uint32_t)p : (uint32_t)(p + (s.nz - 1) * s.sxy);
    const int nb = s.cidx[pvb];
    if (nb < 0) return;
    neem_node<TS, PN, false>(plane, p, nb, pvb, s.nflags[nb], s);
}

// ---------------------------------------------------------------------------
// State transfer and diagnostics

template <typename TS>
__global__ void k_init_eq(DevState s, const double *rho)
{
    using C = typename Traits<TS>::C;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n_fluid) return;
    const uint32_t pv = s.pvox[n];
    TS *A = reinterpret_cast<TS *>(s.f);
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
        const C r = (C)rho[(long long)sg * s.nv + pv];
#pragma unroll
        for (int i = 0; i < 19; ++i)
            Traits<TS>::store(A + ((long long)sg * 19 + i) * s.npad + n, wgt<C>(i) * r, ref_of<TS>(s, sg, i));
    }
}

template <typename TS>
__global__ void k_scatter(DevState s, const double *f)
{
    using C = typename Traits<TS>::C;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n_fluid) return;
    const uint32_t pv = s.pvox[n];
    TS *A = reinterpret_cast<TS *>(s.f);
    for (int k = 0; k < 38; ++k) {
        const int sg = k / 19, i = k % 19;
        Traits<TS>::store(A + (long long)k * s.npad + n, (C)f[(long long)k * s.nv + pv], ref_of<TS>(s, sg, i));
    }
}

template <typename TS, int P>
__global__ void k_gather(DevState s, double *out)
{
    using C = typename Traits<TS>::C;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n_fluid) return;
    const uint32_t pv = s.pvox[n];
    C f[2][19];
    const uint32_t fl = s.nflags[n];
    const Nbr b = make_nbr(fl, s);
    load_pops<TS, P>(f, n, pv, fl, b, s);
#pragma unroll
    for (int sg = 0; sg < 2; ++sg)
#pragma unroll
        for (int i = 0; i < 19; ++i) out[((long long)sg * 19 + i) * s.nv + pv] = (double)f[sg][i];
}

// Frozen values: the initial populations of the non-prescribed component in
// the missing directions of each open plane (parity-0 layout).
template <typename TS>
__global__ void k_capture_frozen(DevState s, double *frozen)
{
    using C = typename Traits<TS>::C;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * s.nxy) return;
    const int plane = t >= s.nxy ? 1 : 0;
    const int p = t - plane * s.nxy;
    const uint32_t pvb = plane == 0 ? (uint32_t)p : (uint32_t)(p + (s.nz - 1) * s.sxy);
    const int nb = s.cidx[pvb];
    const int qc = 1 - plane;
    const TS *A = reinterpret_cast<const TS *>(s.f);
    for (int k = 0; k < 5; ++k) {
        const int i = miss_dir(plane, k);
        double v = 0;
        if (nb >= 0) v = (double)Traits<TS>::load(A + ((long long)qc * 19 + i) * s.npad + nb, ref_of<TS>(s, qc, i));
        frozen[(long long)(plane * 5 + k) * s.nxy + p] = v;
    }
}

template <typename TS, int P>
__global__ void k_fields(DevState s, double *out)
{
    using C = typename Traits<TS>::C;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n_fluid) return;
    const uint32_t pv = s.pvox[n];
    const uint32_t fl = s.nflags[n];
    C f[2][19];
    const Nbr b = make_nbr(fl, s);
    load_pops<TS, P>(f, n, pv, fl, b, s);
    const C rho1 = sum19<C>(f[0]);
    const C rho2 = sum19<C>(f[1]);
    C F1[3], F2[3], u[3], inv_rho;
    forces<TS>(rho1, rho2, pv, fl, b, s, F1, F2);
    mix_velocity<C>(f, rho1, rho2, F1, F2, s, inv_rho, u);
    const C cs2 = C(1) / C(3);
    out[0 * s.nv + pv] = (double)rho1;
    out[1 * s.nv + pv] = (double)rho2;
    out[2 * s.nv + pv] = (double)u[0];
    out[3 * s.nv + pv] = (double)u[1];
    out[4 * s.nv + pv] = (double)u[2];
    out[5 * s.nv + pv] = (double)(cs2 * (rho1 + rho2) + cs2 * (C)s.G * rho1 * rho2);
}

// FP64 reduction of the densities in psi (warp shuffle -> block -> partials).
template <typename TS>
__global__ void __launch_bounds__(kReduceThreads) k_reduce(DevState s, double *partials)
{
    using C2 = typename Traits<TS>::C2;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const C2 *psi = reinterpret_cast<const C2 *>(s.psi);
    const bool all = s.sample_hi <= s.sample_lo;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < s.n_fluid; n += gridDim.x * blockDim.x) {
        const uint32_t pv = s.pvox[n];
        const C2 q = psi[pv];
        const double r1 = (double)q.x, r2 = (double)q.y;
        acc[0] += r1;
        acc[1] += r2;
        const int z = (int)(pv / (uint32_t)s.sxy);
        if (all || (z >= s.sample_lo && z < s.sample_hi)) {
            acc[2] += 1.0;
            acc[3] += (q.y > q.x) ? 1.0 : 0.0;
            acc[4] += r1 / (r1 + r2);
        }
        if (!isfinite(r1 + r2)) acc[5] += 1.0;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    __shared__ double sm[kReduceThreads / 32][6];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 6; ++k) sm[wid][k] = acc[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            double v = lane < kReduceThreads / 32 ? sm[lane][k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) partials[(long long)blockIdx.x * kReduceSlots + k] = v;
        }
    }
}

__global__ void __launch_bounds__(kReduceThreads) k_reduce_final(const double *partials, int nblocks, double *out);

}  // namespace lbm
