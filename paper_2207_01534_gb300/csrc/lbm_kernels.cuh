// lbm_kernels.cuh -- sm_103a kernels of the two-component pseudopotential
// D3Q19 step (Sedahmed et al. 2022, Section 2).  Included by one translation
// unit per population storage type.
//
// Data layout (all in device memory):
//   rest   R[npad]        pairs (f_0^(1), f_0^(2)) of the rest population per
//                         fluid node (compact index n);
//   moving M[18][npad]    pairs (f_i^(1), f_i^(2)), i = 1..18, SoA over n and
//                         stored in place with the A-A pattern (one copy).  The
//                         two components of a direction sit side by side, so
//                         every access moves both with one 8-byte (FP32) load
//                         or store and the arithmetic runs on packed pairs;
//   psi    dense (psi1, psi2) pairs over all nx*ny*nz voxels: rho^sigma on fluid
//          voxels (Eqs. 3, 11), rho-tilde^sigma on wall voxels (Eqs. 14-15), so
//          the force stencil needs no neighbour table;
//   cidx   dense compact index (-1 on solids) for the streaming partner.
//
// A-A slots.  Define slot_j(x), j = 1..18, as the pair cell that holds the
// post-stream f_opp(j)(x) when a step starts and receives the post-collision
// f*_j(x) when it ends.  On even steps slot_j(x) = M[opp(j)][x] (all local); on
// odd steps slot_j(x) = M[j][x + e_j] when x + e_j is fluid, M[opp(j)][x] when
// it is solid (half-way bounce-back), and a boundary cell when x + e_j lies
// beyond an open plane.  Every cell belongs to exactly one (node, direction)
// on a given parity, so a node's reads and writes never race with another's.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdlib>

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

// A model parameter in the compute type: the FP32 copy in DevState for FP32
// arithmetic, the double itself for FP64 (no per-thread conversion).
template <typename C>
__device__ __forceinline__ C pick(double d, float f);
template <>
__device__ __forceinline__ float pick<float>(double, float f)
{
    return f;
}
template <>
__device__ __forceinline__ double pick<double>(double d, float)
{
    return d;
}

// ---------------------------------------------------------------------------
// Pair arithmetic: (component 1, component 2) in one register pair.  FP32
// pairs use the packed FP32 instructions of sm_100+ (one instruction for both
// lanes); FP64 pairs are two scalar operations.
__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
template <typename C2>
__device__ __forceinline__ C2 sub2(C2 a, C2 b)  // a - b
{
    using C = decltype(a.x);
    return fma2(b, mk2(C(-1), C(-1)), a);
}
template <typename C2>
__device__ __forceinline__ C2 bc2(decltype(C2{}.x) k)  // (k, k)
{
    return mk2(k, k);
}

// ---------------------------------------------------------------------------
// Load modes for population and density reads: LD_NC through the read-only
// cache (data the launch never writes), LD_CG through L2 only (data other
// blocks of the same launch wrote), LD_CA an ordinary coherent load (data
// this thread may have written earlier in the launch).
enum : int { LD_NC = 0, LD_CG = 1, LD_CA = 2 };
template <int LD, typename T>
__device__ __forceinline__ T ldm(const T *p)
{
    if constexpr (LD == LD_NC) return __ldg(p);
    else if constexpr (LD == LD_CG) return __ldcg(p);
    else return *p;
}

// Read-only loads of the maps every node reads many times per step (the
// compact index and the dense densities) under an evict-last L2 policy, so
// their lines stay ahead of the streamed populations.  Values are those of an
// ordinary load.  Measured against plain read-only loads: 128^3 pack FP32
// step 0.0930 -> 0.0889 ms (collide-stream 56.3 -> 53.2 us), FP16 0.0736 ->
// 0.0722 ms, 256^3 rock FP32 0.421 -> 0.410 ms; batch and reverse pass
// unchanged within 0.6%.  (A run-time switch between two load forms inside
// the unrolled direction loops doubled the odd-parity passes; the policy is
// therefore fixed.)
__device__ __forceinline__ unsigned long long l2_policy()
{
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int ld_pol(const int32_t *q, unsigned long long pol)
{
    int v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(q), "l"(pol));
    return v;
}
__device__ __forceinline__ float2 ld_pol(const float2 *q, unsigned long long pol)
{
    float2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(q), "l"(pol));
    return v;
}
__device__ __forceinline__ double2 ld_pol(const double2 *q, unsigned long long) { return __ldg(q); }
// Stores of the density map under the same policy (the density and wall
// passes write it; the wall and collide-stream passes read it back at once):
// 128^3 pack FP32 0.0820 -> 0.0814 ms per step, FP16 unchanged.
__device__ __forceinline__ void st_pol(float2 *q, float2 v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(q), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_pol(double2 *q, double2 v, unsigned long long) { *q = v; }
// The same density-map loads for data written earlier in the same launch
// (persistent kernels): ordinary coherent loads, which the compiler orders
// against the launch's barriers like any other memory access.
template <typename C2>
__device__ __forceinline__ C2 ld_pol_coh(const C2 *q, unsigned long long)
{
    return *q;
}
// density-map load in mode LD: LD_NC read-only (data of earlier launches),
// otherwise coherent
template <int LD, typename C2>
__device__ __forceinline__ C2 ld_psi(const C2 *q, unsigned long long pol)
{
    if constexpr (LD == LD_NC) return ld_pol(q, pol);
    else return ld_pol_coh(q, pol);
}

// ---------------------------------------------------------------------------
// Storage traits: how population pairs are kept in memory.  C / C2 are the
// compute scalar and pair; S2 the stored pair of a moving population; R2 the
// stored pair of the rest population.  ref is the per-direction offset
// (w_i rho_ref^1, w_i rho_ref^2) that deviation storage subtracts.
template <typename TS>
struct Traits;

template <>
struct Traits<float> {
    using C = float;
    using C2 = float2;
    using S2 = float2;
    using R2 = float2;
    static constexpr bool kDev = false;
    __device__ static __forceinline__ C2 load(const S2 *p, C2) { return __ldg(p); }
    __device__ static __forceinline__ void store(S2 *p, C2 v, C2) { *p = v; }
    __device__ static __forceinline__ void store1(S2 *p, int sg, C v, C) { (sg ? p->y : p->x) = v; }
    __device__ static __forceinline__ S2 quant(C2 v, C2) { return v; }
    __device__ static __forceinline__ void store_q(S2 *p, S2 q) { *p = q; }
    template <int LD>
    __device__ static __forceinline__ C2 load_dev(const S2 *p) { return ldm<LD>(p); }
    __device__ static __forceinline__ C2 code_value(S2 q) { return q; }
};

template <>
struct Traits<double> {
    using C = double;
    using C2 = double2;
    using S2 = double2;
    using R2 = double2;
    static constexpr bool kDev = false;
    __device__ static __forceinline__ C2 load(const S2 *p, C2) { return __ldg(p); }
    __device__ static __forceinline__ void store(S2 *p, C2 v, C2) { *p = v; }
    __device__ static __forceinline__ void store1(S2 *p, int sg, C v, C) { (sg ? p->y : p->x) = v; }
    __device__ static __forceinline__ S2 quant(C2 v, C2) { return v; }
    __device__ static __forceinline__ void store_q(S2 *p, S2 q) { *p = q; }
    template <int LD>
    __device__ static __forceinline__ C2 load_dev(const S2 *p) { return ldm<LD>(p); }
    __device__ static __forceinline__ C2 code_value(S2 q) { return q; }
};

// 16-bit storage: a moving population is kept as the FP16 / BF16 deviation
// f_i - w_i rho_ref^sigma (one 4-byte pair for both components); arithmetic
// is FP32 and the rest population stays an FP32 pair.
template <typename H2, typename H1>
struct Traits16 {
    using C = float;
    using C2 = float2;
    using S2 = H2;
    using R2 = float2;
    static constexpr bool kDev = true;
    __device__ static __forceinline__ C2 unpack(unsigned u)
    {
        H2 h;
        memcpy(&h, &u, 4);
        return to_float2(h);
    }
    __device__ static __forceinline__ float2 to_float2(__half2 h) { return __half22float2(h); }
    __device__ static __forceinline__ float2 to_float2(__nv_bfloat162 h) { return __bfloat1622float2(h); }
    __device__ static __forceinline__ void from_float2(float2 v, __half2 *h) { *h = __float22half2_rn(v); }
    __device__ static __forceinline__ void from_float2(float2 v, __nv_bfloat162 *h) { *h = __float22bfloat162_rn(v); }
    __device__ static __forceinline__ void from_float(float v, __half *h) { *h = __float2half_rn(v); }
    __device__ static __forceinline__ void from_float(float v, __nv_bfloat16 *h) { *h = __float2bfloat16_rn(v); }
    __device__ static __forceinline__ S2 quant(C2 v, C2 ref)
    {
        S2 h;
        from_float2(sub2(v, ref), &h);  // one packed, explicitly rounded subtraction
        return h;
    }
    __device__ static __forceinline__ C2 load(const S2 *p, C2 ref)
    {
        return add2(ref, unpack(__ldg(reinterpret_cast<const unsigned *>(p))));
    }
    __device__ static __forceinline__ void store(S2 *p, C2 v, C2 ref) { *p = quant(v, ref); }
    __device__ static __forceinline__ void store_q(S2 *p, S2 q) { *p = q; }
    __device__ static __forceinline__ void store1(S2 *p, int sg, C v, C ref)
    {
        H1 *h = reinterpret_cast<H1 *>(p) + sg;
        from_float(__fsub_rn(v, ref), h);
    }
    // the stored deviation itself, as FP32
    template <int LD>
    __device__ static __forceinline__ C2 load_dev(const S2 *p)
    {
        return unpack(ldm<LD>(reinterpret_cast<const unsigned *>(p)));
    }
    __device__ static __forceinline__ C2 code_value(S2 q) { return to_float2(q); }
};

template <>
struct Traits<__half> : Traits16<__half2, __half> {};
template <>
struct Traits<__nv_bfloat16> : Traits16<__nv_bfloat162, __nv_bfloat16> {};

template <typename TS>
__device__ __forceinline__ typename Traits<TS>::C2 ref_of(const DevState &s, int i)
{
    using C = typename Traits<TS>::C;
    if constexpr (!Traits<TS>::kDev) {
        return mk2(C(0), C(0));
    } else {
        // explicitly rounded scalar products (documented never to be merged
        // into a multiply-add), so every kernel that dequantises gets the
        // same bits
        return mk2(__fmul_rn(wgt<C>(i), pick<C>(s.rref1, s.frref1)), __fmul_rn(wgt<C>(i), pick<C>(s.rref2, s.frref2)));
    }
}

// Rest-population pair of node n, kept at compute precision.  With deviation
// storage the array holds f_0 - w_0 rho_ref (FP32); ld_rest returns f_0 and
// ld_rest_dev the stored deviation.
template <typename TS, int LD>
__device__ __forceinline__ typename Traits<TS>::C2 ld_rest_dev(const DevState &s, int n)
{
    const typename Traits<TS>::R2 *R = reinterpret_cast<const typename Traits<TS>::R2 *>(s.rest);
    return ldm<LD>(R + n);
}
template <typename TS, int LD>
__device__ __forceinline__ typename Traits<TS>::C2 ld_rest(const DevState &s, int n)
{
    const typename Traits<TS>::C2 v = ld_rest_dev<TS, LD>(s, n);
    return Traits<TS>::kDev ? add2(v, ref_of<TS>(s, 0)) : v;
}
template <typename TS>
__device__ __forceinline__ void st_rest_dev(const DevState &s, int n, typename Traits<TS>::C2 v)
{
    reinterpret_cast<typename Traits<TS>::R2 *>(s.rest)[n] = v;
}
template <typename TS>
__device__ __forceinline__ void st_rest(const DevState &s, int n, typename Traits<TS>::C2 v)
{
    st_rest_dev<TS>(s, n, Traits<TS>::kDev ? sub2(v, ref_of<TS>(s, 0)) : v);
}

// Density pair from the mass accumulated by load_pops (see there).
template <typename TS>
__device__ __forceinline__ typename Traits<TS>::C2 density_of(typename Traits<TS>::C2 dm, const DevState &s)
{
    using C = typename Traits<TS>::C;
    return Traits<TS>::kDev ? add2(dm, mk2(pick<C>(s.rref1, s.frref1), pick<C>(s.rref2, s.frref2))) : dm;
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a pass launched with the programmatic
// serialization attribute may start while the previous pass finishes; it
// waits for that pass (and the visibility of its writes) before its first
// dependent read, and lets its own successor launch as soon as all of its
// blocks are running.  Both are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Host side: launch with programmatic stream serialization (the kernel waits
// for its predecessor itself); the environment variable LBM_NO_PDL turns it
// off.
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), unsigned grid, int block, size_t smem, cudaStream_t st,
                       Args... args)
{
    static const bool off = std::getenv("LBM_NO_PDL") != nullptr;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = off ? 0 : 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

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

// Pair offset of slot_j(x) in the moving block when x + e_j is not beyond an
// open plane (18 * npad < 2^31 is checked at creation).
template <int P>
__device__ __forceinline__ unsigned slot_in_block(int j, int n, uint32_t pv, const Nbr &b, const DevState &s)
{
    const unsigned np = (unsigned)s.npad;
    if (P == 0) return (unsigned)(opp(j) - 1) * np + (unsigned)n;
    const int c = ld_pol(s.cidx + ((int)pv + nb_off(j, b)), l2_policy());
    return c >= 0 ? (unsigned)(j - 1) * np + (unsigned)c : (unsigned)(opp(j) - 1) * np + (unsigned)n;
}

// Pair offset of the boundary cell that replaces slot_j(x) when j leaves the
// domain through an open plane: bc[plane][k][nxy], k = the missing direction.
__device__ __forceinline__ unsigned bc_cell(int j, uint32_t pv, uint32_t fl, const DevState &s)
{
    const int plane = (fl & F_INLET) ? 0 : 1;
    const int p = plane == 0 ? (int)pv : (int)pv - (s.nz - 1) * s.sxy;
    return (unsigned)((plane * 5 + miss_k(opp(j))) * s.nxy + p);
}

template <typename TS, int P>
__device__ __forceinline__ typename Traits<TS>::S2 *slot_ptr(int j, int n, uint32_t pv, uint32_t fl, const Nbr &b,
                                                            const DevState &s)
{
    using S2 = typename Traits<TS>::S2;
    if (P == 1 && ez(j) != 0 && outside(j, fl)) return reinterpret_cast<S2 *>(s.bc) + bc_cell(j, pv, fl, s);
    return reinterpret_cast<S2 *>(s.f) + slot_in_block<P>(j, n, pv, b, s);
}

// rho^sigma = sum_i f_i^sigma (Eq. 3), in direction order for both components.
template <typename C2>
__device__ __forceinline__ C2 sum19(const C2 f[19])
{
    C2 r = f[0];
#pragma unroll
    for (int i = 1; i < 19; ++i) r = add2(r, f[i]);
    return r;
}

// Post-stream population pairs f[i] of node n at parity P, and its mass dm:
// the density pair sum_i f_i (direction order) for plain storage, or for
// deviation storage the deviation mass (rest deviation + sum of the stored
// deviations), so that mass bookkeeping never adds the large common offsets
// w_i rho_ref (whose identical rounding at every node would bias it); the
// density is then density_of(dm) = rho_ref + dm.  LD selects the load mode
// (LD_CG for data other blocks of the launch wrote, LD_CA for data this
// thread wrote).
// kRec (parity 1 only): also write each in-block slot offset to rec[(j-1)*rs],
// so that store_pops can take it back instead of looking the partner up again.
template <typename TS, int P, int LD = LD_NC, bool kRec = false>
__device__ __forceinline__ void load_pops(typename Traits<TS>::C2 f[19], typename Traits<TS>::C2 &dm, int n,
                                          uint32_t pv, uint32_t fl, const Nbr &b, const DevState &s,
                                          unsigned *rec = nullptr, int rs = 0)
{
    using C2 = typename Traits<TS>::C2;
    using S2 = typename Traits<TS>::S2;
    const S2 *M = reinterpret_cast<const S2 *>(s.f);
    const S2 *B = reinterpret_cast<const S2 *>(s.bc);
    const bool plane = P == 1 && (fl & (F_INLET | F_OUTLET));
    const C2 r0 = ld_rest_dev<TS, LD>(s, n);
    if (Traits<TS>::kDev) {
        dm = r0;
        f[0] = add2(r0, ref_of<TS>(s, 0));
    } else {
        f[0] = r0;
    }
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        const S2 *p;
        if (ez(j) != 0 && plane && outside(j, fl)) {
            p = B + bc_cell(j, pv, fl, s);
        } else {
            const unsigned o = slot_in_block<P>(j, n, pv, b, s);
            if constexpr (kRec) rec[(j - 1) * rs] = o;
            p = M + o;
        }
        if constexpr (Traits<TS>::kDev) {
            const C2 d = Traits<TS>::template load_dev<LD>(p);
            dm = add2(dm, d);
            f[opp(j)] = add2(d, ref_of<TS>(s, j));
        } else {
            f[opp(j)] = ldm<LD>(p);  // plain storage: the stored pair itself
        }
    }
    if (!Traits<TS>::kDev) dm = sum19(f);
}

// Post-collision population pairs f[i] of node n into their slots.  dm is the
// node's mass from load_pops.  For deviation storage the moving populations
// are quantised first and the rest deviation is dm minus the stored moving
// deviations, so the stored mass equals the mass before collision exactly up
// to FP32 rounding of deviation-sized terms; the codes are stored as computed
// (never re-quantised).  kBack: f[] receives the stored values back (the
// dequantised codes and the stored rest population), as a later load would
// return them.
template <typename TS, int P, bool kBack = false, bool kRec = false>
__device__ __forceinline__ void store_pops(typename Traits<TS>::C2 f[19], typename Traits<TS>::C2 dm, int n,
                                           uint32_t pv, uint32_t fl, const Nbr &b, const DevState &s,
                                           const unsigned *rec = nullptr, int rs = 0)
{
    using C2 = typename Traits<TS>::C2;
    using S2 = typename Traits<TS>::S2;
    S2 *M = reinterpret_cast<S2 *>(s.f);
    const bool plane = P == 1 && (fl & (F_INLET | F_OUTLET));
    S2 q[19];
#pragma unroll
    for (int i = 1; i < 19; ++i) q[i] = Traits<TS>::quant(f[i], ref_of<TS>(s, i));
    if (Traits<TS>::kDev) {
        C2 sum = Traits<TS>::code_value(q[1]);
#pragma unroll
        for (int i = 2; i < 19; ++i) sum = add2(sum, Traits<TS>::code_value(q[i]));
        st_rest_dev<TS>(s, n, sub2(dm, sum));
        if constexpr (kBack) {
            f[0] = add2(sub2(dm, sum), ref_of<TS>(s, 0));
#pragma unroll
            for (int i = 1; i < 19; ++i) f[i] = add2(Traits<TS>::code_value(q[i]), ref_of<TS>(s, i));
        }
    } else {
        st_rest_dev<TS>(s, n, f[0]);
    }
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        if (ez(j) != 0 && plane && outside(j, fl)) continue;  // leaves the domain
        const unsigned o = kRec ? rec[(j - 1) * rs] : slot_in_block<P>(j, n, pv, b, s);
        Traits<TS>::store_q(M + o, q[j]);
    }
}

// Force of Eqs. 10, 11, 13 for both components:
// F^sigma = -G psi^sigma(x) sum_i w_i psi^sigma-bar(x+e_i) e_i + rho^sigma g,
// psi being rho on fluid and rho-tilde on wall voxels; beyond an open plane the
// mirrored direction's neighbour is used (Section 2).  The stencil sums
// neighbour minus own value (the same sum, since sum_i w_i e_i = 0, with far
// less cancellation error in FP32).
template <typename TS, int LD = LD_NC>
__device__ __forceinline__ void forces(typename Traits<TS>::C2 rho, uint32_t pv, uint32_t fl, const Nbr &b,
                                       const DevState &s, typename Traits<TS>::C2 F[3])
{
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    const C2 *psi = reinterpret_cast<const C2 *>(s.psi) + pv;
    C2 a[3] = {mk2(C(0), C(0)), mk2(C(0), C(0)), mk2(C(0), C(0))};
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        const int off = (ez(j) != 0 && outside(j, fl)) ? nb_off(mirz(j), b) : nb_off(j, b);
        const C2 d = sub2(ld_psi<LD>(psi + off, l2_policy()), rho);
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

// Eqs. 6-8: tau_s = sum rho^sigma tau^sigma / rho (nu = c_s^2 (tau - 1/2));
// u = (sum_sigma sum_i e_i f_i^sigma [+ F^sigma / 2]) / rho.
template <typename C, typename C2>
__device__ __forceinline__ void mix_velocity(const C2 f[19], C2 rho, const C2 F[3], const DevState &s, C &inv_rho,
                                             C u[3])
{
    C2 m[3] = {mk2(C(0), C(0)), mk2(C(0), C(0)), mk2(C(0), C(0))};
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        if (ex(i)) m[0] = ex(i) > 0 ? add2(m[0], f[i]) : sub2(m[0], f[i]);
        if (ey(i)) m[1] = ey(i) > 0 ? add2(m[1], f[i]) : sub2(m[1], f[i]);
        if (ez(i)) m[2] = ez(i) > 0 ? add2(m[2], f[i]) : sub2(m[2], f[i]);
    }
    inv_rho = C(1) / (rho.x + rho.y);
    const C h = s.velocity_shift ? C(0.5) : C(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const C2 t = fma2(bc2<C2>(h), F[k], m[k]);
        u[k] = (t.x + t.y) * inv_rho;
    }
}

// Eq. 1 with Eq. 2 equilibrium and Eq. 9 forcing, in place on the pairs f[i]:
// f* = (1 - 1/tau_s) f + f^eq / tau_s + (1 - 1/(2 tau_s)) S.  Directions are
// taken in opposite pairs (i, opp(i)): with eu = e_i.u and eF = e_i.F, the
// pair shares sym = 1 + 4.5 eu^2 - 1.5 u^2 and 9 eu eF - 3 u.F and differs
// only in the sign of 3 eu and 3 eF, so each pair is computed once.
template <typename C, typename C2>
__device__ __forceinline__ void collide(C2 f[19], C2 rho, C inv_rho, const C u[3], const C2 F[3], const DevState &s)
{
    const C tau_s = (rho.x * pick<C>(s.tau1, s.ftau1) + rho.y * pick<C>(s.tau2, s.ftau2)) * inv_rho;
    const C om = C(1) / tau_s;
    const C2 keep = bc2<C2>(C(1) - om);
    const C cf = C(1) - C(0.5) * om;
    const C usq = C(1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    C2 uF = mul2(bc2<C2>(u[0]), F[0]);
    uF = fma2(bc2<C2>(u[1]), F[1], uF);
    uF = fma2(bc2<C2>(u[2]), F[2], uF);
    const C2 cuF = mul2(bc2<C2>(C(-3)), uF);
    const C2 ro = mul2(bc2<C2>(om), rho);
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        if (opp(i) < i) continue;  // each pair once, from its first member
        const int o = opp(i);
        const C w = wgt<C>(i);
        C eu = C(0);
        C2 eF = mk2(C(0), C(0));
        if (ex(i)) { eu += ex(i) * u[0]; eF = ex(i) > 0 ? add2(eF, F[0]) : sub2(eF, F[0]); }
        if (ey(i)) { eu += ey(i) * u[1]; eF = ey(i) > 0 ? add2(eF, F[1]) : sub2(eF, F[1]); }
        if (ez(i)) { eu += ez(i) * u[2]; eF = ez(i) > 0 ? add2(eF, F[2]) : sub2(eF, F[2]); }
        const C sym = C(1) + C(4.5) * eu * eu - usq;
        const C2 A = mul2(bc2<C2>(w), fma2(ro, bc2<C2>(sym), mul2(bc2<C2>(cf), fma2(bc2<C2>(C(9) * eu), eF, cuF))));
        const C2 B = mul2(bc2<C2>(w), fma2(ro, bc2<C2>(C(3) * eu), mul2(bc2<C2>(C(3) * cf), eF)));
        f[i] = fma2(keep, f[i], add2(A, B));
        f[o] = fma2(keep, f[o], sub2(A, B));
    }
    // The rest population is written last as rho^sigma minus the 18 moving
    // post-collision populations, accumulated in direction order.  In exact
    // arithmetic this equals Eq. 1 for i = 0 (sum_i f^eq_i = rho, sum_i S_i =
    // 0); in FP32 it removes the mass bias of the rounded weights (their FP32
    // sum exceeds 1 by ~1.5e-8).
    C2 sum = f[1];
#pragma unroll
    for (int i = 2; i < 19; ++i) sum = add2(sum, f[i]);
    f[0] = sub2(rho, sum);
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

// ---------------------------------------------------------------------------
// Kernels of the split schedule

// Density pass of the split schedule at parity P: plane nodes first apply the
// open-plane extrapolation (idempotent: it only reads the interior node), then
// every node sums its populations.  Nodes are taken in reverse order so the
// pass starts on the lines the collide-stream kernel wrote last (still in L2).
template <typename TS, int PN, int LD>
__device__ __forceinline__ void neem_node(int plane, int p, int nb, uint32_t pvb, uint32_t flb, const DevState &s);

// neem = 0 skips the extrapolation (the state is an initial state that the
// first step must see unchanged).
// Density pass at node n: plane nodes first apply the open-plane rule, then
// every node sums its populations.  The loads are ordinary coherent ones: a
// plane node reads back cells it has just written (read-only cache loads may
// be ordered before those writes), and one shared load path keeps the
// common case as lean as before.
template <typename TS, int P, int LDI = LD_NC>
__device__ __forceinline__ void dens_node_geo(int n, uint32_t pv, uint32_t fl, const DevState &s, int neem)
{
    using C2 = typename Traits<TS>::C2;
    if (neem && (fl & (F_INLET | F_OUTLET))) {
        const int plane = (fl & F_INLET) ? 0 : 1;
        const int p = plane == 0 ? (int)pv : (int)pv - (s.nz - 1) * s.sxy;
        neem_node<TS, P, LDI>(plane, p, n, pv, fl, s);  // LDI: how it reads the interior node
    }
    const Nbr b = make_nbr(fl, s);
    C2 f[19], dm;
    load_pops<TS, P, LD_CA>(f, dm, n, pv, fl, b, s);
    st_pol(reinterpret_cast<C2 *>(s.psi) + pv, density_of<TS>(dm, s), l2_policy());
}

template <typename TS, int P>
__device__ __forceinline__ void dens_node_at(int n, const DevState &s, int neem)
{
    dens_node_geo<TS, P>(n, s.pvox[n], s.nflags[n], s, neem);
}

// Resident blocks per SM of the density pass: four for FP32 and 16-bit
// storage (the odd-parity gather otherwise takes 80 registers and three
// blocks: 39.7 vs 36.8 us per pass on the 128^3 pack), two for FP64.
template <typename TS>
struct DensOcc {
    static constexpr int blocks = 4;
};
template <>
struct DensOcc<double> {
    static constexpr int blocks = 2;
};

// nodes [n0, n1), last first
// The node's voxel and flags never change after creation: they are read
// before waiting for the previous pass (programmatic dependent launch), while
// it drains; everything it writes is read after the wait.
template <typename TS, int P>
__global__ void __launch_bounds__(256, DensOcc<TS>::blocks) k_dens(DevState s, int neem, int n0, int n1)
{
    pdl_trigger();
    const int n = n1 - 1 - (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const bool live = n >= n0;
    const uint32_t pv = live ? s.pvox[n] : 0u;
    const uint32_t fl = live ? s.nflags[n] : 0u;
    pdl_wait();
    if (!live) return;
    dens_node_geo<TS, P>(n, pv, fl, s, neem);
}

// Eq. 15 at one wall voxel: rho-tilde^sigma = chi^sigma * (sum of w_i rho^sigma
// over in-domain fluid neighbours) / (sum of those w_i), chi = 1 +/- xi.
template <typename TS, int LD>
__device__ __forceinline__ void wall_node_geo(int w, uint32_t pv, uint32_t mask, typename Traits<TS>::C inv,
                                              const DevState &s, void *psi_out)
{
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    C2 *psi = reinterpret_cast<C2 *>(psi_out);
    const Nbr b = make_nbr(mask >> kWallFaceShift, s);
    C2 acc = mk2(C(0), C(0));
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        if (mask & (1u << j)) {
            const C2 *q = psi + ((int)pv + nb_off(j, b));
            acc = fma2(bc2<C2>(wgt<C>(j)), LD == LD_CG ? __ldcg(q) : *q, acc);
        }
    }
    const C xi = reinterpret_cast<const C *>(s.wxi)[w];
    st_pol(psi + pv, mul2(acc, mk2((C(1) + xi) * inv, (C(1) - xi) * inv)), l2_policy());
}

template <typename TS, int LD>
__device__ __forceinline__ void wall_node(int w, const DevState &s, void *psi_out)
{
    using C = typename Traits<TS>::C;
    wall_node_geo<TS, LD>(w, s.wpvox[w], s.wmask[w], reinterpret_cast<const C *>(s.winv)[w], s, psi_out);
}

// walls [w0, w1)
// The wall's voxel, mask and Eq. 15 denominator never change after creation
// and are read before the wait; xi (lbm_set_xi_field) and the densities after.
template <typename TS>
__global__ void __launch_bounds__(256) k_wall(DevState s, int w0, int w1)
{
    using C = typename Traits<TS>::C;
    pdl_trigger();
    const int w = w0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const bool live = w < w1;
    const uint32_t pv = live ? s.wpvox[w] : 0u;
    const uint32_t mask = live ? s.wmask[w] : 0u;
    const C inv = live ? reinterpret_cast<const C *>(s.winv)[w] : C(0);
    pdl_wait();
    if (!live) return;
    wall_node_geo<TS, LD_NC>(w, pv, mask, inv, s, s.psi);
}

// F: the fused force / collision / streaming update of one node.  The
// node's own density pair is read from the density map, where the density
// pass stored exactly the sum these populations give (the same loads summed
// in the same order), so the force stencil runs before the populations are
// loaded and the stencil's and the populations' loads never hold registers
// at the same time.
// At parity 1 with rec != nullptr, the 18 slot offsets found at the load
// are kept in shared memory (rec[(j-1) * rs], this thread's column) and
// reused for the stores, which then wait on no index loads.
// LD: LD_NC when the populations and densities were written by earlier
// launches, LD_CA inside a persistent launch that wrote them itself.
template <typename TS, int P, bool kRec = false, int LD = LD_NC>
__device__ __forceinline__ void fused_node_geo(int n, uint32_t pv, uint32_t fl, const DevState &s,
                                               unsigned *rec = nullptr, int rs = 0)
{
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    constexpr bool R = kRec && P == 1;
    const Nbr b = make_nbr(fl, s);
    const C2 rho = ld_psi<LD>(reinterpret_cast<const C2 *>(s.psi) + pv, l2_policy());
    C2 F[3];
    forces<TS, LD>(rho, pv, fl, b, s, F);
    C2 f[19], dm;
    load_pops<TS, P, LD, R>(f, dm, n, pv, fl, b, s, rec, rs);
    C u[3], inv_rho;
    mix_velocity<C, C2>(f, rho, F, s, inv_rho, u);
    collide<C, C2>(f, rho, inv_rho, u, F, s);
    store_pops<TS, P, false, R>(f, dm, n, pv, fl, b, s, rec, rs);
}

// Shared memory of the collide-stream kernels at parity 1: 18 slot offsets per thread.
__host__ __device__ constexpr size_t slot_rec_bytes(int parity, int block)
{
    return parity ? (size_t)18 * sizeof(unsigned) * (size_t)block : 0;
}

template <typename TS, int P>
__device__ __forceinline__ void fused_node(int n, const DevState &s)
{
    fused_node_geo<TS, P>(n, s.pvox[n], s.nflags[n], s);
}

// nodes [n0, n1); the node's voxel and flags are read before the wait
// kRec: parity-1 slot offsets kept in dynamic shared memory (slot_rec_bytes)
template <typename TS, int P, bool kRec = false>
__global__ void __launch_bounds__(256, PipeOcc<TS>::blocks) k_fused(DevState s, int n0, int n1)
{
    extern __shared__ unsigned slot_rec[];
    pdl_trigger();
    const int n = n0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const bool live = n < n1;
    const uint32_t pv = live ? s.pvox[n] : 0u;
    const uint32_t fl = live ? s.nflags[n] : 0u;
    pdl_wait();
    if (!live) return;
    fused_node_geo<TS, P, kRec>(n, pv, fl, s, slot_rec + threadIdx.x, (int)blockDim.x);
}

// Open planes, for the parity PN of the step that reads next: the prescribed
// component (1 at the inlet, 2 at the outlet) gets all 19 populations by
// non-equilibrium extrapolation from the first interior node,
// f_i(xb) = f^eq_i(rho_b, u) + f_i(xi) - f^eq_i(rho(xi), u) with u the
// barycentric velocity of xi; the other component's missing populations get
// their initial values back (Section 2).
// Zou-He form: the prescribed component's entering populations from the
// node's own known ones, so that its density is rho_b, its tangential
// momentum vanishes and f_i - f_opp(i) = 6 w_i rho_b u_n for the normal pair:
// with j_n = rho_b - (in-plane sum + 2 outgoing sum) and N_t = half the
// in-plane tangential momentum, f_i = f_opp(i) + 6 w_i j_n - e_i,t . N.
// The plane is a template parameter so that every population index below
// is a compile-time constant (the pairs stay in registers).
template <typename TS, int PN, int LD, int PL>
__device__ __forceinline__ void zou_he_node(int nb, uint32_t pvb, uint32_t flb, const DevState &s)
{
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    using S2 = typename Traits<TS>::S2;
    const Nbr bb = make_nbr(flb, s);
    C2 f[19], dm;
    load_pops<TS, PN, LD>(f, dm, nb, pvb, flb, bb, s);
    constexpr int plane = PL;
    constexpr int pc = PL;                // prescribed component
    constexpr int dir = PL == 0 ? 1 : -1;  // e_z of the entering directions
    C s0 = 0, sout = 0, nx = 0, ny = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const C v = pc == 0 ? f[i].x : f[i].y;
        if (ez(i) == 0) {
            s0 += v;
            nx += ex(i) * v;
            ny += ey(i) * v;
        } else if (ez(i) == -dir) {
            sout += v;
        }
    }
    const C rb = (plane == 0 ? pick<C>(s.rho_in1, s.frho_in1) : pick<C>(s.rho_out2, s.frho_out2));
    const C jn = rb - (s0 + C(2) * sout);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int i = miss_dir(plane, k);
        const C fo = pc == 0 ? f[opp(i)].x : f[opp(i)].y;
        const C v = fo + C(6) * wgt<C>(i) * jn - C(0.5) * (ex(i) * nx + ey(i) * ny);
        S2 *q = slot_ptr<TS, PN>(opp(i), nb, pvb, flb, bb, s);
        Traits<TS>::store1(q, pc, v, pc == 0 ? ref_of<TS>(s, i).x : ref_of<TS>(s, i).y);
    }
}

template <typename TS, int PN, int LD>
__device__ __forceinline__ void neem_node(int plane, int p, int nb, uint32_t pvb, uint32_t flb, const DevState &s)
{
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    using S2 = typename Traits<TS>::S2;
    if (s.zou_he) {
        if (plane == 0) zou_he_node<TS, PN, LD, 0>(nb, pvb, flb, s);
        else zou_he_node<TS, PN, LD, 1>(nb, pvb, flb, s);
        // the other component's entering populations keep their initial values
        const Nbr bb = make_nbr(flb, s);
        const int qc = 1 - plane;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int i = miss_dir(plane, k);
            const C v = (C)s.frozen[(long long)(plane * 5 + k) * s.nxy + p];
            S2 *q = slot_ptr<TS, PN>(opp(i), nb, pvb, flb, bb, s);
            Traits<TS>::store1(q, qc, v, qc == 0 ? ref_of<TS>(s, i).x : ref_of<TS>(s, i).y);
        }
        return;
    }
    const uint32_t pvi = plane == 0 ? pvb + s.sxy : pvb - s.sxy;
    const int ni = s.cidx[pvi];
    const uint32_t fli = s.nflags[ni];
    const Nbr bi = make_nbr(fli, s);
    const Nbr bb = make_nbr(flb, s);
    C2 fi[19], dmi;
    load_pops<TS, PN, LD>(fi, dmi, ni, pvi, fli, bi, s);
    const C2 r = density_of<TS>(dmi, s);
    C m[3] = {0, 0, 0};
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const C tt = fi[i].x + fi[i].y;
        if (ex(i)) m[0] += ex(i) * tt;
        if (ey(i)) m[1] += ey(i) * tt;
        if (ez(i)) m[2] += ez(i) * tt;
    }
    const C ir = C(1) / (r.x + r.y);
    const C u[3] = {m[0] * ir, m[1] * ir, m[2] * ir};
    const C usq = C(1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const C rb = (plane == 0 ? pick<C>(s.rho_in1, s.frho_in1) : pick<C>(s.rho_out2, s.frho_out2));
    const C rin = plane == 0 ? r.x : r.y;
    const int pc = plane;  // prescribed component
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const C eu = ex(i) * u[0] + ey(i) * u[1] + ez(i) * u[2];
        const C base = C(1) + C(3) * eu + C(4.5) * eu * eu - usq;
        const C fin = plane == 0 ? fi[i].x : fi[i].y;
        const C v = wgt<C>(i) * rb * base + fin - wgt<C>(i) * rin * base;
        if (i == 0) {
            C2 rv = ld_rest<TS, LD>(s, nb);
            if (pc == 0) rv.x = v; else rv.y = v;
            st_rest<TS>(s, nb, rv);
        } else {
            S2 *q = slot_ptr<TS, PN>(opp(i), nb, pvb, flb, bb, s);
            Traits<TS>::store1(q, pc, v, pc == 0 ? ref_of<TS>(s, i).x : ref_of<TS>(s, i).y);
        }
    }
    const int qc = 1 - pc;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int i = miss_dir(plane, k);
        const C v = (C)s.frozen[(long long)(plane * 5 + k) * s.nxy + p];
        S2 *q = slot_ptr<TS, PN>(opp(i), nb, pvb, flb, bb, s);
        Traits<TS>::store1(q, qc, v, qc == 0 ? ref_of<TS>(s, i).x : ref_of<TS>(s, i).y);
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
    neem_node<TS, PN, LD_NC>(plane, p, nb, pvb, s.nflags[nb], s);
}

// ---------------------------------------------------------------------------
// Batched kernels: one launch covers the blocks of many samples.  map[b] =
// (sample k, block index within the sample); the block copies states[k] to
// shared memory and works on that sample exactly like the single-sample
// kernel (same per-node functions, same results).

__device__ __forceinline__ const DevState &stage_state(const DevState *states, int k, DevState *sh)
{
    const int words = (int)(sizeof(DevState) / 4);
    const unsigned *src = reinterpret_cast<const unsigned *>(states + k);
    unsigned *dst = reinterpret_cast<unsigned *>(sh);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = __ldg(src + w);
    __syncthreads();
    return *sh;
}

template <typename TS, int P>
__global__ void __launch_bounds__(256) k_dens_batch(const DevState *states, const int2 *map, int neem)
{
    pdl_trigger();
    pdl_wait();
    __shared__ __align__(16) DevState sh;
    const int2 m = map[gridDim.x - 1 - blockIdx.x];  // last node of the last sample first, as k_dens_table
    const DevState &s = stage_state(states, m.x, &sh);
    const int n = m.y * blockDim.x + threadIdx.x;
    if (n < s.n_fluid) dens_node_at<TS, P>(n, s, neem && s.open_z);
}

template <typename TS>
__global__ void __launch_bounds__(256) k_wall_batch(const DevState *states, const int2 *map)
{
    pdl_trigger();
    pdl_wait();
    __shared__ __align__(16) DevState sh;
    const int2 m = map[blockIdx.x];
    const DevState &s = stage_state(states, m.x, &sh);
    const int w = m.y * blockDim.x + threadIdx.x;
    if (w < s.n_wall) wall_node<TS, LD_NC>(w, s, s.psi);
}

template <typename TS, int P>
__global__ void __launch_bounds__(256, PipeOcc<TS>::blocks) k_fused_batch(const DevState *states, const int2 *map)
{
    pdl_trigger();
    pdl_wait();
    __shared__ __align__(16) DevState sh;
    const int2 m = map[blockIdx.x];
    const DevState &s = stage_state(states, m.x, &sh);
    const int n = m.y * blockDim.x + threadIdx.x;
    if (n < s.n_fluid) fused_node<TS, P>(n, s);
}

// Batched kernels with the batch table in parameter space (BatchTable): the
// block's sample is the last k with start[k] <= blockIdx.x (binary search in
// parameter memory), its node or wall index the rest; the geometry words are
// read before the dependent-launch wait, as in the solo passes.
__device__ __forceinline__ int table_sample(const int *start, int count, int blk)
{
    int lo = 0, hi = count - 1;  // start[lo] <= blk < start[hi + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int table_sample(const int *start, int count)
{
    return table_sample(start, count, (int)blockIdx.x);
}

template <typename TS, int P>
__global__ void __launch_bounds__(256, DensOcc<TS>::blocks) k_dens_table(const __grid_constant__ BatchTable t, int neem)
{
    pdl_trigger();
    // the whole batch last node first (samples in reverse order too), so the
    // pass starts on the cells the collide-stream pass wrote last and ends on
    // those its next launch reads first
    const int rb = t.start_n[t.count] - 1 - (int)blockIdx.x;
    const int k = table_sample(t.start_n, t.count, rb);
    const DevState &s = t.s[k];
    const int n = (rb - t.start_n[k]) * (int)blockDim.x + (int)threadIdx.x;
    const bool live = n < s.n_fluid;
    const uint32_t pv = live ? s.pvox[n] : 0u;
    const uint32_t fl = live ? s.nflags[n] : 0u;
    pdl_wait();
    if (!live) return;
    dens_node_geo<TS, P>(n, pv, fl, s, neem && s.open_z);
}

template <typename TS>
__global__ void __launch_bounds__(256) k_wall_table(const __grid_constant__ BatchTable t)
{
    using C = typename Traits<TS>::C;
    pdl_trigger();
    const int k = table_sample(t.start_w, t.count);
    const DevState &s = t.s[k];
    const int w = ((int)blockIdx.x - t.start_w[k]) * (int)blockDim.x + (int)threadIdx.x;
    const bool live = w < s.n_wall;
    const uint32_t pv = live ? s.wpvox[w] : 0u;
    const uint32_t mask = live ? s.wmask[w] : 0u;
    const C inv = live ? reinterpret_cast<const C *>(s.winv)[w] : C(0);
    pdl_wait();
    if (!live) return;
    wall_node_geo<TS, LD_NC>(w, pv, mask, inv, s, s.psi);
}

template <typename TS, int P>
__global__ void __launch_bounds__(256, PipeOcc<TS>::blocks) k_fused_table(const __grid_constant__ BatchTable t)
{
    extern __shared__ unsigned slot_rec[];  // parity 1: slot_rec_bytes(1, blockDim.x)
    pdl_trigger();
    const int k = table_sample(t.start_n, t.count);
    const DevState &s = t.s[k];
    const int n = ((int)blockIdx.x - t.start_n[k]) * (int)blockDim.x + (int)threadIdx.x;
    const bool live = n < s.n_fluid;
    const uint32_t pv = live ? s.pvox[n] : 0u;
    const uint32_t fl = live ? s.nflags[n] : 0u;
    pdl_wait();
    if (!live) return;
    fused_node_geo<TS, P, true>(n, pv, fl, s, slot_rec + threadIdx.x, (int)blockDim.x);
}

// ---------------------------------------------------------------------------
// State transfer and diagnostics.  Host-side population arrays are
// [sigma][i][v] doubles over the dense grid.

template <typename TS>
__global__ void k_init_eq(DevState s, const double *rho)
{
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    using S2 = typename Traits<TS>::S2;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n_fluid) return;
    const uint32_t pv = s.pvox[n];
    const C2 r = mk2((C)rho[pv], (C)rho[s.nv + pv]);
    st_rest<TS>(s, n, mul2(bc2<C2>(wgt<C>(0)), r));
    S2 *M = reinterpret_cast<S2 *>(s.f);
#pragma unroll
    for (int i = 1; i < 19; ++i) Traits<TS>::store(M + (long long)(i - 1) * s.npad + n, mul2(bc2<C2>(wgt<C>(i)), r), ref_of<TS>(s, i));
}

template <typename TS>
__global__ void k_scatter(DevState s, const double *f)
{
    using C = typename Traits<TS>::C;
    using S2 = typename Traits<TS>::S2;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n_fluid) return;
    const long long pv = s.pvox[n];
    st_rest<TS>(s, n, mk2((C)f[pv], (C)f[19 * s.nv + pv]));
    S2 *M = reinterpret_cast<S2 *>(s.f);
    for (int i = 1; i < 19; ++i)
        Traits<TS>::store(M + (long long)(i - 1) * s.npad + n, mk2((C)f[i * s.nv + pv], (C)f[(19 + i) * s.nv + pv]),
                          ref_of<TS>(s, i));
}

template <typename TS, int P>
__global__ void k_gather(DevState s, double *out)
{
    using C2 = typename Traits<TS>::C2;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n_fluid) return;
    const uint32_t pv = s.pvox[n];
    const uint32_t fl = s.nflags[n];
    const Nbr b = make_nbr(fl, s);
    C2 f[19], dm;
    load_pops<TS, P>(f, dm, n, pv, fl, b, s);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        out[(long long)i * s.nv + pv] = (double)f[i].x;
        out[(long long)(19 + i) * s.nv + pv] = (double)f[i].y;
    }
}

// Frozen values: the initial populations of the non-prescribed component in
// the missing directions of each open plane (parity-0 layout).
template <typename TS>
__global__ void k_capture_frozen(DevState s, double *frozen)
{
    using C2 = typename Traits<TS>::C2;
    using S2 = typename Traits<TS>::S2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * s.nxy) return;
    const int plane = t >= s.nxy ? 1 : 0;
    const int p = t - plane * s.nxy;
    const uint32_t pvb = plane == 0 ? (uint32_t)p : (uint32_t)(p + (s.nz - 1) * s.sxy);
    const int nb = s.cidx[pvb];
    const int qc = 1 - plane;
    const S2 *M = reinterpret_cast<const S2 *>(s.f);
    for (int k = 0; k < 5; ++k) {
        const int i = miss_dir(plane, k);
        double v = 0;
        if (nb >= 0) {
            const C2 q = Traits<TS>::load(M + (long long)(i - 1) * s.npad + nb, ref_of<TS>(s, i));
            v = (double)(qc == 0 ? q.x : q.y);
        }
        frozen[(long long)(plane * 5 + k) * s.nxy + p] = v;
    }
}

// Fields of the current state at every voxel (zero at solids), packed: the
// fields whose bit is set in `mask` (RHO1, RHO2, UX, UY, UZ, P), in bit order,
// nv doubles each.
template <typename TS, int P>
__global__ void k_fields(DevState s, double *out, uint32_t mask)
{
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= s.nv) return;
    double val[6] = {0, 0, 0, 0, 0, 0};
    const int n = s.cidx[v];
    if (n >= 0) {
        const uint32_t pv = (uint32_t)v;
        const uint32_t fl = s.nflags[n];
        const Nbr b = make_nbr(fl, s);
        C2 f[19], dm;
        load_pops<TS, P>(f, dm, n, pv, fl, b, s);
        const C2 rho = density_of<TS>(dm, s);
        C2 F[3];
        C u[3], inv_rho;
        forces<TS>(rho, pv, fl, b, s, F);
        mix_velocity<C, C2>(f, rho, F, s, inv_rho, u);
        const C cs2 = C(1) / C(3);
        val[0] = (double)rho.x;
        val[1] = (double)rho.y;
        val[2] = (double)u[0];
        val[3] = (double)u[1];
        val[4] = (double)u[2];
        val[5] = (double)(cs2 * (rho.x + rho.y) + cs2 * pick<C>(s.G, s.fG) * rho.x * rho.y);
    }
    int k = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q)
        if (mask & (1u << q)) out[(long long)(k++) * s.nv + v] = val[q];
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
