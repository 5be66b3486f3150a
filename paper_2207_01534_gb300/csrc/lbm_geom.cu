// lbm_geom.cu -- geometry preprocessing of lbm_create on the device: the
// compact fluid index in voxel order (cidx, pvox, flag bytes), the wall list
// of Eq. 15 (voxel, fluid-neighbour mask with face bits, 1 / sum of weights,
// xi), the first node and wall of every z plane, and the geometry checks.
// The results are those of the host preprocessing, entry for entry: the same
// order, the same masks, the Eq. 15 denominators summed in the same order in
// FP64.
//
// Blocks cover 1024-voxel segments that never straddle a z plane; a first
// pass counts each block's fluid voxels and walls, one block turns the
// counts into offsets (and the plane prefixes), and a second pass writes
// every entry at its offset plus its rank among the block's entries in voxel
// order (warp ballots).
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_kernels.cuh"

namespace lbm {

namespace {

constexpr int kGeomThreads = 256;
constexpr int kGeomSeg = 4 * kGeomThreads;  // voxels per block

struct GeomDims {
    int nx, ny, nz;
    int per[3];
    int open_z;
    int bpp;        // blocks per z plane
    long long nxy;
};

// Periodic-face bits of a voxel (as the host's face_bits).
__device__ __forceinline__ uint32_t face_bits_of(int x, int y, int z, const GeomDims &d)
{
    uint32_t f = 0;
    if (d.per[0] && x == 0) f |= F_XLO;
    if (d.per[0] && x == d.nx - 1) f |= F_XHI;
    if (d.per[1] && y == 0) f |= F_YLO;
    if (d.per[1] && y == d.ny - 1) f |= F_YHI;
    if (d.per[2] && z == 0) f |= F_ZLO;
    if (d.per[2] && z == d.nz - 1) f |= F_ZHI;
    return f;
}

struct Voxel {
    bool fluid, wall;
    uint32_t word;  // fluid: flag byte; wall: mask | face bits << kWallFaceShift
    double den;     // wall: sum of w_j over the in-domain fluid neighbours
    int err;        // bit 0: fluid touches a closed face; bit 1: open-plane node with a solid interior neighbour
};

__device__ Voxel classify(const uint8_t *solid, const GeomDims &d, long long v)
{
    Voxel r{false, false, 0u, 0.0, 0};
    const int x = (int)(v % d.nx);
    const int y = (int)((v / d.nx) % d.ny);
    const int z = (int)(v / d.nxy);
    const int c[3] = {x, y, z};
    const int dims[3] = {d.nx, d.ny, d.nz};
    if (!solid[v]) {
        r.fluid = true;
        uint32_t f = face_bits_of(x, y, z, d);
        if (d.open_z && z == 0) f |= F_INLET;
        if (d.open_z && z == d.nz - 1) f |= F_OUTLET;
        r.word = f;
        const bool face = x == 0 || x == d.nx - 1 || y == 0 || y == d.ny - 1 || z == 0 || z == d.nz - 1;
        if (face) {
            for (int j = 1; j < 19; ++j) {
                const int e[3] = {ex(j), ey(j), ez(j)};
                for (int a = 0; a < 3; ++a) {
                    const int m = c[a] + e[a];
                    if ((m < 0 || m >= dims[a]) && !d.per[a] && !(d.open_z && a == 2)) r.err |= 1;
                }
            }
        }
        if (d.open_z && (z == 0 || z == d.nz - 1) && solid[v + (z == 0 ? 1 : -1) * d.nxy]) r.err |= 2;
        return r;
    }
    uint32_t mask = 0;
    double den = 0.0;
    for (int j = 1; j < 19; ++j) {
        int m[3] = {c[0] + ex(j), c[1] + ey(j), c[2] + ez(j)};
        bool in = true;
        for (int a = 0; a < 3; ++a) {
            if (m[a] < 0 || m[a] >= dims[a]) {
                if (!d.per[a]) in = false;
                m[a] = (m[a] + dims[a]) % dims[a];
            }
        }
        if (!in) continue;
        const long long u = m[0] + (long long)d.nx * (m[1] + (long long)d.ny * m[2]);
        if (!solid[u]) {
            mask |= 1u << j;
            den += wgt<double>(j);
        }
    }
    if (mask) {
        r.wall = true;
        r.word = mask | (face_bits_of(x, y, z, d) << kWallFaceShift);
        r.den = den;
    }
    return r;
}

__device__ __forceinline__ void block_range(const GeomDims &d, long long *v0, long long *v1)
{
    const int z = blockIdx.x / d.bpp, s = blockIdx.x % d.bpp;
    *v0 = (long long)z * d.nxy + (long long)s * kGeomSeg;
    const long long end = (long long)(z + 1) * d.nxy;
    *v1 = *v0 + kGeomSeg < end ? *v0 + kGeomSeg : end;
}

__global__ void __launch_bounds__(kGeomThreads) k_geom_count(const uint8_t *solid, GeomDims d, int2 *cnt, int *err)
{
    long long v0, v1;
    block_range(d, &v0, &v1);
    int nf = 0, nw = 0, e = 0;
    for (long long v = v0 + threadIdx.x; v < v1; v += kGeomThreads) {
        const Voxel q = classify(solid, d, v);
        nf += q.fluid;
        nw += q.wall;
        e |= q.err;
    }
    for (int o = 16; o > 0; o >>= 1) {
        nf += __shfl_down_sync(0xffffffffu, nf, o);
        nw += __shfl_down_sync(0xffffffffu, nw, o);
        e |= __shfl_down_sync(0xffffffffu, e, o);
    }
    __shared__ int sf[kGeomThreads / 32], sw[kGeomThreads / 32], se[kGeomThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sf[wid] = nf;
        sw[wid] = nw;
        se[wid] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0, c = 0;
        for (int k = 0; k < kGeomThreads / 32; ++k) {
            a += sf[k];
            b += sw[k];
            c |= se[k];
        }
        cnt[blockIdx.x] = make_int2(a, b);
        if (c) atomicOr(err, c);
    }
}

// One block: exclusive offsets of the block counts, the totals and the
// first node / wall of every z plane.  out = [N, NW, plane_n[0..nz],
// plane_w[0..nz]].
__global__ void __launch_bounds__(1024) k_geom_scan(const int2 *cnt, int nb, GeomDims d, int2 *off, int *out)
{
    __shared__ int wf[32], ww[32];
    __shared__ int carry_f, carry_w;
    if (threadIdx.x == 0) carry_f = carry_w = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += 1024) {
        const int b = base + (int)threadIdx.x;
        const int2 v = b < nb ? cnt[b] : make_int2(0, 0);
        int f = v.x, w = v.y;  // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const int tf = __shfl_up_sync(0xffffffffu, f, o), tw = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) {
                f += tf;
                w += tw;
            }
        }
        if (lane == 31) {
            wf[wid] = f;
            ww[wid] = w;
        }
        __syncthreads();
        if (wid == 0) {
            int a = wf[lane], c = ww[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int ta = __shfl_up_sync(0xffffffffu, a, o), tc = __shfl_up_sync(0xffffffffu, c, o);
                if (lane >= o) {
                    a += ta;
                    c += tc;
                }
            }
            wf[lane] = a;  // inclusive over warps
            ww[lane] = c;
        }
        __syncthreads();
        const int pf = carry_f + (wid ? wf[wid - 1] : 0) + f - v.x;
        const int pw = carry_w + (wid ? ww[wid - 1] : 0) + w - v.y;
        if (b < nb) {
            off[b] = make_int2(pf, pw);
            if (b % d.bpp == 0) {
                out[2 + b / d.bpp] = pf;
                out[2 + (d.nz + 1) + b / d.bpp] = pw;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_f += wf[31];
            carry_w += ww[31];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = carry_f;
        out[1] = carry_w;
        out[2 + d.nz] = carry_f;
        out[2 + (d.nz + 1) + d.nz] = carry_w;
    }
}

template <typename C>
__global__ void __launch_bounds__(kGeomThreads) k_geom_fill(const uint8_t *solid, const float *xi_field, double xi0,
                                                            GeomDims d, const int2 *off, int32_t *cidx, uint32_t *pvox,
                                                            uint8_t *nflags, uint32_t *wpvox, uint32_t *wmask,
                                                            C *winv, C *wxi)
{
    long long v0, v1;
    block_range(d, &v0, &v1);
    __shared__ int sf[kGeomThreads / 32], sw[kGeomThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    int nf = off[blockIdx.x].x, nw = off[blockIdx.x].y;
    for (long long r0 = v0; r0 < v1; r0 += kGeomThreads) {  // rounds of 256 voxels, in voxel order
        const long long v = r0 + threadIdx.x;
        Voxel q{false, false, 0u, 0.0, 0};
        if (v < v1) q = classify(solid, d, v);
        const unsigned bf = __ballot_sync(0xffffffffu, q.fluid), bw = __ballot_sync(0xffffffffu, q.wall);
        if (lane == 0) {
            sf[wid] = __popc(bf);
            sw[wid] = __popc(bw);
        }
        __syncthreads();
        int pf = nf, pw = nw, tf = 0, tw = 0;
        for (int k = 0; k < kGeomThreads / 32; ++k) {
            if (k < wid) {
                pf += sf[k];
                pw += sw[k];
            }
            tf += sf[k];
            tw += sw[k];
        }
        pf += __popc(bf & below);
        pw += __popc(bw & below);
        if (v < v1) {
            cidx[v] = q.fluid ? pf : -1;
            if (q.fluid) {
                pvox[pf] = (uint32_t)v;
                nflags[pf] = (uint8_t)q.word;
            }
            if (q.wall) {
                wpvox[pw] = (uint32_t)v;
                wmask[pw] = q.word;
                winv[pw] = (C)(1.0 / q.den);
                wxi[pw] = (C)(xi_field ? (double)xi_field[v] : xi0);
            }
        }
        nf += tf;
        nw += tw;
        __syncthreads();
    }
}

}  // namespace

// Host entry points (declared in lbm_internal.h).
GeomPlan geom_plan(const uint8_t *d_solid, int nx, int ny, int nz, const int per[3], int open_z)
{
    GeomPlan g{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    for (int a = 0; a < 3; ++a) g.per[a] = per[a];
    g.open_z = open_z;
    const long long nxy = (long long)nx * ny;
    g.bpp = (int)((nxy + kGeomSeg - 1) / kGeomSeg);
    g.nblocks = g.bpp * nz;
    g.d_solid = d_solid;
    return g;
}

static GeomDims dims_of(const GeomPlan &g)
{
    GeomDims d{};
    d.nx = g.nx;
    d.ny = g.ny;
    d.nz = g.nz;
    for (int a = 0; a < 3; ++a) d.per[a] = g.per[a];
    d.open_z = g.open_z;
    d.bpp = g.bpp;
    d.nxy = (long long)g.nx * g.ny;
    return d;
}

void geom_count(const GeomPlan &g, int2 *d_cnt, int2 *d_off, int *d_err, int *d_out, cudaStream_t st)
{
    const GeomDims d = dims_of(g);
    k_geom_count<<<g.nblocks, kGeomThreads, 0, st>>>(g.d_solid, d, d_cnt, d_err);
    k_geom_scan<<<1, 1024, 0, st>>>(d_cnt, g.nblocks, d, d_off, d_out);
}

void geom_fill(const GeomPlan &g, const float *d_xi, double xi0, const int2 *d_off, int32_t *cidx, uint32_t *pvox,
               uint8_t *nflags, uint32_t *wpvox, uint32_t *wmask, void *winv, void *wxi, bool fp64, cudaStream_t st)
{
    const GeomDims d = dims_of(g);
    if (fp64)
        k_geom_fill<double><<<g.nblocks, kGeomThreads, 0, st>>>(g.d_solid, d_xi, xi0, d, d_off, cidx, pvox, nflags,
                                                                wpvox, wmask, (double *)winv, (double *)wxi);
    else
        k_geom_fill<float><<<g.nblocks, kGeomThreads, 0, st>>>(g.d_solid, d_xi, xi0, d, d_off, cidx, pvox, nflags,
                                                               wpvox, wmask, (float *)winv, (float *)wxi);
}

}  // namespace lbm
