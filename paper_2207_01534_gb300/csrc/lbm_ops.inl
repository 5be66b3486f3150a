// lbm_ops.inl -- launchers of the split-schedule kernels for one storage type.
// Included by lbm_fp32.cu / lbm_fp64.cu after lbm_kernels.cuh.
#pragma once

#include <cstdlib>

#include "lbm_persist.cuh"

namespace lbm {

static inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <typename TS>
void Ops<TS>::dens(const DevState &s, int parity, int neem, cudaStream_t st, int block, int n0, int n1)
{
    if (n1 < 0) n1 = s.n_fluid;
    if (n1 <= n0) return;
    const int ne = neem && s.open_z;
    const unsigned g = grid_for(n1 - n0, block);
    if (parity) launch_pdl(k_dens<TS, 1>, g, block, 0, st, s, ne, n0, n1);
    else launch_pdl(k_dens<TS, 0>, g, block, 0, st, s, ne, n0, n1);
}

template <typename TS>
void Ops<TS>::wall(const DevState &s, cudaStream_t st, int block, int w0, int w1)
{
    if (w1 < 0) w1 = s.n_wall;
    if (w1 <= w0) return;
    launch_pdl(k_wall<TS>, grid_for(w1 - w0, block), block, 0, st, s, w0, w1);
}

template <typename TS>
void Ops<TS>::fused(const DevState &s, int parity, cudaStream_t st, int block, int n0, int n1)
{
    if (n1 < 0) n1 = s.n_fluid;
    if (n1 <= n0) return;
    const unsigned g = grid_for(n1 - n0, block);
    // parity 1 keeps its slot offsets in shared memory between the loads and
    // the stores (128^3 pack: FP32 50.0 -> 48.7 us, FP16 43.0 -> 40.4 us)
    if (parity) launch_pdl(k_fused<TS, 1, true>, g, block, slot_rec_bytes(1, block), st, s, n0, n1);
    else launch_pdl(k_fused<TS, 0>, g, block, 0, st, s, n0, n1);
}

template <typename TS>
void Ops<TS>::dens_batch(const DevState *states, const int2 *map, int nblocks, int parity, int neem, cudaStream_t st,
                         int block)
{
    if (nblocks <= 0) return;
    if (parity) launch_pdl(k_dens_batch<TS, 1>, (unsigned)nblocks, block, 0, st, states, map, neem);
    else launch_pdl(k_dens_batch<TS, 0>, (unsigned)nblocks, block, 0, st, states, map, neem);
}

template <typename TS>
void Ops<TS>::wall_batch(const DevState *states, const int2 *map, int nblocks, cudaStream_t st, int block)
{
    if (nblocks <= 0) return;
    launch_pdl(k_wall_batch<TS>, (unsigned)nblocks, block, 0, st, states, map);
}

template <typename TS>
void Ops<TS>::fused_batch(const DevState *states, const int2 *map, int nblocks, int parity, cudaStream_t st, int block)
{
    if (nblocks <= 0) return;
    if (parity) launch_pdl(k_fused_batch<TS, 1>, (unsigned)nblocks, block, 0, st, states, map);
    else launch_pdl(k_fused_batch<TS, 0>, (unsigned)nblocks, block, 0, st, states, map);
}

template <typename TS>
void Ops<TS>::dens_table(const BatchTable &t, int parity, int neem, cudaStream_t st, int block)
{
    const int nb = t.start_n[t.count];
    if (nb <= 0) return;
    if (parity) launch_pdl(k_dens_table<TS, 1>, (unsigned)nb, block, 0, st, t, neem);
    else launch_pdl(k_dens_table<TS, 0>, (unsigned)nb, block, 0, st, t, neem);
}

template <typename TS>
void Ops<TS>::wall_table(const BatchTable &t, cudaStream_t st, int block)
{
    const int nb = t.start_w[t.count];
    if (nb <= 0) return;
    launch_pdl(k_wall_table<TS>, (unsigned)nb, block, 0, st, t);
}

template <typename TS>
void Ops<TS>::fused_table(const BatchTable &t, int parity, cudaStream_t st, int block)
{
    const int nb = t.start_n[t.count];
    if (nb <= 0) return;
    if (parity) launch_pdl(k_fused_table<TS, 1>, (unsigned)nb, block, slot_rec_bytes(1, block), st, t);
    else launch_pdl(k_fused_table<TS, 0>, (unsigned)nb, block, 0, st, t);
}

template <typename TS>
void Ops<TS>::plane(const DevState &s, int parity_next, cudaStream_t st)
{
    if (!s.open_z || s.nxy == 0) return;
    if (parity_next) k_plane<TS, 1><<<grid_for(2LL * s.nxy, 128), 128, 0, st>>>(s);
    else k_plane<TS, 0><<<grid_for(2LL * s.nxy, 128), 128, 0, st>>>(s);
}

template <typename TS>
void Ops<TS>::init_eq(const DevState &s, const double *rho, cudaStream_t st)
{
    if (s.n_fluid == 0) return;
    k_init_eq<TS><<<grid_for(s.n_fluid, 256), 256, 0, st>>>(s, rho);
}

template <typename TS>
void Ops<TS>::scatter(const DevState &s, const double *f, cudaStream_t st)
{
    if (s.n_fluid == 0) return;
    k_scatter<TS><<<grid_for(s.n_fluid, 256), 256, 0, st>>>(s, f);
}

template <typename TS>
void Ops<TS>::gather(const DevState &s, int parity, double *f, cudaStream_t st)
{
    if (s.n_fluid == 0) return;
    if (parity) k_gather<TS, 1><<<grid_for(s.n_fluid, 256), 256, 0, st>>>(s, f);
    else k_gather<TS, 0><<<grid_for(s.n_fluid, 256), 256, 0, st>>>(s, f);
}

template <typename TS>
void Ops<TS>::capture_frozen(const DevState &s, double *frozen, cudaStream_t st)
{
    if (!s.open_z || s.nxy == 0) return;
    k_capture_frozen<TS><<<grid_for(2LL * s.nxy, 128), 128, 0, st>>>(s, frozen);
}

template <typename TS>
void Ops<TS>::fields(const DevState &s, int parity, double *out, uint32_t mask, cudaStream_t st)
{
    if (s.nv == 0 || !(mask & 63u)) return;
    if (parity) k_fields<TS, 1><<<grid_for(s.nv, 256), 256, 0, st>>>(s, out, mask & 63u);
    else k_fields<TS, 0><<<grid_for(s.nv, 256), 256, 0, st>>>(s, out, mask & 63u);
}

template <typename TS>
void Ops<TS>::reduce(const DevState &s, double *partials, int nblocks, double *out, cudaStream_t st)
{
    k_reduce<TS><<<nblocks, kReduceThreads, 0, st>>>(s, partials);
    k_reduce_final<<<1, kReduceThreads, 0, st>>>(partials, nblocks, out);
}

template <typename TS>
void Ops<TS>::pipe(const DevState &s, const PipeState &ps, int parity, int grid, cudaStream_t st)
{
    if (ps.n_chunks <= 0 || grid <= 0) return;
    DevState a = s;
    PipeState b = ps;
    void *args[] = {&a, &b};
    const void *fn = parity ? (const void *)k_pipe<TS, 1> : (const void *)k_pipe<TS, 0>;
    cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kChunk), args, 0, st);
}

template <typename TS>
void Ops<TS>::flow(const DevState &s, const FlowState &fs, int parity, cudaStream_t st)
{
    if (fs.n_slots <= 0) return;
    if (parity) launch_pdl(k_flow<TS, 1>, (unsigned)fs.n_slots, kFlowThreads, 0, st, s, fs);
    else launch_pdl(k_flow<TS, 0>, (unsigned)fs.n_slots, kFlowThreads, 0, st, s, fs);
}

template <typename TS>
int Ops<TS>::pipe_blocks_per_sm()
{
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pipe<TS, 0>, kChunk, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pipe<TS, 1>, kChunk, 0);
    return a < b ? a : b;
}

template <typename TS>
cudaError_t Ops<TS>::persist(const BatchTable &t, const PersistArgs &pa, int grid, int block, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = slot_rec_bytes(1, block);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_persist<TS>, t, pa);
}

template <typename TS>
int Ops<TS>::persist_grid(int block)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persist<TS>, block, slot_rec_bytes(1, block)) !=
        cudaSuccess)
        return 0;
    return per * sms;
}

}  // namespace lbm
