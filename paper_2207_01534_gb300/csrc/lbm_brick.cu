// Launchers of the brick schedule (FP32 and 16-bit storage).
#include "lbm_brick.cuh"

namespace lbm {

template <typename TS>
void brick_step(const DevState &s, const BrickBufs &bb, int nbricks, int parity, cudaStream_t st)
{
    if (nbricks <= 0) return;
    if (parity) launch_pdl(k_brick<TS, 1>, (unsigned)nbricks, kBrickThreads, 0, st, s, bb);
    else launch_pdl(k_brick<TS, 0>, (unsigned)nbricks, kBrickThreads, 0, st, s, bb);
}

template <typename TS>
void brick_plane(const DevState &s, unsigned long long *acc, int parity_next, cudaStream_t st)
{
    if (!s.open_z || s.nxy == 0) return;
    const unsigned g = (unsigned)((2LL * s.nxy + 127) / 128);
    if (parity_next) launch_pdl(k_plane_acc<TS, 1>, g, 128, 0, st, s, acc);
    else launch_pdl(k_plane_acc<TS, 0>, g, 128, 0, st, s, acc);
}

void brick_coef(const DevState &s, const int32_t *wid, int n, float2 *coef, bool fp64, cudaStream_t st)
{
    if (n <= 0) return;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (fp64)
        k_brick_coef<double><<<g, 256, 0, st>>>(wid, n, (const double *)s.winv, (const double *)s.wxi, coef);
    else
        k_brick_coef<float><<<g, 256, 0, st>>>(wid, n, (const float *)s.winv, (const float *)s.wxi, coef);
}

template void brick_step<float>(const DevState &, const BrickBufs &, int, int, cudaStream_t);
template void brick_step<__half>(const DevState &, const BrickBufs &, int, int, cudaStream_t);
template void brick_step<__nv_bfloat16>(const DevState &, const BrickBufs &, int, int, cudaStream_t);
template void brick_plane<float>(const DevState &, unsigned long long *, int, cudaStream_t);
template void brick_plane<__half>(const DevState &, unsigned long long *, int, cudaStream_t);
template void brick_plane<__nv_bfloat16>(const DevState &, unsigned long long *, int, cudaStream_t);

}  // namespace lbm
