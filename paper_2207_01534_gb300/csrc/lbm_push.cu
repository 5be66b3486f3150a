// Launchers of the push schedule (FP32 storage).
#include "lbm_push.cuh"

namespace lbm {

void push_fused(const DevState &s, const PushBufs &pb, int parity, cudaStream_t st)
{
    if (s.n_fluid == 0) return;
    const int g = (s.n_fluid + 255) / 256;
    if (parity) k_fused_push<1><<<g, 256, 0, st>>>(s, pb);
    else k_fused_push<0><<<g, 256, 0, st>>>(s, pb);
}

void push_plane(const DevState &s, unsigned long long *acc, int parity_next, cudaStream_t st)
{
    if (!s.open_z || s.nxy == 0) return;
    const int g = (2 * s.nxy + 127) / 128;
    if (parity_next) k_plane_push<1><<<g, 128, 0, st>>>(s, acc);
    else k_plane_push<0><<<g, 128, 0, st>>>(s, acc);
}

void push_wall(const DevState &s, unsigned long long *acc, cudaStream_t st)
{
    if (s.n_wall == 0) return;
    k_wall_push<<<(s.n_wall + 255) / 256, 256, 0, st>>>(s, acc);
}

void push_prime(const DevState &s, unsigned long long *acc, cudaStream_t st, bool walls)
{
    const int nw = walls ? s.n_wall : 0;
    const long long n = s.nv > nw ? s.nv : nw;
    k_psi_to_acc<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float2 *>(s.psi), s.cidx,
                                                              s.wpvox, nw, s.nv, acc);
}

}  // namespace lbm
