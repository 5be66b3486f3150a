// Launchers of the push schedule (FP32 storage).
#include "lbm_push.cuh"

namespace lbm {

void push_fused(const DevState &s, const PushBufs &pb, int parity, cudaStream_t st)
{
    if (s.n_fluid == 0) return;
    const int g = (s.n_fluid + 255) / 256;
    if (parity) launch_pdl(k_fused_push<1>, (unsigned)g, 256, 0, st, s, pb);
    else launch_pdl(k_fused_push<0>, (unsigned)g, 256, 0, st, s, pb);
}

int push_finish(const DevState &s, unsigned long long *acc, unsigned long long *clr, int parity_next, int w_lo,
                int w_hi, cudaStream_t st)
{
    if (!s.open_z) w_lo = 0, w_hi = s.n_wall;
    const int nbp = s.open_z ? (2 * s.nxy + 255) / 256 : 0;
    const int nbw = (w_hi - w_lo + 255) / 256;
    const int nbz = (int)(((s.nv + 1) / 2 + 255) / 256);
    if (parity_next) launch_pdl(k_pw_push<1>, (unsigned)(nbp + nbw + nbz), 256, 0, st, s, acc, clr, nbp, nbw, w_lo, w_hi);
    else launch_pdl(k_pw_push<0>, (unsigned)(nbp + nbw + nbz), 256, 0, st, s, acc, clr, nbp, nbw, w_lo, w_hi);
    int launches = 1;
    const int rest = w_lo + (s.n_wall - w_hi);
    if (rest > 0) {
        launch_pdl(k_wall_push, (unsigned)((rest + 255) / 256), 256, 0, st, s, acc, 0, w_lo, w_hi, s.n_wall);
        ++launches;
    }
    return launches;
}

void push_prime(const DevState &s, unsigned long long *acc, cudaStream_t st, bool walls)
{
    const int nw = walls ? s.n_wall : 0;
    const long long n = s.nv > nw ? s.nv : nw;
    k_psi_to_acc<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float2 *>(s.psi), s.cidx,
                                                              s.wpvox, nw, s.nv, acc);
}

}  // namespace lbm
