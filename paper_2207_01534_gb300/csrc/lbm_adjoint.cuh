// lbm_adjoint.cuh -- reverse pass of the split-schedule step (FP32 and FP64
// storage): the discrete adjoint of one time step, node by node, for
// gradients of the smooth non-wetting saturation with respect to the
// per-voxel wettability xi (Eq. 15) and the inlet density of the
// non-equilibrium extrapolation (Section 2).
//
// The forward step maps the post-stream state f_t to f_t+1 through moments
// (Eqs. 3-4), virtual wall densities (Eq. 15), forces (Eqs. 10, 11, 13),
// collision (Eqs. 1, 2, 6-9), streaming with bounce-back, and the open-plane
// extrapolation.  Its adjoint is applied in reverse, as gathers (every thread
// writes only its own node, so the pass is deterministic):
//   k_adj_plane  the extrapolation: the prescribed component of a plane node
//                was overwritten, its adjoint moves to the interior node xI
//                through f_eq(rho_b, u_I) + f(xI) - f_eq(rho(xI), u_I);
//   k_adj_node   streaming (the adjoint of f*_i(y) is that of the population
//                it became: f_i(y + e_i), or f_opp(i)(y) at a solid, nothing
//                beyond an open plane), then collision with tau(rho), u and the
//                forcing term, then the local part of the moments; it leaves
//                the adjoint of the stencil sums A^s of the force on a dense
//                grid;
//   k_adj_wall   the adjoint of each wall's virtual density (the stencil sums
//                of its fluid neighbours, with the mirrored neighbours of the
//                open planes), its xi gradient, and the weight it passes back
//                to the densities of its fluid neighbours;
//   k_adj_dens   the non-local density adjoint of each fluid node (force
//                stencils of its neighbours, virtual densities of adjacent
//                walls), added to every direction of the node.
// The adjoint of a state is held as Lam_i(n) + Rb(voxel of n): the local part
// per population and the density part per node, so the density part is never
// broadcast to 19 cells.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

struct AdjState {
    void *lam_in;    // [19][npad] pairs: local adjoint of the state after the step
    void *lam_out;   // [19][npad] pairs: local adjoint of the state before it
    void *rb_in;     // [nv] pairs: density adjoint after the step (dense, fluid voxels)
    void *rb_out;    // [nv] pairs: density adjoint before it
    void *abar;      // [3][nv] pairs: adjoint of the stencil sums A^sigma (dense)
    void *wbar;      // [nv] pairs: wall adjoint times chi / D (dense, walls only)
    double *gxi;     // [n_wall] dJ/dxi accumulated over steps
    double *grin;    // [nxy] dJ/drho_in1 accumulated per inlet column
};

template <typename C2>
__device__ __forceinline__ C2 swap2(C2 a)
{
    return mk2(a.y, a.x);
}

// adjoint of the final state for J = mean over the sample of rho1/(rho1+rho2):
// (d/d rho1, d/d rho2) = (rho2, -rho1) / (R^2 count), identical for every direction
template <typename TS>
__global__ void k_adj_seed(DevState s, AdjState a, double inv_count)
{
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= s.n_fluid) return;
    const uint32_t pv = s.pvox[n];
    const int z = (int)(pv / (uint32_t)s.sxy);
    const bool all = s.sample_hi <= s.sample_lo;
    C2 v = mk2(C(0), C(0));
    if (all || (z >= s.sample_lo && z < s.sample_hi)) {
        const C2 r = reinterpret_cast<const C2 *>(s.psi)[pv];
        const C R = r.x + r.y;
        const C k = (C)inv_count / (R * R);
        v = mk2(r.y * k, -r.x * k);
    }
    reinterpret_cast<C2 *>(a.rb_in)[pv] = v;
}

// Adjoint of the extrapolation at one plane.  sn is the state after the step
// (its interior node holds the values the extrapolation read), PN its parity.
// plane = 0 or 1 adjoins that plane; plane = 2 adjoins both in one launch
// (only when nz > 3: then the two planes and their interior nodes are four
// distinct layers and the two orders give the same result).
template <typename TS, int PN>
__global__ void __launch_bounds__(64) k_adj_plane(DevState sn, AdjState a, int planes)
{
    pdl_trigger();
    pdl_wait();
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    int plane = planes;
    if (planes == 2) {
        plane = p >= sn.nxy ? 0 : 1;
        if (plane == 0) p -= sn.nxy;
    }
    if (p >= sn.nxy) return;
    const uint32_t pvb = plane == 0 ? (uint32_t)p : (uint32_t)(p + (sn.nz - 1) * sn.sxy);
    const int nb = sn.cidx[pvb];
    if (nb < 0) return;
    const uint32_t pvi = plane == 0 ? pvb + sn.sxy : pvb - sn.sxy;
    const int ni = sn.cidx[pvi];
    const uint32_t fli = sn.nflags[ni];
    const Nbr bi = make_nbr(fli, sn);
    C2 fi[19], dmi;
    load_pops<TS, PN>(fi, dmi, ni, pvi, fli, bi, sn);
    const C2 r = density_of<TS>(dmi, sn);
    C m[3] = {0, 0, 0};
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const C tt = fi[i].x + fi[i].y;
        m[0] += ex(i) * tt;
        m[1] += ey(i) * tt;
        m[2] += ez(i) * tt;
    }
    const C R = r.x + r.y;
    const C u[3] = {m[0] / R, m[1] / R, m[2] / R};
    const C usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const C rb = (C)(plane == 0 ? sn.rho_in1 : sn.rho_out2);
    const C rin = plane == 0 ? r.x : r.y;
    C2 *L = reinterpret_cast<C2 *>(a.lam_in);
    C2 *Rb = reinterpret_cast<C2 *>(a.rb_in);
    const long long np = sn.npad;
    // everything is read first, then written (the plane node and its interior
    // node are distinct cells; keeping the values in registers lets all loads
    // be in flight at once)
    C2 lb[19], li[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        lb[i] = L[i * np + nb];
        li[i] = L[i * np + ni];
    }
    // fold the plane node's density part into its populations
    const C2 rbb = Rb[pvb];
    C gb = 0, rbar = 0, ub[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        C2 l = add2(lb[i], rbb);
        const C mu = plane == 0 ? l.x : l.y;
        if (plane == 0) l.x = C(0); else l.y = C(0);
        lb[i] = l;
        const C eu = ex(i) * u[0] + ey(i) * u[1] + ez(i) * u[2];
        const C feq1 = wgt<C>(i) * (C(1) + C(3) * eu + C(4.5) * eu * eu - C(1.5) * usq);
        gb += mu * feq1;
        rbar -= mu * feq1;
        const C k = mu * (rb - rin) * wgt<C>(i);
        ub[0] += k * (C(3) * ex(i) + C(9) * eu * ex(i) - C(3) * u[0]);
        ub[1] += k * (C(3) * ey(i) + C(9) * eu * ey(i) - C(3) * u[1]);
        ub[2] += k * (C(3) * ez(i) + C(9) * eu * ez(i) - C(3) * u[2]);
        // the f(xI) term
        if (plane == 0) li[i].x += mu; else li[i].y += mu;
    }
    const C ubu = ub[0] * u[0] + ub[1] * u[1] + ub[2] * u[2];
#pragma unroll
    for (int j = 0; j < 19; ++j) {
        const C du = (ex(j) * ub[0] + ey(j) * ub[1] + ez(j) * ub[2] - ubu) / R;
        C2 v = add2(li[j], mk2(du, du));
        if (plane == 0) v.x += rbar; else v.y += rbar;
        L[j * np + ni] = v;
        L[j * np + nb] = lb[j];
    }
    Rb[pvb] = mk2(C(0), C(0));
    if (plane == 0) a.grin[p] += (double)gb;
}

// Adjoint of the force-stencil sums gathered at voxel y: sum over the fluid
// nodes x that read psi(y) of w_i e_i . Abar(x), including the mirrored reads
// of open-plane nodes.  `in(j)` says whether y - e_j is an in-domain fluid
// voxel and `off(j)` gives its offset.  The result is the adjoint of
// psi^sbar(y) for the force of component s, so callers swap it.
template <typename C, typename C2, typename InFn, typename OffFn>
__device__ __forceinline__ C2 gather_abar(const C2 *ab, long long nv, uint32_t py, int z, int nz, int open_z, InFn in,
                                          OffFn off)
{
    C2 g = mk2(C(0), C(0));
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        if (!in(j)) continue;
        const long long x = (long long)py + off(j);
        const C w = wgt<C>(j);
        if (ex(j)) g = fma2(bc2<C2>(w * ex(j)), ab[x], g);
        if (ey(j)) g = fma2(bc2<C2>(w * ey(j)), ab[nv + x], g);
        if (ez(j)) g = fma2(bc2<C2>(w * ez(j)), ab[2 * nv + x], g);
        // x on an open plane also reads y through the mirror of the direction
        // that leaves the domain there: x + e_mirz(j) would be outside
        if (open_z && ez(j) != 0 && ((ez(j) > 0 && z == 1) || (ez(j) < 0 && z == nz - 2))) {
            const int i = mirz(j);
            if (ex(i)) g = fma2(bc2<C2>(w * ex(i)), ab[x], g);
            if (ey(i)) g = fma2(bc2<C2>(w * ey(i)), ab[nv + x], g);
            g = fma2(bc2<C2>(w * ez(i)), ab[2 * nv + x], g);
        }
    }
    return g;
}

// Streaming, collision and local moments in reverse at node n; P is the parity
// of the step's state st (psi holds its densities and wall densities).  The
// forward populations are only needed through the momenta and the sum
// sum_i L_i . f_i of the tau derivative, so they are folded as they load and
// the kernel keeps just the 19 adjoint pairs live (two blocks per SM).
// The 19 adjoint pairs of a thread live in shared memory ([19][blockDim]
// pairs, dynamic) rather than registers, which leaves room for three blocks
// of 256 threads per SM in FP32.
template <typename TS>
struct AdjOcc {  // resident blocks per SM the register budget is sized for
    static constexpr int blocks = 3;
};
template <>
struct AdjOcc<double> {
    static constexpr int blocks = 1;
};

template <typename TS, int P>
__global__ void __launch_bounds__(256, AdjOcc<TS>::blocks) k_adj_node(DevState st, AdjState a)
{
    pdl_trigger();
    pdl_wait();
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    using S2 = typename Traits<TS>::S2;
    extern __shared__ __align__(16) unsigned char adj_smem[];
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= st.n_fluid) return;
    C2 *ls = reinterpret_cast<C2 *>(adj_smem) + threadIdx.x;  // ls[i * blockDim.x]
    const int ld = blockDim.x;
    const uint32_t pv = st.pvox[n];
    const uint32_t fl = st.nflags[n];
    const Nbr b = make_nbr(fl, st);
    const long long np = st.npad;
    // the adjoints of the state after the step, the densities and the state
    // are only read here (the outputs are lam_out and abar), so every gather
    // goes through the read-only data path (reverse pass of the 96^3 pack
    // 63.9 -> 63.4 ms for 500 steps against ordinary loads)
    const C2 *Lin = reinterpret_cast<const C2 *>(a.lam_in);
    const C2 *Rin = reinterpret_cast<const C2 *>(a.rb_in);
    // adjoint of the post-collision populations (streaming transposed)
    const C2 ry = __ldg(Rin + pv);
    ls[0] = add2(__ldg(Lin + n), ry);
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        if (ez(i) != 0 && outside(i, fl)) {
            ls[i * ld] = mk2(C(0), C(0));
            continue;
        }
        const int off = nb_off(i, b);
        const int c = __ldg(st.cidx + ((int)pv + off));
        ls[i * ld] = c >= 0 ? add2(__ldg(Lin + i * np + c), __ldg(Rin + ((int)pv + off))) : add2(__ldg(Lin + opp(i) * np + n), ry);
    }
    // the forward quantities of the node: rho from the density pass, the
    // momenta and L.f from the populations
    const C2 *psi = reinterpret_cast<const C2 *>(st.psi) + pv;
    const C2 rho = __ldg(psi);
    C2 m[3] = {mk2(C(0), C(0)), mk2(C(0), C(0)), mk2(C(0), C(0))};
    C2 lf = mul2(ls[0], ld_rest<TS, LD_NC>(st, n));
    {
        const S2 *M = reinterpret_cast<const S2 *>(st.f);
        const S2 *B = reinterpret_cast<const S2 *>(st.bc);
        const bool plane = P == 1 && (fl & (F_INLET | F_OUTLET));
#pragma unroll
        for (int j = 1; j < 19; ++j) {
            const S2 *q = (ez(j) != 0 && plane && outside(j, fl)) ? B + bc_cell(j, pv, fl, st)
                                                                   : M + slot_in_block<P>(j, n, pv, b, st);
            const C2 fi = Traits<TS>::load(q, ref_of<TS>(st, opp(j)));  // f_opp(j)
            const int i = opp(j);
            lf = fma2(ls[i * ld], fi, lf);
            if (ex(i)) m[0] = ex(i) > 0 ? add2(m[0], fi) : sub2(m[0], fi);
            if (ey(i)) m[1] = ey(i) > 0 ? add2(m[1], fi) : sub2(m[1], fi);
            if (ez(i)) m[2] = ez(i) > 0 ? add2(m[2], fi) : sub2(m[2], fi);
        }
    }
    C2 A[3] = {mk2(C(0), C(0)), mk2(C(0), C(0)), mk2(C(0), C(0))};  // (.x: psi1 sums, .y: psi2 sums)
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        const int off = (ez(j) != 0 && outside(j, fl)) ? nb_off(mirz(j), b) : nb_off(j, b);
        const C2 d = sub2(__ldg(psi + off), rho);
        const C w = wgt<C>(j);
        if (ex(j)) A[0] = fma2(bc2<C2>(w * ex(j)), d, A[0]);
        if (ey(j)) A[1] = fma2(bc2<C2>(w * ey(j)), d, A[1]);
        if (ez(j)) A[2] = fma2(bc2<C2>(w * ez(j)), d, A[2]);
    }
    const C G = pick<C>(st.G, st.fG);
    const C g[3] = {pick<C>(st.gx, st.fgx), pick<C>(st.gy, st.fgy), pick<C>(st.gz, st.fgz)};
    // F^1 = rho1 (-G A.y + g), F^2 = rho2 (-G A.x + g)
    C2 F[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) F[k] = mk2(rho.x * (-G * A[k].y + g[k]), rho.y * (-G * A[k].x + g[k]));
    const C R = rho.x + rho.y;
    const C h = st.velocity_shift ? C(0.5) : C(0);
    C u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = (m[k].x + m[k].y + h * (F[k].x + F[k].y)) / R;
    const C tau = (rho.x * pick<C>(st.tau1, st.ftau1) + rho.y * pick<C>(st.tau2, st.ftau2)) / R;
    const C om = C(1) / tau;
    const C cf = C(1) - C(0.5) * om;
    const C usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    // collision transposed; d f*/d tau = ((f - feq) + S / 2) / tau^2
    C2 rb = mk2(C(0), C(0));
    C ub[3] = {0, 0, 0};
    C2 Fb[3] = {mk2(C(0), C(0)), mk2(C(0), C(0)), mk2(C(0), C(0))};
    C taub = lf.x + lf.y;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const C2 L = ls[i * ld];
        const C w = wgt<C>(i);
        const C eu = ex(i) * u[0] + ey(i) * u[1] + ez(i) * u[2];
        const C feq1 = w * (C(1) + C(3) * eu + C(4.5) * eu * eu - C(1.5) * usq);
        const C2 eF = mk2(ex(i) * F[0].x + ey(i) * F[1].x + ez(i) * F[2].x, ex(i) * F[0].y + ey(i) * F[1].y + ez(i) * F[2].y);
        const C2 uF = mk2(u[0] * F[0].x + u[1] * F[1].x + u[2] * F[2].x, u[0] * F[0].y + u[1] * F[1].y + u[2] * F[2].y);
        // S^s = w (3 (e - u).F^s + 9 eu e.F^s)
        const C2 S = mk2(w * (C(3) * (eF.x - uF.x) + C(9) * eu * eF.x), w * (C(3) * (eF.y - uF.y) + C(9) * eu * eF.y));
        rb = fma2(bc2<C2>(feq1 * om), L, rb);
        const C Lr = L.x * rho.x + L.y * rho.y;  // sum_s L^s rho^s
        const C LeFs = L.x * eF.x + L.y * eF.y;
        ub[0] += w * (om * Lr * (C(3) * ex(i) + C(9) * eu * ex(i) - C(3) * u[0]) +
                      cf * (C(-3) * (L.x * F[0].x + L.y * F[0].y) + C(9) * ex(i) * LeFs));
        ub[1] += w * (om * Lr * (C(3) * ey(i) + C(9) * eu * ey(i) - C(3) * u[1]) +
                      cf * (C(-3) * (L.x * F[1].x + L.y * F[1].y) + C(9) * ey(i) * LeFs));
        ub[2] += w * (om * Lr * (C(3) * ez(i) + C(9) * eu * ez(i) - C(3) * u[2]) +
                      cf * (C(-3) * (L.x * F[2].x + L.y * F[2].y) + C(9) * ez(i) * LeFs));
        const C k0 = cf * w * (C(3) * (ex(i) - u[0]) + C(9) * eu * ex(i));
        const C k1 = cf * w * (C(3) * (ey(i) - u[1]) + C(9) * eu * ey(i));
        const C k2 = cf * w * (C(3) * (ez(i) - u[2]) + C(9) * eu * ez(i));
        Fb[0] = fma2(bc2<C2>(k0), L, Fb[0]);
        Fb[1] = fma2(bc2<C2>(k1), L, Fb[1]);
        Fb[2] = fma2(bc2<C2>(k2), L, Fb[2]);
        taub += -Lr * feq1 + C(0.5) * (L.x * S.x + L.y * S.y);
    }
    taub *= om * om;
    // tau = (rho1 tau1 + rho2 tau2) / R
    rb = add2(rb, mk2(taub * (pick<C>(st.tau1, st.ftau1) - tau) / R, taub * (pick<C>(st.tau2, st.ftau2) - tau) / R));
    // u = (m1 + m2 + h (F1 + F2)) / R
    C2 mb[3];
    const C ubu = (ub[0] * u[0] + ub[1] * u[1] + ub[2] * u[2]) / R;
    rb = sub2(rb, bc2<C2>(ubu));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        mb[k] = bc2<C2>(ub[k] / R);
        Fb[k] = add2(Fb[k], bc2<C2>(h * ub[k] / R));
    }
    // F^1 = rho1 (-G A.y + g): rho-bar and the adjoint of the stencil sums
    C2 *ab = reinterpret_cast<C2 *>(a.abar);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        rb.x += Fb[k].x * (-G * A[k].y + g[k]);
        rb.y += Fb[k].y * (-G * A[k].x + g[k]);
        // Abar^s: adjoint of the sum over psi^sbar read by the force of s
        ab[k * st.nv + pv] = mk2(-G * rho.x * Fb[k].x, -G * rho.y * Fb[k].y);
    }
    // pre-collision populations: direct term, density and momentum; stored
    // with the evict-last L2 policy, since the next reversed step gathers them
    // right away (96^3 pack, 500 steps: reverse 63.3 -> 61.9 ms)
    C2 *Lout = reinterpret_cast<C2 *>(a.lam_out);
    const C2 keep = bc2<C2>(C(1) - om);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        C2 v = fma2(keep, ls[i * ld], rb);
        if (ex(i)) v = ex(i) > 0 ? add2(v, mb[0]) : sub2(v, mb[0]);
        if (ey(i)) v = ey(i) > 0 ? add2(v, mb[1]) : sub2(v, mb[1]);
        if (ez(i)) v = ez(i) > 0 ? add2(v, mb[2]) : sub2(v, mb[2]);
        st_pol(Lout + i * np + n, v, l2_policy());
    }
}

// Wall voxels: adjoint of rho~^s (the stencil sums of the fluid neighbours
// that read it), the xi gradient, and wbar = rho~-bar chi / D.
template <typename TS>
__global__ void __launch_bounds__(256) k_adj_wall(DevState st, AdjState a)
{
    pdl_trigger();
    pdl_wait();
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= st.n_wall) return;
    const uint32_t pw = st.wpvox[w];
    const uint32_t mask = st.wmask[w];
    const Nbr b = make_nbr(mask >> kWallFaceShift, st);
    const int z = (int)(pw / (uint32_t)st.sxy);
    const C2 *ab = reinterpret_cast<const C2 *>(a.abar);
    // y - e_j = y + e_opp(j) is an in-domain fluid voxel iff mask bit opp(j)
    const C2 gsum = gather_abar<C, C2>(
        ab, st.nv, pw, z, st.nz, st.open_z, [&](int j) { return (mask >> opp(j)) & 1u; },
        [&](int j) { return nb_off(opp(j), b); });
    const C2 pb = swap2(gsum);  // adjoint of (rho~1, rho~2)
    const C2 *psi = reinterpret_cast<const C2 *>(st.psi);
    C2 acc = mk2(C(0), C(0));
#pragma unroll
    for (int j = 1; j < 19; ++j)
        if (mask & (1u << j)) acc = fma2(bc2<C2>(wgt<C>(j)), psi[(int)pw + nb_off(j, b)], acc);
    const C inv = reinterpret_cast<const C *>(st.winv)[w];
    const C xi = reinterpret_cast<const C *>(st.wxi)[w];
    a.gxi[w] += (double)(pb.x * acc.x * inv) - (double)(pb.y * acc.y * inv);
    reinterpret_cast<C2 *>(a.wbar)[pw] = mk2(pb.x * (C(1) + xi) * inv, pb.y * (C(1) - xi) * inv);
}

// Fluid voxels: non-local density adjoint into rb_out.
template <typename TS>
__global__ void __launch_bounds__(256) k_adj_dens(DevState st, AdjState a)
{
    pdl_trigger();
    pdl_wait();
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= st.n_fluid) return;
    const uint32_t pv = st.pvox[n];
    const uint32_t fl = st.nflags[n];
    const Nbr b = make_nbr(fl, st);
    const int z = (int)(pv / (uint32_t)st.sxy);
    const C2 *ab = reinterpret_cast<const C2 *>(a.abar);
    const C2 *wb = reinterpret_cast<const C2 *>(a.wbar);
    // y - e_j: in the domain unless it crosses an open plane.  abar is zero
    // on solid voxels and wbar on fluid ones (both are cleared before the
    // pass and only written on their own voxels), so neither gather needs to
    // look the neighbour's kind up.
    auto in_dom = [&](int j) { return !(ez(j) != 0 && outside(opp(j), fl)); };
    const C2 gsum = gather_abar<C, C2>(ab, st.nv, pv, z, st.nz, st.open_z, in_dom,
                                       [&](int j) { return nb_off(opp(j), b); });
    C2 r = swap2(gsum);
#pragma unroll
    for (int j = 1; j < 19; ++j) {
        if (!in_dom(j)) continue;
        r = fma2(bc2<C2>(wgt<C>(j)), wb[(int)pv + nb_off(opp(j), b)], r);
    }
    reinterpret_cast<C2 *>(a.rb_out)[pv] = r;
}

// Out-of-place forward step for the recompute: reads the state of st and
// writes the next one into f_out / rest_out.  Every population cell is
// written exactly once per step (the A-A slots of a parity are a bijection
// onto the cells), so the new buffers are complete but for the open-plane
// boundary cells, which the extrapolation of the next density pass writes.
template <typename TS, int P>
__global__ void __launch_bounds__(256, PipeOcc<TS>::blocks) k_fused_to(DevState st, void *f_out, void *rest_out)
{
    pdl_trigger();
    pdl_wait();
    using C = typename Traits<TS>::C;
    using C2 = typename Traits<TS>::C2;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= st.n_fluid) return;
    const uint32_t pv = st.pvox[n];
    const uint32_t fl = st.nflags[n];
    const Nbr b = make_nbr(fl, st);
    C2 f[19], dm;
    load_pops<TS, P>(f, dm, n, pv, fl, b, st);
    const C2 rho = density_of<TS>(dm, st);
    C2 F[3];
    C u[3], inv_rho;
    forces<TS>(rho, pv, fl, b, st, F);
    mix_velocity<C, C2>(f, rho, F, st, inv_rho, u);
    collide<C, C2>(f, rho, inv_rho, u, F, st);
    DevState so = st;
    so.f = f_out;
    so.rest = rest_out;
    store_pops<TS, P>(f, dm, n, pv, fl, b, so);
}

// dJ/dxi on the dense grid (zero off the walls), scaled by the incoming gradient
template <typename TS>
__global__ void k_adj_xi_out(DevState st, AdjState a, double scale, float *grad)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= st.n_wall) return;
    grad[st.wpvox[w]] = (float)(a.gxi[w] * scale);
}

template <typename TS>
struct Adj {
    static void seed(const DevState &s, const AdjState &a, double inv_count, cudaStream_t st);
    // plane 0 (inlet), 1 (outlet) or 2 (both in one launch; needs nz > 3)
    static void plane(const DevState &sn, const AdjState &a, int parity_next, int plane, cudaStream_t st);
    static void node(const DevState &s, const AdjState &a, int parity, cudaStream_t st);
    static void wall(const DevState &s, const AdjState &a, cudaStream_t st);
    static void dens(const DevState &s, const AdjState &a, cudaStream_t st);
    static void xi_out(const DevState &s, const AdjState &a, double scale, float *grad, cudaStream_t st);
    static void fused_to(const DevState &s, int parity, void *f_out, void *rest_out, cudaStream_t st);
};

template <typename TS>
void Adj<TS>::fused_to(const DevState &s, int parity, void *f_out, void *rest_out, cudaStream_t st)
{
    if (s.n_fluid == 0) return;
    const int g = (s.n_fluid + 255) / 256;
    if (parity) launch_pdl(k_fused_to<TS, 1>, (unsigned)g, 256, 0, st, s, f_out, rest_out);
    else launch_pdl(k_fused_to<TS, 0>, (unsigned)g, 256, 0, st, s, f_out, rest_out);
}

template <typename TS>
void Adj<TS>::seed(const DevState &s, const AdjState &a, double inv_count, cudaStream_t st)
{
    if (s.n_fluid > 0) k_adj_seed<TS><<<(s.n_fluid + 255) / 256, 256, 0, st>>>(s, a, inv_count);
}
template <typename TS>
void Adj<TS>::plane(const DevState &sn, const AdjState &a, int parity_next, int plane, cudaStream_t st)
{
    if (!sn.open_z || sn.nxy == 0) return;
    const int g = ((plane == 2 ? 2 : 1) * sn.nxy + 63) / 64;
    if (parity_next) launch_pdl(k_adj_plane<TS, 1>, (unsigned)g, 64, 0, st, sn, a, plane);
    else launch_pdl(k_adj_plane<TS, 0>, (unsigned)g, 64, 0, st, sn, a, plane);
}
template <typename TS>
void Adj<TS>::node(const DevState &s, const AdjState &a, int parity, cudaStream_t st)
{
    if (s.n_fluid == 0) return;
    using C2 = typename Traits<TS>::C2;
    const size_t smem = (size_t)19 * 256 * sizeof(C2);
    static bool attr = false;  // above the 48 KB default for FP64
    if (!attr) {
        cudaFuncSetAttribute(k_adj_node<TS, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_adj_node<TS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int g = (s.n_fluid + 255) / 256;
    if (parity) launch_pdl(k_adj_node<TS, 1>, (unsigned)g, 256, smem, st, s, a);
    else launch_pdl(k_adj_node<TS, 0>, (unsigned)g, 256, smem, st, s, a);
}
template <typename TS>
void Adj<TS>::wall(const DevState &s, const AdjState &a, cudaStream_t st)
{
    if (s.n_wall > 0) launch_pdl(k_adj_wall<TS>, (unsigned)((s.n_wall + 255) / 256), 256, 0, st, s, a);
}
template <typename TS>
void Adj<TS>::dens(const DevState &s, const AdjState &a, cudaStream_t st)
{
    if (s.n_fluid > 0) launch_pdl(k_adj_dens<TS>, (unsigned)((s.n_fluid + 255) / 256), 256, 0, st, s, a);
}
template <typename TS>
void Adj<TS>::xi_out(const DevState &s, const AdjState &a, double scale, float *grad, cudaStream_t st)
{
    if (s.n_wall > 0) k_adj_xi_out<TS><<<(s.n_wall + 255) / 256, 256, 0, st>>>(s, a, scale, grad);
}

}  // namespace lbm
