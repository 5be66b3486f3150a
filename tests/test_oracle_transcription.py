"""The oracle's time step against a second, independent transcription.

A short NumPy restatement of one step of the method (Section 2, in the step
order of the readings: moments, virtual wall densities, forces, collision,
streaming with half-way bounce-back and frozen missing populations, then the
open-plane extrapolation), written with whole-array shifts instead of the
oracle's per-voxel neighbour search, is run beside the C oracle on small
porous grids (4^3 to 8^3) from random states.  The two must agree to round-off
after one and after a few steps.  This is a cross-check of the oracle's
indexing, streaming direction, wrap-around and plane handling; the physics
itself is pinned elsewhere (Laplace law, contact angles, duct flow, exact
invariants).
"""
import numpy as np
import pytest

import oracle
from conftest import golden

_G = golden("d3q19_section2.txt")
E = np.array([_G["ex"][0], _G["ey"][0], _G["ez"][0]], dtype=int).T  # (19, 3): x, y, z
W = np.array(_G["w"][0])
OPP = np.array([int(np.flatnonzero((E == -E[i]).all(axis=1))[0]) for i in range(19)])
CS2 = 1.0 / 3.0


def _shift(a, d, periodic):
    """b[z, y, x] = a[(z, y, x) + d] with d = (dx, dy, dz), and a mask of the
    voxels whose neighbour lies inside the domain (non-periodic axes end)."""
    b = a
    ok = np.ones(a.shape[-3:], bool)
    for ax_xyz, k in ((0, -1), (1, -2), (2, -3)):  # array axis of x, y, z
        s = d[ax_xyz]
        if s == 0:
            continue
        b = np.roll(b, -s, axis=k)
        if not periodic[ax_xyz]:
            n = a.shape[k]
            idx = np.arange(n) + s
            bad = (idx < 0) | (idx >= n)
            shape = [1, 1, 1]
            shape[k] = n
            ok = ok & ~bad.reshape(shape)
    return b, ok


def _feq(rho, u):
    eu = np.einsum("ia,a...->i...", E.astype(float), u)
    usq = (u ** 2).sum(axis=0)
    return W[:, None, None, None] * rho * (1.0 + 3.0 * eu + 4.5 * eu ** 2 - 1.5 * usq)


def _source(u, F):
    e = E.astype(float)
    eu = np.einsum("ia,a...->i...", e, u)
    eF = np.einsum("ia,a...->i...", e, F)
    uF = (u * F).sum(axis=0)
    return W[:, None, None, None] * (3.0 * (eF - uF) + 9.0 * eu * eF)


class Transcription:
    """One two-component lattice: f[s] has shape (19, nz, ny, nx)."""

    def __init__(self, solid, tau, G, xi_field, periodic, open_z, rho_in1, rho_out2, g, f1, f2):
        self.solid = solid.astype(bool)
        self.fluid = ~self.solid
        self.tau, self.G, self.xi, self.per = tau, G, xi_field, periodic
        self.open_z, self.rho_b = open_z, (rho_in1, rho_out2)
        self.g = np.array(g, float)
        self.f = [f1.copy(), f2.copy()]
        self.f0 = [f1.copy(), f2.copy()]  # the missing populations keep these values

    def step(self):
        fl, so = self.fluid, self.solid
        # moments (Eqs. 3-4) on fluid voxels
        rho = [np.where(fl, f.sum(axis=0), 0.0) for f in self.f]
        mom = [np.where(fl, np.einsum("ia,i...->a...", E.astype(float), f), 0.0) for f in self.f]
        # virtual wall densities (Eqs. 14-15): chi^(1) = 1 + xi, chi^(2) = 1 - xi
        num = [np.zeros(so.shape), np.zeros(so.shape)]
        den = np.zeros(so.shape)
        for i in range(1, 19):
            fl_nb, ok = _shift(fl.astype(float), E[i], self.per)
            wgt = W[i] * fl_nb * ok
            den += wgt
            for s in range(2):
                r_nb, _ = _shift(rho[s], E[i], self.per)
                num[s] += wgt * r_nb
        chi = (1.0 + self.xi, 1.0 - self.xi)
        psi = []
        for s in range(2):
            tilde = np.where(den > 0, chi[s] * num[s] / np.where(den > 0, den, 1.0), 0.0)
            psi.append(np.where(so, tilde, rho[s]))
        # forces (Eqs. 10, 11, 13): the other component's psi over the stencil;
        # a direction leaving through an open z plane reads its mirrored one
        F = []
        for s in range(2):
            acc = np.zeros((3,) + so.shape)
            for i in range(1, 19):
                v_nb, ok = _shift(psi[1 - s], E[i], self.per)
                if self.open_z and E[i][2] != 0:
                    m = E[i].copy()
                    m[2] = -m[2]
                    v_m, _ = _shift(psi[1 - s], m, self.per)
                    v_nb = np.where(ok, v_nb, v_m)
                for a in range(3):
                    acc[a] += W[i] * E[i][a] * v_nb
            F.append(-self.G * rho[s] * acc + rho[s] * self.g[:, None, None, None])
        # mixture relaxation (Eqs. 6-7, nu = c_s^2 (tau - 1/2)) and velocity (Eq. 8 with F/2)
        R = rho[0] + rho[1]
        Rs = np.where(fl, R, 1.0)
        nu = rho[0] * CS2 * (self.tau[0] - 0.5) + rho[1] * CS2 * (self.tau[1] - 0.5)
        tau_s = nu / (Rs * CS2) + 0.5
        u = (mom[0] + mom[1] + 0.5 * (F[0] + F[1])) / Rs
        # collision (Eqs. 1, 2, 9)
        fs = []
        for s in range(2):
            fe = _feq(rho[s], u)
            fs.append(self.f[s] - (self.f[s] - fe) / tau_s + (1.0 - 0.5 / tau_s) * _source(u, F[s]))
        # pull streaming: from x - e_i; a solid source bounces back half-way,
        # a source beyond an open plane leaves the population as it was first set
        new = []
        for s in range(2):
            g_ = np.empty_like(fs[s])
            g_[0] = fs[s][0]
            for i in range(1, 19):
                src, ok = _shift(fs[s][i], -E[i], self.per)
                src_solid, _ = _shift(so.astype(float), -E[i], self.per)
                v = np.where(src_solid > 0, fs[s][OPP[i]], src)
                g_[i] = np.where(ok, v, self.f0[s][i])
            new.append(np.where(fl[None], g_, self.f[s]))
        self.f = new
        # non-equilibrium extrapolation: component 1 at z = 0 from z = 1, component 2 at z = nz-1 from nz-2
        if self.open_z:
            for comp, zb, zi in ((0, 0, 1), (1, -1, -2)):
                r_i = [self.f[s][:, zi].sum(axis=0) for s in range(2)]
                m_i = sum(np.einsum("ia,i...->a...", E.astype(float), self.f[s][:, zi]) for s in range(2))
                u_i = m_i / (r_i[0] + r_i[1])
                fe_b = _feq(self.rho_b[comp] * np.ones_like(r_i[0])[None], u_i[:, None])[:, 0]
                fe_i = _feq(r_i[comp][None], u_i[:, None])[:, 0]
                upd = fe_b + self.f[comp][:, zi] - fe_i
                self.f[comp][:, zb] = np.where(self.fluid[zb][None], upd, self.f[comp][:, zb])


def _random_state(solid, seed):
    rng = np.random.default_rng(seed)
    shape = solid.shape
    r1 = rng.uniform(0.05, 1.0, shape)
    r2 = rng.uniform(0.05, 1.0, shape)
    f = []
    for r in (r1, r2):
        u = rng.uniform(-0.04, 0.04, (3,) + shape)
        fe = _feq(r[None], u[:, None])[:, 0]
        f.append(fe * (1.0 + rng.uniform(-0.05, 0.05, fe.shape)))
    return f


CASES = {
    # open z, periodic x and y, solids inside, a per-voxel xi field and a body force
    "open_porous": dict(shape=(8, 5, 6), porosity=0.7, periodic=(1, 1, 0), open_z=True, g=(1e-4, -2e-4, 3e-4),
                        seed=3),
    # all faces periodic, solids, no planes
    "periodic_porous": dict(shape=(5, 6, 4), porosity=0.65, periodic=(1, 1, 1), open_z=False, g=(0.0, 0.0, 0.0),
                            seed=5),
    # a 4^3 periodic box, few solids
    "small_dense": dict(shape=(4, 4, 4), porosity=0.9, periodic=(1, 1, 1), open_z=False, g=(0.0, 2e-4, 0.0), seed=11),
    # open z with solid walls on the lateral x faces (non-periodic x), 7 x 6 x 8
    "open_walled_x": dict(shape=(8, 6, 7), porosity=0.75, periodic=(0, 1, 0), open_z=True, g=(0.0, 0.0, -1e-4),
                          seed=13),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_step_matches_the_numpy_transcription(name):
    c = CASES[name]
    rng = np.random.default_rng(c["seed"])
    nz, ny, nx = c["shape"]
    solid = (rng.random(c["shape"]) > c["porosity"]).astype(np.uint8)
    if c["open_z"]:  # two fluid slices at each open plane (the plane and its interior node)
        solid[:2] = 0
        solid[-2:] = 0
    if not c["periodic"][0]:  # a closed lateral face is lined with solid voxels
        solid[:, :, 0] = 1
        solid[:, :, -1] = 1
    xi = np.where(solid == 1, rng.uniform(-0.4, 0.4, solid.shape), 0.0)
    tau = (1.3, 0.7)
    f1, f2 = _random_state(solid, 7)
    kw = dict(tau=tau, G=2.0, periodic=c["periodic"], open_axis=2 if c["open_z"] else -1, rho_in1=1.05,
              rho_out2=0.95, body_force=c["g"])
    o = oracle.Oracle(solid, xi_field=xi, **kw)
    o.set_pops(f1, f2)
    t = Transcription(solid, tau, 2.0, xi, c["periodic"], c["open_z"], 1.05, 0.95, c["g"], f1, f2)
    fluid = solid == 0
    for nsteps in (1, 3):
        while o.step_count < nsteps:
            o.step(1)
            t.step()
        a1, a2 = o.get_pops()
        for got, ref in ((a1, t.f[0]), (a2, t.f[1])):
            err = np.abs(got[:, fluid] - ref[:, fluid]).max() / np.abs(ref[:, fluid]).max()
            assert err <= 1e-12, (name, nsteps, err)
