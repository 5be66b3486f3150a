"""Oracle pins against physics the paper prints or the mathematics fixes:
viscosity of the mixture relaxation (Eqs. 6-7), flat-interface coexistence
(continuum limit of Eq. 11), Laplace's law with the paper's surface tension
(Section 3.1), the contact-angle calibration (Section 3.2), square-duct
Poiseuille flow with half-way bounce-back, and layered two-component channel
flow against the continuum momentum balance."""
import math

import numpy as np
import pytest

import oracle
import physics
from conftest import golden
from paper_2207_01534_gb300 import inputs

REF = golden("physics_section3.txt")
GAMMA = REF["gamma"][0][0]
G = REF["G"][0][0]


def _shear_wave_nu(tau, rho1, rho2, n=64, steps=300, amp=1e-4):
    """Decay rate of u_x = A sin(k z) in a periodic column, returned as nu."""
    solid = np.zeros((n, 1, 1), np.uint8)
    k = 2 * math.pi / n
    z = np.arange(n)
    f1 = np.zeros((19, n, 1, 1))
    f2 = np.zeros((19, n, 1, 1))
    for zi in range(n):
        u = np.array([amp * math.sin(k * z[zi]), 0.0, 0.0])
        f1[:, zi, 0, 0] = oracle.feq(rho1, u)
        f2[:, zi, 0, 0] = oracle.feq(rho2, u)
    o = oracle.Oracle(solid, tau=tau, G=0.0)
    o.set_pops(f1, f2)
    s = np.sin(k * z)

    def mode():
        return float(o.fields()["ux"][:, 0, 0] @ s) * 2 / n

    a0 = mode()
    o.step(steps)
    a1 = mode()
    return -math.log(a1 / a0) / (k * k * steps)


@pytest.mark.parametrize("tau,rho", [((0.8, 0.8), (1.0, 0.0)), ((1.7, 0.62), (0.5, 0.5)), ((3.5, 0.62), (0.2, 0.8))])
def test_mixture_viscosity(tau, rho):
    """Eqs. 6-7 with nu = c_s^2 (tau - 1/2): the mixture relaxes with
    tau_s = sum rho tau / rho and its viscosity is c_s^2 (tau_s - 1/2)."""
    tau_s = (rho[0] * tau[0] + rho[1] * tau[1]) / (rho[0] + rho[1])
    nu_expected = (tau_s - 0.5) / 3.0
    nu = _shear_wave_nu(tau, *rho)
    assert abs(nu / nu_expected - 1) < 0.01


def test_viscosity_ratio_pairs():
    """The tau pairs of Section 3.1 give M = 25 and 1/25 only with nu = c_s^2 (tau - 1/2)."""
    t = REF["tau_M25"][0]
    assert abs((t[0] - 0.5) / (t[1] - 0.5) - 25.0) < 1e-12
    t = REF["tau_M1_25"][0]
    assert abs((t[1] - 0.5) / (t[0] - 0.5) - 25.0) < 1e-12
    assert abs((t[1] + 0.5) / (t[0] + 0.5) - 25.0) > 20  # the printed '+1/2' would not


def _slab(Gc, tau, steps, nz=128):
    solid = np.zeros((nz, 1, 1), np.uint8)
    z = np.arange(nz)
    inside = (z >= nz // 4) & (z < 3 * nz // 4)
    r1 = np.where(inside, 1.0, 0.03)[:, None, None]
    r2 = np.where(inside, 0.03, 1.0)[:, None, None]
    o = oracle.Oracle(solid, tau=tau, G=Gc)
    o.init_densities(r1, r2)
    o.step(steps)
    f = o.fields()
    return f["rho1"][nz // 2, 0, 0], f["rho1"][0, 0, 0], np.abs(f["uz"]).max()


def test_flat_interface_coexistence_law():
    """Continuum limit of Eq. 11 for a flat interface at rest: each component
    balances c_s^2 grad rho = F, i.e. ln(a/b) = G (a - b) between the bulk
    densities a, b (lattice corrections are below 1% at G = 2.5)."""
    a, b, umax = _slab(2.5, (1.0, 1.0), 20000)
    assert a > 0.5 > b  # segregated
    assert abs(math.log(a / b) / (2.5 * (a - b)) - 1) < 0.02
    assert umax < 1e-4


def test_coexistence_independent_of_viscosity_ratio():
    """The interface does not depend on the viscosity ratio (Section 3.1):
    identical bulk densities for M = 1, 25 and 1/25 at G = 3.5."""
    res = [_slab(G, tuple(REF[k][0]), 16000, nz=64) for k in ("tau_M1", "tau_M25", "tau_M1_25")]
    for a, b, umax in res:
        assert abs(a - res[0][0]) < 1e-5 * res[0][0]
        assert abs(b - res[0][1]) < 1e-4 * res[0][1]
        assert umax < 1e-7


def _cylinder(R, tau, n=80, steps=4500):
    shape = (n, 1, n)
    solid = np.zeros(shape, np.uint8)
    r1, r2 = inputs.cylinder_densities(shape, (n / 2, n / 2), R, 5.0, 1.0, 0.03)
    o = oracle.Oracle(solid, tau=tau, G=G)
    o.init_densities(r1, r2)
    o.step(steps)
    return physics.laplace_cylinder(o.fields(), (n / 2, n / 2))


def test_laplace_law_surface_tension():
    """Section 3.1: the pressure jump of Eq. 12 is linear in the curvature with
    slope gamma = 0.071 at G = 3.5, independent of the viscosity ratio.  The
    droplets are y-invariant cylinders (jump gamma / R), which share the
    interface of the paper's spheres (jump 2 gamma / R) at lower cost."""
    R1, dP1 = _cylinder(14, (1.0, 1.0))
    R2, dP2 = _cylinder(24, (1.0, 1.0))
    slope = (dP1 - dP2) / (1 / R1 - 1 / R2)
    assert abs(slope / GAMMA - 1) < 0.10
    for R, dP in ((R1, dP1), (R2, dP2)):
        assert abs(dP * R / GAMMA - 1) < 0.12
    R3, dP3 = _cylinder(24, tuple(REF["tau_M25"][0]))
    assert abs(dP3 * R3 - dP2 * R2) < 0.05 * dP2 * R2


def _droplet_gamma(n, R0, cylinder, steps, tau=(1.0, 1.0)):
    """gamma of a sphere (dP = 2 gamma / R) or y-invariant cylinder (dP =
    gamma / R) of component 1 in a periodic box of edge n, initialised by
    Eq. 16 with the Section 3.1 densities and width."""
    shape = (n, 1, n) if cylinder else (n, n, n)
    rin, rout, W = REF["laplace_rho_in"][0][0], REF["laplace_rho_out"][0][0], REF["laplace_W"][0][0]
    if cylinder:
        r1, r2 = inputs.cylinder_densities(shape, (n / 2, n / 2), R0, W, rin, rout)
        c = (n / 2, 0, n / 2)
    else:
        r1, r2 = inputs.droplet_densities(shape, (n / 2, n / 2, n / 2), R0, W, rin, rout)
        c = (n / 2, n / 2, n / 2)
    o = oracle.Oracle(np.zeros(shape, np.uint8), tau=tau, G=G)
    o.init_densities(r1, r2)
    o.step(steps)
    R, dP = physics.laplace_jump(o.fields(), c, cylinder)
    return dP * R / (1.0 if cylinder else 2.0)


def test_laplace_total_curvature_sphere_and_cylinder():
    """Laplace's law in three dimensions (Section 3.1 measures it on spheres):
    the jump is gamma times the total curvature, 2/R for a sphere and 1/R for
    a y-invariant cylinder, so the two give one gamma in the same periodic box
    (40^3, R0 = 12; measured 0.0825 and 0.0837).  A box this small reads
    above the printed 0.071, which the Section 3.1 box of 128^3 reproduces
    (0.0715 for R >= 20 on the GPU; the slow pin below checks 64^3)."""
    gs = _droplet_gamma(40, 12, False, 2500)
    gc = _droplet_gamma(40, 12, True, 2500)
    assert abs(gs / gc - 1) < 0.04, (gs, gc)
    assert GAMMA < gs < 1.25 * GAMMA


@pytest.mark.slow
def test_laplace_sphere_surface_tension_64():
    """Spheres in a 64^3 periodic box (R0 = 12, 16; densities of Eq. 16):
    gamma = dP R / 2 within 10% of the printed 0.071 (about 7-8% high in this
    box; it falls to the printed value as the box grows to the paper's 128^3;
    measured 0.0766 and 0.0760).  Ten to twenty minutes of the oracle."""
    for R0 in (12, 16):
        g = _droplet_gamma(64, R0, False, 6000)
        print("R0 %d: gamma %.5f" % (R0, g))
        assert abs(g / GAMMA - 1) < 0.10


def _cap_angle(xi, tau, nx=96, nz=40, R=16, steps=4000):
    shape = (nz, 1, nx)
    solid = np.zeros(shape, np.uint8)
    solid[0] = 1
    solid[-1] = 1
    r1, r2 = inputs.cylinder_densities(shape, (nx / 2, 1.0), R, 5.0, 1.0, 0.03)
    fl = solid == 0
    o = oracle.Oracle(solid, tau=tau, G=G, xi=xi, periodic=(1, 1, 0))
    o.init_densities(r1 * fl, r2 * fl)
    o.step(steps)
    return physics.contact_angle_water(o.fields(), 0.5)


@pytest.mark.parametrize("xi", [-0.2, 0.2])
def test_contact_angle_calibration(xi):
    """Section 3.2 calibration at G = 3.5, M = 25: theta(xi) from the printed
    cubic, and the quoted pairs xi = -0.2 -> ~70 deg, 0.2 -> ~108 deg."""
    c3, c2, c1, c0 = REF["theta_cubic"][0]
    theta_fit = ((c3 * xi + c2) * xi + c1) * xi + c0
    theta = _cap_angle(xi, tuple(REF["tau_M25"][0]))
    assert abs(theta - theta_fit) < 3.0
    quoted = {round(p[0], 3): p[1] for p in REF["theta_pair"]}[round(xi, 3)]
    assert abs(theta - quoted) < 4.0


def test_contact_angle_neutral_is_ninety_degrees():
    """xi = 0, M = 1, symmetric densities: swapping the components maps theta
    to 180 - theta, so the equilibrium angle is 90 degrees."""
    assert abs(_cap_angle(0.0, (1.0, 1.0)) - 90.0) < 1.0


def test_square_duct_poiseuille():
    """Single component (rho2 = 0, so no interaction force) driven by a body
    acceleration g along z in a square duct with half-way bounce-back walls:
    the series solution with walls half a voxel outside the outermost fluid
    nodes.  tau = 1/2 + sqrt(3/16) puts the bounce-back wall exactly half way."""
    m = 16
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    nu = (tau - 0.5) / 3.0
    g = 1e-6
    solid = np.ones((1, m + 2, m + 2), np.uint8)
    solid[:, 1:-1, 1:-1] = 0
    o = oracle.Oracle(solid, tau=(tau, tau), G=G, periodic=(0, 0, 1), body_force=(0, 0, g))
    o.init_densities(1.0 * (solid == 0), 0.0)
    o.step(3000)
    uz = o.fields()["uz"][0, 1:-1, 1:-1]
    ref = physics.duct_series_velocity(m, m, g, nu)
    assert np.abs(uz - ref).max() / ref.max() < 0.01


def _enclosed_droplet(n=16, r=4.0):
    """A droplet of component 1 in a closed cubic pore (one-voxel solid shell),
    surrounded by component 2, viscosity ratio 10, neutral walls."""
    solid = np.zeros((n, n, n), np.uint8)
    solid[0] = solid[-1] = 1
    solid[:, 0] = solid[:, -1] = 1
    solid[:, :, 0] = solid[:, :, -1] = 1
    c = (n - 1) / 2.0
    r1, r2 = inputs.droplet_densities(solid.shape, (c, c, c), r, 2.0, 1.0, 0.03)
    fl = solid == 0
    return solid, r1 * fl, r2 * fl


def test_enclosed_droplet_keeps_its_volume():
    """Section 4.1's point that the model preserves trapped volume: a droplet
    sealed in a closed pore keeps its volume (count of nodes where component 1
    is the majority) within 1% from step 500 to step 10^4."""
    solid, r1, r2 = _enclosed_droplet()
    o = oracle.Oracle(solid, tau=inputs.tau_for_viscosity_ratio(10.0), G=G, periodic=(0, 0, 0))
    o.init_densities(r1, r2)
    o.step(500)
    f = o.fields()
    v0 = int(((f["rho1"] > f["rho2"]) & (solid == 0)).sum())
    o.step(9500)
    f = o.fields()
    v1 = int(((f["rho1"] > f["rho2"]) & (solid == 0)).sum())
    assert v0 > 100
    assert abs(v1 - v0) <= 0.01 * v0, (v0, v1)


def test_parallel_flow_solver_closed_forms():
    """The momentum-balance solver the layered-flow pins use, against closed
    forms: one viscosity gives the Poiseuille parabola with the walls half a
    node beyond the fluid, and two layers with the jump on a cell face give
    the two-layer solution (outer parabola, inner parabola plus the outer
    layer's velocity at the interface), both to 0.2%."""
    nz, g = 66, 1e-6
    fluid = np.ones(nz, bool)
    fluid[0] = fluid[-1] = False
    y = np.arange(nz)[fluid] - (nz - 1) / 2.0
    h, a = (nz - 2) / 2.0, 16.0
    R = np.ones(nz)
    u = physics.parallel_flow_profile(R, np.full(nz, 0.1), g, fluid)
    ref = g / 0.2 * (h * h - y * y)
    assert np.abs(u - ref).max() <= 2e-3 * ref.max()
    mu_in, mu_out = 0.02, 0.2
    mu = np.where(np.abs(np.arange(nz) - (nz - 1) / 2.0) < a, mu_in, mu_out)
    u = physics.parallel_flow_profile(R, mu, g, fluid)
    ref = np.where(np.abs(y) >= a, g / (2 * mu_out) * (h * h - y * y),
                   g / (2 * mu_in) * (a * a - y * y) + g / (2 * mu_out) * (h * h - a * a))
    assert np.abs(u - ref).max() <= 2e-3 * ref.max()


@pytest.mark.parametrize("tau", [(1.0, 0.55), (0.5433, 0.9330)])
def test_layered_channel_flow(tau):
    """Two immiscible layers driven along x between flat walls: component 1 in
    the middle half of the channel, component 2 against the walls, viscosity
    ratio about 8 or 1/8.  At steady state the momentum balance is d/dz(mu du/dz)
    = -R g, where R = rho1 + rho2 carries the body force (each component gets
    rho_s g) and mu = rho1 nu1 + rho2 nu2 is the dynamic viscosity of the
    mixture relaxation (Eqs. 6-7, nu = c_s^2 (tau - 1/2)).  Solved on the
    oracle's own R(z) and mu(z), including the diffuse interface, where R dips
    by a third, that balance gives the oracle's velocity profile to 1%; the
    sharp-interface parabolas, which ignore the dip, are off by 4-6%.  A
    relaxation time averaged without the density weights, or a body force on
    one component only, is off by tens of percent."""
    nz, g = 66, 1e-7
    solid = np.zeros((nz, 1, 1), np.uint8)
    solid[0] = 1
    solid[-1] = 1
    z = np.arange(nz)
    inner = np.abs(z - (nz - 1) / 2.0) < (nz - 2) / 4.0
    fluid = solid[:, 0, 0] == 0
    r1 = (np.where(inner, 1.0, 0.03) * fluid)[:, None, None]
    r2 = (np.where(inner, 0.03, 1.0) * fluid)[:, None, None]
    o = oracle.Oracle(solid, tau=tau, G=G, periodic=(1, 1, 0), body_force=(g, 0.0, 0.0))
    o.init_densities(r1, r2)
    o.step(240000)
    f = o.fields()
    rho1, rho2, ux = f["rho1"][:, 0, 0], f["rho2"][:, 0, 0], f["ux"][:, 0, 0]
    nu1, nu2 = (tau[0] - 0.5) / 3.0, (tau[1] - 0.5) / 3.0
    mu = rho1 * nu1 + rho2 * nu2
    ref = physics.parallel_flow_profile(rho1 + rho2, mu, g, fluid)
    assert np.abs(ux[fluid] - ref).max() <= 0.01 * ref.max()
    assert abs(ux[nz // 2] / ref[nz // 2 - 1] - 1) <= 0.01
    assert np.abs(f["uz"]).max() < 1e-6 * ref.max() + 1e-12
