"""Oracle pins: exact invariants of the step (conservation, rest states,
symmetry, open-boundary rules of Section 2)."""
import numpy as np
import pytest

import oracle
from paper_2207_01534_gb300 import inputs


def _momentum(o):
    e, _, _ = oracle.lattice()
    f1, f2 = o.get_pops()
    f = (f1 + f2).reshape(19, -1).sum(axis=1)
    return e.astype(float).T @ f


def test_uniform_mixture_is_a_fixed_point_to_roundoff():
    solid = np.zeros((8, 8, 8), np.uint8)
    o = oracle.Oracle(solid, tau=(1.7, 0.62), G=3.5)
    o.init_densities(0.7, 0.3)
    f1a, f2a = o.get_pops()
    o.step(20)
    f1b, f2b = o.get_pops()
    assert np.abs(f1a - f1b).max() < 1e-15 and np.abs(f2a - f2b).max() < 1e-15


def test_single_component_at_rest_in_porous_solid_stays_at_rest():
    rng = np.random.default_rng(1)
    solid = (rng.random((12, 12, 12)) < 0.25).astype(np.uint8)
    o = oracle.Oracle(solid, tau=(0.8, 0.8), G=3.5, xi=-0.3)
    o.init_densities(1.0 * (solid == 0), 0.0)
    o.step(30)
    f = o.fields()
    assert max(np.abs(f[k]).max() for k in ("ux", "uy", "uz")) < 1e-15
    assert np.abs(f["rho1"] - 1.0 * (solid == 0)).max() < 1e-14


def _walled(nz=12, nx=8):
    solid = np.zeros((nz, 4, nx), np.uint8)
    solid[0] = 1
    solid[-1] = 1
    return solid


def test_neutral_wall_keeps_uniform_mixture_at_rest():
    """xi = 0: rho-tilde equals the neighbouring fluid density (Eq. 15), so the
    adhesion force completes the cohesion stencil and a uniform mixture feels
    no force next to a flat wall."""
    solid = _walled()
    o = oracle.Oracle(solid, tau=(1.0, 1.0), G=3.5, xi=0.0, periodic=(1, 1, 0))
    o.init_densities(0.5 * (solid == 0), 0.5 * (solid == 0))
    o.step(50)
    f = o.fields()
    assert max(np.abs(f[k]).max() for k in ("ux", "uy", "uz")) < 1e-13


@pytest.mark.parametrize("xi,wetting1", [(-0.3, False), (0.3, True)])
def test_adhesion_sign(xi, wetting1):
    """Section 2: component 1 is non-wetting for xi < 0 and wetting for xi > 0,
    so it is depleted (enriched) in the layer next to the wall."""
    solid = _walled()
    o = oracle.Oracle(solid, tau=(1.0, 1.0), G=3.5, xi=xi, periodic=(1, 1, 0))
    o.init_densities(0.5 * (solid == 0), 0.5 * (solid == 0))
    o.step(200)
    f = o.fields()
    d = f["rho1"][1].mean() - f["rho2"][1].mean()
    assert (d > 1e-3) if wetting1 else (d < -1e-3)


def _porous_droplet_case(tau):
    n = 16
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    solid = np.zeros((n, n, n), np.uint8)
    for c, r in (((3, 4, 12), 3.0), ((12, 12, 3), 2.5), ((8, 2, 2), 2.0)):
        solid[(xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= r * r] = 1
    r1, r2 = inputs.droplet_densities((n, n, n), (8.3, 9.1, 7.6), 4.0, 3.0, 1.0, 0.03)
    rng = np.random.default_rng(3)
    r1 = (r1 * (1 + 0.01 * rng.uniform(-1, 1, r1.shape))) * (solid == 0)
    r2 = (r2 * (1 + 0.01 * rng.uniform(-1, 1, r2.shape))) * (solid == 0)
    o = oracle.Oracle(solid, tau=tau, G=3.5, xi=-0.3)
    o.init_densities(r1, r2)
    return o


def test_mass_conserved_per_component_to_roundoff():
    o = _porous_droplet_case((1.7, 0.62))
    _, _, m1a, m2a = o.saturation()
    o.step(200)
    _, _, m1b, m2b = o.saturation()
    assert abs(m1b - m1a) / m1a < 1e-12
    assert abs(m2b - m2a) / m2a < 1e-12


def test_total_momentum_conserved_without_solids_equal_tau():
    """With tau1 = tau2 on a periodic solid-free domain the pairwise cohesion
    forces cancel in the sum over nodes, and the F/2 velocity shift makes the
    collision inject exactly F per node, so total momentum stays zero."""
    n = 14
    solid = np.zeros((n, n, n), np.uint8)
    r1, r2 = inputs.droplet_densities((n, n, n), (6.2, 7.7, 5.4), 4.0, 3.0, 1.0, 0.03)
    rng = np.random.default_rng(5)
    r1 *= 1 + 0.02 * rng.uniform(-1, 1, r1.shape)
    o = oracle.Oracle(solid, tau=(1.0, 1.0), G=3.5)
    o.init_densities(r1, r2)
    o.step(100)
    p = _momentum(o)
    mass = sum(o.saturation()[2:])
    assert np.abs(p).max() / mass < 1e-13
    # a nonzero check that momentum is actually being exchanged locally
    f = o.fields()
    assert np.abs(f["ux"]).max() > 1e-6


@pytest.mark.parametrize("tau", [(1.0, 1.0), (1.7, 0.62)])
def test_body_force_injects_exactly_its_momentum(tau):
    """Periodic, solid-free, a droplet (so cohesion forces act) under a body
    acceleration g: each step adds exactly F = sum_x R g to the total momentum,
    whatever the relaxation times, because the velocity of the equilibrium
    carries half the force (Eq. 8 with F/2) and the source term its factor
    1 - 1/(2 tau) (Eq. 9): -(m - R u)/tau + (1 - 1/(2 tau)) F = F.  Without the
    half-force shift at tau = 1 the collision keeps only F/2 per step."""
    n, steps = 14, 100
    solid = np.zeros((n, n, n), np.uint8)
    r1, r2 = inputs.droplet_densities((n, n, n), (6.2, 7.7, 5.4), 4.0, 3.0, 1.0, 0.03)
    g = np.array([2e-5, -1e-5, 3e-5])
    o = oracle.Oracle(solid, tau=tau, G=3.5, body_force=tuple(g))
    o.init_densities(r1, r2)
    o.step(steps)
    mass = sum(o.saturation()[2:])
    assert np.abs(_momentum(o) / (steps * mass * g) - 1).max() < 1e-12
    if tau == (1.0, 1.0):
        q = oracle.Oracle(solid, tau=tau, G=3.5, body_force=tuple(g), velocity_shift=0)
        q.init_densities(r1, r2)
        q.step(steps)
        assert np.abs(_momentum(q) / (steps * mass * g) - 0.5).max() < 1e-12


def test_centred_droplet_keeps_cubic_symmetry():
    """A droplet centred on a node of a periodic cube keeps the 48 symmetries of
    the cube; any wrong component in the velocity table breaks it."""
    n = 20
    solid = np.zeros((n, n, n), np.uint8)
    r1, r2 = inputs.droplet_densities((n, n, n), (10, 10, 10), 5.0, 4.0, 1.0, 0.03)
    o = oracle.Oracle(solid, tau=(1.0, 1.0), G=3.5)
    o.init_densities(r1, r2)
    o.step(40)
    rho = o.fields()["rho1"]
    ref = np.roll(rho, (-10, -10, -10), axis=(0, 1, 2))  # centre to index 0
    for perm in ((0, 2, 1), (1, 0, 2), (2, 1, 0)):
        assert np.abs(np.transpose(ref, perm) - ref).max() < 1e-12
    flip = np.roll(ref[:, :, ::-1], 1, axis=2)  # x -> -x about index 0
    assert np.abs(flip - ref).max() < 1e-12


def _open_channel(rho_in1=1.05, rho_out2=1.0, nz=24):
    solid = np.zeros((nz, 8, 8), np.uint8)
    r1, r2 = inputs.drainage_init(solid, 4)
    o = oracle.Oracle(solid, tau=(1.7, 0.62), G=3.5, periodic=(1, 1, 0), open_axis=2,
                      rho_in1=rho_in1, rho_out2=rho_out2)
    o.init_densities(r1, r2)
    return o


def test_inlet_outlet_densities_are_exact():
    o = _open_channel()
    o.step(30)
    f = o.fields()
    assert np.abs(f["rho1"][0] - 1.05).max() < 1e-14
    assert np.abs(f["rho2"][-1] - 1.0).max() < 1e-14


def test_missing_populations_keep_initial_values():
    """Section 2, open-boundary rule 2: the missing populations of the
    non-prescribed component keep their initial values forever."""
    o = _open_channel()
    f1a, f2a = o.get_pops()
    o.step(40)
    f1b, f2b = o.get_pops()
    inlet_missing = [5, 11, 12, 15, 16]   # e_z = +1: enter the z = 0 plane from outside
    outlet_missing = [6, 13, 14, 17, 18]  # e_z = -1: enter the z = nz-1 plane from outside
    assert np.array_equal(f2b[inlet_missing, 0], f2a[inlet_missing, 0])
    assert np.array_equal(f1b[outlet_missing, -1], f1a[outlet_missing, -1])
    # and the other populations there did change
    assert not np.array_equal(f2b[:, 0], f2a[:, 0])


def test_uniform_state_with_matching_open_planes_stays_at_rest():
    """The mirrored pseudopotential of Section 2 balances the force at the open
    planes: a uniform mixture whose prescribed densities equal its own keeps
    zero velocity (without the mirror rule the planes would feel a force)."""
    solid = np.zeros((16, 6, 6), np.uint8)
    o = oracle.Oracle(solid, tau=(1.0, 1.0), G=3.5, periodic=(1, 1, 0), open_axis=2, rho_in1=0.6, rho_out2=0.4)
    o.init_densities(0.6, 0.4)
    o.step(50)
    f = o.fields()
    assert max(np.abs(f[k]).max() for k in ("ux", "uy", "uz")) < 1e-14


def test_geometry_validation():
    solid = np.zeros((6, 6, 6), np.uint8)
    with pytest.raises(ValueError):
        oracle.Oracle(solid, periodic=(0, 1, 1))  # fluid on a closed x face
    with pytest.raises(ValueError):
        oracle.Oracle(solid, periodic=(1, 1, 1), open_axis=2)  # open axis must not be periodic
    s2 = solid.copy()
    s2[1, 2, 2] = 1
    with pytest.raises(ValueError):
        oracle.Oracle(s2, periodic=(1, 1, 0), open_axis=2)  # inlet node with a solid interior neighbour
