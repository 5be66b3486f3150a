"""Pins of the oracle's hand-derived discrete adjoint (FP64, CPU).

The adjoint is pinned to something other than itself: central finite
differences of the oracle's own forward step in FP64 (eps = 1e-6), for the
per-voxel wettability xi, the inlet density rho_in1, the initial populations
(with the frozen open-boundary values they imply) and a random linear
functional of the final state.  A dropped term in any reverse stage (the
extrapolation, streaming, collision, tau(rho), u, the force stencil with its
mirrored neighbours, the virtual density) breaks one of them."""
import numpy as np
import pytest

import oracle
from paper_2207_01534_gb300 import inputs

EPS = 1e-6


def _slab(seed=3, nz=14, ny=7, nx=8, frac=0.25):
    rng = np.random.default_rng(seed)
    solid = (rng.random((nz, ny, nx)) < frac).astype(np.uint8)
    solid[:3] = 0
    solid[-3:] = 0
    solid = inputs.keep_percolating(solid)
    r1, r2 = inputs.drainage_init(solid, 3)
    # a little noise so that every term of the step is active
    fl = solid == 0
    r1 = r1 * (1 + 0.05 * rng.uniform(-1, 1, r1.shape)) * fl
    r2 = r2 * (1 + 0.05 * rng.uniform(-1, 1, r2.shape)) * fl
    xi = np.where(solid == 1, rng.uniform(-0.4, 0.4, solid.shape), 0.0)
    kw = dict(tau=(1.3, 0.7), G=3.5, periodic=(1, 1, 0), open_axis=2, rho_in1=1.12, rho_out2=1.0,
              body_force=(1e-5, -2e-5, 3e-5))
    return solid, r1, r2, xi, kw


NSTEPS = 25
SAMPLE = (3, 11)


def _loss(solid, r1, r2, xi, kw, pops=None):
    o = oracle.Oracle(solid, xi_field=xi, **kw)
    if pops is None:
        o.init_densities(r1, r2)
    else:
        o.set_pops(pops[0], pops[1])
    o.step(NSTEPS)
    return o.saturation(*SAMPLE)[1]


@pytest.fixture(scope="module")
def case():
    solid, r1, r2, xi, kw = _slab()
    o = oracle.Oracle(solid, xi_field=xi, **kw)
    o.init_densities(r1, r2)
    o.record(NSTEPS)
    g = o.adjoint(*SAMPLE, want_state=True)
    # the reverse pass leaves the oracle at the final state
    assert abs(o.saturation(*SAMPLE)[1] - _loss(solid, r1, r2, xi, kw)) < 1e-15
    return solid, r1, r2, xi, kw, g


def test_xi_gradient_matches_finite_differences(case):
    solid, r1, r2, xi, kw, g = case
    gx = g["xi"]
    assert np.all(gx[solid == 0] == 0)
    walls = np.argsort(-np.abs(gx).ravel())[:6]
    rng = np.random.default_rng(0)
    cand = np.flatnonzero((solid.ravel() == 1) & (gx.ravel() != 0))
    picks = list(walls) + list(rng.choice(cand, 4, replace=False))
    scale = np.abs(gx).max()
    assert scale > 1e-6
    for v in picks:
        xp, xm = xi.copy(), xi.copy()
        xp.ravel()[v] += EPS
        xm.ravel()[v] -= EPS
        fd = (_loss(solid, r1, r2, xp, kw) - _loss(solid, r1, r2, xm, kw)) / (2 * EPS)
        assert abs(fd - gx.ravel()[v]) <= 1e-6 * scale + 1e-5 * abs(fd), (v, fd, gx.ravel()[v])


def test_inlet_density_gradient_matches_finite_differences(case):
    solid, r1, r2, xi, kw, g = case
    kp = dict(kw, rho_in1=kw["rho_in1"] + EPS)
    km = dict(kw, rho_in1=kw["rho_in1"] - EPS)
    fd = (_loss(solid, r1, r2, xi, kp) - _loss(solid, r1, r2, xi, km)) / (2 * EPS)
    assert abs(g["rho_in1"]) > 1e-6
    assert abs(fd - g["rho_in1"]) <= 1e-6 * abs(fd)


def test_initial_population_gradient_matches_finite_differences(case):
    solid, r1, r2, xi, kw, g = case
    o = oracle.Oracle(solid, xi_field=xi, **kw)
    o.init_densities(r1, r2)
    f1, f2 = o.get_pops()
    rng = np.random.default_rng(5)
    fl = (solid == 0)[None]
    for trial in range(3):
        d1 = rng.standard_normal(f1.shape) * fl * 1e-2
        d2 = rng.standard_normal(f2.shape) * fl * 1e-2
        jp = _loss(solid, r1, r2, xi, kw, pops=(f1 + EPS * d1, f2 + EPS * d2))
        jm = _loss(solid, r1, r2, xi, kw, pops=(f1 - EPS * d1, f2 - EPS * d2))
        fd = (jp - jm) / (2 * EPS)
        # set_pops also sets the frozen boundary values: total derivative
        tot = g["f"] + g["frozen"]
        ad = float((tot[0] * d1).sum() + (tot[1] * d2).sum())
        assert abs(fd - ad) <= 1e-6 * abs(fd) + 1e-12, (trial, fd, ad)


def test_random_functional_of_the_final_state():
    """J = <seed, f_n> for a random seed: every output population's adjoint
    path is exercised, not just the densities that the saturation reads."""
    solid, r1, r2, xi, kw = _slab(seed=9, nz=10, ny=6, nx=6)
    n = 6
    rng = np.random.default_rng(7)
    seed = rng.standard_normal((2, 19) + solid.shape) * (solid == 0)[None, None]
    o = oracle.Oracle(solid, xi_field=xi, **kw)
    o.init_densities(r1, r2)
    f1, f2 = o.get_pops()
    o.record(n)
    g = o.adjoint(seed=seed, want_state=True)

    def J(p1, p2, x=xi, k=kw):
        q = oracle.Oracle(solid, xi_field=x, **k)
        q.set_pops(p1, p2)
        q.step(n)
        a, b = q.get_pops()
        return float((seed[0] * a).sum() + (seed[1] * b).sum())

    d1 = rng.standard_normal(f1.shape) * (solid == 0)[None] * 1e-2
    d2 = rng.standard_normal(f2.shape) * (solid == 0)[None] * 1e-2
    fd = (J(f1 + EPS * d1, f2 + EPS * d2) - J(f1 - EPS * d1, f2 - EPS * d2)) / (2 * EPS)
    tot = g["f"] + g["frozen"]
    ad = float((tot[0] * d1).sum() + (tot[1] * d2).sum())
    assert abs(fd - ad) <= 1e-7 * abs(fd)
    # and one wettability direction
    dx = rng.standard_normal(solid.shape) * (solid == 1)
    fdx = (J(f1, f2, x=xi + EPS * dx) - J(f1, f2, x=xi - EPS * dx)) / (2 * EPS)
    adx = float((g["xi"] * dx).sum())
    assert abs(fdx - adx) <= 1e-7 * abs(fdx) + 1e-12


def test_closed_periodic_droplet_has_no_inlet_gradient():
    solid = np.zeros((8, 8, 8), np.uint8)
    r1, r2 = inputs.droplet_densities(solid.shape, (4, 4, 4), 2.5)
    o = oracle.Oracle(solid, tau=(1.0, 1.0), G=3.5)
    o.init_densities(r1, r2)
    o.record(5)
    g = o.adjoint()
    assert g["rho_in1"] == 0.0 and not g["xi"].any()
