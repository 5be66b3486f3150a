"""The brick schedule (one block per 8^3 brick: densities of the brick and its
halo, wall virtual densities and next-step density accumulators in shared
memory; one launch per step plus the plane pass) against the FP64 oracle at
the FP32 parity bounds, on shapes that exercise partial bricks, short
periodic axes, closed faces and open planes; 16-bit storage against the FP32
path; bitwise reproducibility."""
import os

import numpy as np
import pytest

import oracle
from paper_2207_01534_gb300 import inputs
from test_gpu_parity import TOL_FP32_RHO, TOL_MASS, _compare_rho, _open_porous, _porous_periodic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "these tests need a GPU"
    from paper_2207_01534_gb300 import lbm as m

    m.load()
    return m


def _pair(lbm, solid, storage="fp32", **kw):
    g = lbm.Lattice(solid, storage=storage, kernel="brick", **kw)
    o = oracle.Oracle(solid, **{k: v for k, v in kw.items() if k not in ("sample",)})
    return g, o


@pytest.mark.parametrize("steps", [1, 2, 5])
def test_random_state_all_populations(lbm, steps):
    """Every population after a few steps from a random state on a periodic
    porous domain of 22 x 18 x 20 (partial bricks on every axis)."""
    solid = _porous_periodic()
    f1, f2 = inputs.random_pops_state(solid, inputs.SEED_BASE + 100, rho_lo=0.05, rho_hi=0.9, noise=0.05)
    g, o = _pair(lbm, solid, tau=(1.7, 0.62), G=3.5, xi=-0.3)
    g.set_populations(f1, f2)
    o.set_pops(f1, f2)
    g.step(steps)
    o.step(steps)
    a1, a2 = g.get_populations()
    b1, b2 = o.get_pops()
    assert np.abs(a1 - b1).max() <= 2e-6 and np.abs(a2 - b2).max() <= 2e-6


def test_laplace_48_thousand_steps(lbm):
    solid, r1, r2 = inputs.laplace_48()
    g, o = _pair(lbm, solid, tau=(1.0, 1.0), G=3.5)
    g.init_densities(r1, r2)
    o.init_densities(r1, r2)
    m0 = g.saturation()
    g.step(1000)
    o.step(1000)
    _compare_rho(g, o, TOL_FP32_RHO)
    m1 = g.saturation()
    assert abs(m1[2] - m0[2]) / m0[2] <= TOL_MASS and abs(m1[3] - m0[3]) / m0[3] <= TOL_MASS


@pytest.mark.parametrize("bc", ["neem", "zou_he"])
def test_open_drainage_porous(lbm, bc):
    solid = _open_porous()
    r1, r2 = inputs.drainage_init(solid, 4)
    kw = dict(tau=inputs.tau_for_viscosity_ratio(10.0), G=3.5, xi=inputs.xi_of_theta(45.0), periodic=(1, 1, 0),
              open_axis=2, rho_in1=1.08, rho_out2=1.0, bc=bc)
    g, o = _pair(lbm, solid, **kw)
    g.init_densities(r1, r2)
    o.init_densities(r1, r2)
    for chunk in (1, 1, 98, 100):
        g.step(chunk)
        o.step(chunk)
        _compare_rho(g, o, TOL_FP32_RHO)
    fg = g.fields(("rho1", "rho2"))
    fl = solid == 0
    assert np.abs(fg["rho1"][0][fl[0]] - 1.08).max() < 1e-5
    assert np.abs(fg["rho2"][-1][fl[-1]] - 1.0).max() < 1e-5


def test_walled_lateral_faces_and_xi_field(lbm):
    """Non-periodic x closed by solid faces, a per-voxel xi field, open z."""
    nz, ny, nx = 24, 10, 12
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:, :, 0] = 1
    solid[:, :, -1] = 1
    solid[8:14, 3:7, 4:8] = 1
    rng = np.random.default_rng(5)
    xi = rng.uniform(-0.4, 0.3, solid.shape).astype(np.float32).astype(np.float64)
    r1, r2 = inputs.drainage_init(solid, 3)
    kw = dict(tau=(1.1, 0.62), G=3.5, xi_field=xi, periodic=(0, 1, 0), open_axis=2, rho_in1=1.05, rho_out2=1.0)
    g, o = _pair(lbm, solid, **kw)
    g.init_densities(r1, r2)
    o.init_densities(r1, r2)
    g.step(301)
    o.step(301)
    _compare_rho(g, o, TOL_FP32_RHO)


def test_set_xi_field_updates_the_wall_coefficients(lbm):
    """A new xi field after creation reaches the brick wall entries: the brick
    lattice follows the split lattice given the same field."""
    solid = _porous_periodic((20, 16, 24), 13)
    r1, r2 = inputs.droplet_densities(solid.shape, (12, 8, 10), 5.0, 4.0, 1.0, 0.03)
    fl = solid == 0
    xi = np.where(solid == 1, np.random.default_rng(3).uniform(-0.5, 0.5, solid.shape), 0.0).astype(np.float32)
    out = {}
    for sched in ("split", "brick"):
        g = lbm.Lattice(solid, kernel=sched, tau=(1.3, 0.7), G=3.5, xi=0.0)
        g.init_densities(r1 * fl, r2 * fl)
        g.step(50)
        g.set_xi_field(xi)
        g.step(150)
        out[sched] = g.fields(("rho1", "rho2"))
    o = oracle.Oracle(solid, tau=(1.3, 0.7), G=3.5, xi=0.0)
    o.init_densities(r1 * fl, r2 * fl)
    o.step(50)
    fx = oracle.Oracle(solid, tau=(1.3, 0.7), G=3.5, xi_field=xi.astype(np.float64))
    fx.set_pops(*o.get_pops())
    fx.step(150)
    fo = fx.fields()
    for sched in ("split", "brick"):
        for k in ("rho1", "rho2"):
            assert np.abs(out[sched][k] - fo[k]).max() <= TOL_FP32_RHO * np.abs(fo[k]).max(), (sched, k)


def test_body_force_and_ragged_size(lbm):
    solid = _porous_periodic((17, 23, 29), 9)
    r1, r2 = inputs.droplet_densities(solid.shape, (14, 11, 8), 5.0, 4.0, 1.0, 0.03)
    fl = solid == 0
    g, o = _pair(lbm, solid, tau=(1.7, 0.62), G=3.5, xi=0.2, body_force=(1e-5, -2e-5, 3e-5))
    g.init_densities(r1 * fl, r2 * fl)
    o.init_densities(r1 * fl, r2 * fl)
    g.step(333)
    o.step(333)
    _compare_rho(g, o, TOL_FP32_RHO)


def test_degenerate_domains(lbm):
    """Periodic axes shorter than a brick (one voxel: every neighbour is the
    node itself; a 40 x 1 x 1 column), a thin slab with walls, no fluid."""
    solid = np.zeros((1, 1, 1), np.uint8)
    g, o = _pair(lbm, solid, tau=(1.2, 0.8), G=3.5)
    g.init_densities(np.full((1, 1, 1), 0.7), np.full((1, 1, 1), 0.3))
    o.init_densities(0.7, 0.3)
    g.step(7)
    o.step(7)
    _compare_rho(g, o, TOL_FP32_RHO)
    solid = np.zeros((40, 1, 1), np.uint8)
    z = np.arange(40)[:, None, None]
    r1 = np.where((z > 10) & (z < 30), 1.0, 0.03) + 0 * solid
    r2 = np.where((z > 10) & (z < 30), 0.03, 1.0) + 0 * solid
    g, o = _pair(lbm, solid, tau=(1.0, 1.0), G=3.5)
    g.init_densities(r1, r2)
    o.init_densities(r1, r2)
    g.step(300)
    o.step(300)
    _compare_rho(g, o, TOL_FP32_RHO)
    # a cap on a wall, periodic x and a one-voxel periodic y (walls seen
    # through the short axis at several halo cells)
    shape = (20, 1, 30)
    solid = np.zeros(shape, np.uint8)
    solid[0] = 1
    solid[-1] = 1
    r1, r2 = inputs.cylinder_densities(shape, (15.0, 1.0), 6, 5.0, 1.0, 0.03)
    fl = solid == 0
    g, o = _pair(lbm, solid, tau=(1.0, 1.0), G=3.5, xi=0.3, periodic=(1, 1, 0))
    g.init_densities(r1 * fl, r2 * fl)
    o.init_densities(r1 * fl, r2 * fl)
    g.step(200)
    o.step(200)
    _compare_rho(g, o, TOL_FP32_RHO)
    g = lbm.Lattice(np.ones((4, 4, 4), np.uint8), kernel="brick")
    g.init_densities(np.zeros((4, 4, 4)), np.zeros((4, 4, 4)))
    g.step(13)
    assert g.saturation() == (0.0, 0.0, 0.0, 0.0)
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(solid, kernel="brick", storage="fp64")


def test_enclosed_droplet_closed_on_every_face(lbm):
    from test_oracle_physics import _enclosed_droplet

    solid, r1, r2 = _enclosed_droplet()
    kw = dict(tau=inputs.tau_for_viscosity_ratio(10.0), G=3.5, periodic=(0, 0, 0))
    g, o = _pair(lbm, solid, **kw)
    g.init_densities(r1, r2)
    o.init_densities(r1, r2)
    m0 = g.saturation()
    g.step(300)
    o.step(300)
    _compare_rho(g, o, TOL_FP32_RHO)
    m1 = g.saturation()
    assert abs(m1[2] - m0[2]) / m0[2] <= TOL_MASS and abs(m1[3] - m0[3]) / m0[3] <= TOL_MASS


def test_bitwise_reproducible_with_and_without_graphs(lbm):
    solid = _open_porous()
    r1, r2 = inputs.drainage_init(solid, 4)
    kw = dict(tau=(1.7, 0.62), G=3.5, xi=-0.3, periodic=(1, 1, 0), open_axis=2, rho_in1=1.1, rho_out2=1.0)
    out = []
    for env in ({}, {"LBM_NO_GRAPH": "1"}, {}):
        os.environ.update(env)
        try:
            g = lbm.Lattice(solid, kernel="brick", **kw)
            g.init_densities(r1, r2)
            for n in (1, 4, 29, 13, 70):  # off-period starts, short and long replays, ragged tails
                g.step(n)
            out.append(g.get_populations())
        finally:
            os.environ.pop("LBM_NO_GRAPH", None)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    for a, b in zip(out[0], out[2]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["fp16dev", "bf16dev"])
def test_sixteen_bit_against_fp32(lbm, storage):
    """16-bit storage on the brick schedule stays as close to the FP32 path
    as on the split schedule (open drainage through a porous slab, 300 steps:
    the moving front magnifies the storage error to about 2e-2 on either
    schedule)."""
    solid = _open_porous()
    r1, r2 = inputs.drainage_init(solid, 4)
    kw = dict(tau=inputs.tau_for_viscosity_ratio(10.0), G=3.5, xi=inputs.xi_of_theta(45.0), periodic=(1, 1, 0),
              open_axis=2, rho_in1=1.08, rho_out2=1.0)
    f = {}
    for sched, st in (("split", "fp32"), ("split", storage), ("brick", storage)):
        g = lbm.Lattice(solid, kernel=sched, storage=st, **kw)
        g.init_densities(r1, r2)
        g.step(300)
        f[(sched, st)] = g.fields(("rho1", "rho2"))
    ref = f[("split", "fp32")]
    err = {k: max(np.abs(v[c] - ref[c]).max() / np.abs(ref[c]).max() for c in ("rho1", "rho2")) for k, v in f.items()}
    print(storage, err)
    assert err[("brick", storage)] <= 1.25 * err[("split", storage)] + 1e-4
