"""The push schedule (no density pass; next densities accumulated in integer
fixed point by the collide-stream pass) against the FP64 oracle, at the FP32
parity bounds, plus its bitwise reproducibility."""
import os

import numpy as np
import pytest

import oracle
from paper_2207_01534_gb300 import inputs
from test_gpu_parity import (TOL_FP32_RHO, TOL_MASS, _compare_rho, _open_porous, _porous_periodic)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "these tests need a GPU"
    from paper_2207_01534_gb300 import lbm as m

    m.load()
    return m


def _pair(lbm, solid, **kw):
    g = lbm.Lattice(solid, storage="fp32", kernel="push", **kw)
    o = oracle.Oracle(solid, **{k: v for k, v in kw.items() if k not in ("sample",)})
    return g, o


@pytest.mark.parametrize("steps", [1, 2, 5])
def test_random_state_all_populations(lbm, steps):
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


def test_open_drainage_walled_lateral_faces(lbm):
    """Walled x and y faces reach the open planes, so some walls read plane
    nodes (they are finished after them); the fluid rows end at walls, so
    the warp-combined pushes see rows that end inside a warp."""
    solid = inputs.add_lateral_walls(_open_porous((30, 18, 21), seed=5))
    r1, r2 = inputs.drainage_init(solid, 4)
    kw = dict(tau=inputs.tau_for_viscosity_ratio(10.0), G=3.5, xi=inputs.xi_of_theta(60.0), periodic=(0, 0, 0),
              open_axis=2, rho_in1=1.08, rho_out2=1.0, bc="neem")
    g, o = _pair(lbm, solid, **kw)
    g.init_densities(r1, r2)
    o.init_densities(r1, r2)
    for chunk in (1, 2, 97, 200):
        g.step(chunk)
        o.step(chunk)
        _compare_rho(g, o, TOL_FP32_RHO)


def test_walls_body_force_and_ragged_size(lbm):
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
    solid = np.zeros((1, 1, 1), np.uint8)  # every neighbour is the node itself
    g, o = _pair(lbm, solid, tau=(1.2, 0.8), G=3.5)
    g.init_densities(np.full((1, 1, 1), 0.7), np.full((1, 1, 1), 0.3))
    o.init_densities(0.7, 0.3)
    g.step(7)
    o.step(7)
    _compare_rho(g, o, TOL_FP32_RHO)
    g = lbm.Lattice(np.ones((4, 4, 4), np.uint8), kernel="push")
    g.init_densities(np.zeros((4, 4, 4)), np.zeros((4, 4, 4)))
    g.step(13)
    assert g.saturation() == (0.0, 0.0, 0.0, 0.0)
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(solid, kernel="push", storage="fp64")


def test_bitwise_reproducible_with_and_without_graphs(lbm):
    solid = _open_porous()
    r1, r2 = inputs.drainage_init(solid, 4)
    kw = dict(tau=(1.7, 0.62), G=3.5, xi=-0.3, periodic=(1, 1, 0), open_axis=2, rho_in1=1.1, rho_out2=1.0)
    out = []
    for env in ({}, {"LBM_NO_GRAPH": "1"}, {}):
        os.environ.update(env)
        try:
            g = lbm.Lattice(solid, kernel="push", **kw)
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


def test_restart_from_populations_matches_continuous_run(lbm):
    """Re-priming the accumulators from a saved state continues the same run
    up to the fixed-point rounding of the densities."""
    solid = _open_porous()
    r1, r2 = inputs.drainage_init(solid, 4)
    kw = dict(tau=(1.7, 0.62), G=3.5, xi=-0.3, periodic=(1, 1, 0), open_axis=2, rho_in1=1.1, rho_out2=1.0)
    g = lbm.Lattice(solid, kernel="push", **kw)
    g.init_densities(r1, r2)
    g.step(40)
    f1, f2 = g.get_populations()
    g.step(20)
    h = lbm.Lattice(solid, kernel="push", **kw)
    h.set_populations(f1, f2)  # frozen boundary values now come from this state
    h.step(20)
    a = g.fields(("rho1", "rho2"))
    b = h.fields(("rho1", "rho2"))
    assert np.abs(a["rho1"] - b["rho1"]).max() < 1e-4 and np.abs(a["rho2"] - b["rho2"]).max() < 1e-4
