"""Failure detection on the GPU without a GPU fault: the failures are made on
the host (a non-finite population, an impossibly tight drift limit, a device
wait for a round that never completes) and the library must report them as
status codes and stay usable."""
import time

import numpy as np
import pytest

import oracle
from paper_2207_01534_gb300 import inputs

pytestmark = pytest.mark.gpu

LBM_ERR_NONFINITE, LBM_ERR_DRIFT, LBM_ERR_TIMEOUT = -4, -5, -6


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "these tests need a GPU"
    from paper_2207_01534_gb300 import lbm as m

    m.load()
    return m


def _droplet(n=20):
    solid = np.zeros((n, n, n), np.uint8)
    r1, r2 = inputs.droplet_densities(solid.shape, (n / 2, n / 2, n / 2), n / 4)
    return solid, r1, r2


@pytest.mark.parametrize("kernel", ["split", "fused"])
def test_nonfinite_population_is_reported(lbm, kernel):
    solid, r1, r2 = _droplet()
    g = lbm.Lattice(solid, kernel=kernel, reduce_every=1)
    g.init_densities(r1, r2)
    f1, f2 = g.get_populations()
    f1[3, 5, 6, 7] = np.nan
    g.set_populations(f1, f2)
    with pytest.raises(lbm.LbmError) as ei:
        g.step(2)
        g.synchronize()
    assert ei.value.code == LBM_ERR_NONFINITE
    # a fresh state clears it
    g.init_densities(r1, r2)
    g.step(4)
    g.synchronize()


def test_mass_drift_limit(lbm):
    solid, r1, r2 = _droplet()
    ok = lbm.Lattice(solid, reduce_every=5)  # default limit 1e-6: FP32 rounding stays far below
    ok.init_densities(r1, r2)
    ok.step(200)
    ok.synchronize()
    tight = lbm.Lattice(solid, reduce_every=5, drift_limit=1e-300)
    tight.init_densities(r1, r2)
    with pytest.raises(lbm.LbmError) as ei:
        tight.step(200)
        tight.synchronize()
    assert ei.value.code == LBM_ERR_DRIFT


def test_device_wait_timeout_and_recovery(lbm):
    """A single-pass step told to wait for a round that never completes gives
    up after the wait limit, reports LBM_ERR_TIMEOUT, and the context runs
    correctly again after reinitialisation."""
    solid, r1, r2 = _droplet(24)
    g = lbm.Lattice(solid, kernel="fused", tau=(1.0, 1.0), G=3.5)
    g.set_wait_limit(0.05)
    g.init_densities(r1, r2)
    g.step(3)
    g.inject_stall()
    t0 = time.perf_counter()
    with pytest.raises(lbm.LbmError) as ei:
        g.step(1)
        g.synchronize()
    dt = time.perf_counter() - t0
    assert ei.value.code == LBM_ERR_TIMEOUT
    assert dt < 5.0
    # recovery: reinitialise and compare with the oracle
    g.init_densities(r1, r2)
    g.step(40)
    g.synchronize()
    o = oracle.Oracle(solid, tau=(1.0, 1.0), G=3.5)
    o.init_densities(r1, r2)
    o.step(40)
    fg, fo = g.fields(("rho1", "rho2")), o.fields()
    for k in ("rho1", "rho2"):
        assert np.abs(fg[k] - fo[k]).max() <= 1e-5 * np.abs(fo[k]).max()


def test_inject_stall_needs_the_single_pass_schedule(lbm):
    solid, r1, r2 = _droplet(8)
    g = lbm.Lattice(solid, kernel="split")
    with pytest.raises(lbm.LbmError):
        g.inject_stall()
    with pytest.raises(lbm.LbmError):
        g.set_wait_limit(0.0)
