"""The flow schedule (one launch per step: collide-stream, then the next
densities and wall densities from L2, ordered by per-chunk flags) against the
split schedule, through the C ABI.

Every item of the flow launch runs the split passes' per-node arithmetic, so
the two schedules must agree bit for bit: populations, densities and
saturation, on both A-A parities, with and without CUDA graphs, for every
storage type, with open planes (extrapolation and Zou-He), a periodic z axis
(dependencies that wrap around the chunk order), walls with a xi field, a
changed inlet density between steps, and lags from one slot to many.  The
oracle comparisons of the flow schedule are in test_gpu_parity.py (its
`sched` fixture includes it).
"""
import numpy as np
import pytest

from paper_2207_01534_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "these tests need a GPU"
    from paper_2207_01534_gb300 import lbm as m

    m.load()
    return m


def _drainage(n=(40, 26, 30), seed=11):
    nz, ny, nx = n
    rng = np.random.default_rng(seed)
    solid = (rng.random(n) < 0.32).astype(np.uint8)
    solid[:4] = 0
    solid[-4:] = 0
    r1, r2 = inputs.drainage_init(solid, 4)
    kw = dict(tau=(1.7, 0.62), G=3.5, xi=-0.3, periodic=(1, 1, 0), open_axis=2, rho_in1=1.06, rho_out2=1.0)
    return solid, r1, r2, kw


def _pair(lbm, solid, storage, **kw):
    a = lbm.Lattice(solid, storage=storage, kernel="split", **kw)
    b = lbm.Lattice(solid, storage=storage, kernel="flow", **kw)
    assert b.info()["kernel"] == 6
    return a, b


def _same_state(a, b):
    pa, pb = a.get_populations(), b.get_populations()
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y), np.abs(x - y).max()
    fa, fb = a.fields(("rho1", "rho2")), b.fields(("rho1", "rho2"))
    for k in fa:
        assert np.array_equal(fa[k], fb[k])
    assert np.array_equal(np.asarray(a.saturation()), np.asarray(b.saturation()))


@pytest.mark.parametrize("storage", ["fp32", "fp64", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("bc", ["neem", "zou_he"])
def test_open_drainage_bitwise_equal_to_split(lbm, storage, bc):
    solid, r1, r2, kw = _drainage()
    a, b = _pair(lbm, solid, storage, bc=bc, **kw)
    for g in (a, b):
        g.init_densities(r1, r2)
    for n in (1, 1, 2, 7, 40):  # odd and even starts, plain steps and graph replays
        a.step(n)
        b.step(n)
        _same_state(a, b)


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_periodic_droplet_bitwise_equal_to_split(lbm, storage):
    """Fully periodic 48^3 droplet: chunks on the first and last z planes
    depend on each other through the wrap."""
    solid, r1, r2 = inputs.laplace_48()
    a, b = _pair(lbm, solid, storage, tau=(1.0, 1.0), G=3.5)
    for g in (a, b):
        g.init_densities(r1, r2)
    for n in (3, 64, 5):
        a.step(n)
        b.step(n)
        _same_state(a, b)


def test_parameter_changes_between_steps(lbm):
    """A new inlet density or xi field between steps applies from the next
    step in both schedules (the flow schedule recomputes its densities)."""
    solid, r1, r2, kw = _drainage(seed=12)
    a, b = _pair(lbm, solid, "fp32", **kw)
    for g in (a, b):
        g.init_densities(r1, r2)
        g.step(9)
        g.set_inlet(1.1)
        g.step(10)
    _same_state(a, b)
    xi = np.where(solid > 0, np.linspace(-0.4, 0.3, solid.size).reshape(solid.shape), 0).astype(np.float32)
    for g in (a, b):
        g.set_xi_field(xi)
        g.step(33)
    _same_state(a, b)
    # reinitialisation at an odd step count restarts the parity
    for g in (a, b):
        g.init_densities(r1, r2)
        g.step(3)
    _same_state(a, b)


@pytest.mark.parametrize("lags", [("1", "1"), ("4", "200"), ("400", "3")])
def test_lags_do_not_change_results(lbm, monkeypatch, lags):
    monkeypatch.setenv("LBM_FLOW_LAG_D", lags[0])
    monkeypatch.setenv("LBM_FLOW_LAG_W", lags[1])
    solid, r1, r2, kw = _drainage(n=(36, 30, 34), seed=13)
    a, b = _pair(lbm, solid, "fp32", **kw)
    for g in (a, b):
        g.init_densities(r1, r2)
        g.step(21)
    _same_state(a, b)


def test_reduce_every_and_timed_steps(lbm):
    solid, r1, r2, kw = _drainage(seed=14)
    a, b = _pair(lbm, solid, "fp32", reduce_every=5, **kw)
    for g in (a, b):
        g.init_densities(r1, r2)
        g.step(12)
        ms = g.step_timed(5)
        assert np.all(ms >= 0)
    _same_state(a, b)
    assert b.step_timed(2)[4] > 0  # the flow launch is timed in the pipeline slot


def test_ragged_single_chunk_and_tiny_domains(lbm):
    # fewer fluid nodes than one chunk, a one-voxel domain, a 40 x 1 x 1 column
    for shape, per in (((5, 4, 3), (1, 1, 1)), ((1, 1, 1), (1, 1, 1)), ((1, 1, 40), (1, 1, 1))):
        solid = np.zeros(shape, np.uint8)
        rng = np.random.default_rng(sum(shape))
        r1 = rng.uniform(0.05, 0.9, shape)
        r2 = rng.uniform(0.05, 0.9, shape)
        a, b = _pair(lbm, solid, "fp64", tau=(1.2, 0.8), G=3.5, periodic=per)
        for g in (a, b):
            g.init_densities(r1, r2)
            g.step(6)
        _same_state(a, b)


def test_bounded_wait_times_out_and_recovers(lbm):
    """lbm_inject_stall makes one D item of the next flow launch wait for a
    stamp that never comes: the wait gives up after the time limit, the step
    reports LBM_ERR_TIMEOUT, and a reinitialised lattice runs correctly."""
    solid, r1, r2, kw = _drainage(seed=15)
    a, b = _pair(lbm, solid, "fp32", **kw)
    b.set_wait_limit(0.05)
    for g in (a, b):
        g.init_densities(r1, r2)
        g.step(4)
    b.inject_stall()
    with pytest.raises(lbm.LbmError) as ei:
        b.step(1)
        b.synchronize()
    assert ei.value.code == -6
    for g in (a, b):
        g.init_densities(r1, r2)
        g.step(11)
    _same_state(a, b)
