"""Batches of independent lattices, CUDA-graph replay and the autotuner.

A batch runs each sample's nodes through the same per-node arithmetic as a
solo lattice, so every sample must match its solo run bit for bit (FP32 and
16-bit storage alike); graph replay and the block size chosen by the
autotuner must not change a single bit either."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2207_01534_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "these tests need a GPU"
    from paper_2207_01534_gb300 import lbm as m

    m.load()
    return m


def _open_slab(seed, nz=26, ny=12, nx=14, theta=45.0, pin=1.12):
    """A porous slab between an inlet and an outlet reservoir (drainage set-up)."""
    rng = np.random.default_rng(seed)
    solid = (rng.random((nz, ny, nx)) < 0.25).astype(np.uint8)
    solid[:3] = 0
    solid[-3:] = 0
    solid = inputs.keep_percolating(solid)
    r1, r2 = inputs.drainage_init(solid, 3)
    kw = dict(solid=solid, tau=inputs.tau_for_viscosity_ratio(10.0), G=3.5, xi=inputs.xi_of_theta(theta),
              periodic=(1, 1, 0), open_axis=2, rho_in1=pin, rho_out2=1.0, sample=(3, nz - 3))
    return kw, (r1, r2)


def _droplet(n=16, G=3.5):
    solid = np.zeros((n, n, n), np.uint8)
    r1, r2 = inputs.droplet_densities(solid.shape, (n / 2, n / 2, n / 2), n / 4)
    return dict(solid=solid, tau=(1.0, 1.0), G=G), (r1, r2)


def _channel(nz=10, ny=9, nx=7):
    """A walled duct (solid lateral faces) driven by a body force along z."""
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:, 0, :] = solid[:, -1, :] = 1
    solid[:, :, 0] = solid[:, :, -1] = 1
    r1 = np.full(solid.shape, 0.05)
    r2 = np.full(solid.shape, 1.0)
    return dict(solid=solid, tau=(0.8, 1.2), G=3.5, xi=0.2, body_force=(0.0, 0.0, 1e-5)), (r1, r2)


def _cases():
    return [_open_slab(1), _droplet(), _open_slab(2, nz=20, ny=10, nx=11, theta=120.0, pin=1.08), _channel()]


def _solo(lbm, kw, rho, nsteps, storage, env=None):
    kw = dict(kw, storage=storage, kernel="split")
    g = lbm.Lattice(**kw)
    g.init_densities(*rho)
    old = {}
    for k, v in (env or {}).items():
        old[k] = os.environ.get(k)
        os.environ[k] = v
    try:
        g.step(nsteps)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return g


@pytest.mark.parametrize("storage", ["fp32", "fp16dev"])
def test_batch_samples_equal_their_solo_runs(lbm, storage):
    cases = _cases()
    b = lbm.Batch([dict(kw, storage=storage) for kw, _ in cases])
    assert len(b) == len(cases)
    for smp, (_, rho) in zip(b.samples, cases):
        smp.init_densities(*rho)
    b.step(1)  # odd start: the plain steps and the graph are both exercised
    b.step(37)
    b.synchronize()
    info = b.info()
    assert info["step"] == 38
    assert info["n_fluid"] == sum(int((kw["solid"] == 0).sum()) for kw, _ in cases)
    for k, (kw, rho) in enumerate(cases):
        solo = _solo(lbm, kw, rho, 38, storage)
        a1, a2 = b[k].get_populations()
        s1, s2 = solo.get_populations()
        assert np.array_equal(a1, s1) and np.array_equal(a2, s2), "sample %d differs from its solo run" % k
        assert b[k].saturation() == solo.saturation()


@pytest.mark.parametrize("storage", ["fp32", "fp16dev"])
def test_persistent_batch_samples_equal_their_solo_runs(lbm, storage):
    """One cooperative launch for many steps of the whole batch (grid barriers
    between the passes): every sample bitwise its solo run, through a
    parameter change of one sample between calls and launches that start on
    either parity."""
    cases = _cases()
    b = lbm.Batch([dict(kw, storage=storage, kernel="persistent") for kw, _ in cases])
    for smp, (_, rho) in zip(b.samples, cases):
        smp.init_densities(*rho)
    l0 = b.info()["launches"]
    b.step(1)
    b.step(37)
    assert b.info()["launches"] - l0 == 2  # one launch per call of up to 256 steps
    b[2].set_inlet(1.15)
    b.step(9)
    b.step(300)  # two launches
    b.synchronize()
    assert b.info()["step"] == 347
    for k, (kw, rho) in enumerate(cases):
        solo = _solo(lbm, kw, rho, 38, storage)
        if k == 2:
            solo.set_inlet(1.15)
        solo.step(309)
        a1, a2 = b[k].get_populations()
        s1, s2 = solo.get_populations()
        assert np.array_equal(a1, s1) and np.array_equal(a2, s2), "sample %d differs from its solo run" % k
        assert b[k].saturation() == solo.saturation()


def test_persistent_batch_barrier_timeout_is_reported(lbm):
    """A block that never reaches its first grid barrier (lbm_inject_stall):
    every wait gives up after the time limit, lbm_step reports
    LBM_ERR_TIMEOUT, and after re-initialisation the batch steps as before."""
    cases = _cases()[:2]
    b = lbm.Batch([dict(kw, kernel="persistent") for kw, _ in cases])
    for smp, (_, rho) in zip(b.samples, cases):
        smp.init_densities(*rho)
    b.step(4)
    b.set_wait_limit(0.05)
    b.inject_stall()
    with pytest.raises(lbm.LbmError) as e:
        b.step(3)
        b.synchronize()
    assert e.value.code == -6
    for smp, (_, rho) in zip(b.samples, cases):
        smp.init_densities(*rho)
    b.step(20)
    b.synchronize()
    for k, (kw, rho) in enumerate(cases):
        solo = _solo(lbm, kw, rho, 20, "fp32")
        a1, a2 = b[k].get_populations()
        s1, s2 = solo.get_populations()
        assert np.array_equal(a1, s1) and np.array_equal(a2, s2)


def test_persistent_launch_takes_batches_only(lbm):
    kw, rho = _droplet()
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(**dict(kw, kernel="persistent"))
    assert e.value.code == -7
    # the batch table of one launch holds at most 96 samples
    tiny = dict(solid=np.zeros((4, 4, 4), np.uint8), tau=(1.0, 1.0), G=3.5, kernel="persistent")
    with pytest.raises(lbm.LbmError) as e:
        lbm.Batch([tiny] * 97)
    assert e.value.code == -7
    b = lbm.Batch([tiny] * 96)
    for smp in b.samples:
        smp.init_densities(np.full((4, 4, 4), 0.5), np.full((4, 4, 4), 0.5))
    b.step(3)
    b.synchronize()
    assert b.info()["step"] == 3


def test_batch_sample_matches_oracle(lbm):
    kw, rho = _open_slab(3)
    b = lbm.Batch([kw, _droplet()[0]])
    b[0].init_densities(*rho)
    b[1].init_densities(*_droplet()[1])
    b.step(60)
    o = oracle.Oracle(kw["solid"], tau=kw["tau"], G=kw["G"], xi=kw["xi"], periodic=kw["periodic"],
                      open_axis=2, rho_in1=kw["rho_in1"], rho_out2=kw["rho_out2"])
    o.init_densities(*rho)
    o.step(60)
    fo = o.fields()
    fg = b[0].fields()
    for key in ("rho1", "rho2"):
        assert np.abs(fg[key] - fo[key]).max() <= 1e-5 * np.abs(fo[key]).max()


def test_graph_replay_is_bitwise_plain(lbm):
    kw, rho = _open_slab(4)
    plain = _solo(lbm, kw, rho, 41, "fp32", env={"LBM_NO_GRAPH": "1"})
    graph = _solo(lbm, kw, rho, 41, "fp32")
    p1, p2 = plain.get_populations()
    g1, g2 = graph.get_populations()
    assert np.array_equal(p1, g1) and np.array_equal(p2, g2)
    # a parameter change after capture must reach the replayed steps
    for g in (plain, graph):
        g.set_inlet(1.2)
    os.environ["LBM_NO_GRAPH"] = "1"
    try:
        plain.step(20)
    finally:
        os.environ.pop("LBM_NO_GRAPH", None)
    graph.step(20)
    p1, p2 = plain.get_populations()
    g1, g2 = graph.get_populations()
    assert np.array_equal(p1, g1) and np.array_equal(p2, g2)


def test_batch_inlet_change_reaches_the_batch(lbm):
    cases = [_open_slab(5), _open_slab(6)]
    b = lbm.Batch([kw for kw, _ in cases])
    for smp, (_, rho) in zip(b.samples, cases):
        smp.init_densities(*rho)
    b.step(10)
    b[1].set_inlet(1.2)
    b.step(10)
    solo = _solo(lbm, cases[1][0], cases[1][1], 10, "fp32")
    solo.set_inlet(1.2)
    solo.step(10)
    a1, _ = b[1].get_populations()
    s1, _ = solo.get_populations()
    assert np.array_equal(a1, s1)


def test_samples_are_stepped_through_the_batch(lbm):
    b = lbm.Batch([_droplet()[0], _droplet(G=3.0)[0]])
    with pytest.raises(lbm.LbmError):
        b[0].step(1)
    with pytest.raises(lbm.LbmError):
        lbm._check(b._lib.lbm_saturation(b._h, np.zeros(4).ctypes.data), b._h)
    for smp in b.samples:
        smp.init_densities(*_droplet()[1])
    b.step(1)
    b[1].init_densities(*_droplet()[1])  # resets sample 1 to step 0
    with pytest.raises(lbm.LbmError):
        b.step(1)


def test_batch_rejects_mixed_storage(lbm):
    with pytest.raises(lbm.LbmError):
        lbm.Batch([dict(_droplet()[0], storage="fp32"), dict(_droplet()[0], storage="fp16dev")])


def test_autotune_restores_state_and_caches(lbm, tmp_path):
    kw, rho = _open_slab(7)
    ref = _solo(lbm, kw, rho, 30, "fp32")
    g = _solo(lbm, kw, rho, 10, "fp32")
    before = g.get_populations()
    cache = str(tmp_path / "tune.json")
    blk = g.autotune(cache)
    assert blk in (64, 128, 256)
    assert g.info()["step"] == 10
    after = g.get_populations()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    data = json.load(open(cache))
    assert list(data.values()) == [blk]
    assert "fp32" in list(data)[0]
    g.step(20)  # at the tuned block size: still bitwise the untuned run
    a = g.get_populations()
    r = ref.get_populations()
    assert np.array_equal(a[0], r[0]) and np.array_equal(a[1], r[1])
    # a cached key is applied without timing: force a value and read it back
    json.dump({list(data)[0]: 64}, open(cache, "w"))
    assert g.autotune(cache) == 64
    g.step(4)
    ref.step(4)
    a, r = g.get_populations(), ref.get_populations()
    assert np.array_equal(a[0], r[0])


def test_batch_autotune(lbm, tmp_path):
    cases = _cases()
    b = lbm.Batch([kw for kw, _ in cases])
    for smp, (_, rho) in zip(b.samples, cases):
        smp.init_densities(*rho)
    b.step(6)
    snap = [smp.get_populations() for smp in b.samples]
    blk = b.autotune(str(tmp_path / "tune.json"))
    assert blk in (64, 128, 256)
    for smp, (p1, p2) in zip(b.samples, snap):
        q1, q2 = smp.get_populations()
        assert np.array_equal(p1, q1) and np.array_equal(p2, q2)
    b.step(10)
    for k, (kw, rho) in enumerate(cases):
        solo = _solo(lbm, kw, rho, 16, "fp32")
        assert np.array_equal(b[k].get_populations()[0], solo.get_populations()[0])
