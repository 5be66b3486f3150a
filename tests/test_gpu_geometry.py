"""Geometry preprocessing of lbm_create on the device (the split and wave
schedules) against the host preprocessing (LBM_HOST_PREP=1, and the path of
the other schedules): the same node and wall counts and bitwise the same
populations, densities and saturations after steps on both A-A parities,
for open and periodic domains, ragged sizes, walled faces, a per-voxel xi
field, FP32 and FP64 storage (the Eq. 15 denominators and xi in the storage
type's compute precision)."""
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


def _cases():
    rng = np.random.default_rng(21)
    out = []
    s = (rng.random((37, 29, 23)) < 0.35).astype(np.uint8)  # ragged, open z, xi field
    s[:3] = 0
    s[-3:] = 0
    xi = np.where(s > 0, rng.uniform(-0.4, 0.4, s.shape), 0.0).astype(np.float32)
    out.append(("open_xi", s, dict(periodic=(1, 1, 0), open_axis=2, rho_in1=1.07, rho_out2=1.0, xi_field=xi)))
    s = (rng.random((20, 33, 41)) < 0.3).astype(np.uint8)  # fully periodic
    out.append(("periodic", s, dict(periodic=(1, 1, 1), xi=0.25)))
    s = (rng.random((24, 18, 16)) < 0.25).astype(np.uint8)
    s[:2] = 0
    s[-2:] = 0
    s = inputs.add_lateral_walls(s)  # walled x and y faces
    out.append(("walled", s, dict(periodic=(0, 0, 0), open_axis=2, rho_in1=1.05, rho_out2=1.0, xi=-0.3)))
    out.append(("one_voxel", np.zeros((1, 1, 1), np.uint8), dict(periodic=(1, 1, 1))))
    out.append(("column", np.zeros((40, 1, 1), np.uint8), dict(periodic=(1, 1, 1))))
    out.append(("no_fluid", np.ones((4, 5, 6), np.uint8), dict(periodic=(1, 1, 1))))
    return out


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
@pytest.mark.parametrize("case", [c[0] for c in _cases()])
def test_device_geometry_equals_host_geometry(lbm, monkeypatch, storage, case):
    name, solid, kw = next(c for c in _cases() if c[0] == case)
    kw = dict(kw, tau=(1.3, 0.7), G=3.5, storage=storage)
    dev = lbm.Lattice(solid, kernel="split", **kw)
    monkeypatch.setenv("LBM_HOST_PREP", "1")
    host = lbm.Lattice(solid, kernel="split", **kw)
    monkeypatch.delenv("LBM_HOST_PREP")
    a, b = dev.info(), host.info()
    assert (a["n_fluid"], a["n_wall"]) == (b["n_fluid"], b["n_wall"])
    if a["n_fluid"] == 0:
        return
    r1, r2 = inputs.drainage_init(solid, 2) if "open_axis" in kw else (np.full(solid.shape, 0.6), np.full(solid.shape, 0.4))
    rng = np.random.default_rng(5)
    if "open_axis" not in kw:
        r1 = r1 * rng.uniform(0.5, 1.5, solid.shape)
    for g in (dev, host):
        g.init_densities(r1, r2)
    for n in (1, 6):
        for g in (dev, host):
            g.step(n)
        pa, pb = dev.get_populations(), host.get_populations()
        for x, y in zip(pa, pb):
            assert np.array_equal(x, y)
        fa, fb = dev.fields(("rho1", "rho2", "P")), host.fields(("rho1", "rho2", "P"))
        for k in fa:
            assert np.array_equal(fa[k], fb[k])
        assert np.array_equal(np.asarray(dev.saturation()), np.asarray(host.saturation()))


def test_device_geometry_rejects_invalid_geometries(lbm):
    # a fluid voxel on a closed face, and a solid voxel behind an open plane
    s = np.zeros((6, 5, 4), np.uint8)
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(s, kernel="split", periodic=(1, 0, 1))
    assert e.value.code == -1
    s = np.zeros((6, 5, 4), np.uint8)
    s[1, 2, 2] = 1
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(s, kernel="split", periodic=(1, 1, 0), open_axis=2)
    assert e.value.code == -1
