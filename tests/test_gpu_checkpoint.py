"""Checkpoint / resume (lbm_save, lbm_load): a lattice saved part-way and
loaded into a fresh context continues bitwise as the uninterrupted run, for
plain and 16-bit storage and with open planes (boundary cells and frozen
populations travel with the state); files of another lattice, and truncated
files, are refused."""
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


def _slab(seed=6, nz=22, ny=11, nx=13):
    rng = np.random.default_rng(seed)
    solid = (rng.random((nz, ny, nx)) < 0.27).astype(np.uint8)
    solid[:3] = 0
    solid[-3:] = 0
    solid = inputs.keep_percolating(solid)
    r1, r2 = inputs.drainage_init(solid, 3)
    kw = dict(tau=(1.4, 0.66), G=3.5, xi=-0.25, periodic=(1, 1, 0), open_axis=2, rho_in1=1.12, rho_out2=1.0,
              sample=(3, nz - 3))
    return solid, r1, r2, kw


@pytest.mark.parametrize("storage", ["fp32", "fp16dev", "fp64"])
def test_saved_state_resumes_bitwise(lbm, storage, tmp_path):
    solid, r1, r2, kw = _slab()
    a = lbm.Lattice(solid, storage=storage, **kw)
    a.init_densities(r1, r2)
    a.step(37)
    path = tmp_path / "state.lbm"
    a.save(path)
    a.step(23)
    fa = a.get_populations()
    b = lbm.Lattice(solid, storage=storage, **kw)  # never initialised: everything comes from the file
    b.load(path)
    assert b.info()["step"] == 37
    b.step(23)
    fb = b.get_populations()
    assert b.info()["step"] == a.info()["step"] == 60
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])
    assert a.saturation() == b.saturation()


def test_other_lattices_and_broken_files_are_refused(lbm, tmp_path):
    solid, r1, r2, kw = _slab()
    a = lbm.Lattice(solid, **kw)
    a.init_densities(r1, r2)
    a.step(4)
    path = tmp_path / "state.lbm"
    a.save(path)
    other = _slab(seed=7)[0]
    for lat in (lbm.Lattice(other, **kw), lbm.Lattice(solid, storage="fp16dev", **kw)):
        with pytest.raises(lbm.LbmError) as e:
            lat.load(path)
        assert e.value.code == -1
    data = path.read_bytes()
    cut = tmp_path / "cut.lbm"
    cut.write_bytes(data[: len(data) // 2])
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(solid, **kw).load(cut)
    junk = tmp_path / "junk.lbm"
    junk.write_bytes(b"not a state file" * 8)
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(solid, **kw).load(junk)
