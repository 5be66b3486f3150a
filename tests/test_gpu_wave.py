"""The wavefront schedule (split passes per z slab in a dependency graph)
gives the split schedule's results bit for bit, for open and periodic z,
several slab counts and graph lengths, and a ragged remainder of steps."""
import os

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


def _open_case(nz=36, ny=14, nx=12, seed=2):
    rng = np.random.default_rng(seed)
    solid = (rng.random((nz, ny, nx)) < 0.25).astype(np.uint8)
    solid[:3] = 0
    solid[-3:] = 0
    solid = inputs.keep_percolating(solid)
    r1, r2 = inputs.drainage_init(solid, 3)
    kw = dict(tau=inputs.tau_for_viscosity_ratio(10.0), G=3.5, xi=-0.2, periodic=(1, 1, 0), open_axis=2,
              rho_in1=1.1, rho_out2=1.0)
    return solid, (r1, r2), kw


def _closed_case(n=24):
    solid = np.zeros((n, n, n), np.uint8)
    solid[5:9, 5:9, 5:9] = 1
    r1, r2 = inputs.droplet_densities(solid.shape, (n / 2, n / 2, n / 2), 5.0)
    fl = solid == 0
    return solid, (r1 * fl, r2 * fl), dict(tau=(1.0, 0.8), G=3.5, xi=0.3)


def _run(lbm, case, kernel, steps, env):
    solid, rho, kw = case
    saved = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        g = lbm.Lattice(solid, kernel=kernel, **kw)
        g.init_densities(*rho)
        for n in steps:
            g.step(n)
        return g.get_populations(), g.info()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("case", ["open", "closed"])
@pytest.mark.parametrize("slabs,gsteps", [("3", "4"), ("5", "2"), ("7", "6")])
def test_wave_equals_split_bitwise(lbm, case, slabs, gsteps):
    c = _open_case() if case == "open" else _closed_case()
    steps = (1, 2, 37, 5)  # odd start, graph replays and a ragged tail
    (a1, a2), _ = _run(lbm, c, "split", steps, {})
    (b1, b2), info = _run(lbm, c, "wave", steps, {"LBM_WAVE_SLABS": slabs, "LBM_WAVE_STEPS": gsteps})
    assert info["kernel"] == 3
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)


def test_wave_falls_back_on_thin_domains(lbm):
    """Fewer than three slabs of two planes: the wave schedule runs the split
    passes (still correct)."""
    solid = np.zeros((5, 6, 6), np.uint8)
    r1, r2 = inputs.droplet_densities(solid.shape, (3, 3, 2.5), 1.5)
    c = (solid, (r1, r2), dict(tau=(1.0, 1.0), G=3.5))
    (a1, _), _ = _run(lbm, c, "split", (9,), {})
    (b1, _), _ = _run(lbm, c, "wave", (9,), {"LBM_WAVE_SLABS": "8"})
    assert np.array_equal(a1, b1)
