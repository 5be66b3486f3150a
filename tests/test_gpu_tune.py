"""The schedule chooser on the GPU: every candidate schedule runs on the
caller's lattice, the fastest is returned and cached, a cached choice needs
no timing, and a lattice built with the chosen schedule matches the split
schedule's densities."""
import json

import numpy as np
import pytest

from paper_2207_01534_gb300 import inputs, tune
from test_gpu_parity import _open_porous

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "these tests need a GPU"
    from paper_2207_01534_gb300 import lbm as m

    m.load()
    return m


@pytest.mark.parametrize("storage", ["fp32", "fp16dev"])
def test_choose_schedule(lbm, tmp_path, storage):
    solid = _open_porous()
    r1, r2 = inputs.drainage_init(solid, 4)
    kw = dict(tau=(1.7, 0.62), G=3.5, xi=-0.3, periodic=(1, 1, 0), open_axis=2, rho_in1=1.1, rho_out2=1.0,
              storage=storage)
    path, blocks = str(tmp_path / "sched.json"), str(tmp_path / "blocks.json")
    e = tune.choose_schedule(solid, (r1, r2), cache_path=path, block_cache=blocks, **kw)
    print(e)
    assert set(e["timings"]) == set(tune.candidates(storage))
    assert e["kernel"] == min(e["timings"], key=e["timings"].get) and all(v > 0 for v in e["timings"].values())
    assert json.load(open(path))[e["key"]]["kernel"] == e["kernel"]

    def no_timing(*a):
        raise AssertionError("a cached choice must not be timed")

    assert tune.choose_schedule(solid, (r1, r2), cache_path=path, timer=no_timing, **kw) == e
    g = lbm.Lattice(solid, kernel=e["kernel"], **kw)
    if e["kernel"] in ("split", "wave"):
        assert g.autotune(blocks) == e["block"]
    h = lbm.Lattice(solid, kernel="split", **kw)
    for lat in (g, h):
        lat.init_densities(r1, r2)
        lat.step(30)
    a, b = g.fields(("rho1", "rho2")), h.fields(("rho1", "rho2"))
    # the fixed-point densities of the push and brick schedules can flip a
    # 16-bit rounding; FP32 agrees to the parity bound
    tol = 1e-5 if storage == "fp32" else 2e-3
    for k in ("rho1", "rho2"):
        assert np.abs(a[k] - b[k]).max() <= tol * np.abs(b[k]).max()
