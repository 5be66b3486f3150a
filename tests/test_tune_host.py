"""Host logic of the schedule chooser (paper_2207_01534_gb300.tune): the
candidate lists, the cache key, the choice of the fastest schedule and the
JSON cache, with a stand-in lattice and timer (no GPU)."""
import json

import numpy as np
import pytest

from paper_2207_01534_gb300 import tune

DEV = ("Test GPU", (10, 3))


class FakeLattice:
    made = []

    def __init__(self, solid, kernel, **kw):
        assert "kernel" not in kw
        self.kernel, self.kw, self.closed, self.rho = kernel, kw, False, None
        FakeLattice.made.append(self)

    def init_densities(self, r1, r2):
        self.rho = (r1, r2)

    def autotune(self, cache=None):
        self.cache = cache
        return 128

    def close(self):
        self.closed = True


def _timer(ms):
    def t(lat, steps, warmup):
        assert lat.rho is not None and steps == 5 and warmup == 2
        return ms[lat.kernel]
    return t


def _solid():
    s = np.zeros((6, 5, 4), np.uint8)
    s[2, 2, 2] = 1
    return s


def test_candidates_per_storage():
    assert tune.candidates("fp32") == ["split", "wave", "push", "brick"]
    assert tune.candidates("fp16dev") == ["split", "wave", "brick"]
    assert tune.candidates("bf16dev") == ["split", "wave", "brick"]
    assert tune.candidates("fp64") == ["split", "wave"]


def test_cache_key_names_what_changes_the_choice():
    s = _solid()
    k = tune.cache_key(DEV, "fp32", s, (1, 1, 0), 2)
    assert k == tune.cache_key(DEV, "fp32", s.copy(), (1, 1, 0), 2)
    assert "grid=4x5x6" in k and "fluid=119" in k and "sm_103" in k and "open=2" in k and "periodic=110" in k
    t = s.copy()
    t[0, 0, 0] = 1
    others = {tune.cache_key(DEV, "fp16dev", s, (1, 1, 0), 2), tune.cache_key(DEV, "fp32", t, (1, 1, 0), 2),
              tune.cache_key(DEV, "fp32", s, (1, 1, 1), -1), tune.cache_key(("Other", (10, 0)), "fp32", s, (1, 1, 0), 2)}
    assert k not in others and len(others) == 4
    assert '"' not in tune.cache_key(('A"B\\C', (9, 0)), "fp32", s, (1, 1, 1), -1)


def test_fastest_is_chosen_and_cached(tmp_path):
    FakeLattice.made = []
    path = str(tmp_path / "sched.json")
    ms = {"split": 0.9, "wave": 0.95, "push": 1.0, "brick": 1.4}
    r1, r2 = np.ones((6, 5, 4)), np.zeros((6, 5, 4))
    e = tune.choose_schedule(_solid(), (r1, r2), steps=5, warmup=2, cache_path=path, block_cache="b.json",
                             lattice=FakeLattice, timer=_timer(ms), device=DEV, storage="fp32", periodic=(1, 1, 0),
                             open_axis=2)
    assert e["kernel"] == "split" and e["block"] == 128 and e["timings"] == ms and e["ms_per_step"] == 0.9
    assert [lat.kernel for lat in FakeLattice.made] == ["split", "wave", "push", "brick"]
    assert all(lat.closed for lat in FakeLattice.made)
    assert FakeLattice.made[0].cache == "b.json" and FakeLattice.made[0].kw["storage"] == "fp32"
    d = json.load(open(path))
    assert d[e["key"]]["kernel"] == "split"
    # a second call reads the cache and builds nothing
    FakeLattice.made = []
    e2 = tune.choose_schedule(_solid(), (r1, r2), steps=5, warmup=2, cache_path=path, lattice=FakeLattice,
                              timer=None, device=DEV, storage="fp32", periodic=(1, 1, 0), open_axis=2)
    assert e2 == e and FakeLattice.made == []
    # another storage type has its own entry; the brick schedule can win
    ms16 = {"split": 0.9, "wave": 0.95, "brick": 0.5}
    e3 = tune.choose_schedule(_solid(), (r1, r2), steps=5, warmup=2, cache_path=path, lattice=FakeLattice,
                              timer=_timer(ms16), device=DEV, storage="fp16dev", periodic=(1, 1, 0), open_axis=2)
    assert e3["kernel"] == "brick" and e3["block"] is None
    assert len(json.load(open(path))) == 2


def test_restricted_candidates_and_errors(tmp_path):
    r = (np.ones((6, 5, 4)), np.zeros((6, 5, 4)))
    e = tune.choose_schedule(_solid(), r, steps=5, warmup=2, kernels=["wave", "brick"], lattice=FakeLattice,
                             timer=_timer({"wave": 2.0, "brick": 1.0}), device=DEV)
    assert e["kernel"] == "brick" and set(e["timings"]) == {"wave", "brick"}
    with pytest.raises(ValueError):
        tune.choose_schedule(_solid(), r, kernels=["push"], lattice=FakeLattice, device=DEV, storage="fp16dev")
    with pytest.raises(ValueError):
        tune.choose_schedule(_solid(), r, lattice=FakeLattice, device=DEV, kernel="split")
    with pytest.raises(ValueError):
        tune.choose_schedule(_solid(), r, lattice=FakeLattice, device=DEV, storage="fp8")
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert tune.read_cache(str(bad)) == {}
    e = tune.choose_schedule(_solid(), r, steps=5, warmup=2, cache_path=str(bad), kernels=["split"],
                             lattice=FakeLattice, timer=_timer({"split": 1.0}), device=DEV)
    assert json.load(open(bad))[e["key"]]["kernel"] == "split"
