"""The seeded input generators (the recipes of the workloads): determinism,
shapes, porosity, reservoir slices, percolation of the pore space (checked
by an independent breadth-first search), initial states, and the parameter
table of the batched sweep."""
from collections import deque

import numpy as np
import pytest

from paper_2207_01534_gb300 import inputs

# the 18 D3Q19 link directions
E18 = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
       if 0 < abs(dx) + abs(dy) + abs(dz) < 3]


def _reach(fluid, start_z):
    """Fluid voxels connected to the fluid of slice start_z by D3Q19 links,
    periodic in x and y, not in z (plain BFS)."""
    nz, ny, nx = fluid.shape
    seen = np.zeros_like(fluid)
    q = deque()
    for y in range(ny):
        for x in range(nx):
            if fluid[start_z, y, x]:
                seen[start_z, y, x] = True
                q.append((start_z, y, x))
    while q:
        z, y, x = q.popleft()
        for dx, dy, dz in E18:
            zz = z + dz
            if zz < 0 or zz >= nz:
                continue
            yy, xx = (y + dy) % ny, (x + dx) % nx
            if fluid[zz, yy, xx] and not seen[zz, yy, xx]:
                seen[zz, yy, xx] = True
                q.append((zz, yy, xx))
    return seen


def _check_percolating(solid):
    fluid = solid == 0
    both = _reach(fluid, 0) & _reach(fluid, solid.shape[0] - 1)
    assert np.array_equal(both, fluid)  # every pore reaches both ends, and nothing else is fluid


def test_sphere_pack_small():
    s = inputs.sphere_pack(32, 4.0, 0.40, inputs.SEED_BASE + 900, reservoir=4)
    assert s.shape == (32, 32, 32) and s.dtype == np.uint8
    assert np.array_equal(s, inputs.sphere_pack(32, 4.0, 0.40, inputs.SEED_BASE + 900, reservoir=4))
    assert not s[:4].any() and not s[-4:].any()
    assert 0.30 <= inputs.porosity(s, 4) <= 0.41
    _check_percolating(s)
    t = inputs.sphere_pack(32, 4.0, 0.40, inputs.SEED_BASE + 901, reservoir=4)
    assert not np.array_equal(s, t)


def test_grf_rock_small():
    s = inputs.grf_rock(32, 3.0, 0.30, inputs.SEED_BASE + 902, reservoir=4)
    assert s.shape == (32, 32, 32)
    assert np.array_equal(s, inputs.grf_rock(32, 3.0, 0.30, inputs.SEED_BASE + 902, reservoir=4))
    assert not s[:4].any() and not s[-4:].any()
    assert 0.20 <= inputs.porosity(s, 4) <= 0.31  # the quantile threshold, less the isolated pores removed
    _check_percolating(s)


def test_keep_percolating_removes_isolated_pores():
    s = np.ones((10, 6, 6), np.uint8)
    s[:, 2, 2] = 0          # a straight channel from end to end
    s[4:6, 4, 4] = 0        # a cavity that reaches neither end
    s[0:3, 0, 4] = 0        # a dead end open at z = 0 only
    k = inputs.keep_percolating(s)
    expect = np.zeros(s.shape, bool)
    expect[:, 2, 2] = True  # only the channel stays fluid
    assert np.array_equal(k == 0, expect)


@pytest.fixture(scope="module")
def named():
    return {"pack128": inputs.drainage_pack_128(), "pack96": inputs.adjoint_pack_96(),
            "rock256": inputs.rock_grf_256()}


@pytest.mark.parametrize("name,n,phi", [("pack128", 128, 0.38), ("pack96", 96, 0.40), ("rock256", 256, 0.22)])
def test_named_workloads(named, name, n, phi):
    solid, r1, r2 = named[name]
    assert solid.shape == (n, n, n)
    assert not solid[:8].any() and not solid[-8:].any()
    assert abs(inputs.porosity(solid, 8) - phi) <= 0.01
    fl = solid == 0
    assert np.all(r1[~fl] == 0) and np.all(r2[~fl] == 0)
    if name == "pack96":  # imbibition start: water (2) in the outlet reservoir, oil (1) elsewhere
        assert np.all(r2[-8:][fl[-8:]] == 1.0) and np.all(r1[:-8][fl[:-8]] == 1.0)
    else:  # drainage start: oil (1) in the inlet reservoir, water (2) elsewhere
        assert np.all(r1[:8][fl[:8]] == 1.0) and np.all(r2[8:][fl[8:]] == 1.0)
    assert set(np.unique(r1[fl])) == {0.03, 1.0}


def test_crop_of_the_rock(named):
    c = inputs.crop(named["rock256"][0], 64, reservoir=4)
    assert c.shape == (64, 64, 64) and not c[:4].any() and not c[-4:].any()
    assert 0.1 <= inputs.porosity(c, 4) <= 0.3


def test_batched_sweep_table():
    t = inputs.batched_sweep()
    assert t == inputs.batched_sweep() and len(t) == 64
    combos = {}
    for k, spec in enumerate(t):
        assert 48 <= spec["n"] <= 112
        assert 4.0 <= spec["radius"] <= min(8.0, spec["n"] / 6.0)
        assert 0.35 <= spec["porosity"] <= 0.45 and spec["reservoir"] == 6
        combos[(spec["M"], spec["theta_deg"])] = combos.get((spec["M"], spec["theta_deg"]), 0) + 1
    assert len(combos) == 16 and set(combos.values()) == {4}
    assert {m for m, _ in combos} == {1.0, 5.0, 10.0, 50.0} and {th for _, th in combos} == {30.0, 60.0, 90.0, 120.0}
    assert len({spec["seed"] for spec in t}) == 64
    small = inputs.batched_sweep(count=8, edge_lo=24, edge_hi=40)
    assert all(24 <= s["n"] <= 40 and s["radius"] <= s["n"] / 6.0 for s in small)


def test_laplace_droplet():
    solid, r1, r2 = inputs.laplace_48()
    assert solid.shape == (48, 48, 48) and not solid.any()
    assert r1[24, 24, 24] > 0.99 and r2[24, 24, 24] < 0.04 and r1[0, 0, 0] < 0.04 and r2[0, 0, 0] > 0.99
    # radius 10: the rho1 = rho2 level crosses the x axis through the centre about 10 voxels out
    prof = (r1 - r2)[24, 24, 24:]
    k = int(np.argmax(prof < 0))
    assert 9 <= k <= 11
