"""Host logic of the experiment drivers and geometry helpers (no GPU)."""
import math

import numpy as np
import pytest

from paper_2207_01534_gb300 import drivers, inputs


@pytest.mark.parametrize("pc", [0.0, 0.01, 0.035])
def test_inlet_density_gives_the_capillary_pressure(pc):
    rin = drivers.inlet_density(pc, G=3.5, minor=0.03, rho_out2=1.0)
    p_in = drivers.pressure(rin, 0.03, 3.5)
    p_out = drivers.pressure(0.03, 1.0, 3.5)
    assert abs((p_in - p_out) - pc) < 1e-15


@pytest.mark.parametrize("theta_water", [60.0, 90.0, 115.0])
def test_cap_angle_of_an_exact_circle(theta_water):
    """A sharp-interface cap cut from a circle whose angle with the wall plane
    is known: the chord-and-height construction recovers it."""
    nx, nz, wall = 160, 60, 0.5
    R = 24.0
    th1 = math.radians(180.0 - theta_water)  # angle inside the cap
    zc = wall - R * math.cos(th1)           # centre height
    z = np.arange(nz)[:, None]
    x = np.arange(nx)[None, :]
    d = np.sqrt((x - nx / 2) ** 2 + (z - zc) ** 2)
    phi = np.where(z > wall, R - d, -1.0)       # > 0 inside the cap, linear across the interface
    rho1 = (1 + np.tanh(phi)) / 2
    rho2 = 1 - rho1
    got = drivers.cap_angle(rho1[:, None, :], rho2[:, None, :], wall_z=wall, base_height=5.0)
    assert abs(got - theta_water) < 1.5


def test_lateral_walls():
    s = np.zeros((5, 4, 6), np.uint8)
    w = inputs.add_lateral_walls(s)
    assert w[:, :, 0].all() and w[:, :, -1].all() and w[:, 0, :].all() and w[:, -1, :].all()
    assert not w[:, 1:-1, 1:-1].any()
    wx = inputs.add_lateral_walls(s, axes=(0,))
    assert wx[:, :, 0].all() and not wx[:, 1:-1, 1:-1].any() and not wx[:, 0, 1:-1].any()


def test_trapped_volume_counts_only_cut_off_water():
    nz, ny, nx = 12, 6, 6
    solid = np.zeros((nz, ny, nx), np.uint8)
    rho1 = np.full(solid.shape, 1.0)  # oil everywhere
    rho2 = np.full(solid.shape, 0.03)
    rho2[-3:] = 1.0  # water in the outlet reservoir: connected, not trapped
    rho1[-3:] = 0.03
    rho2[2:4, 1:3, 1:3] = 1.0  # a cut-off water blob of 8 voxels
    rho1[2:4, 1:3, 1:3] = 0.03
    rho2[6, 4, 4] = 1.0  # a single voxel with no water among its 18 neighbours
    rho1[6, 4, 4] = 0.03
    assert drivers.trapped_volume(rho1, rho2, solid, 3) == 9
    # a water path to the reservoir makes the blob connected
    rho2[4:9, 2, 2] = 1.0
    rho1[4:9, 2, 2] = 0.03
    assert drivers.trapped_volume(rho1, rho2, solid, 3) == 1
    # solid voxels never count
    solid[2:4, 1:3, 1:3] = 1
    assert drivers.trapped_volume(rho1, rho2, solid, 3) == 1


class _StandInLattice:
    """A stand-in with the Lattice calls the drivers use: S_w falls by a fixed
    amount per step until it reaches a floor; the fields are uniform."""

    def __init__(self, solid):
        self.solid = solid
        self.steps = 0
        self.rin = None

    def step(self, n):
        self.steps += n

    def set_inlet(self, rin):
        self.rin = rin

    def saturation(self):
        sw = max(0.3, 1.0 - 1e-4 * self.steps)
        return (sw, 1.0 - sw, 100.0, 200.0)

    def fields(self, names):
        shape = self.solid.shape
        return {"rho1": np.full(shape, 0.03), "rho2": np.full(shape, 1.0)}

    def info(self):
        return {"step": self.steps, "launches": 3 * self.steps}


def test_drivers_write_json_lines(tmp_path):
    import json

    solid = np.zeros((10, 4, 4), np.uint8)
    lat = _StandInLattice(solid)
    log = tmp_path / "hist.jsonl"
    hist = drivers.drainage_history(lat, solid, 1200, every=500, outlet_slices=2, log=log)
    assert [h["step"] for h in hist] == [500, 1000, 1200]
    recs = [json.loads(line) for line in log.read_text().splitlines()]
    assert recs[0]["run"]["driver"] == "drainage_history"
    assert [r["step"] for r in recs[1:]] == [500, 1000, 1200]
    assert [r["lattice_step"] for r in recs[1:]] == [500, 1000, 1200]
    assert recs[-1]["S_w"] == hist[-1]["S_w"] and recs[-1]["mass2"] == 200.0
    log2 = tmp_path / "pc.jsonl"
    out = drivers.pc_sw_curve(lat, [0.0, 0.01], max_steps=3000, check_every=500, tol=0.06, log=log2)
    recs = [json.loads(line) for line in log2.read_text().splitlines()]
    assert len(recs) == 3 and [r["pc"] for r in recs[1:]] == [0.0, 0.01]
    assert recs[1]["settled"] == out[0]["settled"]
    # no path: nothing written, same results
    assert drivers.drainage_history(_StandInLattice(solid), solid, 1200, every=500, outlet_slices=2) == hist
