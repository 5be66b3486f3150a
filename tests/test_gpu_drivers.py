"""Experiment drivers on the GPU path: the flat-wall contact-angle
calibration (Section 3.2) against the paper's printed cubic, and the
capillary-pressure ramp (Sections 4.1-4.2)."""
import numpy as np
import pytest

from conftest import golden
from paper_2207_01534_gb300 import drivers, inputs

pytestmark = pytest.mark.gpu

REF = golden("physics_section3.txt")


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "these tests need a GPU"
    from paper_2207_01534_gb300 import lbm as m

    m.load()
    return m


@pytest.mark.parametrize("xi", [-0.2, 0.2])
def test_contact_angle_driver_matches_the_printed_calibration(lbm, xi):
    c3, c2, c1, c0 = REF["theta_cubic"][0]
    theta_fit = ((c3 * xi + c2) * xi + c1) * xi + c0
    theta = drivers.contact_angle(lbm, xi, tau=tuple(REF["tau_M25"][0]), steps=4000)
    print("xi %+.2f: theta %.2f (cubic %.2f)" % (xi, theta, theta_fit))
    assert abs(theta - theta_fit) < 4.0


def test_contact_angle_driver_neutral(lbm):
    theta = drivers.contact_angle(lbm, 0.0, tau=(1.0, 1.0), steps=3000)
    assert abs(theta - 90.0) < 1.5


@pytest.mark.parametrize("bc", ["neem", "zou_he"])
def test_pc_sw_ramp(lbm, bc):
    """Primary drainage of a water-wet slab: S_w starts near 1 (only the
    widest inlet pores admit oil at P_c = 0), never grows as the inlet
    pressure is raised, and drops well below its start."""
    rng = np.random.default_rng(3)
    nz, ny, nx = 40, 16, 16
    solid = np.zeros((nz, ny, nx), np.uint8)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for _ in range(14):
        c = rng.uniform(0, 1, 3) * np.array([nx, ny, nz - 12]) + np.array([0, 0, 6])
        r = rng.uniform(3.0, 4.5)
        dx = np.minimum(np.abs(xx - c[0]), nx - np.abs(xx - c[0]))
        dy = np.minimum(np.abs(yy - c[1]), ny - np.abs(yy - c[1]))
        solid[dx ** 2 + dy ** 2 + (zz - c[2]) ** 2 <= r * r] = 1
    solid[:4] = 0
    solid[-4:] = 0
    solid = inputs.keep_percolating(solid)
    r1, r2 = inputs.drainage_init(solid, 4)
    g = lbm.Lattice(solid, tau=inputs.tau_for_viscosity_ratio(5.0), G=3.5, xi=-0.2, periodic=(1, 1, 0), open_axis=2,
                    rho_in1=drivers.inlet_density(0.0), rho_out2=1.0, sample=(4, nz - 4), bc=bc)
    g.init_densities(r1, r2)
    curve = drivers.pc_sw_curve(g, [0.0, 0.01, 0.02, 0.04, 0.06], max_steps=4000, check_every=500, tol=2e-3)
    sw = [c["S_w"] for c in curve]
    print(bc, [(c["pc"], round(c["S_w"], 4), c["steps"]) for c in curve])
    assert sw[0] > 0.9
    assert all(b <= a + 0.01 for a, b in zip(sw, sw[1:]))
    assert sw[-1] < sw[0] - 0.1
