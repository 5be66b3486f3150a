"""Pins of the oracle's Zou-He open planes (Section 2, boundary rule 1 with
the Zou-He method).  They check the conditions that define the method, not
its formulas: after every step the prescribed component at each open-plane
node has exactly the prescribed density and no tangential momentum, the
normal pair (5, 6) obeys non-equilibrium bounce-back, the known populations
are the streamed ones, and the other component's missing populations keep
their initial values."""
import numpy as np
import pytest

import oracle
from paper_2207_01534_gb300 import inputs

E, W, OPP = oracle.lattice()


def _case(seed=5, nz=12, ny=6, nx=7):
    rng = np.random.default_rng(seed)
    solid = (rng.random((nz, ny, nx)) < 0.2).astype(np.uint8)
    solid[:2] = 0
    solid[-2:] = 0
    solid = inputs.keep_percolating(solid)
    r1, r2 = inputs.drainage_init(solid, 2)
    kw = dict(tau=(1.2, 0.7), G=3.5, xi=0.1, periodic=(1, 1, 0), open_axis=2, rho_in1=1.1, rho_out2=0.98)
    return solid, r1, r2, kw


@pytest.mark.parametrize("plane,comp,rho_key", [(0, 0, "rho_in1"), (-1, 1, "rho_out2")])
def test_prescribed_density_and_no_tangential_momentum(plane, comp, rho_key):
    solid, r1, r2, kw = _case()
    o = oracle.Oracle(solid, bc="zou_he", **kw)
    o.init_densities(r1, r2)
    for _ in range(4):
        o.step(3)
        f = o.get_pops()[comp]
        fl = solid[plane] == 0
        rho = f[:, plane].sum(axis=0)[fl]
        jx = np.tensordot(E[:, 0], f[:, plane], axes=1)[fl]
        jy = np.tensordot(E[:, 1], f[:, plane], axes=1)[fl]
        jz = np.tensordot(E[:, 2], f[:, plane], axes=1)[fl]
        assert np.abs(rho - kw[rho_key]).max() < 1e-14
        assert np.abs(jx).max() < 1e-14 and np.abs(jy).max() < 1e-14
        # normal non-equilibrium bounce-back: f5 - f6 = (f5 - f6)_eq = j_z / 3
        d56 = (f[5, plane] - f[6, plane])[fl]
        assert np.abs(d56 - jz / 3.0).max() < 1e-14


def test_known_populations_are_streamed_and_others_frozen():
    """The plane rule touches only the prescribed component of plane nodes:
    after one step, Zou-He and the extrapolation agree on every interior node
    and on the other component at the planes, whose entering populations are
    the initial ones."""
    solid, r1, r2, kw = _case(seed=8)
    a = oracle.Oracle(solid, bc="zou_he", **kw)
    a.init_densities(r1, r2)
    f0 = a.get_pops()
    a.step(1)
    fz = a.get_pops()
    b = oracle.Oracle(solid, bc="neem", **kw)
    b.init_densities(r1, r2)
    b.step(1)
    fn = b.get_pops()
    inlet_in = [i for i in range(19) if E[i, 2] > 0]
    outlet_in = [i for i in range(19) if E[i, 2] < 0]
    fl0 = solid[0] == 0
    # the non-prescribed component is identical (streamed or frozen) under both rules
    assert np.array_equal(fz[1][:, 0][:, fl0], fn[1][:, 0][:, fl0])
    for i in inlet_in:
        assert np.array_equal(fz[1][i, 0][fl0], f0[1][i, 0][fl0])
    fln = solid[-1] == 0
    for i in outlet_in:
        assert np.array_equal(fz[0][i, -1][fln], f0[0][i, -1][fln])
    # interior nodes do not depend on the plane rule after one step
    assert np.array_equal(fz[0][:, 1:-1], fn[0][:, 1:-1]) and np.array_equal(fz[1][:, 1:-1], fn[1][:, 1:-1])


def test_uniform_rest_state_is_steady():
    """Equal densities everywhere at rest, prescribed densities equal to the
    initial ones, no solid and G = 0: nothing may move."""
    solid = np.zeros((8, 4, 4), np.uint8)
    r1 = np.full(solid.shape, 0.7)
    r2 = np.full(solid.shape, 0.4)
    o = oracle.Oracle(solid, tau=(0.9, 1.3), G=0.0, periodic=(1, 1, 0), open_axis=2, rho_in1=0.7, rho_out2=0.4,
                      bc="zou_he")
    o.init_densities(r1, r2)
    f0 = o.get_pops()
    o.step(20)
    f = o.get_pops()
    assert np.abs(f[0] - f0[0]).max() < 1e-14 and np.abs(f[1] - f0[1]).max() < 1e-14


def test_pressure_difference_drives_flow_towards_the_outlet():
    """G = 0, component 2 absent: component 1 alone in a straight periodic
    channel flows from the denser inlet towards the outlet side, and the
    steady mass flux is the same through every cross-section."""
    nz = 24
    solid = np.zeros((nz, 3, 3), np.uint8)
    r1 = np.linspace(1.02, 1.0, nz)[:, None, None] * np.ones(solid.shape)
    r2 = np.full(solid.shape, 1e-6)
    o = oracle.Oracle(solid, tau=(1.0, 1.0), G=0.0, periodic=(1, 1, 0), open_axis=2, rho_in1=1.02,
                      rho_out2=1e-6, bc="zou_he")
    o.init_densities(r1, r2)
    o.step(3000)
    f = o.get_pops()[0]
    jz = np.tensordot(E[:, 2], f, axes=1).mean(axis=(1, 2))
    assert (jz[1:-1] > 0).all()
    assert np.abs(jz[2:-2] - jz[2:-2].mean()).max() < 0.02 * jz[2:-2].mean()


def test_adjoint_refuses_zou_he():
    solid, r1, r2, kw = _case()
    o = oracle.Oracle(solid, bc="zou_he", **kw)
    o.init_densities(r1, r2)
    o.record(2)
    with pytest.raises(NotImplementedError):
        o.adjoint()
