"""Physics checks run on the CUDA path itself (the oracle runs the same ones in
tests/test_oracle_physics.py): square-duct Poiseuille flow with half-way
bounce-back against the series solution, and against the oracle's profile."""
import math

import numpy as np
import pytest

import oracle
import physics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "these tests need a GPU"
    from paper_2207_01534_gb300 import lbm as m

    m.load()
    return m


@pytest.mark.parametrize("storage,tol_oracle", [("fp64", 1e-10), ("fp32", 1e-3)])
def test_square_duct_poiseuille(lbm, storage, tol_oracle):
    """Single component (rho2 = 0, so no interaction force) driven by a body
    acceleration along z in a square duct whose walls are solid voxels: the
    fully developed axial velocity is the classical series solution with the
    walls half a voxel outside the outermost fluid nodes (tau = 1/2 +
    sqrt(3/16) puts the half-way bounce-back wall exactly there), within 1%,
    and the oracle's profile after the same steps."""
    m = 16
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    nu = (tau - 0.5) / 3.0
    g = 1e-6
    solid = np.ones((1, m + 2, m + 2), np.uint8)
    solid[:, 1:-1, 1:-1] = 0
    kw = dict(tau=(tau, tau), G=3.5, periodic=(0, 0, 1), body_force=(0.0, 0.0, g))
    lat = lbm.Lattice(solid, storage=storage, **kw)
    r1 = 1.0 * (solid == 0)
    lat.init_densities(r1, 0.0)
    lat.step(3000)
    uz = lat.fields(("uz",))["uz"][0, 1:-1, 1:-1]
    ref = physics.duct_series_velocity(m, m, g, nu)
    assert np.abs(uz - ref).max() / ref.max() < 0.01
    o = oracle.Oracle(solid, **kw)
    o.init_densities(r1, 0.0)
    o.step(3000)
    uo = o.fields()["uz"][0, 1:-1, 1:-1]
    assert np.abs(uz - uo).max() / uo.max() <= tol_oracle
