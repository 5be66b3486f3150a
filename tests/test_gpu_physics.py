"""Physics checks run on the CUDA path itself (the oracle runs the same ones in
tests/test_oracle_physics.py): square-duct Poiseuille flow with half-way
bounce-back against the series solution, layered two-component channel flow
against the continuum momentum balance, and both against the oracle."""
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


@pytest.mark.parametrize("storage,tol_oracle", [("fp64", 1e-9), ("fp32", 5e-3)])
def test_layered_channel_flow(lbm, storage, tol_oracle):
    """Two immiscible layers between flat walls driven along x (component 1
    in the middle half, viscosity ratio about 8): the steady profile solves
    d/dz(mu du/dz) = -R g on the lattice's own R(z) and mu(z) = rho1 nu1 +
    rho2 nu2 to 1%, and is the oracle's profile after the same steps."""
    nz, g, tau, steps = 66, 1e-6, (1.0, 0.55), 240000
    solid = np.zeros((nz, 1, 1), np.uint8)
    solid[0] = 1
    solid[-1] = 1
    z = np.arange(nz)
    inner = np.abs(z - (nz - 1) / 2.0) < (nz - 2) / 4.0
    fluid = solid[:, 0, 0] == 0
    r1 = (np.where(inner, 1.0, 0.03) * fluid)[:, None, None]
    r2 = (np.where(inner, 0.03, 1.0) * fluid)[:, None, None]
    kw = dict(tau=tau, G=3.5, periodic=(1, 1, 0), body_force=(g, 0.0, 0.0))
    lat = lbm.Lattice(solid, storage=storage, **kw)
    lat.init_densities(r1, r2)
    lat.step(steps)
    f = lat.fields(("rho1", "rho2", "ux"))
    rho1, rho2, ux = f["rho1"][:, 0, 0], f["rho2"][:, 0, 0], f["ux"][:, 0, 0]
    mu = rho1 * (tau[0] - 0.5) / 3.0 + rho2 * (tau[1] - 0.5) / 3.0
    ref = physics.parallel_flow_profile(rho1 + rho2, mu, g, fluid)
    assert np.abs(ux[fluid] - ref).max() <= 0.01 * ref.max()
    o = oracle.Oracle(solid, **kw)
    o.init_densities(r1, r2)
    o.step(steps)
    uo = o.fields()["ux"][:, 0, 0]
    assert np.abs(ux[fluid] - uo[fluid]).max() <= tol_oracle * np.abs(uo[fluid]).max()
