"""The CUDA reverse pass (lbm_record / lbm_adjoint) against the FP64 oracle's
adjoint, finite differences of the CUDA forward, and the autograd wrapper."""
import numpy as np
import pytest

import oracle
from paper_2207_01534_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "these tests need a GPU"
    from paper_2207_01534_gb300 import lbm as m

    m.load()
    return m


def _case(n=16, seed=21, nsteps=40):
    """16^3 porous slab between reservoirs, drainage start, random xi on the
    solids (float32 values, shared exactly by both sides)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = n, n, n
    solid = (rng.random((nz, ny, nx)) < 0.25).astype(np.uint8)
    solid[:3] = 0
    solid[-3:] = 0
    solid = inputs.keep_percolating(solid)
    r1, r2 = inputs.drainage_init(solid, 3)
    xi = np.where(solid == 1, rng.uniform(-0.4, 0.4, solid.shape), 0.0).astype(np.float32)
    kw = dict(tau=(1.3, 0.7), G=3.5, periodic=(1, 1, 0), open_axis=2, rho_in1=1.12, rho_out2=1.0,
              body_force=(0.0, 0.0, 2e-5))
    return solid, r1, r2, xi, kw, (3, nz - 3), nsteps


def _gpu_grad(lbm, storage, case, every, kernel="split", **extra):
    import torch

    solid, r1, r2, xi, kw, sample, nsteps = case
    g = lbm.Lattice(solid, storage=storage, kernel=kernel, sample=sample, **dict(kw, **extra))
    g.set_xi_field(xi)
    g.init_densities(r1, r2)
    g.record(nsteps, every)
    gx = torch.zeros(solid.shape, dtype=torch.float32, device="cuda")
    J, grin = g.adjoint(1.0, gx)
    return g, J, gx.cpu().numpy().astype(np.float64), grin


@pytest.fixture(scope="module")
def oracle_grad():
    case = _case()
    solid, r1, r2, xi, kw, sample, nsteps = case
    o = oracle.Oracle(solid, xi_field=xi.astype(np.float64), **kw)
    o.init_densities(r1, r2)
    o.record(nsteps)
    g = o.adjoint(*sample)
    return case, g, o.saturation(*sample)[1]


# (tolerance on J and dJ/drho_in1, tolerance on dJ/dxi): the xi gradient is
# returned as float32, so FP64 storage is held to float32 output rounding there
# The brick schedule records its forward steps itself (densities through the
# fixed-point accumulators) and the reverse pass recomputes segments with the
# split passes: the gradient is held to the FP32 bounds.
@pytest.mark.parametrize("storage,tol,tol_xi,kernel", [("fp64", 1e-9, 2e-7, "split"), ("fp32", 1e-4, 1e-4, "split"),
                                                       ("fp32", 1e-4, 1e-4, "brick")])
def test_adjoint_matches_oracle_adjoint(lbm, oracle_grad, storage, tol, tol_xi, kernel):
    case, go, Jo = oracle_grad
    _, J, gx, grin = _gpu_grad(lbm, storage, case, every=7, kernel=kernel)  # 40 steps: five full segments and a ragged one
    scale = np.abs(go["xi"]).max()
    err = np.abs(gx - go["xi"]).max() / scale
    print("%s: |J - J_oracle| %.2e  grad_xi rel L-inf %.2e  grad_rho_in %.9e vs %.9e" % (
        storage, abs(J - Jo), err, grin, go["rho_in1"]))
    assert scale > 1e-6
    assert abs(J - Jo) <= 10 * tol
    assert err <= tol_xi
    assert abs(grin - go["rho_in1"]) <= tol * abs(go["rho_in1"])
    assert np.all(gx[case[0] == 0] == 0)


def test_checkpoint_interval_does_not_change_the_gradient(lbm):
    case = _case(nsteps=24)
    ref = None
    for every, extra in ((24, {}), (5, {}), (1, {}), (5, {"reduce_every": 3})):
        _, J, gx, grin = _gpu_grad(lbm, "fp32", case, every, **extra)
        if ref is None:
            ref = (J, gx, grin)
        else:
            assert J == ref[0] and grin == ref[2] and np.array_equal(gx, ref[1]), every


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_recorded_densities_give_the_recomputed_gradient(lbm, storage):
    """The recording steps keep every step's densities when they fit, and the
    reverse pass then recomputes only the collide-stream pass of each state;
    with LBM_RECORD_DENSITIES=0 it recomputes the density and wall passes too.
    Both give the same gradient, bit for bit, for full and ragged segments."""
    import os

    case = _case(nsteps=23)
    out = []
    for flag in (None, "0"):
        old = os.environ.pop("LBM_RECORD_DENSITIES", None)
        if flag is not None:
            os.environ["LBM_RECORD_DENSITIES"] = flag
        try:
            _, J, gx, grin = _gpu_grad(lbm, storage, case, 5)
        finally:
            os.environ.pop("LBM_RECORD_DENSITIES", None)
            if old is not None:
                os.environ["LBM_RECORD_DENSITIES"] = old
        out.append((J, gx, grin))
    assert out[0][0] == out[1][0] and out[0][2] == out[1][2] and np.array_equal(out[0][1], out[1][1])
    assert np.abs(out[0][1]).max() > 0


def test_adjoint_against_finite_differences(lbm):
    """Central differences (eps = 1e-3) of the CUDA forward in FP64 storage
    against the FP32 reverse pass: relative error <= 1e-2."""
    case = _case(n=16, seed=4, nsteps=60)
    solid, r1, r2, xi, kw, sample, nsteps = case
    _, J, gx, grin = _gpu_grad(lbm, "fp32", case, every=20)

    def J_of(x, rin):
        g = lbm.Lattice(solid, storage="fp64", kernel="split", sample=sample, **dict(kw, rho_in1=rin))
        g.set_xi_field(x)
        g.init_densities(r1, r2)
        g.step(nsteps)
        return g.saturation()[1]

    eps = 1e-3
    order = np.argsort(-np.abs(gx).ravel())[:4]
    for v in order:
        xp, xm = xi.copy(), xi.copy()
        xp.ravel()[v] += eps
        xm.ravel()[v] -= eps
        fd = (J_of(xp, kw["rho_in1"]) - J_of(xm, kw["rho_in1"])) / (float(xp.ravel()[v]) - float(xm.ravel()[v]))
        assert abs(fd - gx.ravel()[v]) <= 1e-2 * abs(fd), (v, fd, gx.ravel()[v])
    fd = (J_of(xi, kw["rho_in1"] + eps) - J_of(xi, kw["rho_in1"] - eps)) / (2 * eps)
    assert abs(fd - grin) <= 1e-2 * abs(fd), (fd, grin)


def test_dot_product_along_random_directions(lbm):
    """<dJ/dxi, dxi> + dJ/drho_in1 drho against the change of J along a random
    direction of every wall's xi and the inlet density together (FP64 storage,
    central differences of the CUDA forward).  The perturbed xi fields are
    rounded to float32 as the library stores them, so the directional change
    is taken from the rounded fields themselves."""
    case = _case(n=16, seed=8, nsteps=48)
    solid, r1, r2, xi, kw, sample, nsteps = case
    _, J0, gx, grin = _gpu_grad(lbm, "fp64", case, every=16)

    def J_of(x, rin):
        g = lbm.Lattice(solid, storage="fp64", kernel="split", sample=sample, **dict(kw, rho_in1=rin))
        g.set_xi_field(x)
        g.init_densities(r1, r2)
        g.step(nsteps)
        return g.saturation()[1]

    rng = np.random.default_rng(31)
    for trial in range(2):
        dx = rng.standard_normal(solid.shape) * (solid == 1)
        drho = float(rng.standard_normal())
        eps = 1e-5
        xp = (xi + eps * dx).astype(np.float32)
        xm = (xi - eps * dx).astype(np.float32)
        rp, rm = kw["rho_in1"] + eps * drho, kw["rho_in1"] - eps * drho
        fd = J_of(xp, rp) - J_of(xm, rm)
        ad = float((gx * (xp.astype(np.float64) - xm.astype(np.float64))).sum()) + grin * (rp - rm)
        assert abs(fd - ad) <= 1e-4 * abs(fd), (trial, fd, ad)


def test_reverse_pass_leaves_the_final_state(lbm):
    case = _case(nsteps=12)
    solid, r1, r2, xi, kw, sample, nsteps = case
    g, *_ = _gpu_grad(lbm, "fp32", case, every=5)
    a1, a2 = g.get_populations()
    h = lbm.Lattice(solid, storage="fp32", kernel="split", sample=sample, **kw)
    h.set_xi_field(xi)
    h.init_densities(r1, r2)
    h.step(nsteps)
    b1, b2 = h.get_populations()
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)
    # the recording stays usable, and stepping invalidates it
    J2, _ = g.adjoint(1.0, None)
    g.step(1)
    with pytest.raises(lbm.LbmError):
        g.adjoint(1.0, None)


def test_degenerate_cases(lbm):
    import torch

    # closed periodic droplet: no walls, no open planes
    solid = np.zeros((12, 12, 12), np.uint8)
    r1, r2 = inputs.droplet_densities(solid.shape, (6, 6, 6), 3.0)
    g = lbm.Lattice(solid, tau=(1.0, 1.0), G=3.5)
    g.init_densities(r1, r2)
    g.record(6, 4)
    gx = torch.ones(solid.shape, dtype=torch.float32, device="cuda")
    J, grin = g.adjoint(1.0, gx)
    assert grin == 0.0 and not gx.any().item()
    assert 0.0 < J < 1.0
    # 16-bit storage and batches have no reverse pass
    h = lbm.Lattice(solid, storage="fp16dev")
    h.init_densities(r1, r2)
    with pytest.raises(lbm.LbmError):
        h.record(4, 2)


def test_autograd_function(lbm):
    import torch

    from paper_2207_01534_gb300 import autograd

    case = _case(nsteps=20)
    solid, r1, r2, xi, kw, sample, nsteps = case
    g = lbm.Lattice(solid, storage="fp32", kernel="split", sample=sample, **kw)
    x = torch.tensor(xi, device="cuda", requires_grad=True)
    rin = torch.tensor(kw["rho_in1"], dtype=torch.float64, requires_grad=True)
    J = autograd.saturation(g, (r1, r2), x, rin, nsteps, every=6)
    (3.0 * J).backward()
    _, J2, gx, grin = _gpu_grad(lbm, "fp32", case, every=6)
    assert abs(J.item() - J2) < 1e-12
    assert np.allclose(x.grad.cpu().numpy(), 3.0 * gx, rtol=1e-6, atol=0)
    assert abs(rin.grad.item() - 3.0 * grin) <= 1e-9 * abs(grin)
    # a second forward on the same lattice replaces the recording: the first
    # forward's backward refuses instead of returning the second's gradient
    x1 = torch.tensor(xi, device="cuda", requires_grad=True)
    J1 = autograd.saturation(g, (r1, r2), x1, rin.detach(), nsteps, every=6)
    x2 = torch.tensor(xi * 0.5, device="cuda", requires_grad=True)
    autograd.saturation(g, (r1, r2), x2, rin.detach(), nsteps, every=6)
    with pytest.raises(RuntimeError):
        J1.backward()


@pytest.mark.parametrize("storage,tol_xi", [("fp32", 1e-4), ("fp64", 2e-7)])
def test_adjoint_on_the_crop_of_the_96_pack(lbm, storage, tol_xi):
    """The oracle-adjoint check of the adjoint configuration: the 16^3 crop
    [0, 16)^3 of the 96^3 pack with 2-slice reservoirs, imbibition start,
    60 steps, checkpoints every 25."""
    import torch

    solid = inputs.crop(inputs.adjoint_pack_96()[0], 16, reservoir=2, origin=(0, 0, 0))
    r1, r2 = inputs.imbibition_init(solid, 2)
    rng = np.random.default_rng(16)
    xi = np.where(solid == 1, rng.uniform(-0.4, 0.4, solid.shape), 0.0).astype(np.float32)
    kw = dict(tau=inputs.tau_for_viscosity_ratio(10.0), G=3.5, periodic=(1, 1, 0), open_axis=2, rho_in1=1.02,
              rho_out2=1.0)
    o = oracle.Oracle(solid, xi_field=xi.astype(np.float64), **kw)
    o.init_densities(r1, r2)
    o.record(60)
    go = o.adjoint(2, 14)
    g = lbm.Lattice(solid, storage=storage, kernel="split", sample=(2, 14), **kw)
    g.set_xi_field(xi)
    g.init_densities(r1, r2)
    g.record(60, 25)
    gx = torch.zeros(solid.shape, dtype=torch.float32, device="cuda")
    J, grin = g.adjoint(1.0, gx)
    gx = gx.cpu().numpy().astype(np.float64)
    scale = np.abs(go["xi"]).max()
    err = np.abs(gx - go["xi"]).max() / scale
    print("%s crop: grad_xi rel L-inf %.2e  grad_rho_in %.6e vs %.6e" % (storage, err, grin, go["rho_in1"]))
    assert scale > 1e-8 and err <= tol_xi
    assert abs(grin - go["rho_in1"]) <= 1e-4 * abs(go["rho_in1"]) + 1e-12
