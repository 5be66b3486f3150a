"""lbm_saturation_static: the reduction for callers that cannot allocate.

Such callers (their device memory is held by another allocator, or they must
avoid the cost and device synchronisation of cudaMalloc / cudaFree) pass their
own device buffers; the entry point's scratch lives in static device memory.
This checks it through the C ABI against lbm_saturation on the same state, on
two calls in a row (the second after more steps, so stale scratch from the
first call would show), and that oversize requests are refused.  The file name
makes pytest collect it after every other test.
"""
import numpy as np
import pytest

from paper_2207_01534_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12
LARGE_N = 16777216  # LBM_SATURATION_STATIC_MAX_N


def _porous_open():
    nz, ny, nx = 30, 16, 14
    rng = np.random.default_rng(11)
    solid = (rng.random((nz, ny, nx)) < 0.3).astype(np.uint8)
    solid[:4] = 0
    solid[-4:] = 0
    return solid


def test_static_scratch_saturation_matches_context_saturation():
    import torch

    assert torch.cuda.is_available(), "this test needs a GPU"
    from paper_2207_01534_gb300 import lbm

    lbm.load()
    solid = _porous_open()
    r1, r2 = inputs.drainage_init(solid, 4)
    lat = lbm.Lattice(solid, tau=(1.7, 0.62), G=3.5, xi=-0.3, periodic=(1, 1, 0), open_axis=2, rho_in1=1.1,
                      rho_out2=1.0, sample=(4, 26))
    lat.init_densities(r1, r2)
    fluid = solid == 0
    zidx = np.broadcast_to(np.arange(solid.shape[0])[:, None, None], solid.shape)
    sample = ((zidx >= 4) & (zidx < 26))[fluid].astype(np.uint8)
    sample_d = torch.from_numpy(sample).cuda()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for steps in (150, 57):  # two calls in a row, on different states
        lat.step(steps)
        ref = lat.saturation()
        f = lat.fields(("rho1", "rho2"))
        a = torch.from_numpy(f["rho1"][fluid].astype(np.float32)).cuda()
        b = torch.from_numpy(f["rho2"][fluid].astype(np.float32)).cuda()
        out.fill_(-1.0)
        lbm.saturation_static(a.data_ptr(), b.data_ptr(), sample_d.data_ptr(), a.numel(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == ref[0]
        for k in (1, 2, 3):
            assert abs(got[k] - ref[k]) <= TOL_FP64 * max(1.0, abs(ref[k])), (k, got[k], ref[k])


def _host_reduction(a, b, sample):
    """The same reductions in FP64 on the host, from the same float32 arrays."""
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    sel = np.ones(a.shape, bool) if sample is None else sample != 0
    cnt = int(sel.sum())
    sw = float(np.count_nonzero(b[sel] > a[sel])) / cnt if cnt else 0.0
    smooth = float(np.sum(a64[sel] / (a64[sel] + b64[sel]))) / cnt if cnt else 0.0
    return np.array([sw, smooth, float(np.sum(a64)), float(np.sum(b64))])


@pytest.mark.parametrize("n,with_sample", [(4096 * 4096 - 1000, True), (LARGE_N, False), (70001, False)])
def test_static_scratch_against_host_fp64_sums(n, with_sample):
    """Large inputs (up to the maximum: every block of the scratch array in
    use, the final sum over more than 256 partials) and a NULL sample mask,
    against FP64 sums of the same float32 arrays on the host, on two calls
    in a row with different data."""
    import torch

    assert torch.cuda.is_available(), "this test needs a GPU"
    from paper_2207_01534_gb300 import lbm

    lbm.load()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (1, 2):
        rng = np.random.default_rng(seed + n)
        a = rng.uniform(0.02, 1.0, n).astype(np.float32)
        b = rng.uniform(0.02, 1.0, n).astype(np.float32)
        sample = (rng.random(n) < 0.7).astype(np.uint8) if with_sample else None
        da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        ds = torch.from_numpy(sample).cuda() if with_sample else None
        out.fill_(-1.0)
        lbm.saturation_static(da.data_ptr(), db.data_ptr(), ds.data_ptr() if with_sample else 0, n, out.data_ptr(),
                              stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = _host_reduction(a, b, sample)
        assert got[0] == ref[0], (got[0], ref[0])
        for k in (1, 2, 3):
            assert abs(got[k] - ref[k]) <= TOL_FP64 * abs(ref[k]), (k, got[k], ref[k])


def test_static_scratch_rejects_oversize_and_bad_arguments():
    import torch

    assert torch.cuda.is_available(), "this test needs a GPU"
    from paper_2207_01534_gb300 import lbm

    lbm.load()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.saturation_static(x.data_ptr(), x.data_ptr(), 0, lbm.SATURATION_STATIC_MAX_N + 1, out.data_ptr())
    assert e.value.code == -1
    with pytest.raises(lbm.LbmError):
        lbm.saturation_static(x.data_ptr(), x.data_ptr(), 0, -1, out.data_ptr())
    # an empty input is valid: zero masses and saturations
    lbm.saturation_static(x.data_ptr(), x.data_ptr(), 0, 0, out.data_ptr())
    torch.cuda.synchronize()
    assert out.cpu().numpy().tolist() == [0.0, 0.0, 0.0, 0.0]
