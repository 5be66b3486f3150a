"""Device memory from the caller's allocator (lbm_set_allocator).

With PyTorch's caching allocator installed (lbm.use_torch_allocator) a
lattice steps bitwise as with cudaMalloc and gives its memory back on
destruction; an allocator that fails at the k-th request makes lbm_create
report LBM_ERR_ALLOC, after releasing every block it had obtained."""
import ctypes

import numpy as np
import pytest

from paper_2207_01534_gb300 import inputs

pytestmark = pytest.mark.gpu

LBM_ERR_ALLOC = -2


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "these tests need a GPU"
    from paper_2207_01534_gb300 import lbm as m

    m.load()
    yield m
    m.use_torch_allocator(False)


def _slab():
    rng = np.random.default_rng(4)
    nz, ny, nx = 20, 12, 10
    solid = (rng.random((nz, ny, nx)) < 0.25).astype(np.uint8)
    solid[:3] = 0
    solid[-3:] = 0
    solid = inputs.keep_percolating(solid)
    r1, r2 = inputs.drainage_init(solid, 3)
    kw = dict(tau=(1.3, 0.7), G=3.5, xi=-0.2, periodic=(1, 1, 0), open_axis=2, rho_in1=1.1, rho_out2=1.0)
    return solid, r1, r2, kw


def test_torch_allocator_gives_the_same_bits_and_releases_its_memory(lbm):
    import torch

    solid, r1, r2, kw = _slab()
    lbm.use_torch_allocator(False)
    ref = lbm.Lattice(solid, **kw)
    ref.init_densities(r1, r2)
    ref.step(25)
    p_ref = ref.get_populations()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    lbm.use_torch_allocator(True)
    try:
        lat = lbm.Lattice(solid, **kw)
        held = torch.cuda.memory_allocated() - before
        assert held >= lat.info()["device_bytes"] > 0
        lat.init_densities(r1, r2)
        lat.step(25)
        p = lat.get_populations()
        assert np.array_equal(p[0], p_ref[0]) and np.array_equal(p[1], p_ref[1])
        lat.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
    finally:
        lbm.use_torch_allocator(False)


def test_failing_allocator_is_reported_and_releases_what_it_got(lbm):
    import torch

    solid, r1, r2, kw = _slab()
    lib = lbm.load()
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
    live = {}
    state = {"left": 0, "calls": 0}

    def _alloc(nbytes, _user):
        state["calls"] += 1
        if state["left"] <= 0:
            return None
        state["left"] -= 1
        ptr = int(torch.cuda.caching_allocator_alloc(int(max(nbytes, 1)), torch.cuda.current_device()))
        live[ptr] = nbytes
        return ptr

    def _free(ptr, _user):
        live.pop(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC(_alloc), FREE(_free)
    try:
        # how many requests a successful creation makes
        state["left"] = 1 << 30
        lib.lbm_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None)
        ok = lbm.Lattice(solid, **kw)
        n_ok = state["calls"]
        assert n_ok >= 3
        ok.close()
        assert not live
        for k in sorted({0, 1, n_ok // 2, n_ok - 1}):
            state["left"], state["calls"] = k, 0
            with pytest.raises(lbm.LbmError) as e:
                lbm.Lattice(solid, **kw)
            assert e.value.code == LBM_ERR_ALLOC, k
            assert not live, (k, len(live))
    finally:
        lib.lbm_set_allocator(None, None, None)
