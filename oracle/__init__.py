"""FP64 CPU oracle of the two-component pseudopotential D3Q19 LBM step.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its binding) never imports, links or calls it.

A thin ctypes wrapper over ``oracle_lbm.c``: arrays are dense numpy arrays in
(z, y, x) order, i.e. x fastest, matching the C layout ``v = x + nx*(y + ny*z)``.
Populations are (19, nz, ny, nx) per component.
"""
import ctypes
import os

import numpy as np

from . import build as _build

Q = 19
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.ora_create.restype = ctypes.c_void_p
    lib.ora_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ip, ctypes.c_int,
                               ctypes.c_void_p, ctypes.c_double, dp, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, dp, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
    lib.ora_destroy.argtypes = [ctypes.c_void_p]
    lib.ora_init_densities.argtypes = [ctypes.c_void_p, dp, dp]
    lib.ora_set_pops.argtypes = [ctypes.c_void_p, dp, dp]
    lib.ora_get_pops.argtypes = [ctypes.c_void_p, dp, dp]
    lib.ora_set_inlet.argtypes = [ctypes.c_void_p, ctypes.c_double]
    lib.ora_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
    lib.ora_step_count.argtypes = [ctypes.c_void_p]
    lib.ora_step_count.restype = ctypes.c_long
    lib.ora_fields.argtypes = [ctypes.c_void_p] + [dp] * 6
    lib.ora_saturation.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, dp]
    lib.ora_set_bc.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.ora_record.argtypes = [ctypes.c_void_p, ctypes.c_long]
    lib.ora_adjoint.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp]
    lib.ora_lattice.argtypes = [ip, dp, ip]
    lib.ora_mirror_map.argtypes = [ctypes.c_int, ip]
    lib.ora_feq.argtypes = [ctypes.c_double, dp, dp]
    lib.ora_source.argtypes = [dp, dp, dp]
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def set_threads(n: int) -> None:
    """Set the OpenMP thread count used by later oracle calls (this process)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(int(n))
    except OSError:
        pass


def lattice():
    """D3Q19 velocities (19, 3), weights (19,) and opposite-direction table (19,)."""
    lib = _load()
    e = np.zeros(Q * 3, dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    opp = np.zeros(Q, dtype=np.int32)
    lib.ora_lattice(_ip(e), _dp(w), _ip(opp))
    return e.reshape(Q, 3), w, opp


def mirror_map(axis: int):
    lib = _load()
    m = np.zeros(Q, dtype=np.int32)
    lib.ora_mirror_map(int(axis), _ip(m))
    return m


def feq(rho: float, u):
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(Q)
    lib.ora_feq(float(rho), _dp(uu), _dp(out))
    return out


def source(u, F):
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64)
    ff = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(Q)
    lib.ora_source(_dp(uu), _dp(ff), _dp(out))
    return out


class Oracle:
    """One FP64 simulation on a dense nx*ny*nz grid.

    solid: uint8 array of shape (nz, ny, nx), 1 = solid.
    """

    def __init__(self, solid, tau=(1.0, 1.0), G=3.5, xi=0.0, xi_field=None, periodic=(1, 1, 1),
                 open_axis=-1, rho_in1=1.0, rho_out2=1.0, body_force=(0.0, 0.0, 0.0), velocity_shift=1, bc="neem"):
        lib = _load()
        self._lib = lib
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        assert solid.ndim == 3
        self.shape = solid.shape  # (nz, ny, nx)
        nz, ny, nx = solid.shape
        self.solid = solid
        per = np.ascontiguousarray(periodic, dtype=np.int32)
        taus = np.ascontiguousarray(tau, dtype=np.float64)
        g = np.ascontiguousarray(body_force, dtype=np.float64)
        xf = None
        if xi_field is not None:
            xf = np.ascontiguousarray(xi_field, dtype=np.float64)
            assert xf.shape == solid.shape
        err = ctypes.create_string_buffer(256)
        h = lib.ora_create(nx, ny, nz, solid.ctypes.data, _ip(per), int(open_axis),
                           xf.ctypes.data if xf is not None else None, float(xi), _dp(taus), float(G),
                           float(rho_in1), float(rho_out2), _dp(g), int(velocity_shift), err, 256)
        if not h:
            raise ValueError(err.value.decode())
        self._h = h
        self._keep = (xf,)
        assert bc in ("neem", "zou_he")
        lib.ora_set_bc(h, 1 if bc == "zou_he" else 0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.ora_destroy(h)
            self._h = None

    def init_densities(self, rho1, rho2):
        r1 = np.ascontiguousarray(np.broadcast_to(rho1, self.shape), dtype=np.float64)
        r2 = np.ascontiguousarray(np.broadcast_to(rho2, self.shape), dtype=np.float64)
        self._lib.ora_init_densities(self._h, _dp(r1), _dp(r2))

    def set_pops(self, f1, f2):
        a = np.ascontiguousarray(f1, dtype=np.float64).reshape((Q,) + self.shape)
        b = np.ascontiguousarray(f2, dtype=np.float64).reshape((Q,) + self.shape)
        self._lib.ora_set_pops(self._h, _dp(a), _dp(b))

    def get_pops(self):
        a = np.zeros((Q,) + self.shape)
        b = np.zeros((Q,) + self.shape)
        self._lib.ora_get_pops(self._h, _dp(a), _dp(b))
        return a, b

    def set_inlet(self, rho_in1: float):
        self._lib.ora_set_inlet(self._h, float(rho_in1))

    def step(self, n: int = 1):
        self._lib.ora_step(self._h, int(n))

    @property
    def step_count(self) -> int:
        return int(self._lib.ora_step_count(self._h))

    def fields(self):
        """dict of rho1, rho2, ux, uy, uz, P as (nz, ny, nx) arrays."""
        names = ("rho1", "rho2", "ux", "uy", "uz", "P")
        arrs = [np.zeros(self.shape) for _ in names]
        self._lib.ora_fields(self._h, *[_dp(a) for a in arrs])
        return dict(zip(names, arrs))

    def saturation(self, lo: int = 0, hi: int = 0):
        """(S_w, smooth S_nw, mass1, mass2); sample slab [lo, hi) along the open axis."""
        out = np.zeros(4)
        self._lib.ora_saturation(self._h, int(lo), int(hi), _dp(out))
        return tuple(float(x) for x in out)

    def record(self, n: int) -> None:
        """Take n steps keeping every state for ``adjoint`` (tiny grids only)."""
        if self._lib.ora_record(self._h, int(n)) != 0:
            raise MemoryError("oracle tape")

    def adjoint(self, lo: int = 0, hi: int = 0, seed=None, want_state: bool = False):
        """Reverse pass over the recorded steps.  J is the smooth non-wetting
        saturation of the sample slab [lo, hi) (or <seed, f_n> for a seed of
        shape (2, 19, nz, ny, nx)).  Returns dJ/dxi (nz, ny, nx), dJ/drho_in1
        and, with want_state, dJ/df_0 and dJ/d(frozen populations)."""
        gxi = np.zeros(self.shape)
        grin = np.zeros(1)
        sd = None
        if seed is not None:
            sd = np.ascontiguousarray(seed, dtype=np.float64).reshape(-1)
            assert sd.size == 2 * 19 * int(np.prod(self.shape))
        gf = np.zeros((2, 19) + self.shape) if want_state else None
        gz = np.zeros((2, 19) + self.shape) if want_state else None
        rc = self._lib.ora_adjoint(self._h, int(lo), int(hi), _dp(sd) if sd is not None else None, _dp(gxi),
                                   _dp(grin), _dp(gf) if gf is not None else None,
                                   _dp(gz) if gz is not None else None)
        if rc == -2:
            raise NotImplementedError("the oracle adjoint covers the extrapolation boundary only")
        if rc != 0:
            raise RuntimeError("record() first")
        out = {"xi": gxi, "rho_in1": float(grin[0])}
        if want_state:
            out["f"] = gf
            out["frozen"] = gz
        return out
