"""Python binding of liblbm (include/lbm.h): argument marshalling only.

Every step of the method runs in the CUDA library.  PyTorch supplies the CUDA
stream and, optionally, device memory (through its caching allocator).  If the
library cannot be loaded this module raises: there is no CPU fallback.

Arrays are numpy, shape (nz, ny, nx) (x fastest), like the geometry
generators in ``inputs``; populations are (2, 19, nz, ny, nx).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK = 0
STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_ALLOC", -3: "LBM_ERR_CUDA", -4: "LBM_ERR_NONFINITE",
          -5: "LBM_ERR_DRIFT", -6: "LBM_ERR_TIMEOUT", -7: "LBM_ERR_UNSUPPORTED"}
BC = {"neem": 0, "zou_he": 1}
STORAGE = {"fp32": 0, "fp64": 1, "fp16dev": 2, "bf16dev": 3}
KERNEL = {"auto": 0, "split": 1, "fused": 2, "wave": 3, "push": 4, "brick": 5, "flow": 6, "persistent": 7}
FIELDS = ("rho1", "rho2", "ux", "uy", "uz", "P")


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class Geometry(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("solid", ctypes.c_void_p), ("periodic", ctypes.c_int32 * 3), ("open_axis", ctypes.c_int32),
                ("sample_lo", ctypes.c_int32), ("sample_hi", ctypes.c_int32), ("xi_field", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double * 2), ("G", ctypes.c_double), ("xi", ctypes.c_double),
                ("rho_in1", ctypes.c_double), ("rho_out2", ctypes.c_double), ("body_force", ctypes.c_double * 3),
                ("bc", ctypes.c_int32), ("storage", ctypes.c_int32), ("velocity_shift", ctypes.c_int32),
                ("reduce_every", ctypes.c_int32), ("rho_ref", ctypes.c_double * 2), ("kernel", ctypes.c_int32),
                ("drift_limit", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("n_fluid", ctypes.c_int64), ("n_wall", ctypes.c_int64), ("n_voxels", ctypes.c_int64),
                ("step", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("storage", ctypes.c_int32), ("kernel", ctypes.c_int32)]


_lib = None
_ALLOC_CB = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_CB = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_torch_hooks = None


def load(build_if_missing: bool = True):
    """Load liblbm.so (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and (not os.path.exists(path) or _build._stale()):
        _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.lbm_default_params.argtypes = [ctypes.POINTER(Params)]
    lib.lbm_create.argtypes = [ctypes.POINTER(Geometry), ctypes.POINTER(Params), ctypes.POINTER(P)]
    lib.lbm_destroy.argtypes = [P]
    lib.lbm_destroy.restype = None
    lib.lbm_set_allocator.argtypes = [P, P, P]
    lib.lbm_init_densities.argtypes = [P, P, P]
    lib.lbm_set_populations.argtypes = [P, P]
    lib.lbm_get_populations.argtypes = [P, P]
    lib.lbm_step.argtypes = [P, ctypes.c_int64]
    lib.lbm_step_timed.argtypes = [P, ctypes.c_int64, P, ctypes.c_int32]
    lib.lbm_read_fields.argtypes = [P, ctypes.c_uint32, P, ctypes.c_size_t]
    lib.lbm_saturation.argtypes = [P, P]
    lib.lbm_set_inlet.argtypes = [P, ctypes.c_double]
    lib.lbm_set_stream.argtypes = [P, P]
    lib.lbm_synchronize.argtypes = [P]
    lib.lbm_get_info.argtypes = [P, ctypes.POINTER(Info)]
    lib.lbm_saturation_static.argtypes = [P, P, P, ctypes.c_int64, P, P]
    lib.lbm_last_error.argtypes = [P]
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_create_batch.argtypes = [ctypes.c_int32, ctypes.POINTER(Geometry), ctypes.POINTER(Params),
                                     ctypes.POINTER(P)]
    lib.lbm_batch_size.argtypes = [P]
    lib.lbm_batch_size.restype = ctypes.c_int32
    lib.lbm_batch_get.argtypes = [P, ctypes.c_int32, ctypes.POINTER(P)]
    lib.lbm_save.argtypes = [P, ctypes.c_char_p]
    lib.lbm_load.argtypes = [P, ctypes.c_char_p]
    lib.lbm_autotune.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32)]
    lib.lbm_set_xi_field.argtypes = [P, P, ctypes.c_int32]
    lib.lbm_record.argtypes = [P, ctypes.c_int64, ctypes.c_int32]
    lib.lbm_set_wait_limit.argtypes = [P, ctypes.c_double]
    lib.lbm_inject_stall.argtypes = [P]
    lib.lbm_adjoint.argtypes = [P, ctypes.c_double, P, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double)]
    for name in ("lbm_default_params", "lbm_create", "lbm_set_allocator", "lbm_init_densities",
                 "lbm_set_populations", "lbm_get_populations", "lbm_step", "lbm_step_timed", "lbm_read_fields",
                 "lbm_saturation", "lbm_saturation_static", "lbm_set_inlet", "lbm_set_stream", "lbm_synchronize",
                 "lbm_get_info", "lbm_create_batch", "lbm_batch_get", "lbm_autotune", "lbm_set_xi_field",
                 "lbm_record", "lbm_adjoint", "lbm_set_wait_limit", "lbm_inject_stall", "lbm_save", "lbm_load"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def use_torch_allocator(enable: bool = True) -> None:
    """Route later context allocations through PyTorch's caching allocator."""
    global _torch_hooks
    lib = load()
    if not enable:
        lib.lbm_set_allocator(None, None, None)
        _torch_hooks = None
        return
    import torch

    def _alloc(nbytes, _user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device()))
        except Exception:  # reported to the library as an allocation failure
            return None

    def _free(ptr, _user):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_CB(_alloc), _FREE_CB(_free)
    _torch_hooks = (a, f)  # keep the callbacks alive
    lib.lbm_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None)


def _check(code, ctx=None):
    if code != LBM_OK:
        lib = load()
        msg = lib.lbm_last_error(ctx)
        raise LbmError(code, msg.decode() if msg else "")


SATURATION_STATIC_MAX_N = 16777216


def saturation_static(rho1_ptr, rho2_ptr, sample_ptr, n, out_ptr, stream=0):
    """lbm_saturation_static on caller-owned device buffers (integer device
    addresses); enqueues the FP64 reduction on ``stream`` and returns."""
    lib = load()
    code = lib.lbm_saturation_static(ctypes.c_void_p(rho1_ptr), ctypes.c_void_p(rho2_ptr),
                                     ctypes.c_void_p(sample_ptr) if sample_ptr else None, int(n),
                                     ctypes.c_void_p(out_ptr), ctypes.c_void_p(int(stream)) if stream else None)
    if code != LBM_OK:
        raise LbmError(code, "lbm_saturation_static")


def _geometry_params(lib, solid, tau=(1.0, 1.0), G=3.5, xi=0.0, xi_field=None, periodic=(1, 1, 1), open_axis=-1,
                     rho_in1=1.0, rho_out2=1.0, body_force=(0.0, 0.0, 0.0), velocity_shift=1, storage="fp32",
                     kernel="auto", sample=(0, 0), reduce_every=0, drift_limit=1e-6, rho_ref=(0.0, 0.0), bc="neem"):
    """lbm_geometry and lbm_params of one lattice, plus the arrays they point
    to (keep them alive until lbm_create returns)."""
    solid = np.ascontiguousarray(solid, dtype=np.uint8)
    assert solid.ndim == 3
    nz, ny, nx = solid.shape
    g = Geometry()
    g.nx, g.ny, g.nz = nx, ny, nz
    g.solid = solid.ctypes.data
    for a in range(3):
        g.periodic[a] = int(bool(periodic[a]))
    g.open_axis = int(open_axis)
    g.sample_lo, g.sample_hi = int(sample[0]), int(sample[1])
    xf = None
    if xi_field is not None:
        xf = np.ascontiguousarray(xi_field, dtype=np.float32)
        assert xf.shape == solid.shape
        g.xi_field = xf.ctypes.data
    p = Params()
    lib.lbm_default_params(ctypes.byref(p))
    p.tau[0], p.tau[1] = float(tau[0]), float(tau[1])
    p.G = float(G)
    p.xi = float(xi)
    p.rho_in1, p.rho_out2 = float(rho_in1), float(rho_out2)
    for a in range(3):
        p.body_force[a] = float(body_force[a])
    p.velocity_shift = int(velocity_shift)
    p.storage = STORAGE[storage]
    p.kernel = KERNEL[kernel]
    p.reduce_every = int(reduce_every)
    p.drift_limit = float(drift_limit)
    p.rho_ref[0], p.rho_ref[1] = float(rho_ref[0]), float(rho_ref[1])
    p.bc = BC[bc]
    return g, p, (solid, xf)


def _current_stream(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            stream = None
    return stream


class Lattice:
    """One simulation context (``lbm_ctx``) on the current CUDA device."""

    def __init__(self, solid, stream=None, **kw):
        lib = load()
        self._lib = lib
        g, p, keep = _geometry_params(lib, solid, **kw)
        self.shape = keep[0].shape
        self.nv = int(np.prod(self.shape))
        h = ctypes.c_void_p()
        _check(lib.lbm_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(h)))
        self._h = h
        self._owner = None
        stream = _current_stream(stream)
        if stream:
            _check(lib.lbm_set_stream(h, ctypes.c_void_p(int(stream))), h)

    @classmethod
    def _sample(cls, lib, handle, shape, owner):
        """A sample lattice of a batch (owned by the batch)."""
        self = cls.__new__(cls)
        self._lib = lib
        self._h = handle
        self._owner = owner
        self.shape = tuple(shape)
        self.nv = int(np.prod(self.shape))
        return self

    def set_xi_field(self, xi):
        """Wettability xi per voxel (Eq. 15): a numpy array or a CUDA float32 tensor of the grid's shape."""
        if hasattr(xi, "data_ptr"):
            import torch

            assert xi.is_cuda and xi.dtype == torch.float32 and xi.is_contiguous() and tuple(xi.shape) == self.shape
            self._c(self._lib.lbm_set_xi_field(self._h, ctypes.c_void_p(xi.data_ptr()), 1))
        else:
            a = np.ascontiguousarray(np.broadcast_to(xi, self.shape), dtype=np.float32)
            self._c(self._lib.lbm_set_xi_field(self._h, a.ctypes.data, 0))

    def save(self, path: str):
        """lbm_save: the lattice's state (populations, boundary cells, step count) to a file."""
        self._c(self._lib.lbm_save(self._h, str(path).encode()))

    def load(self, path: str):
        """lbm_load: the state saved by ``save`` into a lattice of the same geometry and storage."""
        self._c(self._lib.lbm_load(self._h, str(path).encode()))

    def set_wait_limit(self, seconds: float):
        """lbm_set_wait_limit: time limit of the single-pass schedule's device waits."""
        self._c(self._lib.lbm_set_wait_limit(self._h, float(seconds)))

    def inject_stall(self):
        """lbm_inject_stall: the next single-pass step waits for a round that never completes."""
        self._c(self._lib.lbm_inject_stall(self._h))

    def record(self, nsteps: int, every: int = 50):
        """lbm_record: nsteps steps, keeping a checkpoint every ``every`` steps.
        ``recordings`` counts the calls, so a caller holding an earlier
        recording can tell that it has been replaced."""
        self.recordings = getattr(self, "recordings", 0) + 1
        self._c(self._lib.lbm_record(self._h, int(nsteps), int(every)))

    def adjoint(self, dloss: float = 1.0, grad_xi=None):
        """lbm_adjoint: reverse pass of the recording.  ``grad_xi`` (optional)
        is a CUDA float32 tensor of the grid's shape that receives dloss *
        dJ/dxi.  Returns (J, dloss * dJ/drho_in1)."""
        gr, J = ctypes.c_double(0.0), ctypes.c_double(0.0)
        ptr = None
        if grad_xi is not None:
            assert grad_xi.is_cuda and grad_xi.is_contiguous() and tuple(grad_xi.shape) == self.shape
            ptr = ctypes.c_void_p(grad_xi.data_ptr())
        self._c(self._lib.lbm_adjoint(self._h, float(dloss), ptr, ctypes.byref(gr), ctypes.byref(J)))
        return J.value, gr.value

    def autotune(self, cache_path=None) -> int:
        """lbm_autotune: pick (or read from the JSON cache) the block size of the split schedule."""
        b = ctypes.c_int32(0)
        self._c(self._lib.lbm_autotune(self._h, cache_path.encode() if cache_path else None, ctypes.byref(b)))
        return int(b.value)

    def close(self):
        h = getattr(self, "_h", None)
        if getattr(self, "_owner", None) is not None:  # a sample: the batch destroys it
            self._h = None
            return
        if h is not None and h.value:
            self._lib.lbm_destroy(h)
            self._h = None

    def __del__(self):
        self.close()

    def _c(self, code):
        _check(code, self._h)

    def set_stream(self, stream):
        self._c(self._lib.lbm_set_stream(self._h, ctypes.c_void_p(int(stream))))

    def init_densities(self, rho1, rho2):
        r1 = np.ascontiguousarray(np.broadcast_to(rho1, self.shape), dtype=np.float64)
        r2 = np.ascontiguousarray(np.broadcast_to(rho2, self.shape), dtype=np.float64)
        self._c(self._lib.lbm_init_densities(self._h, r1.ctypes.data, r2.ctypes.data))

    def set_populations(self, f1, f2):
        f = np.ascontiguousarray(np.stack([np.asarray(f1).reshape((19,) + self.shape),
                                           np.asarray(f2).reshape((19,) + self.shape)]), dtype=np.float64)
        self._c(self._lib.lbm_set_populations(self._h, f.ctypes.data))

    def get_populations(self):
        f = np.zeros((2, 19) + self.shape)
        self._c(self._lib.lbm_get_populations(self._h, f.ctypes.data))
        return f[0], f[1]

    def step(self, n: int = 1):
        self._c(self._lib.lbm_step(self._h, int(n)))

    def step_timed(self, n: int = 1):
        """Run n steps; return per-kernel device milliseconds (dens, wall, fused, plane, pipeline)."""
        ms = np.zeros(5)
        self._c(self._lib.lbm_step_timed(self._h, int(n), ms.ctypes.data, 5))
        return ms

    def fields(self, names=FIELDS):
        mask = 0
        for nme in names:
            mask |= 1 << FIELDS.index(nme)
        order = [nme for nme in FIELDS if mask & (1 << FIELDS.index(nme))]
        out = np.zeros((len(order), self.nv))
        self._c(self._lib.lbm_read_fields(self._h, mask, out.ctypes.data, self.nv))
        return {nme: out[k].reshape(self.shape) for k, nme in enumerate(order)}

    def saturation(self):
        """(S_w, smooth S_nw, mass1, mass2)."""
        out = np.zeros(4)
        self._c(self._lib.lbm_saturation(self._h, out.ctypes.data))
        return tuple(float(x) for x in out)

    def set_inlet(self, rho_in1: float):
        self._c(self._lib.lbm_set_inlet(self._h, float(rho_in1)))

    def synchronize(self):
        self._c(self._lib.lbm_synchronize(self._h))

    def info(self) -> dict:
        i = Info()
        self._c(self._lib.lbm_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in Info._fields_}


class Batch:
    """Independent lattices stepped together (``lbm_create_batch``): one
    launch per pass for all samples.  ``samples`` is a list of dicts of
    Lattice keyword arguments, each with its ``solid``."""

    def __init__(self, samples, stream=None):
        lib = load()
        self._lib = lib
        n = len(samples)
        gs, ps, keep = (Geometry * n)(), (Params * n)(), []
        shapes = []
        for k, kw in enumerate(samples):
            kw = dict(kw)
            g, p, kp = _geometry_params(lib, kw.pop("solid"), **kw)
            gs[k], ps[k] = g, p
            keep.append(kp)
            shapes.append(kp[0].shape)
        h = ctypes.c_void_p()
        _check(lib.lbm_create_batch(n, gs, ps, ctypes.byref(h)))
        self._h = h
        stream = _current_stream(stream)
        if stream:
            _check(lib.lbm_set_stream(h, ctypes.c_void_p(int(stream))), h)
        self.samples = []
        for k in range(n):
            sh = ctypes.c_void_p()
            _check(lib.lbm_batch_get(h, k, ctypes.byref(sh)), h)
            self.samples.append(Lattice._sample(lib, sh, shapes[k], self))

    def __len__(self):
        return len(self.samples)

    def __getitem__(self, k):
        return self.samples[k]

    def _c(self, code):
        _check(code, self._h)

    def step(self, n: int = 1):
        self._c(self._lib.lbm_step(self._h, int(n)))

    def synchronize(self):
        self._c(self._lib.lbm_synchronize(self._h))

    def set_stream(self, stream):
        self._c(self._lib.lbm_set_stream(self._h, ctypes.c_void_p(int(stream))))

    def set_wait_limit(self, seconds: float):
        """lbm_set_wait_limit: time limit of the persistent launch's grid barriers."""
        self._c(self._lib.lbm_set_wait_limit(self._h, float(seconds)))

    def inject_stall(self):
        """lbm_inject_stall: one block of the next persistent launch never reaches its first barrier."""
        self._c(self._lib.lbm_inject_stall(self._h))

    def autotune(self, cache_path=None) -> int:
        b = ctypes.c_int32(0)
        self._c(self._lib.lbm_autotune(self._h, cache_path.encode() if cache_path else None, ctypes.byref(b)))
        return int(b.value)

    def info(self) -> dict:
        i = Info()
        self._c(self._lib.lbm_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            for smp in self.samples:
                smp._h = None
            self._lib.lbm_destroy(h)
            self._h = None

    def __del__(self):
        self.close()
