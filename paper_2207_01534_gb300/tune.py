"""Schedule chooser: times the kernel schedules on the caller's own lattice and
keeps the fastest, cached in a JSON file (host logic only; every timed step
runs in liblbm's CUDA kernels).

The candidates differ in kernel structure and in memory layout:

* ``split``: density, wall and collide-stream passes, fluid nodes in voxel
  order; its threads per block are tuned by ``lbm_autotune``;
* ``wave``: the same passes per z slab as a dependency graph (same layout);
* ``push``: the collide-stream pass accumulates the next densities in fixed
  point (FP32 storage only);
* ``brick``: one block per 8^3 brick with the density halo, walls and next
  densities in shared memory; the fluid nodes are numbered brick by brick (a
  different layout), so it needs its own context.

Each candidate gets a fresh lattice with the caller's parameters and initial
densities, ``warmup`` untimed steps (enough for its CUDA graphs to be captured
and replayed once), then ``steps`` steps timed with CUDA events on the
lattice's stream.  The split and wave schedules replay 32-step graphs (then
2-step ones), push and brick 30-step graphs (then 6-step ones): the default 96
timed steps are long-graph replays plus at most one short one.  The cache is a flat JSON object mapping a
key (GPU name, compute capability, storage, grid shape, periodic axes, open
axis, fluid count and a hash of the solid mask) to the chosen entry; a cached
key is returned without creating or timing anything.
"""
from __future__ import annotations

import hashlib
import json
import os

STORAGES = ("fp32", "fp64", "fp16dev", "bf16dev")


def candidates(storage: str):
    """Schedules available for a storage type."""
    out = ["split", "wave"]
    if storage == "fp32":
        out.append("push")
    if storage != "fp64":
        out.append("brick")
    return out


def cache_key(device, storage, solid, periodic, open_axis) -> str:
    """``device`` = (name, (major, minor)); ``solid`` the uint8 mask."""
    import numpy as np

    name, (major, minor) = device
    name = "".join(ch if (ch.isprintable() and ch not in '"\\') else "_" for ch in name)
    m = np.ascontiguousarray(solid, dtype=np.uint8)
    shape = m.shape
    digest = hashlib.sha1(m.tobytes()).hexdigest()[:12]
    return "%s|sm_%d%d|%s|grid=%dx%dx%d|periodic=%d%d%d|open=%d|fluid=%d|mask=%s" % (
        name, major, minor, storage, shape[2], shape[1], shape[0], int(periodic[0]), int(periodic[1]),
        int(periodic[2]), int(open_axis), int((m == 0).sum()), digest)


def read_cache(path):
    if not path or not os.path.exists(path):
        return {}
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return {}
    return d if isinstance(d, dict) else {}


def write_cache(path, d):
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _device():
    import torch

    i = torch.cuda.current_device()
    return torch.cuda.get_device_name(i), tuple(torch.cuda.get_device_capability(i))


def _event_timer(lat, steps, warmup):
    """Milliseconds per step: CUDA events around lat.step(steps) on the
    current stream, after warmup steps."""
    import torch

    lat.step(warmup)
    lat.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    lat.step(steps)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def choose_schedule(solid, rho, steps=96, warmup=40, cache_path=None, block_cache=None, kernels=None, lattice=None,
                    timer=None, device=None, **kw):
    """Time the candidate schedules on this lattice and return the fastest as
    {"kernel", "block", "ms_per_step", "timings": {kernel: ms}, "key"}.

    ``rho`` = (rho1, rho2) initial densities; ``kw`` are the Lattice
    parameters (storage, tau, G, xi, periodic, open_axis, ...; not kernel).
    ``kernels`` restricts the candidates.  ``block_cache`` is handed to
    ``Lattice.autotune`` for the split and wave candidates, so a lattice
    created with the chosen kernel gets the tuned block by calling
    ``autotune(block_cache)``.  ``lattice`` (a Lattice factory), ``timer``
    (lat, steps, warmup -> ms per step) and ``device`` ((name, (major,
    minor))) default to the CUDA library, CUDA events and the current
    device."""
    import numpy as np

    if "kernel" in kw:
        raise ValueError("the kernel is what choose_schedule chooses")
    storage = kw.get("storage", "fp32")
    if storage not in STORAGES:
        raise ValueError("unknown storage %r" % (storage,))
    if lattice is None:
        from . import lbm

        lattice = lbm.Lattice
    timer = timer or _event_timer
    device = device or _device()
    solid = np.asarray(solid)
    cands = list(kernels) if kernels else candidates(storage)
    bad = [k for k in cands if k not in candidates(storage)]
    if bad:
        raise ValueError("schedules %s are not available with %s storage" % (bad, storage))
    key = cache_key(device, storage, solid, kw.get("periodic", (1, 1, 1)), kw.get("open_axis", -1))
    hit = read_cache(cache_path).get(key)
    if isinstance(hit, dict) and hit.get("kernel") in cands:
        return dict(hit, key=key)
    timings, blocks = {}, {}
    for k in cands:
        lat = lattice(solid, kernel=k, **kw)
        try:
            lat.init_densities(*rho)
            blocks[k] = lat.autotune(block_cache) if k in ("split", "wave") else None
            timings[k] = float(timer(lat, steps, warmup))
        finally:
            lat.close()
    best = min(timings, key=timings.get)
    entry = {"kernel": best, "block": blocks[best], "ms_per_step": timings[best], "timings": timings}
    if cache_path:
        cache = read_cache(cache_path)
        cache[key] = entry
        write_cache(cache_path, cache)
    return dict(entry, key=key)
