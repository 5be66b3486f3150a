"""Experiment drivers on top of the lattice (host-side control only; every
time step runs in liblbm's CUDA kernels).

* ``inlet_density``: the inlet density of component 1 that gives a capillary
  pressure P_c = P_in - P_out with the Eq. 12 pressure.
* ``pc_sw_curve``: the capillary-pressure ramp of Sections 4.1-4.2 -- the inlet
  density is raised stage by stage, each stage run until the water saturation
  settles, giving the P_c - S_w curve.
* ``drainage_history``: S_w(t) and the trapped wetting volume every few
  hundred steps of a drainage (Section 4.1 outputs).
* ``contact_angle``: the flat-wall calibration of Section 3.2 at reduced size
  -- a cap of component 1 (oil) on a wall, relaxed, its angle measured through
  component 2 (water) from the base width a few lattice units above the wall
  and the cap height, with the wall surface half way between the solid and
  the first fluid layer.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import inputs

CS2 = 1.0 / 3.0


class JsonLines:
    """Append one JSON object per line to ``path`` (a run's time series: one
    record per stage or checkpoint, each stamped with the wall-clock time and
    the lattice's step count and launch count).  ``None`` writes nothing."""

    def __init__(self, path, lattice=None, **run):
        self.path, self.lattice = path, lattice
        if path is not None and run:
            self.write({"run": run})

    def write(self, rec):
        if self.path is None:
            return
        rec = dict(rec)
        rec["time"] = time.time()
        if self.lattice is not None and hasattr(self.lattice, "info"):
            info = self.lattice.info()
            rec.setdefault("lattice_step", int(info["step"]))
            rec.setdefault("launches", int(info["launches"]))
        with open(self.path, "a") as fh:
            fh.write(json.dumps(rec) + "\n")


def pressure(rho1, rho2, G):
    """Eq. 12 over ordered pairs: c_s^2 (rho1 + rho2) + c_s^2 G rho1 rho2."""
    return CS2 * (rho1 + rho2) + CS2 * G * rho1 * rho2


def inlet_density(pc, G=3.5, minor=0.03, rho_out2=1.0):
    """rho_in1 such that P(rho_in1, minor) - P(minor, rho_out2) = pc, with the
    other component at the dissolved level ``minor`` on each side."""
    p_out = pressure(minor, rho_out2, G)
    return (p_out + pc - CS2 * minor) / (CS2 * (1.0 + G * minor))


def pc_sw_curve(lattice, pcs, G=3.5, minor=0.03, rho_out2=1.0, max_steps=20000, check_every=500, tol=1e-3,
                log=None):
    """Raise the inlet density through the capillary pressures ``pcs`` (in
    order).  At each stage the lattice steps in chunks of ``check_every`` until
    the water saturation changes by less than ``tol`` over a chunk, or
    ``max_steps`` have run.  Returns one dict per stage: pc, rho_in1, S_w,
    smooth S_nw, steps, settled; with ``log`` (a path) each stage is also
    appended to that file as a JSON line."""
    jl = JsonLines(log, lattice, driver="pc_sw_curve", pcs=[float(p) for p in pcs], G=G, tol=tol)
    out = []
    for pc in pcs:
        rin = inlet_density(pc, G, minor, rho_out2)
        lattice.set_inlet(rin)
        prev = lattice.saturation()[0]
        steps, settled = 0, False
        while steps < max_steps:
            lattice.step(check_every)
            steps += check_every
            sw, snw = lattice.saturation()[:2]
            if abs(sw - prev) < tol:
                settled = True
                break
            prev = sw
        sw, snw = lattice.saturation()[:2]
        out.append({"pc": float(pc), "rho_in1": float(rin), "S_w": float(sw), "S_nw_smooth": float(snw),
                    "steps": int(steps), "settled": settled})
        jl.write(out[-1])
    return out


def trapped_volume(rho1, rho2, solid, outlet_slices, periodic_xy=(True, True)):
    """Wetting-phase voxels (component 2 the majority, rho2 > rho1) in
    18-connected clusters that reach neither the outlet reservoir (the last
    ``outlet_slices`` z slices) nor, through it, the outlet: the volume the
    displacing phase has cut off.  Clusters joined across a periodic lateral
    face (``periodic_xy`` for x and y) are one cluster, as on the lattice."""
    from scipy import ndimage

    water = (rho2 > rho1) & (solid == 0)
    lab, n = ndimage.label(water, structure=ndimage.generate_binary_structure(3, 2))
    if n == 0:
        return 0
    # labels that touch across a periodic face: compare each voxel with its
    # D3Q19 neighbours through the wrap, and join the two clusters
    parent = np.arange(n + 1)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    px, py = bool(periodic_xy[0]), bool(periodic_xy[1])
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if not 0 < abs(dz) + abs(dy) + abs(dx) <= 2:
                    continue
                if not ((px and dx) or (py and dy)):
                    continue  # this offset never crosses a periodic face
                nb = np.roll(lab, (-dy if py else 0, -dx if px else 0), axis=(1, 2))
                if dz:
                    nb = np.roll(nb, -dz, axis=0)
                    edge = np.ones(lab.shape[0], bool)
                    edge[-1 if dz > 0 else 0] = False  # z is not periodic
                    nb = nb * edge[:, None, None]
                a, b = lab.ravel(), nb.ravel()
                m = (a > 0) & (b > 0) & (a != b)
                for u, v in set(zip(a[m].tolist(), b[m].tolist())):
                    ru, rv = find(u), find(v)
                    if ru != rv:
                        parent[max(ru, rv)] = min(ru, rv)
    root = np.array([find(k) for k in range(n + 1)])
    tail = lab[-outlet_slices:]
    connected = np.unique(root[np.unique(tail[tail > 0])])
    return int(((lab > 0) & ~np.isin(root[lab], connected)).sum())


def drainage_history(lattice, solid, nsteps, every=500, outlet_slices=8, periodic_xy=(True, True), log=None):
    """Step a drainage ``nsteps`` steps, recording every ``every`` steps the
    water saturation S_w, the smooth non-wetting saturation, the component
    masses and the trapped wetting volume (Section 4.1 outputs).  Returns a
    list of dicts; with ``log`` (a path) each record is also appended to that
    file as a JSON line."""
    jl = JsonLines(log, lattice, driver="drainage_history", nsteps=int(nsteps), every=int(every))
    out = []
    done = 0
    while done < nsteps:
        k = min(every, nsteps - done)
        lattice.step(k)
        done += k
        sw, snw, m1, m2 = (list(lattice.saturation()) + [float("nan")] * 4)[:4]
        f = lattice.fields(("rho1", "rho2"))
        out.append({"step": done, "S_w": float(sw), "S_nw_smooth": float(snw), "mass1": float(m1),
                    "mass2": float(m2),
                    "trapped": trapped_volume(f["rho1"], f["rho2"], solid, outlet_slices, periodic_xy)})
        jl.write(out[-1])
    return out


def _crossings(phi, coord0=0.0):
    """Sub-cell positions where a 1-D profile changes sign (linear interpolation)."""
    out = []
    for k in range(len(phi) - 1):
        a, b = phi[k], phi[k + 1]
        if a == 0.0:
            out.append(coord0 + k)
        elif a * b < 0:
            out.append(coord0 + k + a / (a - b))
    return out


def cap_angle(rho1, rho2, wall_z=0.5, base_height=5.0):
    """Contact angle in degrees through component 2 of a y-invariant cap of
    component 1 standing on a wall whose surface is the plane z = wall_z.

    The interface is the rho1 = rho2 level set (linear interpolation).  The
    cap top T is the highest crossing over all columns; the base width 2a is
    measured on the line z = wall_z + base_height.  A circle through the top
    and the chord ends has radius R = (a^2 + H^2) / (2H), H = T - chord line;
    its centre lies R - H below the top, and the angle inside the cap
    satisfies cos(theta_1) = -(centre height above the wall) / R."""
    phi = (rho1 - rho2)[:, 0, :]  # (nz, nx), > 0 inside the cap
    nz, nx = phi.shape
    tops = []
    for x in range(nx):
        col = phi[:, x]
        if col.max() <= 0:
            continue
        tops.extend(c for c in _crossings(col) if c > wall_z)
    T = max(tops)
    zc = wall_z + base_height
    k = int(math.floor(zc))
    t = zc - k
    row = (1 - t) * phi[k] + t * phi[k + 1]
    cr = _crossings(row)
    if len(cr) < 2:
        raise ValueError("the cap does not reach the base line")
    a = 0.5 * (max(cr) - min(cr))
    H = T - zc
    R = (a * a + H * H) / (2.0 * H)
    centre = T - R  # height of the circle centre
    c = max(-1.0, min(1.0, -(centre - wall_z) / R))
    return 180.0 - math.degrees(math.acos(c))


def contact_angle(lbm, xi, tau=(3.5, 0.62), G=3.5, nx=96, nz=40, radius=16, steps=4000, storage="fp32"):
    """Relax a cap of component 1 (radius ``radius``, centred on the lower
    wall) between two solid walls at z = 0 and z = nz - 1, periodic in x and
    y (one voxel deep), and return its angle through component 2."""
    shape = (nz, 1, nx)
    solid = np.zeros(shape, np.uint8)
    solid[0] = 1
    solid[-1] = 1
    r1, r2 = inputs.cylinder_densities(shape, (nx / 2, 1.0), radius, 5.0, 1.0, 0.03)
    fl = solid == 0
    lat = lbm.Lattice(solid, tau=tau, G=G, xi=xi, periodic=(1, 1, 0), storage=storage)
    lat.init_densities(r1 * fl, r2 * fl)
    lat.step(steps)
    f = lat.fields(("rho1", "rho2"))
    return cap_angle(f["rho1"], f["rho2"])
