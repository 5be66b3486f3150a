"""Measurements used by the physics pins (test code; not part of either path).

All fields are numpy arrays of shape (nz, ny, nx) as returned by the oracle's
``fields()`` or the library's ``read_fields()``.
"""
import math

import numpy as np


def laplace_cylinder(f, center_xz):
    """Radius and pressure jump of a y-invariant droplet of component 1.

    R from the area where component 1 is the majority, A = pi R^2; the jump is
    P at the centre minus P at the far corner (periodic far field)."""
    A = float((f["rho1"][:, 0, :] > f["rho2"][:, 0, :]).sum())
    R = math.sqrt(A / math.pi)
    cx, cz = center_xz
    dP = f["P"][int(cz), 0, int(cx)] - f["P"][0, 0, 0]
    return R, float(dP)


def laplace_sphere(f, center):
    """Radius (from the volume, V = 4/3 pi R^3) and pressure jump of a droplet."""
    V = float((f["rho1"] > f["rho2"]).sum())
    R = (3.0 * V / (4.0 * math.pi)) ** (1.0 / 3.0)
    cx, cy, cz = (int(c) for c in center)
    dP = f["P"][cz, cy, cx] - f["P"][0, 0, 0]
    return R, float(dP)


def laplace_jump(f, center, cylinder=False):
    """Radius and pressure jump of a droplet of component 1 centred at
    (cx, cy, cz) in a periodic box (for a y-invariant cylinder pass
    cylinder=True).  R from the majority volume (V = 4/3 pi R^3) or area
    (A = pi R^2); the jump is the mean pressure (Eq. 12) over the nodes more
    than 6 lattice units inside the interface minus the mean over the nodes
    more than 10 units outside it (the periodic far field)."""
    rho1, rho2, P = f["rho1"], f["rho2"], f["P"]
    nz, ny, nx = rho1.shape
    cx, cy, cz = center
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def per(a, c, n):
        d = np.abs(a - c)
        return np.minimum(d, n - d)

    d2 = per(x, cx, nx) ** 2 + per(z, cz, nz) ** 2
    if not cylinder:
        d2 = d2 + per(y, cy, ny) ** 2
    d = np.sqrt(d2)
    inside = rho1 > rho2
    if cylinder:
        R = math.sqrt(float(inside[:, 0, :].sum()) / math.pi)
    else:
        R = (3.0 * float(inside.sum()) / (4.0 * math.pi)) ** (1.0 / 3.0)
    p_in = float(P[d < max(1.0, R - 6.0)].mean())
    p_out = float(P[d > R + 10.0].mean())
    return R, p_in - p_out


def interface_points_xz(rho1, rho2, z_min):
    """Sub-voxel points of the rho1 = rho2 contour of a y-invariant field,
    by linear interpolation along z and x, keeping points with z >= z_min."""
    phi = rho1 - rho2  # > 0 inside the droplet
    pts = []
    nz, nx = phi.shape
    for x in range(nx):
        col = phi[:, x]
        for z in range(nz - 1):
            a, b = col[z], col[z + 1]
            if a * b < 0:
                zz = z + a / (a - b)
                if zz >= z_min:
                    pts.append((float(x), zz))
    for z in range(nz):
        row = phi[z, :]
        if z < z_min:
            continue
        for x in range(nx - 1):
            a, b = row[x], row[x + 1]
            if a * b < 0:
                pts.append((x + a / (a - b), float(z)))
    return np.array(pts)


def fit_circle(pts):
    """Algebraic least-squares circle: returns (xc, zc, R)."""
    x, z = pts[:, 0], pts[:, 1]
    A = np.stack([x, z, np.ones_like(x)], axis=1)
    b = x * x + z * z
    c, *_ = np.linalg.lstsq(A, b, rcond=None)
    xc, zc = c[0] / 2, c[1] / 2
    R = math.sqrt(c[2] + xc * xc + zc * zc)
    return xc, zc, R


def contact_angle_water(f, wall_z, z_min_above_wall=3.0):
    """Contact angle (degrees) of a y-invariant cap of component 1 sitting on a
    flat wall, measured through component 2 (Section 3.2 convention).

    The interface is fitted by a circle away from the wall; the wall surface is
    the half-way plane z = wall_z (the solid layer ends half a voxel below)."""
    rho1 = f["rho1"][:, 0, :]
    rho2 = f["rho2"][:, 0, :]
    pts = interface_points_xz(rho1, rho2, wall_z + z_min_above_wall)
    xc, zc, R = fit_circle(pts)
    h = zc - wall_z  # centre height above the wall surface
    # angle inside the droplet (component 1): cos(theta_1) = -h / R
    c = max(-1.0, min(1.0, -h / R))
    theta1 = math.degrees(math.acos(c))
    return 180.0 - theta1


def duct_series_velocity(nxf, nyf, g, nu, nterms=101):
    """Fully developed flow in a rectangular duct of width a = nxf and height
    b = nyf (walls half a voxel outside the outermost fluid nodes), driven by a
    uniform acceleration g along the axis: the classical Fourier series
    solution of nu (u_xx + u_yy) = -g with u = 0 on the walls.  Returns u at
    the fluid node centres, shape (nyf, nxf)."""
    a, b = float(nxf), float(nyf)
    x = np.arange(nxf) + 0.5  # node centres measured from the wall plane
    y = np.arange(nyf) + 0.5
    X, Y = np.meshgrid(x, y)
    u = np.zeros_like(X)
    for n in range(1, nterms + 1, 2):
        kn = n * math.pi / a
        # particular + homogeneous parts of the sine expansion in x
        coef = 4.0 * g / (nu * a * kn ** 3)
        u += coef * np.sin(kn * X) * (1.0 - np.cosh(kn * (Y - b / 2)) / np.cosh(kn * b / 2))
    return u


def parallel_flow_profile(R, mu, g, fluid):
    """Steady flow along x of a layered mixture between half-way walls:
    d/dz (mu(z) du/dz) = -R(z) g on the fluid nodes of a column, u = 0 half
    a node beyond the first and last fluid node.  Finite volumes with the
    viscosity between two nodes taken as the harmonic mean of theirs (the
    series resistance of two half cells).  R, mu and fluid are 1-D arrays over
    z; returns u on the fluid nodes."""
    idx = np.flatnonzero(fluid)
    m = len(idx)
    A = np.zeros((m, m))
    for k in range(m):
        i = idx[k]
        for nb, kk in ((i - 1, k - 1), (i + 1, k + 1)):
            if 0 <= kk < m:
                mh = 2.0 * mu[i] * mu[nb] / (mu[i] + mu[nb])
                A[k, k] -= mh
                A[k, kk] += mh
            else:
                A[k, k] -= 2.0 * mu[i]  # wall half a node away
    return np.linalg.solve(A, -np.asarray(R, float)[idx] * g)


def trapped_by_dilation(rho1, rho2, solid, outlet_slices, periodic_xy=True):
    """Trapped wetting volume by repeated dilation (an algorithm independent
    of cluster labelling): start from the water voxels (rho2 > rho1, fluid) of
    the outlet reservoir, grow through water voxels over the 18 D3Q19
    neighbours (wrapping in x and y when those faces are periodic) until
    nothing changes, and count the water voxels never reached."""
    water = (rho2 > rho1) & (solid == 0)
    reached = np.zeros_like(water)
    reached[-outlet_slices:] = water[-outlet_slices:]
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if 0 < abs(dz) + abs(dy) + abs(dx) <= 2]

    def shifted(a, dz, dy, dx):
        b = np.roll(a, (dy, dx), axis=(1, 2)) if periodic_xy else a
        if not periodic_xy:
            b = np.zeros_like(a)
            ys = slice(max(dy, 0), a.shape[1] + min(dy, 0))
            yd = slice(max(-dy, 0), a.shape[1] + min(-dy, 0))
            xs = slice(max(dx, 0), a.shape[2] + min(dx, 0))
            xd = slice(max(-dx, 0), a.shape[2] + min(-dx, 0))
            b[:, ys, xs] = a[:, yd, xd]
        out = np.zeros_like(b)
        if dz > 0:
            out[dz:] = b[:-dz]
        elif dz < 0:
            out[:dz] = b[-dz:]
        else:
            out = b
        return out

    while True:
        grow = reached.copy()
        for o in offs:
            grow |= shifted(reached, *o)
        grow &= water
        if np.array_equal(grow, reached):
            break
        reached = grow
    return int((water & ~reached).sum())


def trapped_wetting_volume(f, solid, reservoir):
    """Wetting-phase (component 2, rho2 > rho1) fluid nodes in 18-connected
    clusters that do not reach the outlet reservoir (the last `reservoir`
    z slices): the trapped volume of a drainage."""
    from scipy import ndimage

    water = (f["rho2"] > f["rho1"]) & (solid == 0)
    lab, n = ndimage.label(water, structure=ndimage.generate_binary_structure(3, 2))
    if n == 0:
        return 0
    outlet = set(np.unique(lab[-reservoir:][lab[-reservoir:] > 0]).tolist())
    trapped = (lab > 0) & ~np.isin(lab, list(outlet))
    return int(trapped.sum())
