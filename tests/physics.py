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
