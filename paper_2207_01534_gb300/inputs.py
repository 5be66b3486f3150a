"""Seeded synthetic inputs: geometries, initial density fields, parameter maps.

This module holds none of the lattice Boltzmann arithmetic.  It only draws
geometries and initial fields, so both the CUDA path and the FP64 oracle (in
tests) can be fed the same arrays.  All arrays are numpy, shape (nz, ny, nx),
x fastest; ``solid`` is uint8 with 1 = solid.

Stand-ins for the paper's datasets (the Finney sphere pack of Section 4.1 and
the Bentheimer sandstone of Section 4.2 are not available here):
  * ``sphere_pack``: seeded random sequential addition of equal spheres with a
    minimum centre distance that is relaxed by 5% after 10^4 consecutive
    rejections until the voxel porosity reaches the target (non-overlapping
    packing jams near 38% solid, so porosities below ~0.62 need overlap);
  * ``grf_rock``: a periodic Gaussian random field (Gaussian covariance of
    correlation length ``corr_len``) thresholded at the quantile that gives the
    requested porosity.
Both get fluid reservoir slabs at the two ends of the flow axis (z) and lose
pore clusters that do not connect inlet to outlet (isolated-pore removal,
Section 4.2).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 220701534

# Contact-angle calibration of Section 3.2 (degrees, measured through
# component 2): theta = 47.4136 xi^3 - 23.4513 xi^2 + 89.7938 xi + 91.2324.
_THETA_CUBIC = (47.4136, -23.4513, 89.7938, 91.2324)


def theta_of_xi(xi: float) -> float:
    a, b, c, d = _THETA_CUBIC
    return ((a * xi + b) * xi + c) * xi + d


def xi_of_theta(theta_deg: float) -> float:
    """Invert the calibration cubic on its monotone branch (bisection)."""
    lo, hi = -0.62, 0.8
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if theta_of_xi(mid) < theta_deg:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def tau_for_viscosity_ratio(M: float, tau2: float = 0.62) -> tuple[float, float]:
    """tau^(1) giving nu1/nu2 = M with nu = c_s^2 (tau - 1/2) (Section 3.1 pairs)."""
    return (0.5 + M * (tau2 - 0.5), tau2)


def droplet_densities(shape, center, r0, W=5.0, rho_major=1.0, rho_minor=0.03):
    """Eq. 16 tanh profile: component 1 forms the droplet, component 2 the rest."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    t = np.tanh(2.0 * (d - r0) / W)
    rho1 = 0.5 * (rho_major + rho_minor) - 0.5 * (rho_major - rho_minor) * t
    rho2 = 0.5 * (rho_minor + rho_major) - 0.5 * (rho_minor - rho_major) * t
    return rho1, rho2


def cylinder_densities(shape, center_xz, r0, W=5.0, rho_major=1.0, rho_minor=0.03):
    """Eq. 16 profile for a droplet invariant along y (a cylinder)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = np.sqrt((x - center_xz[0]) ** 2 + (z - center_xz[1]) ** 2)
    t = np.tanh(2.0 * (d - r0) / W)
    rho1 = 0.5 * (rho_major + rho_minor) - 0.5 * (rho_major - rho_minor) * t
    rho2 = 0.5 * (rho_minor + rho_major) - 0.5 * (rho_minor - rho_major) * t
    return rho1, rho2


def _ball_offsets(r: float):
    R = int(np.ceil(r))
    g = np.arange(-R, R + 1)
    dz, dy, dx = np.meshgrid(g, g, g, indexing="ij")
    m = dx * dx + dy * dy + dz * dz <= r * r
    return dz[m], dy[m], dx[m]


def _label_pores(pore: np.ndarray, periodic_xy: bool):
    """18-connected labels of the pore space, merged across periodic x/y faces."""
    from scipy import ndimage

    st = ndimage.generate_binary_structure(3, 2)  # 18-connectivity (D3Q19 links)
    lab, n = ndimage.label(pore, structure=st)
    if not periodic_xy or n == 0:
        return lab, n
    nz = pore.shape[0]
    z = np.arange(nz)[:, None, None]
    pairs = set()
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                k = abs(dx) + abs(dy) + abs(dz)
                if k == 0 or k == 3:
                    continue
                other = np.roll(lab, (-dz, -dy, -dx), axis=(0, 1, 2))  # other[v] = lab[v + d]
                zok = (z + dz >= 0) & (z + dz < nz)
                m = (lab > 0) & (other > 0) & (lab != other) & zok
                if m.any():
                    pp = np.unique(np.stack([lab[m], other[m]], axis=1), axis=0)
                    pairs.update(map(tuple, pp.tolist()))
    parent = np.arange(n + 1)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for p, q in pairs:
        rp, rq = find(p), find(q)
        if rp != rq:
            parent[rp] = rq
    roots = np.array([find(i) for i in range(n + 1)])
    return roots[lab], n


def keep_percolating(solid: np.ndarray, periodic_xy: bool = True) -> np.ndarray:
    """Turn into solid every pore cluster that does not touch both z ends."""
    pore = solid == 0
    lab, n = _label_pores(pore, periodic_xy)
    if n == 0:
        return solid.copy()
    top = set(np.unique(lab[0][lab[0] > 0]).tolist())
    bot = set(np.unique(lab[-1][lab[-1] > 0]).tolist())
    keep = np.array(sorted(top & bot), dtype=lab.dtype)
    ok = np.isin(lab, keep) & pore
    return np.where(ok, 0, 1).astype(np.uint8)


def add_reservoirs(solid: np.ndarray, k: int) -> np.ndarray:
    """Clear k slices at each end of z: pure-fluid reservoirs (Section 4.1)."""
    s = solid.copy()
    if k > 0:
        s[:k] = 0
        s[-k:] = 0
    return s


def sphere_pack(n, radius, porosity, seed, reservoir=8, periodic_xy=True, shape=None):
    """Relaxed random sequential addition of equal spheres (see module doc).

    Returns a uint8 solid mask of shape (nz, ny, nx) (default n^3) with
    ``reservoir`` fluid slices at each z end and only percolating pores kept.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if shape is None:
        shape = (n, n, n)
    nz, ny, nx = shape
    solid = np.zeros(shape, dtype=np.uint8)
    zlo, zhi = reservoir, nz - reservoir
    target_solid = (1.0 - porosity) * nx * ny * (zhi - zlo)
    oz, oy, ox = _ball_offsets(radius)
    centers = np.zeros((0, 3))
    dmin = 2.0 * radius
    rejections = 0
    nsolid = 0
    L = np.array([nx, ny, nz], dtype=float)
    while nsolid < target_solid:
        cand = rng.random((256, 3)) * np.array([nx, ny, zhi - zlo]) + np.array([0, 0, zlo])
        # distance of every candidate to the nearest centre placed before this batch
        if len(centers):
            from scipy.spatial import cKDTree

            box = np.array([nx, ny, 64.0 * nz]) if periodic_xy else None
            pts = np.mod(centers, box) if periodic_xy else centers
            tree = cKDTree(pts, boxsize=box)
            dist, _ = tree.query(np.mod(cand, box) if periodic_xy else cand, k=1)
            d2old = dist * dist
        else:
            d2old = np.full(len(cand), np.inf)
        placed = []
        for k, c in enumerate(cand):
            d2 = d2old[k]
            if placed:
                dn = np.array(placed) - c
                if periodic_xy:
                    dn[:, :2] -= L[:2] * np.round(dn[:, :2] / L[:2])
                d2 = min(d2, float(np.min(np.einsum("ij,ij->i", dn, dn))))
            if d2 < dmin * dmin:
                rejections += 1
                if rejections >= 10000:
                    dmin *= 0.95
                    rejections = 0
                continue
            rejections = 0
            placed.append(c)
            ci = np.round(c).astype(int)
            zz = ci[2] + oz
            yy = ci[1] + oy
            xx = ci[0] + ox
            if periodic_xy:
                yy %= ny
                xx %= nx
                m = (zz >= zlo) & (zz < zhi)
            else:
                m = (zz >= zlo) & (zz < zhi) & (yy >= 0) & (yy < ny) & (xx >= 0) & (xx < nx)
            before = solid[zz[m], yy[m], xx[m]].sum()
            solid[zz[m], yy[m], xx[m]] = 1
            nsolid += int(m.sum()) - int(before)
            if nsolid >= target_solid:
                break
        if placed:
            centers = np.vstack([centers, np.array(placed)])
    solid = add_reservoirs(solid, reservoir)
    return keep_percolating(solid, periodic_xy)


def grf_rock(n, corr_len, porosity, seed, reservoir=8, shape=None):
    """Thresholded periodic Gaussian random field (see module doc)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if shape is None:
        shape = (n, n, n)
    noise = rng.standard_normal(shape)
    k = [np.fft.fftfreq(s) * 2 * np.pi for s in shape]
    kz, ky, kx = np.meshgrid(*k, indexing="ij", sparse=True)
    # Gaussian covariance exp(-r^2 / (2 l^2)) has spectrum ~ exp(-k^2 l^2 / 2);
    # the filter is its square root.
    filt = np.exp(-(kx ** 2 + ky ** 2 + kz ** 2) * corr_len ** 2 / 4.0)
    field = np.fft.ifftn(np.fft.fftn(noise) * filt).real
    thr = np.quantile(field, porosity)
    solid = (field > thr).astype(np.uint8)
    solid = add_reservoirs(solid, reservoir)
    return keep_percolating(solid, True)


def add_lateral_walls(solid: np.ndarray, axes=(0, 1)) -> np.ndarray:
    """Close the lateral faces with solid voxels (a core holder, Section 4.2):
    axes 0 / 1 are x / y.  Such a geometry is run with those axes
    non-periodic."""
    s = solid.copy()
    if 0 in axes:
        s[:, :, 0] = 1
        s[:, :, -1] = 1
    if 1 in axes:
        s[:, 0, :] = 1
        s[:, -1, :] = 1
    return s


def drainage_init(solid, inlet_slices, rho_major=1.0, rho_minor=0.03):
    """Component 2 (wetting water) everywhere, component 1 (oil) in the first
    ``inlet_slices`` z slices (Section 4.1 initial state)."""
    nz = solid.shape[0]
    rho1 = np.full(solid.shape, rho_minor)
    rho2 = np.full(solid.shape, rho_major)
    rho1[:inlet_slices] = rho_major
    rho2[:inlet_slices] = rho_minor
    fluid = solid == 0
    return rho1 * fluid, rho2 * fluid


def imbibition_init(solid, outlet_slices, rho_major=1.0, rho_minor=0.03):
    """Component 1 (non-wetting oil) everywhere, component 2 (water) in the
    last ``outlet_slices`` z slices: the start of an imbibition, water entering
    the oil-filled sample from the outlet side."""
    nz = solid.shape[0]
    rho1 = np.full(solid.shape, rho_major)
    rho2 = np.full(solid.shape, rho_minor)
    rho1[nz - outlet_slices:] = rho_minor
    rho2[nz - outlet_slices:] = rho_major
    fluid = solid == 0
    return rho1 * fluid, rho2 * fluid


def porosity(solid: np.ndarray, reservoir: int = 0) -> float:
    s = solid[reservoir: solid.shape[0] - reservoir] if reservoir else solid
    return float((s == 0).mean())


# ---------------------------------------------------------------------------
# Named workloads (seed = SEED_BASE + index)

def laplace_48(minor=0.03):
    """48^3 periodic, droplet of component 1 radius 10 at node (24,24,24)."""
    shape = (48, 48, 48)
    solid = np.zeros(shape, np.uint8)
    r1, r2 = droplet_densities(shape, (24, 24, 24), 10.0, 5.0, 1.0, minor)
    return solid, r1, r2


def drainage_pack_128(seed_offset=1):
    """128^3 sphere pack, radius 8, porosity 0.38, 8-slice reservoirs."""
    solid = sphere_pack(128, 8.0, 0.38, SEED_BASE + seed_offset, reservoir=8)
    r1, r2 = drainage_init(solid, 8)
    return solid, r1, r2


def batched_sweep(count=64, seed_offset=100, edge_lo=48, edge_hi=112):
    """Parameter points of the batched sweep: ``count`` independent sphere
    packs, edge n uniform in edge_lo..edge_hi (48..112), sphere radius uniform
    in [4, 8] (at most n / 6), porosity
    uniform in [0.35, 0.45], 6 reservoir slices per end; sample k takes the
    (viscosity ratio, contact angle) combination k mod 16 of {1, 5, 10, 50} x
    {30, 60, 90, 120} deg (so 64 samples are 4 seeds of every combination).
    Returns one dict per sample; ``batched_sample`` builds its geometry and
    initial state."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed_offset))
    ms, thetas = (1.0, 5.0, 10.0, 50.0), (30.0, 60.0, 90.0, 120.0)
    out = []
    for k in range(count):
        n = int(rng.integers(edge_lo, edge_hi + 1))
        out.append({"n": n, "radius": min(float(rng.uniform(4.0, 8.0)), n / 6.0),
                    "porosity": float(rng.uniform(0.35, 0.45)), "M": ms[k % 4], "theta_deg": thetas[(k // 4) % 4],
                    "reservoir": 6, "seed": SEED_BASE + seed_offset + 1 + k})
    return out


def batched_sample(spec):
    """(solid, rho1, rho2) of one sample of ``batched_sweep``."""
    solid = sphere_pack(spec["n"], spec["radius"], spec["porosity"], spec["seed"], reservoir=spec["reservoir"])
    r1, r2 = drainage_init(solid, spec["reservoir"])
    return solid, r1, r2


def rock_grf_256(seed_offset=3):
    """256^3 sandstone stand-in: periodic Gaussian random field, correlation
    length 6, thresholded to porosity 0.22, 8-slice reservoirs, drainage start."""
    solid = grf_rock(256, 6.0, 0.22, SEED_BASE + seed_offset, reservoir=8)
    r1, r2 = drainage_init(solid, 8)
    return solid, r1, r2


def crop(solid, n, reservoir=4, origin=None):
    """An n^3 sub-block of a rock (from its centre unless ``origin`` (z, y, x) is
    given) with ``reservoir`` fluid slices added at both z ends (inside the n
    slices) and only percolating pores kept."""
    nz, ny, nx = solid.shape
    if origin is None:
        origin = ((nz - n) // 2, (ny - n) // 2, (nx - n) // 2)
    z, y, x = origin
    c = solid[z:z + n, y:y + n, x:x + n].copy()
    c = add_reservoirs(c, reservoir)
    return keep_percolating(c, True)


def adjoint_pack_96(seed_offset=2):
    """96^3 sphere pack, radius 6, porosity 0.40, 8-slice reservoirs, with the
    imbibition start (oil everywhere, water in the outlet reservoir)."""
    solid = sphere_pack(96, 6.0, 0.40, SEED_BASE + seed_offset, reservoir=8)
    r1, r2 = imbibition_init(solid, 8)
    return solid, r1, r2


def random_pops_state(solid, seed, rho_lo=0.02, rho_hi=1.0, noise=0.05):
    """Non-equilibrium populations for parity tests: per-node random component
    densities spread evenly over the 19 directions with a random relative
    perturbation.  Returns two (19, nz, ny, nx) arrays (zeros on solids)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(2):
        rho = rng.uniform(rho_lo, rho_hi, solid.shape)
        pert = 1.0 + noise * rng.uniform(-1, 1, (19,) + solid.shape)
        f = (rho[None] / 19.0) * pert
        f[:, solid != 0] = 0.0
        out.append(f)
    return out[0], out[1]
