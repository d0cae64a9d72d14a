"""Voxelised geometries.

Arrays are C-ordered with shape (nz, ny, nx), so the linear cell index is
``x + nx * (y + ny * z)``.  Cell centres sit at integer + 1/2.

Flag values (uint8): SOLID=0, FLUID=1, INLET=2, OUTLET=3.
"""

import numpy as np

SOLID, FLUID, INLET, OUTLET = 0, 1, 2, 3


def _centres(nx, ny, nz):
    z, y, x = np.meshgrid(
        np.arange(nz, dtype=np.float64) + 0.5,
        np.arange(ny, dtype=np.float64) + 0.5,
        np.arange(nx, dtype=np.float64) + 0.5,
        indexing="ij",
    )
    return x, y, z


def pipe_flags(nx=32, ny=32, nz=64, radius=14.0, cx=16.0, cy=16.0):
    """Straight circular pipe along z: fluid where the cell centre lies within
    ``radius`` of (cx, cy); walls elsewhere.  Periodic in z by configuration."""
    x, y, _ = _centres(nx, ny, nz)
    fluid = (x - cx) ** 2 + (y - cy) ** 2 <= radius ** 2
    flags = np.zeros((nz, ny, nx), dtype=np.uint8)
    flags[fluid] = FLUID
    return flags


def channel_flags(ny, nx=2, nz=2):
    """Plane channel between two walls normal to y (solid rows y=0 and y=ny-1);
    periodic in x and z by configuration.  Fluid occupies y=1..ny-2."""
    flags = np.full((nz, ny, nx), FLUID, dtype=np.uint8)
    flags[:, 0, :] = SOLID
    flags[:, ny - 1, :] = SOLID
    return flags


def periodic_box_flags(nx, ny, nz, obstacles=0, seed=0):
    """Fully fluid box (periodic on all axes by configuration) with an optional
    number of randomly placed solid voxels."""
    flags = np.full((nz, ny, nx), FLUID, dtype=np.uint8)
    if obstacles:
        rng = np.random.default_rng(seed)
        sel = rng.choice(nx * ny * nz, size=obstacles, replace=False)
        flags.reshape(-1)[sel] = SOLID
    return flags


def _aneurysm_shape(n, small=False):
    """Radii of vessel, sac and neck plus the sac gap for an n^3 box."""
    if small:
        return 3.0, 6.0, 2.5, 1.0
    s = n / 256.0
    return 20.0 * s, 40.0 * s, 15.0 * s, 4.0 * s


def _aneurysm_geom(n, small=False):
    r_v, r_s, r_n, gap = _aneurysm_shape(n, small)
    rc = n / 2.0
    y0 = n / 2.0
    e = np.array([-1.0, 0.0, 1.0]) / np.sqrt(2.0)
    dist = rc + r_v + gap + r_s
    sc = np.array([n, y0, 0.0]) + dist * e
    p0 = np.array([n, y0, 0.0]) + rc * e
    return dict(r_v=r_v, r_s=r_s, r_n=r_n, rc=rc, y0=y0, e=e, dist=dist, sc=sc, p0=p0)


def _aneurysm_parts(n, small=False, z0=0, z1=None):
    """Boolean (vessel, sac, neck) masks for the z-slab [z0, z1) of the box."""
    g = _aneurysm_geom(n, small)
    z1 = n if z1 is None else z1
    z, y, x = np.meshgrid(
        np.arange(z0, z1, dtype=np.float64) + 0.5,
        np.arange(n, dtype=np.float64) + 0.5,
        np.arange(n, dtype=np.float64) + 0.5,
        indexing="ij",
    )
    # Quarter-circle centreline of radius rc around the bend centre (n, y0, 0)
    # in the x-z plane, from (n/2, y0, 0) (tangent +z) to (n, y0, n/2) (tangent +x).
    # Inside the box every point lies in the quarter's angular range.
    dx = x - n
    rho = np.sqrt(dx * dx + z * z)
    vessel = (rho - g["rc"]) ** 2 + (y - g["y0"]) ** 2 <= g["r_v"] ** 2
    del rho, dx
    # Sac: sphere on the outer side of the bend at 45 degrees.
    sc = g["sc"]
    sac = (x - sc[0]) ** 2 + (y - sc[1]) ** 2 + (z - sc[2]) ** 2 <= g["r_s"] ** 2
    # Neck: cylinder along the radial from the centreline point to the sac centre.
    e, p0 = g["e"], g["p0"]
    rx, ry, rz = x - p0[0], y - p0[1], z - p0[2]
    t = rx * e[0] + ry * e[1] + rz * e[2]
    perp2 = rx * rx + ry * ry + rz * rz - t * t
    neck = (t >= 0.0) & (t <= g["dist"] - g["rc"]) & (perp2 <= g["r_n"] ** 2)
    return vessel, sac, neck


def _slabs(n, cells_per_slab=1 << 22):
    step = max(1, cells_per_slab // (n * n))
    for z0 in range(0, n, step):
        yield z0, min(n, z0 + step)


def aneurysm_flags(n, small=False):
    """Synthetic saccular aneurysm in an n^3 box.

    A tube (radius 20*n/256) follows a quarter circle of radius n/2 in the x-z
    plane; a sphere (radius 40*n/256) sits on the outer side of the bend at 45
    degrees, joined to the tube by a neck cylinder (radius 15*n/256).  The inlet
    is the tube's disk on the face z=0, the outlet its disk on the face x=n-1.
    ``small=True`` gives the 24^3 variant (radii 3/6/2.5, gap 1).

    Outlet cells are the fluid cells of the face x=n-1 whose upstream neighbour
    (x=n-2) is fluid; other fluid cells of that face become solid so that every
    outlet cell has an interior neighbour to extrapolate from.
    """
    flags = np.zeros((n, n, n), dtype=np.uint8)
    for z0, z1 in _slabs(n):
        vessel, sac, neck = _aneurysm_parts(n, small, z0, z1)
        flags[z0:z1][vessel | sac | neck] = FLUID
    face = flags[0, :, :]
    face[face == FLUID] = INLET
    last = flags[:, :, n - 1]
    prev = flags[:, :, n - 2]
    out = (last == FLUID) & (prev == FLUID)
    last[(last == FLUID) & ~out] = SOLID
    last[out] = OUTLET
    return flags


def aneurysm_inlet(n, small=False):
    """(centre_x, centre_y, radius) of the inlet disk on z=0, in lattice units."""
    g = _aneurysm_geom(n, small)
    return (n / 2.0, g["y0"], g["r_v"])


def sac_mask(n, small=False):
    """uint8 mask of the sac sphere (the objective / diagnostic region)."""
    m = np.zeros((n, n, n), dtype=np.uint8)
    for z0, z1 in _slabs(n):
        _, sac, _ = _aneurysm_parts(n, small, z0, z1)
        m[z0:z1][sac] = 1
    return m


def sac_sphere(n, small=False):
    """(centre (x, y, z), radius) of the sac sphere."""
    g = _aneurysm_geom(n, small)
    return g["sc"], g["r_s"]
