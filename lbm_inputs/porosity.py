"""Seeded porosity fields (the coil represented as a porous medium).

All fields are float32 arrays of shape (nz, ny, nx) with values in (0, 1].
"""

import numpy as np

from . import geometry as geo


def plug_porosity(flags, z0=24, z1=40, value=0.75):
    """Porosity 1 everywhere except a plug of layers z0..z1 (inclusive)."""
    phi = np.ones(flags.shape, dtype=np.float32)
    phi[z0 : z1 + 1] = np.float32(value)
    return phi


def sac_random_porosity(n, small=False, seed=0, sigma=6.0, mean=0.75, amp=0.1,
                        lo=0.6, hi=1.0):
    """Coil porosity inside the sac: a Gaussian-smoothed random field.

    i.i.d. N(0, 1) noise is drawn on the sac's bounding box padded by 4*sigma
    (default_rng(seed)), filtered with a Gaussian of standard deviation
    ``sigma`` voxels, rescaled to unit standard deviation, mapped to
    ``mean + amp * z`` and clipped to [lo, hi].  It is applied inside the sac
    sphere only; porosity is 1 elsewhere.
    """
    from scipy.ndimage import gaussian_filter

    sc, r_s = geo.sac_sphere(n, small)
    pad = int(np.ceil(r_s + 4 * sigma))
    lo_c = [max(0, int(np.floor(c)) - pad) for c in sc]
    hi_c = [min(n, int(np.ceil(c)) + pad + 1) for c in sc]
    shape = (hi_c[2] - lo_c[2], hi_c[1] - lo_c[1], hi_c[0] - lo_c[0])
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    field = gaussian_filter(noise, sigma=sigma, mode="reflect")
    field /= field.std()
    val = np.clip(mean + amp * field, lo, hi).astype(np.float32)
    phi = np.ones((n, n, n), dtype=np.float32)
    sub = phi[lo_c[2] : hi_c[2], lo_c[1] : hi_c[1], lo_c[0] : hi_c[0]]
    sac = geo.sac_mask(n, small)[lo_c[2] : hi_c[2], lo_c[1] : hi_c[1], lo_c[0] : hi_c[0]] > 0
    sub[sac] = val[sac]
    return phi


def wire_coil(n, packing=0.25, seed=0, thickness_radius=1, small=False):
    """Seeded random-walk helical wire filling ``packing`` of the sac volume.

    Unit steps; each direction is the previous one plus a helical bias (rotation
    about the sac's radial axis) plus Gaussian jitter, reflected back when the
    walker leaves the sac sphere.  The wire is deposited with a dilation radius
    ``thickness_radius`` (a 2-voxel-thick wire for radius 1).  Returns a uint8
    mask of wire voxels (inside the sac only).
    """
    return (wire_coil_order(n, packing, seed, thickness_radius, small) >= 0).astype(np.uint8)


def coil_packings(n, packings, seed=0, thickness_radius=1, small=False):
    """Wires of several packing densities from one walk, the way a coil is
    inserted: the wire of packing p is the first p |sac| voxels the walk of the
    largest packing deposits.  Returns {p: uint8 mask}."""
    order = wire_coil_order(n, max(packings), seed, thickness_radius, small)
    n_sac = int((geo.sac_mask(n, small) > 0).sum())
    return {p: ((order >= 0) & (order < int(p * n_sac))).astype(np.uint8) for p in packings}


def wire_coil_order(n, packing=0.25, seed=0, thickness_radius=1, small=False):
    """The walk of :func:`wire_coil`; returns an int32 array holding the
    deposition index of every wire voxel and -1 elsewhere."""
    sc, r_s = geo.sac_sphere(n, small)
    sac = geo.sac_mask(n, small) > 0
    target = int(packing * sac.sum())
    wire = np.full(sac.shape, -1, dtype=np.int32)
    rng = np.random.default_rng(seed)
    p = np.array(sc, dtype=np.float64)
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    axis = np.array([0.0, 1.0, 0.0])
    offs = [
        (dz, dy, dx)
        for dz in range(-thickness_radius, thickness_radius + 1)
        for dy in range(-thickness_radius, thickness_radius + 1)
        for dx in range(-thickness_radius, thickness_radius + 1)
        if dx * dx + dy * dy + dz * dz <= thickness_radius * thickness_radius
    ]
    count = 0
    max_steps = 200 * target + 1000
    for _ in range(max_steps):
        if count >= target:
            break
        helix = np.cross(axis, d)
        d = d + 0.35 * helix + 0.25 * rng.standard_normal(3)
        d /= np.linalg.norm(d)
        q = p + d
        if np.linalg.norm(q - sc) > r_s - thickness_radius - 0.5:
            # reflect the direction about the sphere normal
            nrm = (q - sc) / np.linalg.norm(q - sc)
            d = d - 2.0 * np.dot(d, nrm) * nrm
            q = p + d
            if np.linalg.norm(q - sc) > r_s - thickness_radius - 0.5:
                q = p
        p = q
        ix, iy, iz = (int(np.floor(c)) for c in p)
        for dz, dy, dx in offs:
            z, y, x = iz + dz, iy + dy, ix + dx
            if 0 <= x < n and 0 <= y < n and 0 <= z < n and sac[z, y, x] and wire[z, y, x] < 0:
                wire[z, y, x] = count
                count += 1
    return wire


def coil_shape_tensor(shape, ratio=4.0, sigma=3.0, seed=0):
    """Seeded shape tensor S of an anisotropic coil medium, (6, nz, ny, nx)
    float32, components xx yy zz xy xz yz: S = t t^T / ratio + (Id - t t^T)
    with t(x) a smooth random unit vector (i.i.d. normal vector components
    filtered with a Gaussian of ``sigma`` voxels, then normalised), the local
    wire direction.  Eigenvalues 1/ratio along t and 1 across it: the medium
    is ``ratio`` times more permeable along the wire than across it."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    t = np.stack([gaussian_filter(rng.standard_normal(shape, dtype=np.float32), sigma=sigma, mode="wrap")
                  for _ in range(3)])
    t /= np.maximum(np.sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]), np.float32(1e-12))
    a = np.float32(1.0 / ratio - 1.0)
    S = np.empty((6,) + tuple(shape), dtype=np.float32)
    for k, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
        S[k] = a * t[i] * t[j] + np.float32(1.0 if i == j else 0.0)
    return S
