"""Volume-averaged porosity of a voxelised coil (Sec. 4: the porosity field is
the windowed convolution of the voxelised coil with a uniform averaging kernel;
Table 1: averaging window 1.23 mm, 28 cells at the Table 1 spacing).

TEST INFRASTRUCTURE ONLY: used by the tests and the CPU baseline; the library
path never imports it.

Definition (written out, no blocking or reordering):
  count(x) = number of wire voxels v with x_a - lo <= v_a <= x_a + hi on every
             axis a, lo = window // 2, hi = window - 1 - lo (cells outside the
             box count as no wire);
  phi(x)   = max(phi_min, (window^3 - count(x)) / window^3): the quotient of
             two exact integers, divided in FP64 and rounded to FP32 (no FP32
             midpoint lies within FP64 rounding of such a quotient, so this is
             its correctly rounded FP32 value), phi_min rounded to FP32;
  phi(x)   = 1 on solid cells (flags == 0) when flags are given.
"""

import numpy as np


def window_bounds(window):
    """(lo, hi): the window of cell x along an axis is [x - lo, x + hi]."""
    lo = window // 2
    return lo, window - 1 - lo


def wire_count(wire, window):
    """count(x) of the definition above, as int64, through the summed-volume
    table S (S[i, j, k] = number of wire voxels with index < (i, j, k)): the box
    sum is the eight-term inclusion-exclusion of S at the clipped corners."""
    w = (np.asarray(wire) != 0).astype(np.int64)
    nz, ny, nx = w.shape
    S = np.zeros((nz + 1, ny + 1, nx + 1), np.int64)
    S[1:, 1:, 1:] = w.cumsum(0).cumsum(1).cumsum(2)
    lo, hi = window_bounds(window)

    def edges(n):
        i = np.arange(n)
        return np.clip(i - lo, 0, n), np.clip(i + hi + 1, 0, n)

    z0, z1 = edges(nz)
    y0, y1 = edges(ny)
    x0, x1 = edges(nx)
    Z0, Y0, X0 = np.ix_(z0, y0, x0)
    Z1, Y1, X1 = np.ix_(z1, y1, x1)
    return (S[Z1, Y1, X1] - S[Z0, Y1, X1] - S[Z1, Y0, X1] - S[Z1, Y1, X0]
            + S[Z0, Y0, X1] + S[Z0, Y1, X0] + S[Z1, Y0, X0] - S[Z0, Y0, X0])


def porosity_average(wire, window, phi_min, flags=None):
    """phi of the definition above: float32 array of the wire's shape."""
    w3 = float(window) ** 3
    phi = ((w3 - wire_count(wire, window)) / w3).astype(np.float32)
    phi = np.maximum(phi, np.float32(phi_min))
    if flags is not None:
        phi[np.asarray(flags) == 0] = np.float32(1.0)
    return phi


def wire_count_at(wire, window, points):
    """count(x) at the given (z, y, x) points, each summed directly over its
    clipped window box (for sampled checks on large boxes)."""
    nz, ny, nx = wire.shape
    lo, hi = window_bounds(window)
    out = np.empty(len(points), np.int64)
    for k, (z, y, x) in enumerate(points):
        box = wire[max(0, z - lo):min(nz, z + hi + 1), max(0, y - lo):min(ny, y + hi + 1),
                   max(0, x - lo):min(nx, x + hi + 1)]
        out[k] = int(np.count_nonzero(box))
    return out
