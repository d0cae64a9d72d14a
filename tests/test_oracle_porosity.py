"""Pins of the oracle's volume-averaged porosity (oracle/porosity.py): the
windowed convolution of the voxelised coil with a uniform kernel (Sec. 4,
Table 1 averaging window).

* brute force: the window count summed cell by cell in plain loops on tiny
  boxes, odd and even windows, windows wider than the box;
* orientation: a single wire voxel counts exactly on the box [v - hi, v + lo]
  (an even window is asymmetric, so a swapped lo / hi fails);
* library: scipy.ndimage.uniform_filter (FP64, zero outside) times window^3;
* conservation: a wire away from the faces contributes window^3 to the total;
* the quotient is the correctly rounded FP32 value of (W^3 - c) / W^3 (checked
  with exact rationals), clamped at phi_min; solid cells get 1.
"""

from fractions import Fraction

import numpy as np
import pytest

from oracle.porosity import porosity_average, window_bounds, wire_count, wire_count_at


def brute_count(wire, window):
    nz, ny, nx = wire.shape
    lo, hi = window_bounds(window)
    out = np.zeros(wire.shape, np.int64)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                c = 0
                for k in range(z - lo, z + hi + 1):
                    for j in range(y - lo, y + hi + 1):
                        for i in range(x - lo, x + hi + 1):
                            if 0 <= k < nz and 0 <= j < ny and 0 <= i < nx and wire[k, j, i]:
                                c += 1
                out[z, y, x] = c
    return out


@pytest.mark.parametrize("window", [1, 2, 3, 4, 9])
def test_count_equals_brute_force(window):
    rng = np.random.default_rng(window)
    wire = (rng.random((5, 6, 7)) < 0.3).astype(np.uint8) * rng.integers(1, 256, (5, 6, 7)).astype(np.uint8)
    assert np.array_equal(wire_count(wire, window), brute_count(wire, window))
    pts = [(0, 0, 0), (4, 5, 6), (2, 3, 1)]
    assert np.array_equal(wire_count_at(wire, window, pts), brute_count(wire, window)[tuple(np.array(pts).T)])


@pytest.mark.parametrize("window", [3, 4, 28])
def test_single_voxel_orientation(window):
    n = 40
    v = (17, 11, 23)
    wire = np.zeros((n, n, n), np.uint8)
    wire[v] = 1
    c = wire_count(wire, window)
    lo, hi = window_bounds(window)
    expect = np.zeros_like(c)
    expect[tuple(slice(max(0, c - hi), c + lo + 1) for c in v)] = 1
    assert np.array_equal(c, expect)


@pytest.mark.parametrize("window", [5, 6, 28])
def test_count_equals_uniform_filter(window):
    from scipy.ndimage import uniform_filter

    rng = np.random.default_rng(3)
    wire = (rng.random((30, 33, 35)) < 0.2).astype(np.uint8)
    ref = uniform_filter(wire.astype(np.float64), size=window, mode="constant") * window ** 3
    assert np.abs(wire_count(wire, window) - ref).max() < 1e-6


def test_conservation_away_from_the_faces():
    window, n = 6, 30
    rng = np.random.default_rng(5)
    wire = np.zeros((n, n, n), np.uint8)
    wire[8:22, 8:22, 8:22] = rng.random((14, 14, 14)) < 0.25
    assert wire_count(wire, window).sum() == window ** 3 * int(wire.sum())


def test_quotient_rounding_clamp_and_solid_override():
    window = 28
    w3 = window ** 3
    n = 40
    rng = np.random.default_rng(7)
    wire = (rng.random((n, n, n)) < 0.5).astype(np.uint8)
    wire[2:38, 2:38, 2:38] = 1  # a solid block of wire: count = W^3 deep inside
    c = wire_count(wire, window)
    phi = porosity_average(wire, window, 0.0)
    for v in np.unique(c)[:: max(1, len(np.unique(c)) // 200)]:
        exact = Fraction(int(w3 - v), w3)
        got = phi[c == v][0]
        up = np.nextafter(got, np.float32(2))
        dn = np.nextafter(got, np.float32(-1))
        # no other float32 is closer to the exact quotient
        assert abs(Fraction(float(got)) - exact) <= abs(Fraction(float(up)) - exact)
        assert abs(Fraction(float(got)) - exact) <= abs(Fraction(float(dn)) - exact)
    assert phi.min() == 0.0 and (c == w3).any()
    clamped = porosity_average(wire, window, 0.05)
    assert np.array_equal(clamped, np.maximum(phi, np.float32(0.05)))
    assert clamped.min() == np.float32(0.05)
    flags = np.ones(wire.shape, np.uint8)
    flags[:3] = 0
    withflags = porosity_average(wire, window, 0.05, flags)
    assert np.all(withflags[:3] == 1.0) and np.array_equal(withflags[3:], clamped[3:])
    assert np.all(porosity_average(np.zeros((4, 5, 6), np.uint8), 3, 0.05) == 1.0)
