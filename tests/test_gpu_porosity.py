"""lbm_porosity_average (through the C ABI) against the oracle's volume-averaged
porosity (oracle/porosity.py).  The count is exact integer work and the
quotient is correctly rounded on both sides, so the comparison is bit-exact.

Cases: odd and even windows up to 40 cells (the y and z passes keep the
trailing edge of their running sums in a shared-memory ring) and of 60 and
100 cells (the passes that would need a ring over 48 KB re-read it instead),
a window wider than the box,
window 1 (the wire itself), ragged x extents (scalar path), segments along y
and z that end mid-way, unaligned output (scalar path), solid override; the
512^3 box of the coil study at the paper's 28-cell window on sampled cells;
the documented argument errors.
"""

import numpy as np
import pytest

from oracle.porosity import porosity_average, window_bounds, wire_count_at

pytestmark = pytest.mark.gpu


def gpu_phi(lbm, wire, window, phi_min, flags=None, offset=0):
    import torch

    w = torch.from_numpy(wire).cuda()
    f = torch.from_numpy(flags).cuda() if flags is not None else None
    if offset == 0:
        out = lbm.porosity_average(w, window, phi_min, f)
    else:
        nz, ny, nx = wire.shape
        nbytes = lbm.lbm_porosity_workspace_size(nx, ny, nz)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        buf = torch.empty(wire.size + offset, dtype=torch.float32, device="cuda")
        out = buf[offset:].view(wire.shape)
        lbm.lbm_porosity_average(nx, ny, nz, w.data_ptr(), f.data_ptr() if f is not None else 0, window, phi_min,
                                 out.data_ptr(), ws.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [
    ((24, 24, 24), 28, 0.05, 0.3, False),
    ((37, 19, 23), 5, 0.0, 0.4, True),
    ((64, 48, 40), 6, 0.05, 0.2, False),
    ((130, 70, 90), 28, 0.05, 0.3, True),
    ((16, 8, 12), 1, 0.0, 0.5, False),
    ((3, 2, 1), 2, 0.1, 0.5, True),
    ((200, 3, 130), 9, 0.2, 0.6, False),
    ((96, 70, 300), 32, 0.05, 0.02, True),   # long z: several running-sum segments per line
    ((70, 45, 60), 40, 0.05, 0.3, True),
    ((68, 40, 33), 33, 0.0, 0.1, False),
    ((40, 36, 70), 60, 0.05, 0.3, True),     # z pass without the ring (its ring would exceed 48 KB)
    ((44, 30, 20), 100, 0.0, 0.3, False),    # neither pass with the ring
]


@pytest.mark.parametrize("dims,window,phi_min,density,with_flags", CASES)
def test_matches_oracle_exactly(lbm, dims, window, phi_min, density, with_flags):
    nx, ny, nz = dims
    rng = np.random.default_rng(nx * 7 + window)
    wire = ((rng.random((nz, ny, nx)) < density) * rng.integers(1, 256, (nz, ny, nx))).astype(np.uint8)
    flags = (rng.random((nz, ny, nx)) < 0.8).astype(np.uint8) if with_flags else None
    ref = porosity_average(wire, window, phi_min, flags)
    got = gpu_phi(lbm, wire, window, phi_min, flags)
    assert got.dtype == np.float32 and np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("window", [6, 36])
def test_unaligned_output(lbm, window):
    """An output pointer off the 16-byte grid takes the scalar form of the passes."""
    rng = np.random.default_rng(11)
    wire = (rng.random((20, 12, 32)) < 0.3).astype(np.uint8)
    ref = porosity_average(wire, window, 0.05)
    assert np.array_equal(gpu_phi(lbm, wire, window, 0.05, offset=1), ref)


def test_coil_study_box_sampled(lbm):
    """512^3 at the 28-cell window, the launch configuration of the coil study:
    4096 random cells plus the corners and face centres, each counted directly
    by the oracle."""
    n, window, phi_min = 512, 28, 0.05
    rng = np.random.default_rng(2)
    wire = np.zeros((n, n, n), np.uint8)
    wire[150:380, 200:440, 100:330] = rng.random((230, 240, 230)) < 0.25
    flags = np.ones((n, n, n), np.uint8)
    flags[:, :, :3] = 0
    got = gpu_phi(lbm, wire, window, phi_min, flags)
    pts = rng.integers(0, n, (4096, 3))
    edge = [0, n // 2, n - 1]
    pts = np.concatenate([pts, np.array([(a, b, c) for a in edge for b in edge for c in edge])])
    w3 = float(window) ** 3
    c = wire_count_at(wire, window, [tuple(p) for p in pts])
    ref = np.maximum(((w3 - c) / w3).astype(np.float32), np.float32(phi_min))
    ref[flags[tuple(pts.T)] == 0] = 1.0
    assert np.array_equal(got[tuple(pts.T)], ref)
    # every cell: phi in [phi_min, 1], and 1 wherever the window holds no wire
    assert got.min() >= np.float32(phi_min) and got.max() <= 1.0
    lo, hi = window_bounds(window)
    assert np.all(got[:150 - hi] == 1.0) and np.all(got[380 + lo:] == 1.0)


def test_argument_errors(lbm):
    import torch

    w = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
    for window, phi_min in ((0, 0.05), (256, 0.05), (3, -1.0)):
        with pytest.raises(lbm.LBMError) as e:
            lbm.porosity_average(w, window, phi_min)
        assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(ValueError):
        lbm.porosity_average(w.float(), 3, 0.05)
