"""lbm_diag_noalloc: the diagnostics entry point for callers that cannot
allocate device memory where they need the numbers (for example a monitoring
thread whose device allocator belongs to another framework).  It must give the
same diagnostics as lbm_diag, which reduces in the caller's workspace, on
consecutive calls, and refuse contexts beyond its fixed capacity.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""

import numpy as np
import pytest

from lbm_inputs import aneurysm_problem, periodic_box_problem

pytestmark = pytest.mark.gpu


def _close(a, b):
    # the two paths run the same kernels in the same order: expect equality,
    # allow the FP64 round-off of a reordering anyway
    assert a[3] == b[3] and a[7] == b[7]
    assert np.allclose(a, b, rtol=1e-12, atol=0.0), (a, b)


def test_noalloc_diag_matches_workspace_diag_twice(lbm):
    import torch

    prob = aneurysm_problem(64, q=27, u0=0.05, period=200.0)
    sim = lbm.Simulation(prob, storage="f32")
    region = torch.from_numpy(np.ascontiguousarray(prob.region)).cuda()
    sim.step(60)
    ref1 = lbm.lbm_diag(sim.ctx, region.data_ptr(), 1)
    got1 = lbm.lbm_diag_noalloc(sim.ctx, region.data_ptr())
    _close(got1, ref1)
    assert ref1[3] > 0 and ref1[2] > 0
    sim.step(25)
    got2 = lbm.lbm_diag_noalloc(sim.ctx, region.data_ptr())
    ref2 = lbm.lbm_diag(sim.ctx, region.data_ptr(), 1)
    _close(got2, ref2)
    assert not np.array_equal(got1, got2)  # the state moved on; nothing stale returned
    got3 = lbm.lbm_diag_noalloc(sim.ctx, None)
    ref3 = lbm.lbm_diag(sim.ctx, None, 0)
    _close(got3, ref3)


def test_noalloc_diag_limits(lbm):
    import torch

    prob = aneurysm_problem(24, q=19, small=True, u0=0.05, period=100.0)
    sim = lbm.Simulation(prob, storage="f16dev")
    sim.step(10)
    host_region = np.ascontiguousarray(prob.region)
    with pytest.raises(lbm.LBMError) as e:  # host regions would need scratch to copy
        lbm.lbm_diag_noalloc(sim.ctx, host_region.ctypes.data)
    assert e.value.status == lbm.LBM_EINVAL
    big = periodic_box_problem(212, 210, 190, q=19)  # 8,458,800 cells > 8,388,608
    simb = lbm.Simulation(big, storage="f16dev")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_diag_noalloc(simb.ctx, None)
    assert e.value.status == lbm.LBM_EINVAL
    assert "at most 8388608" in str(e.value)
    d = lbm.lbm_diag(simb.ctx, None, 0)  # the workspace path still serves it
    assert d[7] == 0
