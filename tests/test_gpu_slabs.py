"""z-slab decomposition on one GPU: the problem split into 2 or 3 slab
contexts with halo planes, faces exchanged after every step, must give the
unsharded run's fields bit for bit (every cell computes the same arithmetic on
the same values) and its diagnostics up to the FP64 order of the sums; the
packed-message path (pack, copy, unpack) must equal the direct exchange."""

import numpy as np
import pytest

from lbm_inputs import aneurysm_problem, periodic_box_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f32", "f16dev"])
@pytest.mark.parametrize("nslabs", [2, 3])
def test_slabs_match_the_unsharded_box(lbm, storage, nslabs):
    from paper_2402_10809_gb300 import slabs

    prob = aneurysm_problem(64, q=27, u0=0.05, period=200.0)
    ref = lbm.Simulation(prob, storage=storage)
    ref.step(120)
    a = ref.moments()
    da = ref.diag(prob.region)
    ref.close()
    sl = slabs.SlabSimulation(prob, nslabs, storage=storage)
    sl.step(120)
    b = sl.moments()
    db = sl.diag(prob.region)
    sl.close()
    for k in ("rho", "u", "gdot", "omega"):
        assert np.array_equal(a[k], b[k]), k
    assert np.allclose(da, db, rtol=1e-12, atol=0.0), (da, db)
    assert da[3] == db[3] and da[7] == db[7] == 0


def test_packed_messages_equal_the_direct_exchange(lbm):
    import torch

    from paper_2402_10809_gb300 import slabs

    prob = aneurysm_problem(48, q=19, u0=0.05, period=100.0)
    direct = slabs.SlabSimulation(prob, 2)  # concurrent slabs, lbm_step_slabs
    packed = slabs.SlabSimulation(prob, 2, concurrent=False)  # one stream, stepped by hand
    lo, hi = packed.sims
    n_up = lbm.lbm_halo_message_size(lo.ctx, 1)
    n_dn = lbm.lbm_halo_message_size(hi.ctx, 0)
    assert n_up > 0 and n_dn > 0
    assert lbm.lbm_halo_message_size(lo.ctx, 0) == 0 and lbm.lbm_halo_message_size(hi.ctx, 1) == 0
    up = torch.empty(n_up, dtype=torch.uint8, device="cuda")
    dn = torch.empty(n_dn, dtype=torch.uint8, device="cuda")
    direct.step(60)
    for _ in range(60):
        lbm.lbm_step(lo.ctx, 1)
        lbm.lbm_step(hi.ctx, 1)
        lbm.lbm_halo_pack(lo.ctx, 1, up.data_ptr())
        lbm.lbm_halo_pack(hi.ctx, 0, dn.data_ptr())
        lbm.lbm_halo_unpack(hi.ctx, 0, up.data_ptr())
        lbm.lbm_halo_unpack(lo.ctx, 1, dn.data_ptr())
    a, b = direct.moments(), packed.moments()
    for k in ("rho", "u", "gdot", "omega"):
        assert np.array_equal(a[k], b[k]), k
    direct.close()
    packed.close()


def test_halo_arguments_are_checked(lbm):
    box = lbm.Simulation(periodic_box_problem(8, 8, 8))
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_set_halo(box.ctx, 1, 0)  # periodic in z
    assert e.value.status == lbm.LBM_EINVAL
    box.close()
    prob = aneurysm_problem(24, q=27, small=True)
    s = lbm.Simulation(prob)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_set_halo(s.ctx, 2, 0)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_halo_pack(s.ctx, 1, 0)  # no halo on that side
    other = lbm.Simulation(aneurysm_problem(24, q=19, small=True))
    lbm.lbm_set_halo(s.ctx, 0, 1)
    lbm.lbm_set_halo(other.ctx, 1, 0)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_halo_exchange(s.ctx, other.ctx)  # different lattices
    with pytest.raises(lbm.LBMError):
        lbm.lbm_step_slabs([s.ctx, other.ctx], 1)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_step_slabs([other.ctx, s.ctx], 1)  # not bottom to top
    s.close()
    other.close()


def test_halo_planes_can_be_restored(lbm):
    """Unsetting the halo planes gives the context back its own masks: the
    box then steps exactly like a fresh one."""
    prob = aneurysm_problem(48, q=27, u0=0.05, period=100.0)
    a = lbm.Simulation(prob)
    b = lbm.Simulation(prob)
    lbm.lbm_set_halo(a.ctx, 1, 1)
    lbm.lbm_set_halo(a.ctx, 0, 1)
    lbm.lbm_set_halo(a.ctx, 0, 0)
    a.step(40)
    b.step(40)
    ma, mb = a.moments(), b.moments()
    for k in ("rho", "u", "gdot", "omega"):
        assert np.array_equal(ma[k], mb[k]), k
    a.close()
    b.close()
