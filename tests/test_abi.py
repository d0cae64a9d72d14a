"""The C-ABI library builds, loads and exports every function include/lbm.h
declares; host-only argument handling (no CUDA work) behaves as documented."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2402_10809_gb300 import lbm

    L = lbm.load()
    declared = _declared()
    assert declared, "no declarations found"
    assert declared == set(lbm.SYMBOLS)
    for name in declared:
        assert hasattr(L, name), name


def test_workspace_size_host_logic():
    from paper_2402_10809_gb300 import lbm

    g = lbm.make_grid((32, 32, 64), 19, "f32", (0, 0, 1))
    full = lbm.lbm_workspace_size(g, -1)
    from lbm_inputs import pipe_problem
    import numpy as np

    flags = np.ascontiguousarray(pipe_problem().flags)
    n_list = lbm.lbm_list_length(g, flags.ctypes.data)
    assert n_list == 39424  # a circular cross-section: every row span is all fluid
    tight = lbm.lbm_workspace_size(g, n_list)
    assert full > tight > 2 * 19 * n_list * 4
    g16 = lbm.make_grid((32, 32, 64), 19, "f16dev", (0, 0, 1))
    assert lbm.lbm_workspace_size(g16, 39424) < tight
    bad = lbm.make_grid((32, 32, 64), 20, "f32", (0, 0, 1))
    assert lbm.lbm_workspace_size(bad, 10) == 0
    huge = lbm.make_grid((2048, 2, 2), 19, "f32", (0, 0, 0))
    assert lbm.lbm_workspace_size(huge, 10) == 0


def test_list_length_counts_row_spans():
    """Spans run from the first to the last non-solid cell of each x-row; solid
    cells inside a span count, rows without fluid do not."""
    from paper_2402_10809_gb300 import lbm
    import numpy as np

    flags = np.zeros((3, 4, 10), np.uint8)
    flags[0, 1, 2:5] = 1          # span 3
    flags[1, 2, [1, 7]] = 1       # span 7 (five solid cells inside)
    flags[2, 3, 9] = 3            # span 1
    g = lbm.make_grid((10, 4, 3), 19, "f32", (0, 0, 0))
    assert lbm.lbm_list_length(g, flags.ctypes.data) == 11
    flags[2, 0, 0] = 7            # not a valid flag: not counted
    assert lbm.lbm_list_length(g, flags.ctypes.data) == 11


def test_init_rejects_bad_arguments_before_any_device_work():
    from paper_2402_10809_gb300 import lbm
    from lbm_inputs import pipe_problem

    prob = pipe_problem()
    r, p, b = lbm.make_params(prob.rheology, prob.porous, prob.bc)
    g = lbm.make_grid(prob.dims, 23, "f32", prob.periodic)  # q must be 19 or 27
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_init(g, 1, 1, 0, r, p, b, 256, 1 << 20, 0)
    assert e.value.status == lbm.LBM_EINVAL
    g = lbm.make_grid(prob.dims, 19, "f32", prob.periodic)
    with pytest.raises(lbm.LBMError) as e:  # misaligned workspace
        lbm.lbm_init(g, 1, 1, 0, r, p, b, 257, 1 << 20, 0)
    assert e.value.status == lbm.LBM_EINVAL
    r.mu0 = -1.0
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_init(g, 1, 1, 0, r, p, b, 256, 1 << 20, 0)
    assert e.value.status == lbm.LBM_EINVAL


def test_null_context_calls_are_safe():
    from paper_2402_10809_gb300 import lbm

    L = lbm.load()
    assert L.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert L.lbm_time(None) == -1
    assert L.lbm_state_size(None) == 0
    L.lbm_destroy(None)


def test_porosity_average_host_checks():
    """Workspace size and the argument checks of lbm_porosity_average, all of
    which return before any device work."""
    from paper_2402_10809_gb300 import lbm

    L = lbm.load()
    assert lbm.lbm_porosity_workspace_size(10, 4, 3) == 256 + 256
    assert lbm.lbm_porosity_workspace_size(100, 100, 100) == 1000192 + 2000128
    assert lbm.lbm_porosity_workspace_size(0, 4, 3) == 0
    assert lbm.lbm_porosity_workspace_size(16385, 1, 1) == 0
    ws = lbm.lbm_porosity_workspace_size(8, 8, 8)

    def call(window=3, phi_min=0.05, wire=256, phi=256, work=256, nbytes=ws, dims=(8, 8, 8)):
        return L.lbm_porosity_average(*dims, C.c_void_p(wire), None, window, C.c_float(phi_min),
                                      C.c_void_p(phi), C.c_void_p(work), nbytes, None)

    assert call(window=0) == lbm.LBM_EINVAL
    assert call(window=256) == lbm.LBM_EINVAL
    assert call(phi_min=-0.1) == lbm.LBM_EINVAL
    assert call(phi_min=float("nan")) == lbm.LBM_EINVAL
    assert call(phi_min=1.5) == lbm.LBM_EINVAL
    assert call(wire=0) == lbm.LBM_EINVAL
    assert call(phi=0) == lbm.LBM_EINVAL
    assert call(work=0) == lbm.LBM_EINVAL
    assert call(work=257) == lbm.LBM_EINVAL
    assert call(nbytes=ws - 1) == lbm.LBM_ENOMEM
    assert call(dims=(0, 8, 8)) == lbm.LBM_EINVAL


def test_anisotropy_entry_points_host_checks():
    """lbm_set_anisotropy / lbm_anisotropy_buffer_size without a context: the
    checks that return before any device work."""
    from paper_2402_10809_gb300 import lbm

    L = lbm.load()
    assert L.lbm_anisotropy_buffer_size(None) == 0
    assert L.lbm_set_anisotropy(None, C.c_void_p(256), C.c_void_p(256), 1 << 20, 16, C.c_float(1e-6)) == lbm.LBM_EINVAL
    assert L.lbm_set_anisotropy(None, None, None, 0, 16, C.c_float(1e-6)) == lbm.LBM_EINVAL
