"""Pins of the oracles' velocity sets against the isotropy conditions every
lattice with c_s^2 = 1/3 must satisfy (Sec. 3: D3Q27 with c_s = 1/sqrt(3);
D3Q19 for the 19-velocity workload)."""

import itertools

import numpy as np
import pytest

from lbm_inputs import periodic_box_problem
from oracle.oracle import Oracle
from oracle.torch_ref import velocity_set


def _tables(q, which):
    if which == "c":
        o = Oracle(periodic_box_problem(2, 2, 2, q=q))
        c, w, opp = o.lattice()
        o.close()
        return c.astype(float), w, opp
    c, w, opp = velocity_set(q)
    return c.astype(float), w, opp


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("which", ["c", "torch"])
def test_isotropy(q, which):
    c, w, opp = _tables(q, which)
    assert len(w) == q
    assert len({tuple(v) for v in c.astype(int)}) == q
    cs2 = 1.0 / 3.0
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(w @ c).max() < 1e-15
    d = np.eye(3)
    for a, b in itertools.product(range(3), repeat=2):
        assert abs((w * c[:, a] * c[:, b]).sum() - cs2 * d[a, b]) < 1e-15
    for a, b, g in itertools.product(range(3), repeat=3):
        assert abs((w * c[:, a] * c[:, b] * c[:, g]).sum()) < 1e-15
    for a, b, g, h in itertools.product(range(3), repeat=4):
        ref = cs2 * cs2 * (d[a, b] * d[g, h] + d[a, g] * d[b, h] + d[a, h] * d[b, g])
        assert abs((w * c[:, a] * c[:, b] * c[:, g] * c[:, h]).sum() - ref) < 1e-15
    for i in range(q):
        assert np.array_equal(c[opp[i]], -c[i])
        assert w[opp[i]] == w[i]


def test_d3q27_is_tensor_product_of_d1q3():
    """D3Q27 weights are the product of the 1-D weights (2/3, 1/6, 1/6)."""
    c, w, _ = _tables(27, "c")
    w1 = {0: 2 / 3, 1: 1 / 6, -1: 1 / 6}
    for ci, wi in zip(c.astype(int), w):
        assert abs(wi - w1[ci[0]] * w1[ci[1]] * w1[ci[2]]) < 1e-16
