"""CUDA graphs of time steps (lbm_step on a problem without a velocity
inlet replays captured graphs of 32 steps): the state must equal, byte for
byte, the same steps launched one call at a time (lbm_step(ctx, 1) never
uses a graph).  Covers both starting buffers (an odd step first), instability
checks that cut the runs into pieces, and a change of the step's parameters
(the anisotropic solve switched on) between runs, after which the graphs
must be captured again."""

import numpy as np
import pytest

from lbm_inputs import coil_shape_tensor, periodic_box_problem, pipe_problem

pytestmark = pytest.mark.gpu


def one_by_one(lbm, prob, schedule, check=0, shape_after=None, storage="f32"):
    sim = lbm.Simulation(prob, storage=storage)
    if check:
        lbm.lbm_set_check(sim.ctx, check)
    for k, n in enumerate(schedule):
        if shape_after is not None and k == shape_after[0]:
            sim.set_anisotropy(shape_after[1])
        for _ in range(n):
            sim.step(1)
    state = sim.save()
    sim.close()
    return state


def batched(lbm, prob, schedule, check=0, shape_after=None, storage="f32"):
    sim = lbm.Simulation(prob, storage=storage)
    if check:
        lbm.lbm_set_check(sim.ctx, check)
    for k, n in enumerate(schedule):
        if shape_after is not None and k == shape_after[0]:
            sim.set_anisotropy(shape_after[1])
        sim.step(n)
    assert sim.t == sum(schedule)
    state = sim.save()
    sim.close()
    return state


@pytest.mark.parametrize("storage", ["f32", "f16dev"])
def test_graphs_equal_single_launches_pipe(lbm, storage):
    prob = pipe_problem(q=19)
    schedule = [200, 1, 70, 33]  # even and odd starting buffers, remainders
    a = one_by_one(lbm, prob, schedule, storage=storage)
    b = batched(lbm, prob, schedule, storage=storage)
    assert np.array_equal(a, b), f"first differing byte {int(np.argmax(a != b))}"


def test_graphs_with_checks(lbm):
    prob = pipe_problem(q=19)
    a = one_by_one(lbm, prob, [150], check=40)
    b = batched(lbm, prob, [150], check=40)
    assert np.array_equal(a, b)


def test_graphs_recaptured_after_a_parameter_change(lbm):
    rng = np.random.default_rng(3)
    phi = rng.uniform(0.6, 1.0, (16, 16, 16)).astype(np.float32)
    prob = periodic_box_problem(16, 16, 16, q=27, body_force=(2e-5, 0.0, 0.0), obstacles=20, seed=1, phi=phi)
    shape = coil_shape_tensor(prob.flags.shape, ratio=4.0, seed=2)
    a = one_by_one(lbm, prob, [64, 64], shape_after=(1, shape))
    b = batched(lbm, prob, [64, 64], shape_after=(1, shape))
    assert np.array_equal(a, b)
