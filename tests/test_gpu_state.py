"""emt_save_state / emt_load_state: a run resumed in a new context from a
saved state continues bit for bit as the uninterrupted run."""
import numpy as np
import pytest

from paper_1903_01081_b300 import emt, netgen as g
from test_gpu_combined import combined_network

pytestmark = pytest.mark.gpu


def straight(net, N, sc=None):
    ctx = emt.emt_build_network(net, sc)
    emt.emt_prefactor(ctx)
    emt.emt_set_recording(ctx, None, 1, N)
    emt.emt_step_n(ctx, N)
    emt.emt_sync(ctx)
    S = 1 if sc is None else sc.n_scenarios
    w = emt.emt_read_waveforms(ctx, np.arange(net.n_nodes, dtype=np.int32), 1, N, 0, S)
    emt.emt_destroy(ctx)
    return w


def resumed(net, N, half, sc=None):
    a = emt.emt_build_network(net, sc)
    emt.emt_prefactor(a)
    emt.emt_step_n(a, half)
    emt.emt_sync(a)
    state = emt.emt_save_state(a)
    emt.emt_destroy(a)
    b = emt.emt_build_network(net, sc)
    emt.emt_prefactor(b)
    emt.emt_set_recording(b, None, 1, N)
    emt.emt_load_state(b, state)
    assert emt.emt_get_info(b, "step") == half
    emt.emt_step_n(b, N - half)
    emt.emt_sync(b)
    S = 1 if sc is None else sc.n_scenarios
    w = emt.emt_read_waveforms(b, np.arange(net.n_nodes, dtype=np.int32), half + 1, N - half, 0, S)
    emt.emt_destroy(b)
    return w


def test_resume_with_every_feature():
    net = combined_network()
    N, half = 2000, 1137
    assert np.array_equal(resumed(net, N, half), straight(net, N)[half:])


def test_resume_with_states_factorised_at_run_time():
    base = g.multi_subsystem(41, [3, 5, 4], n_lines=4, n_sources=2, dt=20e-6)
    net = g.with_converter_stations(base, n_stations=1)
    N, half = 3000, 1500
    assert np.array_equal(resumed(net, N, half), straight(net, N)[half:])


def test_resume_of_a_scenario_set():
    net, sc = g.n1_contingency(seed=77, n_scenarios=12, n_buses=40, n_sub=8, n_lines=12, n_sources=3,
                               n_steps=1500, fault_step=500, target_branches=240)
    N, half = 1500, 700
    assert np.array_equal(resumed(net, N, half, sc), straight(net, N, sc)[half:])


def test_state_is_checked_against_the_context():
    net = combined_network()
    a = emt.emt_build_network(net)
    emt.emt_prefactor(a)
    emt.emt_step_n(a, 10)
    state = emt.emt_save_state(a)
    other = emt.emt_build_network(g.single_rlc(n_steps=10))
    emt.emt_prefactor(other)
    for bad in (state[:100], np.zeros_like(state)):
        with pytest.raises(emt.EmtError) as ei:
            emt.emt_load_state(a, bad)
        assert ei.value.status == emt.EMT_EINVAL
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_load_state(other, state)
    assert ei.value.status == emt.EMT_EINVAL and "another network" in str(ei.value)
    fresh = emt.emt_build_network(net)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_load_state(fresh, state)
    assert ei.value.status == emt.EMT_ESTATE
    for c in (a, other, fresh):
        emt.emt_destroy(c)
