"""The multi-scenario solve in digit form on the bf16 tensor cores
(option digit_solve): for a subsystem whose matrix a whole scenario tile
shares, V = X [i^(1) .. i^(S_t)] as exact products of base-256 digits
(emt_digits.cuh), one rounding to double per entry.

Held to the oracle (peak-normalised 1e-10) on the shared-G study, where
the faulted subsystem's matrices differ per scenario after the fault (so
they stay on the FP64 path beside the digit ones), on an N-1 study, and
over the full 10,000-step shared-G run for drift; against the FP64 path of
the same set.
"""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import emt, netgen as g

pytestmark = pytest.mark.gpu
TOL = 1e-10


def rel_err(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def run(net, sc, n_steps, digit, decim=1, shape=None, min_rows=1):
    """min_rows=1: every shared matrix in digit form (the default leaves
    subsystems below 24 rows on the FP64 path)."""
    ctx = emt.emt_build_network(net, sc)
    emt.emt_prefactor(ctx)
    if shape:
        emt.emt_set_option(ctx, "scenarios_per_cta", shape[0])
        emt.emt_set_option(ctx, "batch_threads", shape[1])
    emt.emt_set_option(ctx, "digit_solve", digit)
    if min_rows is not None:
        emt.emt_set_option(ctx, "digit_min_rows", min_rows)
    info = {k: emt.emt_get_info(ctx, k) for k in ("digit_solve", "digit_matrices", "scenarios_per_cta")}
    emt.emt_set_recording(ctx, None, decim, n_steps // decim)
    emt.emt_step_n(ctx, n_steps)
    emt.emt_sync(ctx)
    w = emt.emt_read_waveforms(ctx, np.arange(net.n_nodes, dtype=np.int32), decim, n_steps // decim, 0,
                               sc.n_scenarios)
    emt.emt_destroy(ctx)
    return w, info


def test_shared_g_small_matches_the_oracle_and_the_fp64_path():
    base = g.multi_subsystem(91, [3, 5, 2, 4, 6], n_lines=9, n_sources=3, dt=20e-6, n_series_extra=2)
    net, sc = g.shared_g(seed=92, n_scenarios=40, n_steps=1500, fault_step=500, base=base)
    N = 1500
    got, info = run(net, sc, N, 1)
    assert info["digit_solve"] == 1 and info["digit_matrices"] > 0
    ref64, info0 = run(net, sc, N, 0)
    assert info0["digit_solve"] == 0
    for s in (0, 17, 39):
        ref = oracle.simulate(sc.expand(net, s), N)
        assert rel_err(got[:, s, :], ref) <= TOL, s
    assert rel_err(got, ref64) <= TOL


def test_n1_contingency_mixes_digit_and_fp64_subsystems():
    net, sc = g.n1_contingency(seed=77, n_scenarios=48, n_buses=40, n_sub=8, n_lines=12, n_sources=3,
                               n_steps=1500, fault_step=500, target_branches=240)
    N = 1500
    got, info = run(net, sc, N, 1)
    assert info["digit_matrices"] > 0
    for s in (0, 23, 47):
        ref = oracle.simulate(sc.expand(net, s), N)
        assert rel_err(got[:, s, :], ref) <= TOL, s


@pytest.mark.parametrize("shape", [(16, 512), (28, 1024), (7, 256)])
def test_launch_shapes(shape):
    base = g.multi_subsystem(91, [3, 5, 2, 4, 6], n_lines=9, n_sources=3, dt=20e-6, n_series_extra=2)
    net, sc = g.shared_g(seed=92, n_scenarios=40, n_steps=600, fault_step=200, base=base)
    got, info = run(net, sc, 600, 1, shape=shape)
    assert info["scenarios_per_cta"] == shape[0]
    ref64, _ = run(net, sc, 600, 0, shape=shape)
    assert rel_err(got, ref64) <= TOL


def test_shared_g_full_length_sampled_scenarios():
    """The 3,000-node network, 10,000 steps across the fault at step 2,500,
    64 scenarios; four compared with the oracle at every 10th step."""
    net, sc = g.shared_g(n_scenarios=64)
    N = net.n_steps
    got, info = run(net, sc, N, 1, decim=10, min_rows=None)   # the default split between the two paths
    assert info["digit_solve"] == 1
    for s in (0, 21, 42, 63):
        ref = oracle.simulate(sc.expand(net, s), N)[9::10]
        assert rel_err(got[:, s, :], ref) <= TOL, s


def test_min_rows_option_range():
    base = g.multi_subsystem(91, [3, 5, 2, 4, 6], n_lines=9, n_sources=3, dt=20e-6, n_series_extra=2)
    net, sc = g.shared_g(seed=92, n_scenarios=40, n_steps=100, fault_step=50, base=base)
    ctx = emt.emt_build_network(net, sc)
    assert emt.emt_get_info(ctx, "digit_min_rows") == 24
    for bad in (0, 65):
        with pytest.raises(emt.EmtError) as ei:
            emt.emt_set_option(ctx, "digit_min_rows", bad)
        assert ei.value.status == emt.EMT_EINVAL
    emt.emt_destroy(ctx)


def test_option_is_for_scenario_sets_only():
    ctx = emt.emt_build_network(g.single_rlc(n_steps=10))
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_set_option(ctx, "digit_solve", 1)
    assert ei.value.status == emt.EMT_EINVAL
    emt.emt_destroy(ctx)
