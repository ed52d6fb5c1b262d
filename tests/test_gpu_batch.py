"""GPU parity of the multi-scenario path against the CPU oracle.

Each scenario of a set is written out as a plain network (removed elements
dropped, fault switches added, sources overridden) and run by the oracle;
the batched CUDA run of the whole set must match every checked scenario to
the same peak-normalised 1e-10 as the single-network path.
"""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import emt, netgen as g

pytestmark = pytest.mark.gpu
TOL = 1e-10


def rel_err(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def batch_run(net, sc, n_steps, channels=None, decim=1, check=None):
    sim = emt.Simulator(net, sc, n_steps=n_steps, channels=channels, decim=decim)
    sim.run(n_steps)
    sim.sync()
    out = {}
    for s in (range(sc.n_scenarios) if check is None else check):
        out[s] = sim.waveforms(scen0=s, n_scen=1)[:, 0, :]
    info = {k: sim.info(k) for k in ("n_scenarios", "n_matrix_variants", "scenarios_per_cta")}
    sim.close()
    return out, info


def test_small_n1_contingency_all_scenarios():
    net, sc = g.n1_contingency(seed=77, n_scenarios=12, n_buses=40, n_sub=8, n_lines=12, n_sources=3,
                               n_steps=1500, fault_step=500, target_branches=240)
    N = 1500
    got, info = batch_run(net, sc, N)
    assert info["n_scenarios"] == 12 and info["n_matrix_variants"] > 8
    for s in range(12):
        ref = oracle.simulate(sc.expand(net, s), N)
        assert rel_err(got[s], ref) <= TOL, s


def test_small_shared_g_all_scenarios():
    base = g.multi_subsystem(91, [3, 5, 2, 4, 6], n_lines=9, n_sources=3, dt=20e-6, n_series_extra=2)
    net, sc = g.shared_g(seed=92, n_scenarios=10, n_steps=1200, fault_step=400, base=base)
    N = 1200
    got, info = batch_run(net, sc, N)
    for s in range(10):
        ref = oracle.simulate(sc.expand(net, s), N)
        assert rel_err(got[s], ref) <= TOL, s


def test_one_scenario_set_equals_the_plain_network():
    net = g.multi_subsystem(93, [4, 3, 5], n_lines=5, n_sources=2, dt=20e-6)
    sc = g.Scenarios(n_scenarios=1)
    N = 800
    got, _ = batch_run(net, sc, N)
    assert rel_err(got[0], oracle.simulate(net, N)) <= TOL


def test_scenario_tiles_with_a_ragged_tail():
    # 300 scenarios: tiles of 2, the last tile holds a ragged count only if S_t does not divide S
    net, sc = g.n1_contingency(seed=78, n_scenarios=300, n_buses=30, n_sub=6, n_lines=8, n_sources=2,
                               n_steps=600, fault_step=200, target_branches=180)
    N = 600
    check = [0, 1, 149, 298, 299]
    got, info = batch_run(net, sc, N, check=check)
    for s in check:
        assert rel_err(got[s], oracle.simulate(sc.expand(net, s), N)) <= TOL, s


def test_n1_full_size_sampled_scenarios():
    """1,024 N-1 scenarios of the 200-bus network, 10,000 steps, in one launch;
    sixteen scenarios checked against the oracle on every 10th step."""
    net, sc = g.n1_contingency()
    N = net.n_steps
    rng = np.random.default_rng(5)
    check = sorted(rng.choice(sc.n_scenarios, size=16, replace=False).tolist())
    got, info = batch_run(net, sc, N, decim=10, check=check)
    assert info["n_scenarios"] == 1024
    for s in check:
        ref = oracle.simulate(sc.expand(net, s), N)[9::10]
        assert rel_err(got[s], ref) <= TOL, s


def test_shared_g_full_length_sampled_scenarios():
    """The shared-G study at its stated network and length: the 3,000-node
    large-scale network, 10,000 steps across the fault at step 2,500, the
    first 256 of its scenarios (scenario s is the same whatever the count) in
    one launch of the autotuned shape.  Four seeded scenarios are compared
    with the oracle on all 3,000 nodes at every 10th step, so a drift over the
    long recursion shows."""
    net, sc = g.shared_g(n_scenarios=256)
    N = net.n_steps
    assert N == 10000 and net.n_nodes == 3000
    rng = np.random.default_rng(6)
    check = sorted({0, 255} | set(rng.choice(np.arange(1, 255), size=2, replace=False).tolist()))
    sim = emt.Simulator(net, sc, n_steps=N, decim=10)
    emt.emt_autotune(sim.ctx, 20)
    sim.run(N)
    sim.sync()
    for s in check:
        got = sim.waveforms(scen0=s, n_scen=1)[:, 0, :]
        assert got.shape == (N // 10, net.n_nodes)
        ref = oracle.simulate(sc.expand(net, s), N)[9::10]
        assert rel_err(got, ref) <= TOL, s
    sim.close()


def run_shape(net, sc, N, shape=None, graph=True, autotune=0):
    ctx = emt.emt_build_network(net, sc)
    emt.emt_prefactor(ctx)
    if not graph:
        emt.emt_set_option(ctx, "batch_graph", 0)
    if shape:
        emt.emt_set_option(ctx, "scenarios_per_cta", shape[0])
        emt.emt_set_option(ctx, "batch_threads", shape[1])
    if autotune:
        emt.emt_autotune(ctx, autotune)
        assert emt.emt_get_info(ctx, "autotuned") == 1
        assert emt.emt_get_info(ctx, "step") == 0
    emt.emt_set_recording(ctx, None, 1, N)
    emt.emt_step_n(ctx, N // 2)
    emt.emt_step_n(ctx, N - N // 2)
    emt.emt_sync(ctx)
    w = emt.emt_read_waveforms(ctx, np.arange(net.n_nodes, dtype=np.int32), 1, N, 0, sc.n_scenarios)
    info = {k: emt.emt_get_info(ctx, k) for k in ("scenarios_per_cta", "batch_threads", "batch_groups",
                                                  "graph_launches")}
    emt.emt_destroy(ctx)
    return w, info


def test_launch_shapes_graph_and_autotune_give_identical_results():
    """Every (node, scenario) item runs the same arithmetic whatever the
    tile, block size or launch route, so the results are bit-identical."""
    net, sc = g.n1_contingency(seed=80, n_scenarios=45, n_buses=40, n_sub=8, n_lines=12, n_sources=3,
                               n_steps=700, fault_step=300, target_branches=240)
    N = 700
    ref, info = run_shape(net, sc, N)
    assert info["graph_launches"] == 2
    for shape in ((1, 256), (3, 1024), (7, 512), (16, 256), (32, 1024)):
        w, info = run_shape(net, sc, N, shape)
        assert info["scenarios_per_cta"] == shape[0] and info["batch_threads"] == shape[1]
        assert np.array_equal(w, ref), shape
    w, info = run_shape(net, sc, N, graph=False)
    assert info["graph_launches"] == 0 and np.array_equal(w, ref)
    w, info = run_shape(net, sc, N, autotune=20)
    assert np.array_equal(w, ref)
    for s in (0, 22, 44):
        assert rel_err(ref[:, s, :], oracle.simulate(sc.expand(net, s), N)) <= TOL, s


def test_small_shared_memory_budget_splits_subsystems_into_groups():
    # 32 scenarios per CTA of a 3,000-node network cannot hold one group
    net, sc = g.shared_g(seed=94, n_scenarios=64, n_steps=300, fault_step=100)
    N = 300
    w, info = run_shape(net, sc, N, (32, 1024))
    assert info["batch_groups"] > 1
    for s in (0, 63):
        assert rel_err(w[:, s, :], oracle.simulate(sc.expand(net, s), N)) <= TOL, s


def test_launch_shape_options_are_checked():
    net, sc = g.n1_contingency(seed=81, n_scenarios=4, n_buses=20, n_sub=4, n_lines=5, n_sources=2,
                               n_steps=100, fault_step=50, target_branches=120)
    ctx = emt.emt_build_network(net, sc)
    for key, val in (("batch_threads", 100), ("batch_threads", 2048), ("scenarios_per_cta", 0)):
        with pytest.raises(emt.EmtError) as ei:
            emt.emt_set_option(ctx, key, val)
        assert ei.value.status == emt.EMT_EINVAL
    emt.emt_destroy(ctx)
    ctx = emt.emt_build_network(g.single_rlc(n_steps=10))
    with pytest.raises(emt.EmtError):
        emt.emt_set_option(ctx, "scenarios_per_cta", 4)
    emt.emt_destroy(ctx)


def test_pipelined_read_of_a_scenario_set():
    """run_to_host on a scenario set (every scenario, decimated rows) equals
    the synchronous read of the same run."""
    import torch
    net, sc = g.n1_contingency(n_scenarios=12, n_buses=40, n_sub=8, n_lines=12, n_sources=3, n_steps=3000,
                               target_branches=240)
    N, decim = 3000, 4
    a = emt.Simulator(net, sc, n_steps=N, decim=decim)
    a.run(N)
    a.sync()
    want = a.waveforms()
    a.close()
    b = emt.Simulator(net, sc, n_steps=N, decim=decim)
    out = torch.empty((N // decim, 12, net.n_nodes), dtype=torch.float64, pin_memory=True)
    b.run_to_host(N, out, chunk=900)
    b.close()
    assert np.array_equal(out.numpy(), want)
