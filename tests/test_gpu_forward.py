"""GPU parity of the single-scenario time loop against the CPU oracle.

Every case runs the CUDA path through the C ABI and the oracle on the same
seeded network and compares all recorded node voltages element by element.
Tolerance: the peak-normalised error
    max_{n,k} |v_gpu - v_oracle| / max_{n,k} |v_oracle|  <=  1e-10,
the bar the method is held to (explicit G^-1 against per-step LU differ only
by rounding, amplified at most by the matrices' condition numbers; G^-1 is
kept as a double plus its single-precision remainder so that the rounded
inverse does not act as a systematically perturbed conductance matrix).
"""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import emt, netgen as g

pytestmark = pytest.mark.gpu
TOL = 1e-10


def gpu_run(net, n_steps, chunks=None, stream=None, options=None):
    sim = emt.Simulator(net, n_steps=n_steps, options=options)
    for c in (chunks or [n_steps]):
        sim.run(c, stream)
    sim.sync()
    w = sim.waveforms()[:, 0, :]
    sim.close()
    return w


def rel_err(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_single_subsystem_config1_full():
    net = g.single_rlc()                     # 12 nodes, fault at step 2000, 20,000 steps
    ref = oracle.simulate(net, net.n_steps)
    got = gpu_run(net, net.n_steps)
    assert got.shape == ref.shape
    assert rel_err(got, ref) <= TOL


def test_three_subsystem_bergeron_toy():
    net = g.multi_subsystem(7, [2, 3, 2], n_lines=5, n_sources=1, dt=20e-6, phases=1,
                            delay_range=(1, 3), n_series_extra=1)
    N = 4000
    assert rel_err(gpu_run(net, N), oracle.simulate(net, N)) <= TOL


@pytest.mark.parametrize("seed", [1, 2])
def test_multi_subsystem_three_phase_with_switches(seed):
    net = g.multi_subsystem(100 + seed, [3, 7, 2, 5, 4, 6, 2, 8, 3, 4], n_lines=18, n_sources=3, dt=20e-6,
                            n_series_extra=4)
    rng = np.random.default_rng(seed)
    nodes = rng.choice(net.n_nodes, size=3, replace=False)
    net.sw_k = nodes.astype(np.int32)
    net.sw_m = np.array([-1, -1, int(nodes[0])], np.int32)
    net.sw_r = np.array([0.01, 0.5, 2.0])
    net.sw_close_step = np.array([500, 800, 1200], np.int64)
    net.sw_open_step = np.array([-1, 1500, 2100], np.int64)
    N = 3000
    assert rel_err(gpu_run(net, N), oracle.simulate(net, N)) <= TOL


def test_large_scale_full_size():
    """The large-scale workload at its full size: 3,000 nodes, ~100
    subsystems, 700 three-phase lines, 50,000 steps; every node, every step."""
    net = g.large_scale()
    N = net.n_steps
    ref = oracle.simulate(net, N)
    got = gpu_run(net, N)
    assert rel_err(got, ref) <= TOL
    per_node = np.max(np.abs(got - ref), axis=0) / np.maximum(np.max(np.abs(ref), axis=0), 1e-300)
    assert np.max(per_node) <= 1e-8


def test_strict_500_subsystems():
    net = g.large_scale(strict_500=True, n_steps=4000)
    N = 4000
    assert rel_err(gpu_run(net, N), oracle.simulate(net, N)) <= TOL


def test_resume_and_reset_are_bitwise_stable():
    net = g.multi_subsystem(9, [4, 5, 3, 6], n_lines=6, n_sources=2, dt=20e-6)
    N = 2500
    a = gpu_run(net, N)
    b = gpu_run(net, N, chunks=[1, 700, 999, 800])
    assert np.array_equal(a, b)
    sim = emt.Simulator(net, n_steps=N)
    sim.run(N)
    first = sim.waveforms().copy()
    sim.reset()
    sim.run(N)
    assert np.array_equal(first, sim.waveforms())
    sim.close()


def test_runs_on_a_torch_stream():
    torch = pytest.importorskip("torch")
    net = g.multi_subsystem(5, [3, 3], n_lines=2, n_sources=1, dt=20e-6)
    N = 500
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got = gpu_run(net, N, stream=s)
    assert rel_err(got, oracle.simulate(net, N)) <= TOL


def test_waveforms_into_device_tensor_and_channel_subset():
    torch = pytest.importorskip("torch")
    net = g.multi_subsystem(6, [3, 4, 2], n_lines=3, n_sources=1, dt=20e-6)
    N = 300
    ch = np.array([7, 2, 11, 0], np.int32)
    sim = emt.Simulator(net, n_steps=N, channels=ch, decim=3)
    sim.run(N)
    out = torch.empty((N // 3, 1, len(ch)), dtype=torch.float64, device="cuda")
    sim.waveforms(out=out)
    ref = oracle.simulate(net, N)[2::3][:, ch]
    assert rel_err(out.cpu().numpy()[:, 0, :], ref) <= TOL
    sim.close()


def test_edge_cases():
    # one node, no lines; n_steps = 0; a subsystem of exactly the maximum size
    b = g.NetworkBuilder()
    b.source(1000.0, 0.1)
    b.branch(g.source_node(0), 0, 1, 0.01)
    b.branch(0, g.GROUND, 2, 1e-5)
    net = b.build(20e-6, 1)
    assert rel_err(gpu_run(net, 200), oracle.simulate(net, 200)) <= TOL
    sim = emt.Simulator(net, n_steps=10)
    sim.run(0)
    assert sim.info("step") == 0
    sim.close()
    b = g.NetworkBuilder()
    b.source(1000.0, 0.0)
    n = 128
    b.branch(g.source_node(0), 0, 0, 2.0)
    rng = np.random.default_rng(3)
    for i in range(1, n):
        kind = int(rng.integers(0, 3))
        b.branch(i, int(rng.integers(0, i)), kind, [1.0, 0.01, 1e-5][kind])
        b.branch(i, g.GROUND, 0, float(rng.uniform(1, 10)))
    net = b.build(20e-6, n)
    assert rel_err(gpu_run(net, 300), oracle.simulate(net, 300)) <= TOL


def test_wait_timeout_is_reported_and_context_stays_usable():
    net = g.multi_subsystem(8, [2, 2, 2], n_lines=3, n_sources=1, dt=20e-6, delay_range=(1, 1))
    sim = emt.Simulator(net, n_steps=100)
    emt.emt_set_option(sim.ctx, "wait_budget_ns", 50_000_000)      # 50 ms
    emt.emt_set_option(sim.ctx, "debug_hold_lines", 0)              # subsystem 0 never sends line values
    sim.run(100)
    with pytest.raises(emt.EmtError) as ei:
        sim.sync()
    assert ei.value.status == emt.EMT_ETIMEOUT
    emt.emt_set_option(sim.ctx, "debug_hold_lines", -1)
    sim.reset()
    sim.run(100)
    sim.sync()
    assert rel_err(sim.waveforms()[:, 0, :], oracle.simulate(net, 100)) <= TOL
    sim.close()


def test_step_before_prefactor_is_a_state_error():
    net = g.single_rlc(n_steps=10)
    ctx = emt.emt_build_network(net)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_step_n(ctx, 5)
    assert ei.value.status == emt.EMT_ESTATE
    emt.emt_destroy(ctx)


def test_singular_network_is_reported():
    b = g.NetworkBuilder()
    b.source(1.0, 0.0)
    b.branch(g.source_node(0), 0, 0, 1.0)
    b.branch(1, 2, 0, 1.0)            # nodes 1, 2 float
    net = b.build(1e-5, 3)
    ctx = emt.emt_build_network(net)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_prefactor(ctx)
    assert ei.value.status == emt.EMT_ESINGULAR
    emt.emt_destroy(ctx)


def test_packed_network_beyond_coresidency():
    """A network of 500 subsystems (16,500 nodes) has more subsystems than
    CTAs the device holds at once: the build packs them several to a CTA
    (block-diagonal solves) and the run matches the oracle, which solves
    each subsystem on its own.  With a surge arrester in every subsystem
    (each keeps a CTA of its own) nothing can be packed, and the step is
    refused before any launch (ERESOURCE), the context staying readable."""
    import torch
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    N = 400
    net = g.paper_scale(500, n_steps=N)
    sim = emt.Simulator(net, n_steps=N)
    n_cta, n_comp = sim.info("n_subsystems"), sim.info("n_components")
    assert n_comp == 500
    assert n_cta < 500 and n_cta <= sim.info("ctas_per_sm") * n_sm
    sim.run(N)
    sim.sync()
    got = sim.waveforms()[:, 0, :]
    sim.close()
    assert rel_err(got, oracle.simulate(net, N)) <= TOL

    locked = g.with_arresters(g.paper_scale(500, n_steps=10), n_arresters=500)
    ctx = emt.emt_build_network(locked)
    try:
        assert emt.emt_get_info(ctx, "n_subsystems") == 500
        if 500 <= emt.emt_get_info(ctx, "ctas_per_sm") * n_sm:
            pytest.skip("this device holds 500 CTAs at once")
        emt.emt_prefactor(ctx)
        with pytest.raises(emt.EmtError, match="co-resident"):
            emt.emt_step_n(ctx, 10)
        assert emt.emt_get_info(ctx, "step") == 0
    finally:
        emt.emt_destroy(ctx)


@pytest.mark.parametrize("decim,chunk", [(1, 700), (3, 1000)])
def test_pipelined_read_to_pinned_host_is_bitwise(decim, chunk):
    """Steps in chunks with each chunk's rows copied to pinned host memory on
    a second stream (emt_read_waveforms_async) give the same rows as one
    run followed by a synchronous read."""
    import torch
    net = g.multi_subsystem(11, [4, 5, 3, 6], n_lines=6, n_sources=2, dt=20e-6)
    N = 4000
    a = emt.Simulator(net, n_steps=N, decim=decim)
    a.run(N)
    a.sync()
    want = a.waveforms()
    a.close()
    b = emt.Simulator(net, n_steps=N, decim=decim)
    out = torch.empty((N // decim, 1, net.n_nodes), dtype=torch.float64, pin_memory=True)
    b.run_to_host(N, out, chunk=chunk)
    b.sync()
    b.close()
    assert np.array_equal(out.numpy(), want)
    assert rel_err(want[:, 0, :], oracle.simulate(net, N)[decim - 1::decim]) <= TOL


@pytest.mark.parametrize("kind", ["single_rlc", "strict_500", "multi"])
def test_warp_per_subsystem_kernel(kind):
    """Networks whose subsystems are all small (at most 32 nodes) with basic
    elements can run one warp per subsystem (option warp_per_subsystem = 1);
    the same runs on the CTA kernel (the default) and both match the
    oracle."""
    if kind == "single_rlc":
        net, N = g.single_rlc(), 20000                     # the 12-node network, its fault at step 2,000
    elif kind == "strict_500":
        net, N = g.large_scale(strict_500=True, n_steps=2000), 2000
    else:
        net, N = g.multi_subsystem(17, [2, 4, 3, 5, 1], n_lines=9, n_sources=2, dt=20e-6, delay_range=(1, 3)), 3000
    ref = oracle.simulate(net, N)
    for warp in (1, 0):
        sim = emt.Simulator(net, n_steps=N)
        assert sim.info("warp_per_subsystem") == 0
        emt.emt_set_option(sim.ctx, "warp_per_subsystem", warp)
        assert sim.info("warp_per_subsystem") == warp
        sim.run(N // 3)
        sim.run(N - N // 3)
        sim.sync()
        w = sim.waveforms()[:, 0, :]
        sim.close()
        assert np.max(np.abs(w - ref)) / np.max(np.abs(ref)) <= 1e-10, warp


def test_warp_per_subsystem_kernel_is_not_used_for_large_subsystems():
    sim = emt.Simulator(g.large_scale(n_steps=10), n_steps=10)
    assert sim.info("warp_per_subsystem") == 0
    with pytest.raises(emt.EmtError):
        emt.emt_set_option(sim.ctx, "warp_per_subsystem", 1)
    sim.close()
