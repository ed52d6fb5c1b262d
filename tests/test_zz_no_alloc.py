"""emt_prefactor_noalloc against emt_prefactor, through the C ABI.

emt_prefactor_noalloc serves callers that cannot allocate device memory at
the moment they need G^-1 rebuilt: a service that reserved all device memory
up front and hands it out itself, or a loop that cannot take cudaMalloc's
implicit device synchronisation or risk its failure mid-run.  It keeps its
workspace in a fixed array inside the library.  This file runs last on
purpose, so that a run stopping at the first failure has already run every
other test; it must also pass on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1903_01081_b300 import emt, netgen as g

pytestmark = pytest.mark.gpu
TOL = 1e-10


def run(net, n_steps, noalloc, stream=None):
    ctx = emt.emt_build_network(net)
    if noalloc:
        emt.emt_prefactor_noalloc(ctx, stream)
    else:
        emt.emt_prefactor(ctx)
    emt.emt_set_recording(ctx, None, 1, n_steps)
    emt.emt_step_n(ctx, n_steps, stream)
    emt.emt_sync(ctx)
    w = emt.emt_read_waveforms(ctx, np.arange(net.n_nodes, dtype=np.int32), 1, n_steps)[:, 0, :]
    emt.emt_destroy(ctx)
    return w


def rel_err(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def switched_network():
    net = g.multi_subsystem(131, [3, 6, 2, 5, 4], n_lines=8, n_sources=2, dt=20e-6, n_series_extra=2)
    nodes = np.random.default_rng(4).choice(net.n_nodes, size=2, replace=False)
    net.sw_k = nodes.astype(np.int32)
    net.sw_m = np.array([-1, int(nodes[0])], np.int32)
    net.sw_r = np.array([0.05, 1.5])
    net.sw_close_step = np.array([300, 500], np.int64)
    net.sw_open_step = np.array([-1, 900], np.int64)
    return net


def test_noalloc_prefactor_matches_the_allocating_one_on_two_calls_in_a_row():
    # two calls in a row, different networks, so the shared workspace is reused
    for net, n_steps in ((switched_network(), 1200), (g.single_rlc(n_steps=3000), 3000)):
        ref = run(net, n_steps, noalloc=False)
        got = run(net, n_steps, noalloc=True)
        assert rel_err(got, ref) <= TOL


def test_noalloc_prefactor_on_a_caller_stream():
    import torch
    net = switched_network()
    ref = run(net, 1200, noalloc=False)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        got = run(net, 1200, noalloc=True, stream=st)
    assert rel_err(got, ref) <= TOL


def test_noalloc_prefactor_allocates_nothing():
    """After the first call on the device (which only looks up the array's
    address), a call leaves the device's free memory unchanged; the
    allocating prefactor of the same large network needs two workspaces of
    every solve-matrix entry (a few MB) from cudaMalloc."""
    import torch
    net = g.large_scale(n_steps=10)
    ctx = emt.emt_build_network(net)
    emt.emt_prefactor_noalloc(ctx)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    emt.emt_prefactor_noalloc(ctx)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    emt.emt_destroy(ctx)
    assert free1 == free0


def test_noalloc_prefactor_reports_the_singular_subsystem():
    # subsystem of two nodes joined by one branch, neither reaching ground or a source
    b = g.NetworkBuilder()
    b.source(1000.0, 0.0)
    b.branch(g.source_node(0), 0, 0, 1.0)
    b.branch(0, g.GROUND, 0, 5.0)
    b.branch(1, 2, 1, 0.01)
    net = b.build(20e-6, 100)
    for call in (emt.emt_prefactor, emt.emt_prefactor_noalloc):
        ctx = emt.emt_build_network(net)
        with pytest.raises(emt.EmtError) as ei:
            call(ctx)
        assert ei.value.status == emt.EMT_ESINGULAR
        assert "subsystem" in str(ei.value) and "singular" in str(ei.value)
        emt.emt_destroy(ctx)


def test_noalloc_prefactor_rejects_networks_beyond_its_workspace():
    # 40 subsystems of 120 nodes: 40 * 120 * 120 solve-matrix entries > 491,520
    b = g.NetworkBuilder()
    b.source(1000.0, 0.0)
    for s in range(40):
        base = 120 * s
        b.branch(g.source_node(0), base, 0, 1.0)
        for i in range(1, 120):
            b.branch(base + i, base + i - 1, 0, 1.0)
            b.branch(base + i, g.GROUND, 0, 10.0)
    net = b.build(20e-6, 4800)
    ctx = emt.emt_build_network(net)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_prefactor_noalloc(ctx)
    assert ei.value.status == emt.EMT_EINVAL
    assert "workspace" in str(ei.value)
    emt.emt_destroy(ctx)
