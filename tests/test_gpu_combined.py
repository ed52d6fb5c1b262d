"""All network features in one run: Bergeron lines, coupled three-phase lines,
frequency-dependent lines, runtime switches (diodes, a breaker), scheduled
switches, nonlinear resistors and control blocks with controlled
injections, against the oracle over several launches."""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import emt, netgen as g

pytestmark = pytest.mark.gpu


def combined_network():
    base = g.multi_subsystem(31, [5, 4, 6, 3, 5], n_lines=8, n_sources=3, dt=2.0 ** -16)
    coupled = g.with_coupled_lines(base)                 # every three-phase line becomes a coupled line
    net = g.with_converter_controls(coupled, n_converters=4)
    net = g.with_rectifier_loads(net, n_rectifiers=3, n_breakers=1, trip_range=(300, 600))
    net = g.with_arresters(net, n_arresters=3)
    sub, n_sub = oracle.partition(net)
    rng = np.random.default_rng(5)
    # three frequency-dependent lines and one plain Bergeron line between subsystems
    pairs = []
    while len(pairs) < 4:
        a, b = rng.choice(base.n_nodes, size=2, replace=False)
        if sub[a] != sub[b]:
            pairs.append((int(a), int(b)))
    fb = g.NetworkBuilder()
    for (a, b), tau in zip(pairs[:3], (3.5, 9.0, 1.25)):
        fb.fd_line(a, b, tau * net.dt, 1 / 310.0, yq=[-5e3], yc=[1e3 / 310], a0=0.1, ap=[-4e3, -6e4],
                   ar=[0.5 * 4e3, 0.3 * 6e4])
    fd = fb.build(net.dt, 0)
    for f in ("fl_k", "fl_m", "fl_tau", "fl_y0", "fl_ny", "fl_yq", "fl_yc", "fl_a0", "fl_na", "fl_ap", "fl_ar"):
        setattr(net, f, getattr(fd, f))
    a, b = pairs[3]
    net.ln_k = np.array([a], np.int32)
    net.ln_m = np.array([b], np.int32)
    net.ln_zc = np.array([280.0])
    net.ln_delay = np.array([4], np.int32)
    net.sw_k = np.array([int(base.meta["bus_nodes"][2][0])], np.int32)
    net.sw_m = np.array([g.GROUND], np.int32)
    net.sw_r = np.array([5.0])
    net.sw_close_step = np.array([700], np.int64)
    net.sw_open_step = np.array([1400], np.int64)
    return net


def test_all_features_together():
    net = combined_network()
    assert net.n_coupled_lines > 0 and net.n_fd_lines == 3 and net.n_lines == 1
    assert net.n_runtime_switches == 4 and net.n_control_blocks == 96 and net.n_switches == 1
    assert net.n_nonlinear == 3
    N = 2400
    ref = oracle.simulate(net, N)
    # no diode decision within rounding of its threshold on the oracle's run
    node = lambda x: ref[:, x] if x >= 0 else np.zeros(N)
    for w in range(net.n_runtime_switches):
        if net.rs_kind[w] == 0:
            va, vb = node(int(net.rs_k[w])), node(int(net.rs_m[w]))
            sc = np.maximum(np.abs(va), np.abs(vb))
            ok = sc > 0
            assert np.min(np.abs(va - vb)[ok] / sc[ok]) > 1e-9
    sim = emt.Simulator(net, n_steps=N)
    for c in (700, 1, 699, 1000):
        sim.run(c)
    sim.sync()
    got = sim.waveforms()[:, 0, :]
    y = sim.controls()
    sim.close()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-10
    yr = oracle.controls(net, N)[-1]
    assert np.max(np.abs(y - yr)) <= 1e-9 * np.max(np.abs(yr))


def test_packed_network_with_controls_and_arresters():
    """A 400-subsystem network with converter controls and surge arresters
    (their subsystems keep CTAs of their own): the controls' shared memory
    leaves room for two CTAs per SM, fewer than the subsystems, so the build
    packs the others several to a CTA; against the oracle."""
    import torch
    N = 300
    base = g.paper_scale(400, n_steps=N)
    net = g.with_arresters(g.with_converter_controls(base, n_converters=100), n_arresters=40)
    sim = emt.Simulator(net, n_steps=N)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    assert sim.info("n_components") == 400
    assert sim.info("n_subsystems") < 400 and sim.info("n_subsystems") <= sim.info("ctas_per_sm") * n_sm
    sim.run(N)
    sim.sync()
    got = sim.waveforms()[:, 0, :]
    sim.close()
    ref = oracle.simulate(net, N)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
