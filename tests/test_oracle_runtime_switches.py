"""Pins of the oracle's runtime switches (two-state resistors whose state
in force at step n is decided from step n-1's solution).

* resistive half-wave rectifier: closed form v_load(n) = v_src(n) R_L /
  (R_s + R_d(n) + R_L) with the diode conducting at step n iff
  v_src(n-1) > 0;
* a runtime-switched run equals the same network with the switch written
  as an always-present r_off branch plus time-scheduled switches (an
  independent, already pinned code path) closed on the decided intervals;
* the breaker opens at the first current sign change at or after its
  trip step, and the diode state at every step follows the sign of the
  previous step's diode voltage in the oracle's own waveform;
* monolithic and partitioned solves agree with switches in several
  subsystems.
"""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import netgen as g

A, F, PHI = 1000.0, 60.0, 0.3


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def rectifier(r_s=1.0, r_l=10.0, r_on=0.01, r_off=1e6, dt=50e-6, on0=False, cap=None):
    b = g.NetworkBuilder()
    b.source(A, PHI, F)
    b.branch(g.source_node(0), 0, 0, r_s)
    b.diode(0, 1, r_on, r_off, on0=on0)
    b.branch(1, g.GROUND, 0, r_l)
    if cap is not None:
        b.branch(1, g.GROUND, 2, cap)
    return b.build(dt, 2, 2000)


def src(n, dt):
    return A * np.sin(2.0 * np.pi * F * (n * dt) + PHI)


def test_half_wave_rectifier_closed_form():
    net = rectifier()
    N, dt = 2000, net.dt
    v = oracle.simulate(net, N)
    n = np.arange(1, N + 1)
    vs = src(n, dt)
    prev = src(n - 1, dt)
    assert np.min(np.abs(prev[1:])) > 1e-6 * A          # no decision sits on a rounding tie
    on = np.concatenate([[False], prev[1:] > 0.0])       # step 1 uses the initial state (off)
    r_d = np.where(on, 0.01, 1e6)
    expect = vs * 10.0 / (1.0 + r_d + 10.0)
    assert rel(v[:, 1], expect) <= 1e-13
    st = oracle.runtime_switch_states(net, N)[:, 0].astype(bool)
    assert np.array_equal(st, on)
    assert 0 < st.sum() < N


def intervals(states):
    """[close, open) step intervals (steps 1..N) where the state is on."""
    out, start = [], None
    for i, s in enumerate(states, start=1):
        if s and start is None:
            start = i
        if not s and start is not None:
            out.append((start, i))
            start = None
    if start is not None:
        out.append((start, -1))
    return out


def scheduled_equivalent(net, states):
    """The network with runtime switch w written as an r_off branch plus one
    scheduled switch of resistance 1/(1/r_on - 1/r_off) per on-interval."""
    b = g.NetworkBuilder()
    for a in range(net.n_sources):
        b.source(net.src_amp[a], net.src_phase[a], net.src_freq[a])
    for i in range(net.n_branches):
        b.branch(net.br_k[i], net.br_m[i], net.br_kind[i], net.br_value[i])
    for i in range(net.n_lines):
        b.line(net.ln_k[i], net.ln_m[i], net.ln_zc[i], net.ln_delay[i])
    for i in range(net.n_switches):
        b.switch(net.sw_k[i], net.sw_m[i], net.sw_r[i], net.sw_close_step[i], net.sw_open_step[i])
    for w in range(net.n_runtime_switches):
        k, m = int(net.rs_k[w]), int(net.rs_m[w])
        b.branch(k, m, 0, net.rs_roff[w]) if k >= 0 else b.branch(m, k, 0, net.rs_roff[w])
        r_x = 1.0 / (1.0 / net.rs_ron[w] - 1.0 / net.rs_roff[w])
        for (c, o) in intervals(states[:, w]):
            b.switch(k, m, r_x, c, o)
    return b.build(net.dt, net.n_nodes, net.n_steps)


def test_rectifier_with_filter_capacitor_equals_scheduled_switching():
    net = rectifier(cap=200e-6)
    N = 2000
    v = oracle.simulate(net, N)
    st = oracle.runtime_switch_states(net, N)
    # the diode state follows the sign of the previous step's diode voltage
    vb_prev = v[:-1, 0] - v[:-1, 1]
    assert np.array_equal(st[1:, 0].astype(bool), vb_prev > 0.0)
    assert np.min(np.abs(vb_prev)) > 1e-9 * np.max(np.abs(v))
    # with the capacitor the diode conducts only near the source peaks
    assert 0.05 < st[:, 0].mean() < 0.5
    ref = oracle.simulate(scheduled_equivalent(net, st), N)
    assert rel(v, ref) <= 1e-12


def rl_breaker(trip):
    b = g.NetworkBuilder()
    b.source(A, PHI, F)
    b.branch(g.source_node(0), 0, 0, 1.0)
    b.branch(0, 1, 1, 10e-3)
    b.breaker(1, g.GROUND, 1e-3, 1e5, trip)
    b.branch(1, g.GROUND, 2, 1e-6)     # small stray capacitance across the breaker
    return b.build(20e-6, 2, 3000)


@pytest.mark.parametrize("trip", [400, 1234])
def test_breaker_opens_at_the_first_current_zero_after_trip(trip):
    net = rl_breaker(trip)
    N = 3000
    v = oracle.simulate(net, N)
    st = oracle.runtime_switch_states(net, N)[:, 0]
    i = v[:, 1] / 1e-3                      # breaker current while closed, steps 1..N
    prod = np.concatenate([[0.0], i[:-1]]) * i
    n_open = next(n for n in range(trip, N + 1) if prod[n - 1] <= 0.0)
    assert np.all(st[:n_open] == 1) and np.all(st[n_open:] == 0)
    assert n_open < N
    ref = oracle.simulate(scheduled_equivalent(net, st[:, None]), N)
    assert rel(v, ref) <= 1e-12


def test_monolithic_equals_partitioned_with_runtime_switches():
    base = g.multi_subsystem(151, [3, 4, 2, 3], n_lines=5, n_sources=2, dt=20e-6)
    rng = np.random.default_rng(9)
    net = base.copy()
    nodes = rng.choice(net.n_nodes, size=6, replace=False)
    net.rs_k = np.array([nodes[0], nodes[2], nodes[4]], np.int32)
    net.rs_m = np.array([nodes[1], -1, nodes[5]], np.int32)
    net.rs_kind = np.array([0, 1, 0], np.uint8)
    net.rs_ron = np.array([0.05, 0.01, 0.1])
    net.rs_roff = np.array([1e5, 1e6, 1e4])
    net.rs_on0 = np.array([0, 1, 1], np.uint8)
    net.rs_trip = np.array([-1, 600, -1], np.int64)
    N = 1500
    a = oracle.simulate(net, N, monolithic=True)
    b = oracle.simulate(net, N, monolithic=False)
    assert rel(a, b) <= 1e-12
    st = oracle.runtime_switch_states(net, N)
    assert st[:, 0].min() != st[:, 0].max() or st[:, 2].min() != st[:, 2].max()
