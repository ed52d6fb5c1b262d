"""Pins of the oracle's control blocks (the paper's control components as
basic processes of its computation graph, Sec. III-A) and of their
coupling to the electrical network.

* INTEG driven by a constant: the ramp k c dt (n - 1/2) of the trapezoidal
  integral with a zero initial input;
* LAG and PI driven by a measured node voltage: scipy.signal.lfilter of the
  Tustin (scipy.signal.bilinear) discretisations of k / (1 + sT) and
  kp + ki / s applied to the node's closed-form waveform (a resistive
  divider), zero initial state;
* GAIN, SUM, MUL, LIMIT on two measured dividers: their closed forms;
* loop breaking: a block reading itself and a block of higher index sees
  the previous step's outputs (geometric series in closed form), in both
  block orders;
* a controlled current injection enters at the next step with the sign of
  a current into the node: a scalar recurrence written out by hand;
* monolithic and partitioned solves agree with converter controls in
  several subsystems; invalid descriptions are rejected.
"""
import numpy as np
import pytest
import scipy.signal as sig

import oracle
from paper_1903_01081_b300 import netgen as g

A, F, PHI = 1000.0, 60.0, 0.4
DT = 50e-6


def divider(b, r1, r2, node):
    """node = source 0 through r1, r2 to ground: v = v_src r2 / (r1 + r2)."""
    b.branch(g.source_node(0), node, g.KIND_R, r1)
    b.branch(node, g.GROUND, g.KIND_R, r2)


def vsrc(n):
    return A * np.sin(2 * np.pi * F * n * DT + PHI)


def test_integrator_ramp():
    b = g.NetworkBuilder()
    b.branch(0, g.GROUND, g.KIND_R, 1.0)
    c0 = b.block(g.CB_CONST, p0=3.0)
    b.block(g.CB_INTEG, c0, p0=2.0)
    net = b.build(DT, 1)
    y = oracle.controls(net, 500)
    n = np.arange(1, 501)
    assert np.allclose(y[:, 0], 3.0, rtol=0, atol=0)
    assert np.max(np.abs(y[:, 1] - 2.0 * 3.0 * DT * (n - 0.5))) <= 1e-13 * 2.0 * 3.0 * DT * 500


def test_lag_and_pi_match_bilinear():
    b = g.NetworkBuilder()
    b.source(A, PHI, F)
    divider(b, 2.0, 3.0, 0)
    m = b.block(g.CB_MEAS, node=0)
    b.block(g.CB_LAG, m, p0=1.5, p1=0.7e-3)
    b.block(g.CB_PI, m, p0=0.3, p1=40.0)
    net = b.build(DT, 1)
    N = 3000
    y = oracle.controls(net, N)
    x = vsrc(np.arange(1, N + 1)) * 3.0 / 5.0
    assert np.max(np.abs(y[:, 0] - x)) <= 1e-13 * A
    bl, al = sig.bilinear([1.5], [0.7e-3, 1.0], fs=1.0 / DT)
    lag = sig.lfilter(bl, al, x)
    assert np.max(np.abs(y[:, 1] - lag)) <= 1e-11 * np.max(np.abs(lag))
    bp, ap = sig.bilinear([0.3, 40.0], [1.0, 0.0], fs=1.0 / DT)
    pi = sig.lfilter(bp, ap, x)
    assert np.max(np.abs(y[:, 2] - pi)) <= 1e-11 * np.max(np.abs(pi))


def test_static_blocks():
    b = g.NetworkBuilder()
    b.source(A, PHI, F)
    divider(b, 1.0, 1.0, 0)
    divider(b, 1.0, 4.0, 1)
    m0 = b.block(g.CB_MEAS, node=0)
    m1 = b.block(g.CB_MEAS, node=1)
    b.block(g.CB_GAIN, m0, p0=-0.25)
    b.block(g.CB_SUM, m0, m1, p0=2.0, p1=-3.0)
    b.block(g.CB_MUL, m0, m1, p0=1e-3)
    b.block(g.CB_LIMIT, m1, p0=-300.0, p1=500.0)
    net = b.build(DT, 2)
    N = 1000
    y = oracle.controls(net, N)
    s = vsrc(np.arange(1, N + 1))
    v0, v1 = 0.5 * s, 0.8 * s
    tol = 1e-13 * A
    assert np.max(np.abs(y[:, 2] + 0.25 * v0)) <= tol
    assert np.max(np.abs(y[:, 3] - (2 * v0 - 3 * v1))) <= 10 * tol
    assert np.max(np.abs(y[:, 4] - 1e-3 * v0 * v1)) <= tol
    assert np.max(np.abs(y[:, 5] - np.clip(v1, -300.0, 500.0))) <= tol
    assert np.any(y[:, 5] == 500.0) and np.any(y[:, 5] == -300.0)


@pytest.mark.parametrize("const_first", [True, False])
def test_loop_breaking(const_first):
    """y = 1 * c + 0.5 * y(n-1) with c a CONST 1: when the constant comes
    first it is read at step n, otherwise (higher index) at step n-1."""
    b = g.NetworkBuilder()
    b.branch(0, g.GROUND, g.KIND_R, 1.0)
    if const_first:
        c = b.block(g.CB_CONST, p0=1.0)
        s = b.block(g.CB_SUM, c, c + 1, p0=1.0, p1=0.5)
    else:
        s = b.block(g.CB_SUM, 1, 0, p0=1.0, p1=0.5)
        b.block(g.CB_CONST, p0=1.0)
    net = b.build(DT, 1)
    y = oracle.controls(net, 60)[:, s]
    n = np.arange(1, 61)
    want = 2.0 - 2.0 ** (1 - n) if const_first else np.where(n == 1, 0.0, 2.0 - 2.0 ** (2 - n))
    assert np.max(np.abs(y - want)) <= 1e-15


def test_injection_timing_and_sign():
    """Node 0: source through R_s, shunt R, controlled current -K v(n-1)
    into the node: v(n) = (v_src(n)/R_s - K v(n-1)) / (1/R_s + 1/R)."""
    rs, r, k = 2.0, 5.0, 0.3
    b = g.NetworkBuilder()
    b.source(A, PHI, F)
    divider(b, rs, r, 0)
    m = b.block(g.CB_MEAS, node=0)
    gk = b.block(g.CB_GAIN, m, p0=-k)
    b.injection(gk, 0)
    net = b.build(DT, 1)
    N = 400
    v = oracle.simulate(net, N)[:, 0]
    want = np.zeros(N)
    prev = 0.0
    for i in range(N):
        want[i] = (vsrc(i + 1) / rs - k * prev) / (1.0 / rs + 1.0 / r)
        prev = want[i]
    assert np.max(np.abs(v - want)) <= 1e-13 * A
    # without the injection the node is the plain divider
    net0 = net.copy()
    net0.ci_block = net0.ci_block[:0]
    net0.ci_node = net0.ci_node[:0]
    assert np.max(np.abs(oracle.simulate(net0, N)[:, 0] - vsrc(np.arange(1, N + 1)) * r / (rs + r))) <= 1e-13 * A


def converter_net(n_steps=1500):
    base = g.multi_subsystem(11, [4, 5, 3, 6], n_lines=5, n_sources=3, dt=20e-6, n_steps=n_steps)
    return g.with_converter_controls(base, n_converters=7)


def test_monolithic_equals_partitioned_with_controls():
    net = converter_net()
    assert net.n_control_blocks == 7 * 24
    _, n_sub = oracle.partition(net)
    conv_subs = {int(s) for s in oracle.partition(net)[0][net.ci_node]}
    assert n_sub == 4 and len(conv_subs) >= 3
    a = oracle.simulate(net, 1500)
    m = oracle.simulate(net, 1500, monolithic=True)
    assert np.max(np.abs(a - m)) <= 1e-11 * np.max(np.abs(a))
    y = oracle.controls(net, 1500)
    assert np.max(np.abs(y[:, 21::24])) > 0.1          # the converters draw current


def test_invalid_controls_rejected():
    net = converter_net(10)

    def bad(**kw):
        x = net.copy()
        for k, v in kw.items():
            setattr(x, k, v)
        with pytest.raises(oracle.OracleError):
            oracle.controls(x, 5)

    t = net.cb_type.copy(); t[3] = 9
    bad(cb_type=t)
    i0 = net.cb_in0.copy(); i0[4] = net.n_control_blocks
    bad(cb_in0=i0)
    p1 = net.cb_p1.copy(); p1[21] = 0.0        # a LAG with T = 0
    bad(cb_p1=p1)
    p0 = net.cb_p0.copy(); p0[14] = 1e9        # a LIMIT with lo > hi
    bad(cb_p0=p0)
    nd = net.cb_node.copy(); nd[0] = net.n_nodes
    bad(cb_node=nd)
    cb = net.ci_block.copy(); cb[0] = -1
    bad(ci_block=cb)
    with pytest.raises(oracle.OracleError):
        oracle.adjoint(net, 5, np.zeros((5, net.n_nodes)))
