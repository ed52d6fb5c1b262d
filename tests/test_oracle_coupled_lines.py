"""Pins of the oracle's coupled three-phase lossless lines (modal Bergeron
with linearly interpolated non-integer travel times).

* with T_v = I and integer travel times they are three single-phase
  Bergeron lines (the pinned line model), to rounding;
* a matched line is a pure interpolated delay: v_m(n) = (1 - f) v_k(n - d)
  + f v_k(n - d - 1) for a travel time (d + f) dt;
* a transposed line in Clarke modes with matched modal terminations (built
  from resistors) carries each mode with its own delay: the far-end phase
  voltages are T_v times the interpolated, delayed near-end modal voltages;
* monolithic and partitioned solves agree.
"""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import netgen as g

DT = 2.0 ** -16      # travel times d dt are exact in binary


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def three_line_net(coupled, z=(400.0, 300.0, 250.0), d=(3, 5, 7), tau=None, tv=np.eye(3)):
    """Sources through R into end k; end m loaded by R and C per phase."""
    b = g.NetworkBuilder()
    for p in range(3):
        b.source(1000.0, -2 * np.pi * p / 3, 60.0)
        b.branch(g.source_node(p), p, 0, 50.0)
        b.branch(p, g.GROUND, 2, 2e-6)
        b.branch(3 + p, g.GROUND, 0, 800.0)
        b.branch(3 + p, g.GROUND, 2, 5e-6)
    b.branch(0, 1, 0, 2000.0)            # couple the phases of each end
    b.branch(4, 5, 0, 2000.0)
    if coupled:
        taus = [di * DT for di in d] if tau is None else tau
        b.coupled_line([0, 1, 2], [3, 4, 5], tv, z, taus)
    else:
        for p in range(3):
            b.line(p, 3 + p, z[p], d[p])
    return b.build(DT, 6, 3000)


def test_identity_modes_with_integer_delays_are_single_phase_lines():
    N = 3000
    a = oracle.simulate(three_line_net(True), N)
    b = oracle.simulate(three_line_net(False), N)
    assert rel(a, b) <= 1e-14


@pytest.mark.parametrize("steps", [1.0, 3.25, 6.5, 11.875])
def test_matched_line_is_an_interpolated_delay(steps):
    z = 300.0
    b = g.NetworkBuilder()
    b.source(1000.0, 0.4, 60.0)
    b.branch(g.source_node(0), 0, 0, z)          # matched source
    for p in (1, 2):                              # the idle modes, matched at both ends
        b.branch(p, g.GROUND, 0, z)
        b.branch(3 + p, g.GROUND, 0, z)
    b.branch(3, g.GROUND, 0, z)                   # matched load
    b.coupled_line([0, 1, 2], [3, 4, 5], np.eye(3), [z, z, z], [steps * DT] * 3)
    net = b.build(DT, 6, 2000)
    v = oracle.simulate(net, 2000)
    n = np.arange(1, 2001)
    vs = 1000.0 * np.sin(2 * np.pi * 60.0 * n * DT + 0.4)
    assert rel(v[:, 0], vs / 2) <= 1e-13
    d, f = int(np.floor(steps)), steps - np.floor(steps)
    vk = np.concatenate([np.zeros(d + 1), v[:, 0]])       # v_k at steps n - d - 1, ..., index shift d + 1
    idx = np.arange(2000)
    expect = (1 - f) * vk[idx + 1] + f * vk[idx]
    assert rel(v[:, 3], expect) <= 1e-13


def test_transposed_line_modes_travel_with_their_own_delays():
    T = g.CLARKE
    z = np.array([600.0, 300.0, 300.0])
    y0, y1 = 1 / z[0], 1 / z[1]
    b_off = (y0 - y1) / 3                         # Y_p off-diagonal (< 0)
    b = g.NetworkBuilder()
    for p, amp in enumerate((1000.0, 600.0, 1400.0)):   # unbalanced: every mode is excited
        b.source(amp, 0.2 - 2 * np.pi * p / 3, 60.0)
        b.branch(g.source_node(p), p, 0, 1e-3)
        b.branch(3 + p, g.GROUND, 0, 1 / y0)      # matched termination: Y_p as resistors
    for p, q in ((3, 4), (4, 5), (3, 5)):
        b.branch(p, q, 0, -1 / b_off)
    taus = np.array([7.3, 5.6, 5.6]) * DT
    b.coupled_line([0, 1, 2], [3, 4, 5], T, z, taus)
    net = b.build(DT, 6, 3000)
    N = 3000
    v = oracle.simulate(net, N)
    vk_mode = v[:, :3] @ np.linalg.inv(T).T       # modal voltages at end k, per step
    assert np.max(np.abs(vk_mode[:, 0])) > 0.1 * np.max(np.abs(vk_mode))
    expect = np.zeros((N, 3))
    for j in range(3):
        s = taus[j] / DT
        d, f = int(np.floor(s)), s - np.floor(s)
        pad = np.concatenate([np.zeros((d + 1,)), vk_mode[:, j]])
        idx = np.arange(N)
        expect[:, j] = (1 - f) * pad[idx + 1] + f * pad[idx]
    vm_mode = v[:, 3:] @ np.linalg.inv(T).T
    for j in range(3):   # each mode on its own scale
        assert rel(vm_mode[:, j], expect[:, j]) <= 1e-12, j
    assert rel(v[:, 3:], expect @ T.T) <= 1e-12


def test_monolithic_equals_partitioned_with_coupled_lines():
    net = three_line_net(True, tau=[3.4 * DT, 5.1 * DT, 7.9 * DT], tv=g.CLARKE, z=(550.0, 280.0, 280.0))
    a = oracle.simulate(net, 3000, monolithic=True)
    b = oracle.simulate(net, 3000, monolithic=False)
    assert rel(a, b) <= 1e-12
    sub, ns = oracle.partition(net)
    assert ns == 2 and sub[0] == sub[1] == sub[2] != sub[3] == sub[4] == sub[5]


def test_coupled_line_validation():
    net = three_line_net(True, tau=[0.5 * DT, 3 * DT, 3 * DT])   # shorter than one step
    with pytest.raises(oracle.OracleError):
        oracle.simulate(net, 10)
    net = three_line_net(True, tv=np.ones((3, 3)))               # singular transformation
    with pytest.raises(oracle.OracleError):
        oracle.simulate(net, 10)


def test_adjoint_with_coupled_lines_vs_complex_step():
    """The reverse of the modal line (interpolated delays, T_v, Y_p) against
    complex-step derivatives of every parameter."""
    net = three_line_net(True, tau=[3.4 * DT, 5.1 * DT, 7.9 * DT], tv=g.CLARKE, z=(550.0, 280.0, 280.0))
    N = 600
    br_t, amp_t = g.adjoint_target(net, seed=77)
    tgt = oracle.simulate(net.with_params(br_t, amp_t), N)
    grad, J = oracle.adjoint(net, N, tgt)
    n_par = net.n_branches + net.n_sources
    cs = np.array([oracle.loss_complex_step(net, N, tgt, p)[1] for p in range(n_par)])
    p = np.concatenate([net.br_value, net.src_amp])
    assert np.max(np.abs(p * (grad - cs)) / J) < 1e-9
