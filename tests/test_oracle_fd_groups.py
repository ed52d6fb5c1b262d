"""Pins of the oracle's frequency-dependent line groups (three frequency-
dependent conductors carrying the modes of one three-phase line through
T_v, T_i = T_v^-T):

* with T_v = I a group is its three lines on their own;
* lossless modes (Y_c = 1/Z_j, A = e^{-s tau_j}) are the coupled Bergeron
  line with the same T_v, impedances and (non-integer) travel times;
* with equal modes and an orthogonal T_v the phases decouple: the group is
  three equal frequency-dependent lines;
* monolithic and partitioned solves agree.
"""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import netgen as g


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def base_net():
    return g.multi_subsystem(161, [3, 4, 2, 3, 5], n_lines=8, n_sources=2, dt=20e-6)


def ungrouped(net):
    """The same frequency-dependent lines without the grouping."""
    u = net.copy()
    u.fg_line = np.zeros(0, np.int32)
    u.fg_tv = np.zeros(0, np.float64)
    return u


def test_identity_transformation_is_the_lines_on_their_own():
    net = g.fd_groups_from_coupled(g.with_coupled_lines(base_net(), seed=3), seed=5)
    net.fg_tv = np.tile(np.eye(3).reshape(9), len(net.fg_line) // 3)
    N = 4000
    assert rel(oracle.simulate(net, N), oracle.simulate(ungrouped(net), N)) <= 1e-13


def test_lossless_modes_are_the_coupled_bergeron_line():
    cnet = g.with_coupled_lines(base_net(), seed=3)   # Clarke modes, fractional travel times
    net = g.fd_groups_from_coupled(cnet, lossless=True)
    N = 4000
    ref = oracle.simulate(cnet, N)
    got = oracle.simulate(net, N)
    assert np.max(np.abs(ref)) > 1.0
    assert rel(got, ref) <= 1e-12


def test_equal_modes_with_orthogonal_transformation_decouple():
    cnet = g.with_coupled_lines(base_net(), seed=3)
    tv = cnet.cl_tv[:9].reshape(3, 3)
    assert np.allclose(tv @ tv.T, np.eye(3), atol=1e-15)   # (the Clarke matrix used is orthogonal)
    net = g.fd_groups_from_coupled(cnet, seed=7, same_modes=True)
    N = 4000
    got = oracle.simulate(net, N)
    assert rel(got, oracle.simulate(ungrouped(net), N)) <= 1e-11
    # and the modes' losses matter: not the lossless line
    lossless = g.fd_groups_from_coupled(cnet, lossless=True, same_modes=True)
    assert rel(got, oracle.simulate(lossless, N)) > 1e-3


def test_group_changes_the_waveforms():
    """A general group (lossy Clarke modes of different impedance and travel
    time) differs from its lines without the coupling."""
    net = g.with_fd_line_groups(base_net())
    N = 3000
    assert rel(oracle.simulate(net, N), oracle.simulate(ungrouped(net), N)) > 1e-3


def test_monolithic_equals_partitioned():
    net = g.with_fd_line_groups(base_net())
    N = 3000
    assert rel(oracle.simulate(net, N, monolithic=True), oracle.simulate(net, N)) <= 1e-11


def test_invalid_groups_are_rejected():
    net = g.with_fd_line_groups(base_net())
    bad = net.copy()
    bad.fg_line = bad.fg_line.copy()
    bad.fg_line[1] = bad.fg_line[0]   # a line in a group twice
    with pytest.raises(oracle.OracleError):
        oracle.simulate(bad, 10)
    bad = net.copy()
    bad.fg_tv = np.zeros_like(net.fg_tv)   # singular T_v
    with pytest.raises(oracle.OracleError):
        oracle.simulate(bad, 10)
