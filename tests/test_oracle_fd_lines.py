"""Pins of the oracle's frequency-dependent lines (Y_c and A as pole-residue
sums, trapezoidal recursive convolution, interpolated travel time).

* with Y_c = 1/Z, A = e^{-s tau} and tau a whole number of steps the line is
  the lossless Bergeron line (an independent, already pinned code path);
* with a fractional tau, three such lossless lines equal one coupled line
  with T_v = I (its modes interpolate the same way; pinned separately);
* sinusoidal steady state of a damped network with lossy lines equals a
  complex phasor solve in which each pole term is the Tustin transform of
  r / (s - p) computed by ``scipy.signal.bilinear`` and evaluated by
  ``scipy.signal.freqz``, the delay is z^-d ((1 - phi) + phi z^-1), and the
  line is the two-port I_k = Y_c V_k - A (Y_c V_m + I_m) (and symmetric);
* invalid descriptions are rejected, and so is the adjoint.
"""
import numpy as np
import pytest
import scipy.signal as sig

import oracle
from paper_1903_01081_b300 import netgen as g

DT = 2.0 ** -16          # travel times that are whole steps are exact
W60 = 2 * np.pi * 60.0


def end_loads(b):
    b.source(1000.0, 0.3, 60.0)
    b.branch(g.source_node(0), 0, g.KIND_R, 5.0)
    b.branch(0, g.GROUND, g.KIND_C, 20e-6)
    b.branch(1, g.GROUND, g.KIND_R, 300.0)
    b.branch(1, g.GROUND, g.KIND_L, 0.05)


def test_lossless_reduction_to_bergeron():
    for d in (1, 7, 20):
        nets = []
        for fd in (True, False):
            b = g.NetworkBuilder()
            end_loads(b)
            if fd:
                b.fd_line(0, 1, d * DT, 1 / 350.0, a0=1.0)
            else:
                b.line(0, 1, 350.0, d)
            nets.append(b.build(DT, 2))
        a, r = oracle.simulate(nets[0], 3000), oracle.simulate(nets[1], 3000)
        assert np.max(np.abs(a - r)) <= 1e-14 * np.max(np.abs(r))


def test_fractional_lossless_equals_coupled_identity_modes():
    taus = np.array([3.25, 7.5, 11.8125]) * DT
    zs = np.array([310.0, 420.0, 275.0])
    nets = []
    for fd in (True, False):
        b = g.NetworkBuilder()
        b.source(1000.0, 0.3, 60.0)
        for p in range(3):
            b.branch(g.source_node(0), p, g.KIND_R, 4.0 + p)
            b.branch(p, g.GROUND, g.KIND_C, 30e-6)
            b.branch(3 + p, g.GROUND, g.KIND_R, 200.0 + 50 * p)
            b.branch(3 + p, g.GROUND, g.KIND_L, 0.04)
        b.branch(0, 1, g.KIND_R, 50.0)      # one subsystem per end
        b.branch(1, 2, g.KIND_R, 50.0)
        b.branch(3, 4, g.KIND_R, 50.0)
        b.branch(4, 5, g.KIND_R, 50.0)
        if fd:
            for p in range(3):
                b.fd_line(p, 3 + p, taus[p], 1 / zs[p], a0=1.0)
        else:
            b.coupled_line([0, 1, 2], [3, 4, 5], np.eye(3), zs, taus)
        nets.append(b.build(DT, 6))
    a, r = oracle.simulate(nets[0], 4000), oracle.simulate(nets[1], 4000)
    assert np.max(np.abs(a - r)) <= 1e-13 * np.max(np.abs(r))


def pole_sum(z, direct, poles, residues, dt):
    """direct + sum_i Tustin(r_i / (s - p_i)) at z (scipy's bilinear/freqz)."""
    h = np.full_like(z, direct, dtype=complex)
    for p, r in zip(poles, residues):
        bz, az = sig.bilinear([r], [1.0, -p], fs=1.0 / dt)
        h += sig.freqz(bz, az, worN=[np.angle(z)])[1][0]
    return h


def fd_network():
    b = g.NetworkBuilder()
    b.source(1000.0, 0.3, 60.0)
    b.branch(g.source_node(0), 0, g.KIND_R, 5.0)
    b.branch(0, g.GROUND, g.KIND_C, 20e-6)
    b.branch(0, g.GROUND, g.KIND_R, 200.0)
    b.branch(1, g.GROUND, g.KIND_R, 150.0)
    b.branch(1, g.GROUND, g.KIND_L, 0.05)
    b.branch(2, g.GROUND, g.KIND_R, 90.0)
    b.branch(2, g.GROUND, g.KIND_C, 40e-6)
    b.fd_line(0, 1, 37.3 * DT, 1 / 320.0, yq=[-4e3, -6e4], yc=[0.3e3 / 320, 5e3 / 320],
              a0=0.2, ap=[-5e3, -8e4], ar=[0.6 * 5e3, 0.1 * 8e4])
    b.fd_line(1, 2, 12.0 * DT, 1 / 410.0, yq=[-2e4], yc=[3e3 / 410], a0=0.0, ap=[-3e4], ar=[0.9 * 3e4])
    return b.build(DT, 3)


def test_steady_state_matches_discrete_phasor_solve():
    net = fd_network()
    N = 120000                      # 1.8 s; the slowest transient decays long before
    v = oracle.simulate(net, N)
    z = np.exp(1j * W60 * DT)
    th = W60 * DT
    Y = np.zeros((3, 3), dtype=complex)
    I = np.zeros(3, dtype=complex)
    Vs = 1000.0 * np.exp(0.3j)
    for k, m, kind, val in zip(net.br_k, net.br_m, net.br_kind, net.br_value):
        y = (1.0 / val if kind == 0 else
             1.0 / (1j * (2 * val / DT) * np.tan(th / 2)) if kind == 1 else
             1.0 / (-1j * (DT / (2 * val)) / np.tan(th / 2)))
        if k >= 0 and m == g.GROUND:
            Y[k, k] += y
        elif m >= 0 and k <= -2:
            Y[m, m] += y
            I[m] += y * Vs
    for l in range(net.n_fd_lines):
        k, m = int(net.fl_k[l]), int(net.fl_m[l])
        ny, na = int(net.fl_ny[l]), int(net.fl_na[l])
        yc = pole_sum(z, net.fl_y0[l], net.fl_yq[4 * l:4 * l + ny], net.fl_yc[4 * l:4 * l + ny], DT)
        steps = net.fl_tau[l] / DT
        d, phi = np.floor(steps), steps - np.floor(steps)
        a = z ** (-d) * ((1 - phi) + phi / z) * pole_sum(z, net.fl_a0[l], net.fl_ap[4 * l:4 * l + na],
                                                         net.fl_ar[4 * l:4 * l + na], DT)
        # I_k + A I_m = Y_c (V_k - A V_m), A I_k + I_m = Y_c (V_m - A V_k)
        Y2 = yc * np.linalg.solve(np.array([[1, a], [a, 1]]), np.array([[1, -a], [-a, 1]]))
        for i, x in enumerate((k, m)):
            for j, y_ in enumerate((k, m)):
                Y[x, y_] += Y2[i, j]
    V = np.linalg.solve(Y, I)
    t = np.arange(N - 3000, N) * DT + DT
    ref = np.imag(V[None, :] * np.exp(1j * W60 * t)[:, None])
    err = np.max(np.abs(v[N - 3000:] - ref)) / np.max(np.abs(ref))
    assert err < 1e-10, err
    # the losses are visible: the same lines lossless give another answer
    lossless = net.copy()
    lossless.fl_ny[:] = 0
    lossless.fl_na[:] = 0
    lossless.fl_a0[:] = 1.0
    assert np.max(np.abs(oracle.simulate(lossless, 4000) - v[:4000])) > 1e-2 * np.max(np.abs(v[:4000]))


def test_large_network_lossy_lines_stay_bounded():
    base = g.large_scale(n_steps=6000)
    net = g.with_fd_lines(base)
    assert net.n_fd_lines == 2100 and net.n_lines == 0
    v = oracle.simulate(net, 6000)
    early, late = np.abs(v[:1000]).max(), np.abs(v[5000:]).max()
    assert np.isfinite(v).all() and late < 1.5 * early


def test_invalid_fd_lines_rejected():
    net = fd_network()

    def bad(**kw):
        x = net.copy()
        for k, v in kw.items():
            setattr(x, k, v)
        with pytest.raises(oracle.OracleError):
            oracle.simulate(x, 5)

    bad(fl_tau=np.array([0.5 * DT, 12 * DT]))
    bad(fl_ny=np.array([5, 1], np.int32))
    yq = net.fl_yq.copy(); yq[0] = 10.0
    bad(fl_yq=yq)
    ap = net.fl_ap.copy(); ap[4] = 0.0
    bad(fl_ap=ap)
    bad(fl_y0=np.array([-1.0, 0.0]), fl_ny=np.array([0, 0], np.int32))   # no conductance
    bad(fl_m=np.array([0, 2], np.int32))
    with pytest.raises(oracle.OracleError):
        oracle.adjoint(net, 5, np.zeros((5, 3)))
