"""Pins of the CPU oracle to results fixed by mathematics, not by the oracle.

Each test ties one part of the oracle to an independent closed form, a
library routine used as a different method, exact arithmetic, or an
invariant computed by a different recursion:

* Tustin equivalence: the trapezoidal companion recursion of an LTI circuit
  equals the bilinear transform of its transfer function (scipy.signal).
* discrete sinusoidal steady state: late-time waveforms equal the complex
  phasor solution with the trapezoidal rule's frequency-warped impedances
  and the exact lossless-line two-port.
* exact travel-time delay of a lossless Bergeron line (matched ends).
* KCL at every node with branch currents from the textbook current
  recursions (not the history-source form the oracle uses).
* dense LU against Cramer's rule in exact rational arithmetic.
* resistive switching against the resistive divider.
* partitioning against networkx connected components.
"""
from fractions import Fraction

import networkx as nx
import numpy as np
import pytest
from scipy import signal

import oracle
from paper_1903_01081_b300 import netgen as g

W60 = 2 * np.pi * 60.0


def src_wave(net, s, n_steps):
    t = np.arange(0, n_steps + 1) * net.dt
    w = net.src_amp[s] * np.sin(2 * np.pi * net.src_freq[s] * t + net.src_phase[s])
    w[0] = 0.0   # de-energised start: the source counts as 0 at n = 0
    return w


def series_circuit(elems, dt=50e-6, phase=0.3):
    """source -> elems[0] -> node0 -> elems[1] -> node1 ... -> last -> ground."""
    b = g.NetworkBuilder()
    b.source(1000.0, phase)
    n = len(elems) - 1
    prev = g.source_node(0)
    for i, (kind, val) in enumerate(elems):
        nxt = i if i < n else g.GROUND
        b.branch(prev, nxt, kind, val)
        prev = nxt
    return b.build(dt, n)


# ----------------------------------------------------------------- Tustin

@pytest.mark.parametrize("case", ["RL", "RC", "RLC", "LC_R"])
def test_tustin_equivalence(case):
    dt, N = 50e-6, 6000
    R, L, C = 2.7, 0.033, 47e-6
    if case == "RL":
        net = series_circuit([(0, R), (1, L)], dt)
        b_s, a_s = [L, 0.0], [L, R]                        # V0/Vs = sL/(R+sL)
        node = 0
    elif case == "RC":
        net = series_circuit([(0, R), (2, C)], dt)
        b_s, a_s = [1.0], [R * C, 1.0]                     # 1/(sRC+1)
        node = 0
    elif case == "RLC":
        net = series_circuit([(0, R), (1, L), (2, C)], dt)
        b_s, a_s = [1.0], [L * C, R * C, 1.0]              # V1/Vs = 1/(s^2LC+sRC+1)
        node = 1
    else:
        net = series_circuit([(1, L), (2, C), (0, R)], dt)
        b_s, a_s = [R * C, 0.0], [L * C, R * C, 1.0]       # V1/Vs = sRC/(s^2LC+sRC+1)
        node = 1
    bz, az = signal.bilinear(b_s, a_s, fs=1.0 / dt)
    x = src_wave(net, 0, N)
    y = signal.lfilter(bz, az, x)
    v = oracle.simulate(net, N)[:, node]
    err = np.max(np.abs(v - y[1:])) / np.max(np.abs(y))
    assert err < 1e-11, err


def test_rl_scalar_recurrence():
    # series RL driven by v_s: (1 + gR) i_n = (1 - gR) i_{n-1} + g (v_n + v_{n-1}),  g = dt/(2L)
    dt, N, R, L = 20e-6, 3000, 1.3, 0.021
    net = series_circuit([(0, R), (1, L)], dt)
    vs = src_wave(net, 0, N)
    gl = dt / (2 * L)
    i = np.zeros(N + 1)
    for n in range(1, N + 1):
        i[n] = ((1 - gl * R) * i[n - 1] + gl * (vs[n] + vs[n - 1])) / (1 + gl * R)
    v_node = vs[1:] - R * i[1:]
    v = oracle.simulate(net, N)[:, 0]
    assert np.max(np.abs(v - v_node)) / np.max(np.abs(v_node)) < 1e-12


# ----------------------------------------------------------------- phasor

def damped_network(seed, phases=1):
    net = g.multi_subsystem(seed, [3, 4, 2], n_lines=4, n_sources=2, dt=50e-6, phases=phases,
                            shunt_kinds=(g.KIND_R,), n_series_extra=0)
    # every shunt to ground an R in [100, 400] ohm (near Z_c, so line
    # reflections die out) so that all transients decay within the run
    shunt = (net.br_m == g.GROUND) & (net.br_kind == g.KIND_R)
    net.br_value[shunt] = 100.0 + 300.0 * (net.br_value[shunt] - 0.1) / 9.9
    return net


def phasor_solution(net, omega):
    """Complex node voltages: Y V = I with trapezoidal-warped impedances."""
    n = net.n_nodes
    th = omega * net.dt
    Y = np.zeros((n, n), dtype=complex)
    I = np.zeros(n, dtype=complex)
    Vs = net.src_amp * np.exp(1j * net.src_phase)

    def y_of(kind, val):
        if kind == 0:
            return 1.0 / val
        if kind == 1:
            return 1.0 / (1j * (2 * val / net.dt) * np.tan(th / 2))
        return 1.0 / (-1j * (net.dt / (2 * val)) / np.tan(th / 2))

    for k, m, kind, val in zip(net.br_k, net.br_m, net.br_kind, net.br_value):
        y = y_of(int(kind), float(val))
        for a, c in ((k, m), (m, k)):
            if a >= 0:
                Y[a, a] += y
                if c >= 0:
                    Y[a, c] -= y
                elif c <= -2:
                    I[a] += y * Vs[-2 - c]
    for k, m, zc, d in zip(net.ln_k, net.ln_m, net.ln_zc, net.ln_delay):
        wt = omega * d * net.dt
        ys = -1j / (zc * np.tan(wt))      # self admittance of a lossless line
        ym = 1j / (zc * np.sin(wt))       # transfer admittance (from the ABCD two-port)
        Y[k, k] += ys
        Y[m, m] += ys
        Y[k, m] += ym
        Y[m, k] += ym
    return np.linalg.solve(Y, I)


@pytest.mark.parametrize("seed,phases", [(11, 1), (12, 1), (13, 1)])
def test_phasor_steady_state(seed, phases):
    net = damped_network(seed, phases)
    N = 60000
    v = oracle.simulate(net, N)
    V = phasor_solution(net, W60)
    t = np.arange(1, N + 1) * net.dt
    tail = slice(N - 2000, N)
    ref = np.imag(V[None, :] * np.exp(1j * W60 * t[tail])[:, None])
    err = np.max(np.abs(v[tail] - ref)) / np.max(np.abs(ref))
    assert err < 1e-11, err


# ----------------------------------------------------------------- lines

def line_circuit(rs, load, d, zc=300.0, dt=20e-6):
    """source -Rs- node0 ==line(d)== node1 [-load- ground]."""
    b = g.NetworkBuilder()
    b.source(1000.0, 0.4)
    b.branch(g.source_node(0), 0, 0, rs)
    b.line(0, 1, zc, d)
    if load is not None:
        b.branch(1, g.GROUND, 0, load)
    return b.build(dt, 2)


@pytest.mark.parametrize("d", [1, 3, 17])
def test_line_matched_source_is_pure_delay(d):
    zc, N = 300.0, 400
    net = line_circuit(zc, None, d, zc)      # matched source, open far end
    v = oracle.simulate(net, N)
    vs = src_wave(net, 0, N)
    pad = np.concatenate([np.zeros(2 * d), vs])          # pad[j + 2d] = vs[j], vs[<0] = 0
    n = np.arange(1, N + 1)
    exp_m = pad[n - d + 2 * d]
    exp_k = 0.5 * (pad[n + 2 * d] + pad[n - 2 * d + 2 * d])
    scale = np.max(np.abs(vs))
    assert np.max(np.abs(v[:, 1] - exp_m)) / scale < 1e-13
    assert np.max(np.abs(v[:, 0] - exp_k)) / scale < 1e-13


@pytest.mark.parametrize("d", [2, 9])
def test_line_matched_load_no_reflection(d):
    zc, rs, N = 250.0, 37.0, 300
    net = line_circuit(rs, zc, d, zc)
    v = oracle.simulate(net, N)
    vs = src_wave(net, 0, N)
    scale = np.max(np.abs(vs))
    assert np.max(np.abs(v[:, 0] - vs[1:] * zc / (rs + zc))) / scale < 1e-13
    vk = np.concatenate([np.zeros(d), v[:, 0]])
    assert np.max(np.abs(v[:, 1] - vk[:N])) / scale < 1e-13


# ----------------------------------------------------------------- KCL

def kcl_residual(net, v, n_steps):
    """Max over steps and nodes of |sum of currents leaving the node|,
    relative to the largest branch current; currents from the textbook
    recursions (trapezoidal current form, d'Alembert form for lines)."""
    N = n_steps
    V = np.zeros((N + 1, net.n_nodes))
    V[1:] = v
    vsrc = np.stack([src_wave(net, s, N) for s in range(net.n_sources)], axis=1) if net.n_sources else np.zeros((N + 1, 0))

    def volt(x):
        if x >= 0:
            return V[:, x]
        if x == -1:
            return np.zeros(N + 1)
        return vsrc[:, -2 - x]

    leave = np.zeros((N + 1, net.n_nodes))
    big = 0.0
    for k, m, kind, val in zip(net.br_k, net.br_m, net.br_kind, net.br_value):
        vb = volt(k) - volt(m)
        i = np.zeros(N + 1)
        if kind == 0:
            i = vb / val
        elif kind == 1:
            for n in range(1, N + 1):
                i[n] = i[n - 1] + net.dt / (2 * val) * (vb[n] + vb[n - 1])
        else:
            for n in range(1, N + 1):
                i[n] = -i[n - 1] + 2 * val / net.dt * (vb[n] - vb[n - 1])
        big = max(big, np.max(np.abs(i)))
        if k >= 0:
            leave[:, k] += i
        if m >= 0:
            leave[:, m] -= i
    for k, m, zc, d in zip(net.ln_k, net.ln_m, net.ln_zc, net.ln_delay):
        ik = np.zeros(N + 1)
        im = np.zeros(N + 1)
        for n in range(1, N + 1):
            pk = V[n - d, m] / zc + im[n - d] if n - d >= 1 else 0.0
            pm = V[n - d, k] / zc + ik[n - d] if n - d >= 1 else 0.0
            ik[n] = V[n, k] / zc - pk
            im[n] = V[n, m] / zc - pm
        big = max(big, np.max(np.abs(ik)), np.max(np.abs(im)))
        leave[:, k] += ik
        leave[:, m] += im
    for k, m, r, on, off in zip(net.sw_k, net.sw_m, net.sw_r, net.sw_close_step, net.sw_open_step):
        steps = np.arange(N + 1)
        closed = (steps >= on) & ((off < 0) | (steps < off)) & (on >= 0)
        i = np.where(closed, (volt(k) - volt(m)) / r, 0.0)
        if k >= 0:
            leave[:, k] += i
        if m >= 0:
            leave[:, m] -= i
    return np.max(np.abs(leave[1:])) / big


def test_kcl_single_subsystem_with_fault():
    net = g.single_rlc(seed=1001, n_steps=3000, fault_step=1500)
    N = 3000
    v = oracle.simulate(net, N)
    assert kcl_residual(net, v, N) < 1e-11


def test_kcl_multi_subsystem_three_phase():
    net = g.multi_subsystem(21, [2, 3, 2, 4], n_lines=6, n_sources=2, dt=20e-6, n_series_extra=3)
    N = 1500
    v = oracle.simulate(net, N)
    assert kcl_residual(net, v, N) < 1e-11


# ----------------------------------------------------------------- LU

def cramer(A, b):
    n = len(A)

    def det(M):
        if len(M) == 1:
            return M[0][0]
        return sum(((-1) ** j) * M[0][j] * det([row[:j] + row[j + 1:] for row in M[1:]]) for j in range(len(M)))

    D = det(A)
    return [det([[b[i] if c == j else A[i][c] for c in range(n)] for i in range(n)]) / D for j in range(n)]


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_lu_against_exact_cramer(n):
    rng = np.random.default_rng(100 + n)
    for _ in range(5):
        Ai = rng.integers(-9, 10, size=(n, n))
        if n > 1:
            Ai[0, 0] = 0          # forces a row swap
        bi = rng.integers(-9, 10, size=n)
        A = [[Fraction(int(x)) for x in row] for row in Ai]
        b = [Fraction(int(x)) for x in bi]
        try:
            xe = cramer(A, b)
        except ZeroDivisionError:
            continue
        x = oracle.lu_solve(Ai.astype(float), bi.astype(float))
        xe = np.array([float(q) for q in xe])
        assert np.max(np.abs(x - xe)) <= 1e-13 * max(1.0, np.max(np.abs(xe)))


@pytest.mark.parametrize("n", [5, 6, 12])
def test_lu_against_numpy(n):
    rng = np.random.default_rng(7 + n)
    A = rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    assert np.allclose(oracle.lu_solve(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------- switches

def test_resistive_fault_divider():
    b = g.NetworkBuilder()
    b.source(1000.0, 0.2)
    R1, R2, Rf, ns = 3.0, 7.0, 0.5, 40
    b.branch(g.source_node(0), 0, 0, R1)
    b.branch(0, g.GROUND, 0, R2)
    b.switch(0, g.GROUND, Rf, ns, 90)
    net = b.build(50e-6, 1)
    N = 120
    v = oracle.simulate(net, N)[:, 0]
    vs = src_wave(net, 0, N)[1:]
    n = np.arange(1, N + 1)
    par = R2 * Rf / (R2 + Rf)
    ratio = np.where((n >= ns) & (n < 90), par / (R1 + par), R2 / (R1 + R2))
    assert np.max(np.abs(v - vs * ratio)) < 1e-12 * 1000


# ----------------------------------------------------------------- partition

def test_partition_matches_connected_components():
    net = g.large_scale(n_steps=10)
    sub, ns = oracle.partition(net)
    G = nx.Graph()
    G.add_nodes_from(range(net.n_nodes))
    for k, m in zip(net.br_k, net.br_m):
        if k >= 0 and m >= 0:
            G.add_edge(int(k), int(m))
    comps = list(nx.connected_components(G))
    assert ns == len(comps)
    for c in comps:
        c = list(c)
        assert len(set(sub[c])) == 1


def test_monolithic_equals_partitioned():
    net = g.multi_subsystem(31, [2, 5, 3, 4, 2], n_lines=7, n_sources=2, dt=20e-6, n_series_extra=2)
    net.sw_k = np.array([3], np.int32); net.sw_m = np.array([-1], np.int32)
    net.sw_r = np.array([0.01]); net.sw_close_step = np.array([300], np.int64); net.sw_open_step = np.array([-1], np.int64)
    N = 2000
    a = oracle.simulate(net, N, monolithic=False)
    b = oracle.simulate(net, N, monolithic=True)
    assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-12
