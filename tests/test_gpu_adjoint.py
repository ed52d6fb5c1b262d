"""GPU discrete adjoint (emt_adjoint) against the CPU oracle's adjoint and
against central finite differences.

The oracle's adjoint is itself pinned to complex-step derivatives
(tests/test_oracle_adjoint.py).  Targets v* come from the oracle run with
seeded +-5% parameter perturbations.  Gradients are compared norm-wise:
max_i |g_gpu - g_cpu| <= 1e-9 max_i |g_cpu|.
"""
import numpy as np
import pytest

import oracle
from paper_1903_01081_b300 import emt, netgen as g

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-9


def switched_network():
    net = g.multi_subsystem(141, [3, 6, 2, 5, 4], n_lines=8, n_sources=2, dt=20e-6, n_series_extra=2)
    nodes = np.random.default_rng(6).choice(net.n_nodes, size=2, replace=False)
    net.sw_k = nodes.astype(np.int32)
    net.sw_m = np.array([-1, int(nodes[0])], np.int32)
    net.sw_r = np.array([0.05, 1.5])
    net.sw_close_step = np.array([250, 420], np.int64)
    net.sw_open_step = np.array([-1, 610], np.int64)
    return net


def target_of(net, n_steps, seed=1005):
    br, amp = g.adjoint_target(net, seed=seed)
    pert = net.copy()
    pert.br_value, pert.src_amp = br, amp
    return np.ascontiguousarray(oracle.simulate(pert, n_steps))


def gpu_adjoint(net, tgt, n_steps, ckpt_every, overlap=True):
    ctx = emt.emt_build_network(net)
    if not overlap:
        emt.emt_set_option(ctx, "adjoint_overlap", 0)
    emt.emt_prefactor(ctx)
    out = emt.emt_adjoint(ctx, tgt, n_steps, ckpt_every)
    emt.emt_destroy(ctx)
    return out


def close(got, ref, tol=GRAD_TOL):
    return np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


def test_adjoint_matches_the_cpu_adjoint_with_switches_and_lines():
    net = switched_network()
    N = 700   # ten 64-step segments and a ragged one of 60
    tgt = target_of(net, N)
    g_ref, J_ref = oracle.adjoint(net, N, tgt)
    J, grad = gpu_adjoint(net, tgt, N, 64)
    assert abs(J - J_ref) <= 1e-12 * J_ref
    assert close(grad, g_ref)
    # every parameter kind is exercised
    for kind in (0, 1, 2):
        sel = np.flatnonzero(net.br_kind == kind)
        assert np.max(np.abs(g_ref[sel])) > 0
    assert np.max(np.abs(g_ref[net.n_branches:])) > 0


def test_checkpoint_spacing_gives_bit_identical_results():
    net = switched_network()
    N = 700
    tgt = target_of(net, N)
    ref = gpu_adjoint(net, tgt, N, 0)          # whole tape, no recomputation
    for K in (1, 64, 256, 699, 700, 5000):
        for overlap in (True, False):
            J, grad = gpu_adjoint(net, tgt, N, K, overlap)
            assert J == ref[0], (K, overlap)
            assert np.array_equal(grad, ref[1]), (K, overlap)


def test_device_tensors_and_stream():
    import torch
    net = switched_network()
    N = 300
    tgt = target_of(net, N)
    J_h, g_h = gpu_adjoint(net, tgt, N, 64)
    ctx = emt.emt_build_network(net)
    emt.emt_prefactor(ctx)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        J_d, g_d = emt.emt_adjoint(ctx, torch.from_numpy(tgt).cuda(), N, 64, stream=s)
    emt.emt_destroy(ctx)
    assert g_d.is_cuda and J_d == J_h
    assert np.array_equal(g_d.cpu().numpy(), g_h)


def test_adjoint_with_runtime_switches():
    """Rectifier loads and breakers: the reverse sweep uses the switch states
    the forward run decided (word tape), across checkpoint segments."""
    base = g.multi_subsystem(43, [2, 3, 2], n_lines=4, n_sources=2, dt=20e-6, n_series_extra=2,
                             delay_range=(1, 6))
    net = g.with_rectifier_loads(base, seed=7, n_rectifiers=3, n_breakers=2, trip_range=(100, 300))
    N = 900
    tgt = target_of(net, N)
    g_ref, J_ref = oracle.adjoint(net, N, tgt)
    st = oracle.runtime_switch_states(net, N)
    assert (st.min(axis=0) != st.max(axis=0)).any()
    ref = gpu_adjoint(net, tgt, N, 0)
    assert abs(ref[0] - J_ref) <= 1e-12 * J_ref
    assert close(ref[1], g_ref)
    for K in (1, 64, 300):
        for overlap in (True, False):
            J, grad = gpu_adjoint(net, tgt, N, K, overlap)
            assert J == ref[0] and np.array_equal(grad, ref[1]), (K, overlap)


def test_adjoint_with_coupled_lines():
    """Clarke-mode coupled lines with interpolated travel times: the reverse of
    the modal exchange, across checkpoint segments."""
    base = g.multi_subsystem(44, [2, 3, 2, 2], n_lines=5, n_sources=2, dt=20e-6, n_series_extra=2,
                             delay_range=(1, 6))
    net = g.with_coupled_lines(base, seed=8)
    N = 900
    tgt = target_of(net, N)
    g_ref, J_ref = oracle.adjoint(net, N, tgt)
    ref = gpu_adjoint(net, tgt, N, 0)
    assert abs(ref[0] - J_ref) <= 1e-12 * J_ref
    assert close(ref[1], g_ref)
    for K in (1, 64, 300):
        for overlap in (True, False):
            J, grad = gpu_adjoint(net, tgt, N, K, overlap)
            assert J == ref[0] and np.array_equal(grad, ref[1]), (K, overlap)


def test_single_subsystem_and_one_step():
    net = g.single_rlc(n_steps=400)
    for N, K in ((1, 1), (400, 32)):
        tgt = target_of(net, N)
        g_ref, J_ref = oracle.adjoint(net, N, tgt)
        J, grad = gpu_adjoint(net, tgt, N, K)
        assert abs(J - J_ref) <= 1e-12 * J_ref
        assert close(grad, g_ref)


def test_autograd_function():
    import torch
    from paper_1903_01081_b300.autograd import emt_loss, parameters_of
    net = switched_network()
    N = 400
    tgt = target_of(net, N)
    p = torch.tensor(parameters_of(net), dtype=torch.float64, device="cuda", requires_grad=True)
    J = emt_loss(p, net, torch.from_numpy(tgt).cuda(), N, 64)
    (3.0 * J).backward()
    g_ref, J_ref = oracle.adjoint(net, N, tgt)
    assert abs(J.item() - J_ref) <= 1e-12 * J_ref
    assert close(p.grad.cpu().numpy() / 3.0, g_ref)


def test_adjoint_rejects_what_it_cannot_do():
    net, sc = g.n1_contingency(seed=79, n_scenarios=4, n_buses=20, n_sub=4, n_lines=5, n_sources=2,
                               n_steps=100, fault_step=50, target_branches=120)
    ctx = emt.emt_build_network(net, sc)
    emt.emt_prefactor(ctx)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_adjoint(ctx, np.zeros((10, net.n_nodes)), 10, 4)
    assert ei.value.status == emt.EMT_EINVAL
    emt.emt_destroy(ctx)
    net = switched_network()
    ctx = emt.emt_build_network(net)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_adjoint(ctx, np.zeros((10, net.n_nodes)), 10, 4)
    assert ei.value.status == emt.EMT_ESTATE
    emt.emt_prefactor(ctx)
    with pytest.raises(ValueError):
        emt.emt_adjoint(ctx, np.zeros((9, net.n_nodes)), 10, 4)
    with pytest.raises(emt.EmtError) as ei:
        emt.emt_adjoint(ctx, np.zeros((10, net.n_nodes)), 10, -1)
    assert ei.value.status == emt.EMT_EINVAL
    emt.emt_destroy(ctx)


def test_large_network_matches_the_cpu_adjoint_on_a_short_horizon():
    """The 3,000-node, ~100-subsystem network, 1,000 steps."""
    net = g.large_scale()
    N = 1000
    tgt = target_of(net, N)
    g_ref, J_ref = oracle.adjoint(net, N, tgt)
    J, grad = gpu_adjoint(net, tgt, N, 256)
    assert abs(J - J_ref) <= 1e-12 * J_ref
    assert close(grad, g_ref)


def fd_parameters(grad, params, J, count=20, seed=1005, min_share=1e-2):
    """Seeded draw of `count` parameters whose logarithmic sensitivity
    |p dJ/dp| is at least min_share * J: below that the rounding noise of
    the computed J, divided by the step, approaches the 1e-6 tolerance."""
    ok = np.flatnonzero(np.abs(params * grad) >= min_share * J)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(ok, size=min(count, ok.size), replace=False))


def test_full_size_gradient_against_cpu_adjoint_complex_step_and_differences():
    """3,000 nodes, 20,000 steps, checkpoints every 256 steps.

    (1) the oracle's adjoint, all parameters, norm-wise 1e-9;
    (2) the oracle's complex-step derivative of the most sensitive branch;
    (3) 20 seeded parameters against the fourth-order central difference
        (J(p-2h) - 8 J(p-h) + 8 J(p+h) - J(p+2h)) / 12h with h = 1e-4 |p|,
        relative 1e-6.  Measured on one branch (C, share 1e-2): errors
        1.7e-8 (h = 1e-3 |p|), 4.2e-8 (1e-4), 2.1e-6 (1e-5), 5.8e-6 (1e-6):
        below 1e-4 the rounding noise of J dominates."""
    import torch
    from paper_1903_01081_b300.autograd import parameters_of
    net = g.large_scale()
    N = 20000
    tgt_h = target_of(net, N)
    tgt = torch.from_numpy(tgt_h).cuda()
    J, grad = gpu_adjoint(net, tgt, N, 256)
    grad = grad.cpu().numpy()
    params = parameters_of(net)
    nb = net.n_branches

    g_ref, J_ref = oracle.adjoint(net, N, tgt_h)
    assert abs(J - J_ref) <= 1e-11 * J_ref
    assert close(grad, g_ref)
    top = int(np.argmax(np.abs(params[:nb] * grad[:nb])))
    _, d_cs = oracle.loss_complex_step(net, N, tgt_h, top)
    assert abs(grad[top] - d_cs) <= 1e-9 * abs(d_cs)

    idx = fd_parameters(grad, params, J)
    assert idx.size == 20

    def loss_at(i, delta):
        run = net.copy()
        run.br_value = net.br_value.copy()
        run.src_amp = net.src_amp.copy()
        if i < nb:
            run.br_value[i] += delta
        else:
            run.src_amp[i - nb] += delta
        ctx = emt.emt_build_network(run)
        emt.emt_prefactor(ctx)
        Jx = emt.emt_adjoint(ctx, tgt, N, 256)[0]
        emt.emt_destroy(ctx)
        return Jx

    for i in idx:
        h = 1e-4 * abs(params[i])
        fd = (loss_at(i, -2 * h) - 8 * loss_at(i, -h) + 8 * loss_at(i, h) - loss_at(i, 2 * h)) / (12 * h)
        assert abs(fd - grad[i]) <= 1e-6 * abs(grad[i]), (i, fd, grad[i])
