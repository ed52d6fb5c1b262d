"""Workloads the checks-build test runs (tests/test_gpu_checks.py): forward
runs of the large-scale network, of a network with every feature, of
converter stations (states factorised at run time), of arrester sets
(several nonlinear resistors per subsystem) and of the 500 x 6-node network
(the 64-register build), frequency-dependent line groups, scenario sets
(one with the shared-matrix solve on the tensor cores) and an adjoint gradient.

    python tests/checks_workload.py OUT.npz

writes every result and the emt_sync status of each run.  Which library it
uses follows EMT_CHECKS (see paper_1903_01081_b300.emt.checks_build)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from paper_1903_01081_b300 import emt, netgen as g  # noqa: E402


def forward(net, N, sc=None, options=None):
    sim = emt.Simulator(net, sc, n_steps=N, options=options)
    sim.run(N)
    status = 0
    try:
        sim.sync()
    except emt.EmtError as e:
        status = e.status
    w = sim.waveforms() if status == 0 else np.zeros(0)
    sim.close()
    return w, status


def run_all():
    from test_gpu_combined import combined_network
    out = {}
    base = g.multi_subsystem(41, [3, 5, 4], n_lines=4, n_sources=2, dt=20e-6)
    cases = {
        "large": (g.large_scale(n_steps=1500), 1500, None),
        "combined": (combined_network(), 1500, None),
        "stations": (g.with_converter_stations(base, n_stations=1), 1500, None),
        "bus_arresters": (g.with_bus_arresters(g.multi_subsystem(43, [4, 5, 3], n_lines=4, n_sources=2, dt=20e-6),
                                               n_buses=1, scale=(0.07, 0.09)), 1500, None),
        "strict500": (g.large_scale(strict_500=True, n_steps=600), 600, None),
    }
    net, sc = g.n1_contingency(seed=77, n_scenarios=12, n_buses=40, n_sub=8, n_lines=12, n_sources=3,
                               n_steps=600, fault_step=300, target_branches=240)
    cases["n1"] = (net, 600, sc)
    cases["fd_groups"] = (g.with_fd_line_groups(g.multi_subsystem(161, [3, 4, 2, 3, 5], n_lines=8, n_sources=2,
                                                                    dt=20e-6)), 1500, None)
    # the shared-matrix solve on the tensor cores (every shared matrix in digit form)
    sg_base = g.multi_subsystem(91, [3, 5, 2, 4, 6], n_lines=9, n_sources=3, dt=20e-6, n_series_extra=2)
    net, sc = g.shared_g(seed=92, n_scenarios=40, n_steps=600, fault_step=200, base=sg_base)
    cases["shared_g_tcgen05"] = (net, 600, sc, {"digit_solve": 1, "digit_min_rows": 1})
    for name, case in cases.items():
        net, N, sc = case[:3]
        w, status = forward(net, N, sc, case[3] if len(case) > 3 else None)
        out[name] = w
        out[name + "_status"] = np.array([status])
    # adjoint gradient of a small network
    net = g.multi_subsystem(21, [4, 3, 5], n_lines=5, n_sources=2, dt=20e-6)
    N = 400
    tgt, _ = forward(net, N)
    br, amp = g.adjoint_target(net, seed=3)
    pert = net.copy()
    pert.br_value, pert.src_amp = br, amp
    target, _ = forward(pert, N)
    ctx = emt.emt_build_network(net)
    emt.emt_prefactor(ctx)
    status = 0
    try:
        J, grad = emt.emt_adjoint(ctx, target[:, 0, :], N, 64)
        out["adjoint"] = np.asarray(grad)
    except emt.EmtError as e:
        status = e.status
        out["adjoint"] = np.zeros(0)
    out["adjoint_status"] = np.array([status])
    emt.emt_destroy(ctx)
    return out


if __name__ == "__main__":
    np.savez(sys.argv[1], **run_all())
