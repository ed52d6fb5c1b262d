"""Multi-rank paths of bench.py on CPU (gloo, world size 2, 127.0.0.1):
max-over-ranks timing and the whole-job rate, and the reference arm
printing from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def torchrun(*args, timeout=300):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.join(ROOT, "bench.py"), *args]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    return subprocess.run(cmd, capture_output=True, text=True, timeout=timeout, cwd=ROOT, env=env)


def json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_two_ranks_take_the_slowest_rank_and_count_all_units():
    r = torchrun("--selftest-ranks")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1                      # rank 0 alone prints
    d = lines[0]
    assert d["world"] == 2 and d["t_max"] == 1.5   # ranks report 1.0 and 1.5
    assert d["value"] == pytest.approx(2 * 1000.0 / 1.5)


@pytest.mark.slow
def test_reference_arm_prints_on_rank_zero_only():
    r = torchrun("--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference"
    assert lines[0]["value"] > 0 and lines[0]["cpu_baseline"]["kind"] == "oracle"
