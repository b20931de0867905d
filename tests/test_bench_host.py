"""Host logic of bench.py, no GPU: the launch counts the JSON line claims,
the double-float instruction model, the traffic lookup, and the reference
arm's JSON line (the oracle on the host cores) against the bench contract."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_launches_per_solve():
    # 10000 steps: one launch per `depth` steps; the double-float kernel adds its prescale
    assert bench.launches_per_solve("temporal", 48) == 209
    assert bench.launches_per_solve("temporal", 128) == 79
    assert bench.launches_per_solve("temporal_df", 96) == 105 + 1
    assert bench.launches_per_solve("temporal_df", 1) == 10000 + 1
    assert bench.launches_per_solve("onestep", 48) == 10000
    assert bench.launches_per_solve("canonical", 1) == 10000
    assert bench.launches_per_solve("subdomain16_onestep", 1) == 10000


def test_double_float_instruction_model():
    # 2r an FP32 number: the fast product path (12.5 instructions per update)
    assert bench.two_r_is_fp32(2.0) and bench.two_r_is_fp32(0.375)
    assert not bench.two_r_is_fp32(0.3) and not bench.two_r_is_fp32(1.0 / 3.0)
    assert bench.DF_OPS_PER_UPDATE[True] < bench.DF_OPS_PER_UPDATE[False]


def test_traffic_lookup_is_keyed_by_kernel_and_source():
    assert bench.measured_traffic("no_such_kernel<int>") is None
    got = bench.measured_traffic("tb_kernel<double>")
    # an entry is used only while the kernel's sources are the ones it was captured from
    assert got is None or (isinstance(got, int) and got > 0)
    for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, sha, nbytes = line.split()[:3]
        assert len(sha) >= 12 and int(nbytes) > 0, line


@pytest.mark.timeout(600)
def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 1
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["n"] == bench.N_POINTS


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_prints_once():
    """Two ranks: rank 0 alone runs the oracle and prints the line; the other
    rank exits 0 without work."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def test_shard_problems_balances_points():
    """Config 3 sharded by problem: contiguous blocks covering every problem
    once, at least one per rank, points within one problem's size of an
    equal share."""
    from paper_1310_3422_gb300 import inputs
    bt = inputs.uneven_batch()
    for world in (1, 2, 3, 4, 8):
        cuts = bench.shard_problems(bt.n, world)
        assert cuts[0] == 0 and cuts[-1] == len(bt.n) and len(cuts) == world + 1
        assert all(cuts[q + 1] > cuts[q] for q in range(world))
        share = bt.n.sum() / world
        for q in range(world):
            pts = bt.n[cuts[q]:cuts[q + 1]].sum()
            assert abs(pts - share) <= bt.n.max() + 1
    # more ranks than would balance: still one problem each
    assert bench.shard_problems([1000, 1, 1, 1], 4) == [0, 1, 2, 3, 4]
