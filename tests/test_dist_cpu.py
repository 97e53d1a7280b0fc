"""Multi-rank logic of bench.py on CPU: world size 2 over gloo.

The method shards nothing (replicas only), so the only cross-rank operations
are the max of the timed regions and the sums of whole-job totals; the
reference arm runs on rank 0 alone under torchrun and the other rank exits 0.
"""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch, torch.distributed as dist
dist.init_process_group("gloo")
import bench
r = dist.get_rank(); w = dist.get_world_size()
cpu = torch.device("cpu")
out = {"rank": r, "max": bench.max_over_ranks(float(10 * (r + 1)), w, cpu),
       "sum": bench.sum_over_ranks(float(r + 1), w, cpu), "env": list(bench.dist_env())}
print(json.dumps(out), flush=True)
dist.destroy_process_group()
"""


def test_max_and_sum_over_two_gloo_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["max"] == 20.0 and o["sum"] == 3.0
        assert o["env"] == [o["rank"], 2, o["rank"]]


def test_single_rank_helpers_are_identity():
    import bench
    assert bench.max_over_ranks(1.5, 1, None) == 1.5
    assert bench.sum_over_ranks(2.5, 1, None) == 2.5


def test_reference_arm_prints_once_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "grid2d", "--steps", "1", "--warmup", "1", "--gpus", "2"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
