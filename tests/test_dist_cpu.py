"""The multi-rank (N > 1) bench path on CPU: two gloo ranks agree on the
max-over-ranks time and on the whole-job rate, and the reference arm does
no work on ranks other than 0."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:{port}", rank=int(sys.argv[1]), world_size=2)
r = dist.get_rank()
t = bench.max_over_ranks(1.0 + r, dist, "cpu")
v = bench.whole_job_rate(dist.get_world_size(), 32000, 100, t)
dist.barrier()
print(f"rank {{r}} max {{t}} rate {{v}}", flush=True)
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_agree_on_max_time_and_rate(tmp_path):
    port = _free_port()
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT, port=port))
    procs = [subprocess.Popen([sys.executable, str(script), str(r)], stdout=subprocess.PIPE, stderr=subprocess.PIPE)
             for r in range(2)]
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e.decode()
        outs.append(o.decode().strip())
    for r, o in enumerate(outs):
        assert o == f"rank {r} max 2.0 rate {2 * 32000 * 100 / 2.0}"


def test_reference_arm_other_ranks_do_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, timeout=120)
    assert p.returncode == 0
    assert p.stdout.decode().strip() == ""
