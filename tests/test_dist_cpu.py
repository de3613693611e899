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


PARTITION_WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
from paper_2001_07089_gb300 import workloads as wl
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:{port}", rank=int(sys.argv[1]), world_size=2)
r, w = dist.get_rank(), dist.get_world_size()
spec = wl.ensemble(512, 4)
mine = bench.partition_replicas(spec.n, w)[r]
got = [None] * w
dist.all_gather_object(got, mine)
n_rank = int(spec.n[mine].sum())
total = bench.sum_over_ranks(n_rank, dist, "cpu")
slow = bench.max_over_ranks(1.0 + 0.5 * r, dist, "cpu")
flat = sorted(x for p in got for x in p)
assert flat == list(range(512)), "partition not complete/disjoint"
assert total == int(spec.n.sum())
loads = [int(spec.n[p].sum()) for p in got]
assert max(loads) - min(loads) <= int(spec.n.max())
dist.barrier()
print(f"rank {{r}} ok {{len(mine)}} {{n_rank}} {{int(total)}} {{slow}}", flush=True)
dist.destroy_process_group()
"""


def test_two_gloo_ranks_split_the_ensemble():
    """The 512-replica ensemble on two ranks: each rank takes its share of the greedy N-balanced
    partition; together the shares are the whole ensemble, once, with loads within one replica's N;
    the whole-job atom count and the slowest rank's time come from collectives."""
    import tempfile
    port = _free_port()
    with tempfile.TemporaryDirectory() as td:
        script = os.path.join(td, "worker.py")
        with open(script, "w") as f:
            f.write(PARTITION_WORKER.format(root=ROOT, port=port))
        procs = [subprocess.Popen([sys.executable, script, str(r)], stdout=subprocess.PIPE, stderr=subprocess.PIPE)
                 for r in range(2)]
        outs = []
        for p in procs:
            o, e = p.communicate(timeout=120)
            assert p.returncode == 0, e.decode()
            outs.append(o.decode().split())
    assert [o[:2] for o in outs] == [["rank", "0"], ["rank", "1"]]
    assert all(o[2] == "ok" for o in outs)
    assert int(outs[0][4]) + int(outs[1][4]) == int(outs[0][5]) == int(outs[1][5])
    assert float(outs[0][6]) == float(outs[1][6]) == 1.5
