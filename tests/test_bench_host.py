"""Host-side pieces of the benchmark (no GPU): the drift fit, the clock-record
parser, and the rule that a committed ncu summary only supplies the roofline's
DRAM traffic while the kernel sources and the tuning it was taken with are
the current ones."""
import os

import numpy as np

import bench


def _log(steps, etot):
    dt = np.dtype([("step", "<i8", (1,)), ("etot_per_n", "<f8", (1,))])
    log = np.zeros(len(steps), dtype=dt)
    log["step"][:, 0] = steps
    log["etot_per_n"][:, 0] = etot
    return log


def test_drift_fit_recovers_a_known_slope():
    dt = 0.005
    steps = np.arange(10, 1010, 10)
    e = -5.0 + 2e-4 * steps * dt + 1e-7 * np.sin(steps)
    slope, fluct = bench.drift_per_tau(_log(steps, e), dt)
    assert abs(slope - 2e-4) < 1e-7
    assert 0.0 < fluct < 2e-7
    assert bench.drift_per_tau(_log([10, 20], [0.0, 1.0]), dt) == (None, None)


def test_clock_record_parsing():
    rows = [
        "0, 2070, 2070, 1200.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1250.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    rec = bench.parse_clock_samples(rows)
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples"] == 3
    assert bench.parse_clock_samples([])["reasons"] == ["no samples"]


def _fake_tree(root, source):
    csrc = root / "paper_2001_07089_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(source)
    (root / "profiles").mkdir()


def test_traffic_only_for_current_sources_and_tuning(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _fake_tree(tmp_path, "__global__ void k() {}\n")
    tuning = {"threads_per_atom": 4, "block_size": 512, "skin": 0.3, "skin_outer": 1.2}
    assert bench.profiled_traffic("ka32k", tuning) is None  # no summary yet
    summary = tmp_path / "profiles" / "md_persistent_ka32k.md"
    summary.write_text(
        "# summary\n\n"
        f"- `kernel_sources_sha256`: `{bench.kernel_sources_digest()}`\n"
        "- `tuning`: `4,512,0.3,1.2`\n"
        "- `dram_bytes_per_launch`: `216729856`\n")
    assert bench.profiled_traffic("ka32k", tuning) == 216729856.0
    assert bench.profiled_traffic("ka32k", dict(tuning, skin_outer=0.3)) is None
    assert bench.profiled_traffic("ka1m", tuning) is None
    (tmp_path / "paper_2001_07089_gb300" / "csrc" / "k.cu").write_text("__global__ void k() { }\n")
    assert bench.profiled_traffic("ka32k", tuning) is None  # the kernel changed since the capture


def test_committed_summaries_carry_the_fields_the_bench_reads():
    prof = os.path.join(bench.ROOT, "profiles")
    # the per-workload launch summaries that profiled_traffic reads (other summaries, such as a
    # phase timed alone, carry no traffic fields)
    names = [n for n in os.listdir(prof) if n in {f"md_persistent_{w}.md" for w in bench.WORKLOADS}]
    assert names
    for n in names:
        text = open(os.path.join(prof, n)).read()
        for key in ("kernel_sources_sha256", "tuning", "dram_bytes_per_launch"):
            assert f"- `{key}`: `" in text, (n, key)
        assert "--clock-control none" in text


def test_drift_equal_or_better_rule():
    a = {"slope": 1e-6, "err": 1e-7}
    assert bench.drift_equal_or_better(a, {"slope": -2e-6, "err": 1e-7}) is True
    assert bench.drift_equal_or_better({"slope": 5e-6, "err": 1e-7}, {"slope": 1e-6, "err": 1e-7}) is False
    # within two combined error bars counts as equal
    assert bench.drift_equal_or_better({"slope": 1.2e-6, "err": 1e-7}, {"slope": 1e-6, "err": 1e-7}) is True
    assert bench.drift_equal_or_better(None, a) is None


def test_drift_stats_window_and_error():
    dt = 0.005
    steps = np.arange(10, 2010, 10)
    rng = np.random.default_rng(1)
    e = -5.4 + 3e-6 * steps * dt + rng.normal(0, 1e-5, size=len(steps))
    d = bench.drift_stats(_log(steps, e), dt)
    assert d["window_steps"] == 1990
    assert abs(d["slope"] - 3e-6) < 4 * d["err"] and 0 < d["err"] < 1e-5
    assert bench.drift_stats(_log([10, 20, 30], [0.0, 1.0, 2.0]), dt)["slope"] is None


def test_replica_partition_is_complete_disjoint_and_balanced():
    from paper_2001_07089_gb300 import workloads as wl
    n = wl.ensemble(512, 4).n
    for world in (1, 2, 3, 4, 8):
        parts = bench.partition_replicas(n, world)
        flat = sorted(r for p in parts for r in p)
        assert flat == list(range(len(n)))
        loads = [int(n[p].sum()) for p in parts]
        assert max(loads) - min(loads) <= int(n.max())
        assert all(p == sorted(p) for p in parts)
