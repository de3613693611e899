"""Host logic of the autotuning cache (no GPU)."""
from paper_2001_07089_gb300 import autotune


class FakeSystem:
    precision = "mixed"
    n_per = [32000]
    L_per = [29.876]

    def __init__(self):
        self.applied = None
        self.probed = 0

    def set_tuning(self, **kw):
        self.applied = kw

    def autotune(self, dt, probe_steps):
        self.probed += 1
        return {"threads_per_atom": 4, "block_size": 256, "skin": 0.3, "skin_outer": 0.8}, 2.5e-5


def test_key_buckets_size_density_and_gpu():
    k1 = autotune.cache_key("GB300", "mixed", [32000], [29.876])
    k2 = autotune.cache_key("GB300", "mixed", [33000], [30.19])
    k3 = autotune.cache_key("GB300", "fp64", [32000], [29.876])
    k4 = autotune.cache_key("GB300", "mixed", [1_000_000], [94.104])
    assert k1 == k2 and k1 != k3 and k1 != k4
    assert "rho1.20" in k1 and "r1" in k1


def test_tune_probes_once_then_reuses(tmp_path):
    path = str(tmp_path / "t.json")
    s = FakeSystem()
    t1 = autotune.tune(s, 0.005, "GB300", path=path)
    assert s.probed == 1 and s.applied is None
    s2 = FakeSystem()
    t2 = autotune.tune(s2, 0.005, "GB300", path=path)
    assert s2.probed == 0 and t2 == t1
    assert s2.applied == {"threads_per_atom": 4, "block_size": 256, "skin": 0.3, "skin_outer": 0.8}
    s3 = FakeSystem()
    autotune.tune(s3, 0.005, "GB300", path=path, refresh=True)
    assert s3.probed == 1
