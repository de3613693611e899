"""Failure detection on the GPU without a GPU fault.

* a barrier wait that is made to run out (one block never arrives) returns
  MD_ERR_TIMEOUT within its limit, and the system stays usable;
* a NaN velocity is reported as MD_ERR_UNSTABLE;
* a neighbour list that starts far too small overflows, is regrown on the
  host and the run continues bitwise identical to an unconstrained run.
"""
import os
import time

import numpy as np
import pytest

import oracle
from paper_2001_07089_gb300 import kamd
from paper_2001_07089_gb300 import workloads as wl
from tests.helpers import force_errors, ka_params, melted

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kamd.load()


def _sys(n, L, types, prec="mixed"):
    return kamd.System(n, L, types, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, 1.0, 0.3, prec)


def test_barrier_wait_runs_out_and_context_stays_usable():
    pos, vel, types, L = melted(1000, 101, nsteps=50)
    with _sys(1000, L, types) as s:
        s.set_state(pos, vel)
        t0 = time.perf_counter()
        st = kamd.md_selftest_barrier(s.handle, 0.5)
        el = time.perf_counter() - t0
        assert st == kamd.MD_ERR_TIMEOUT
        assert 0.4 < el < 10.0
        assert "ran out" in kamd.md_last_error(s.handle)
        f, pe, _ = s.forces()
    f_ref, v_ref, _ = oracle.forces(pos, types, ka_params(), L)
    emax, e2 = force_errors(f, f_ref)
    assert emax < 1e-5 and e2 < 1e-5


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nan_velocity_reported_unstable(prec):
    pos, vel, types, L = melted(1000, 102, nsteps=50)
    bad = vel.copy()
    bad[17, 1] = np.nan
    with _sys(1000, L, types, prec) as s:
        s.set_state(pos, bad)
        with pytest.raises(kamd.KamdError) as ei:
            s.step_nve(0.005, 10)
        assert ei.value.status == kamd.MD_ERR_UNSTABLE
        # a fresh state makes the handle usable again
        s.set_state(pos, vel)
        s.step_nve(0.005, 10)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_runaway_move_reported_unstable(prec):
    pos, vel, types, L = melted(1000, 103, nsteps=50)
    fast = vel.copy()
    fast[5] = [L * 100.0, 0.0, 0.0]
    with _sys(1000, L, types, prec) as s:
        s.set_state(pos, fast)
        with pytest.raises(kamd.KamdError) as ei:
            s.step_nve(0.005, 5)
        assert ei.value.status == kamd.MD_ERR_UNSTABLE


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_list_overflow_regrows_and_matches(prec, monkeypatch):
    pos, vel, types, L = melted(1000, 104, nsteps=100)
    runs = []
    for cap in (None, "6"):
        if cap is None:
            monkeypatch.delenv("KAMD_LIST_CAPACITY", raising=False)
        else:
            monkeypatch.setenv("KAMD_LIST_CAPACITY", cap)
        with _sys(1000, L, types, prec) as s:
            s.set_state(pos, vel)
            log = s.step_nve(0.005, 120, log_every=10)
            p, v, _ = s.get_state()
            info = s.info()
        runs.append((p, v, log, info))
    monkeypatch.delenv("KAMD_LIST_CAPACITY", raising=False)
    assert runs[1][3]["list_capacity"] > 6
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert np.array_equal(runs[0][2], runs[1][2])
