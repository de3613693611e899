"""Measurement schedules: the log-spaced MSD grid against the paper's loop."""
import math

import numpy as np
import pytest

import oracle
from paper_2001_07089_gb300 import analysis


@pytest.mark.parametrize("n_md,t0,kmax", [(1000, 1.0, 60), (10000, 1.0, 60), (100000, 2.0, 40), (50, 1.0, 10)])
def test_log_grid_matches_oracle_loop(n_md, t0, kmax):
    assert analysis.log_time_grid(n_md, t0, kmax) == oracle.log_time_grid(n_md, t0, kmax)


def test_log_grid_shape_follows_eq_A():
    """Eq. (A): the k_max-th point lands on n_MD; points are distinct, increasing, and
    once they are far apart their ratios approach A."""
    n_md, kmax = 100000, 60
    g = analysis.log_time_grid(n_md, 1.0, kmax)
    A = n_md ** (1.0 / kmax)
    assert g[0] == 1 and g[-1] == n_md
    assert all(b > a for a, b in zip(g, g[1:]))
    assert len(g) <= kmax + 1
    tail = np.array(g[-10:], dtype=float)
    assert np.allclose(tail[1:] / tail[:-1], A, rtol=2e-3)
    # the first steps are consecutive integers while A*t grows by less than 1
    assert g[:5] == [1, 2, 3, 4, 5]


class _Clock:
    """Stand-in system: a step counter whose 'MSD' against a slot is the time since that slot's reset."""

    ntypes = 2

    def __init__(self):
        self.step = 0
        self.ref = {}
        self.calls = []

    def advance(self, n):
        assert n > 0
        self.step += n

    def msd_tw(self, slot, reset_reference=False):
        self.calls.append((self.step, slot, reset_reference))
        if reset_reference:
            self.ref[slot] = self.step
        return np.array([self.step - self.ref[slot], 2.0 * (self.step - self.ref[slot])], dtype=float)


def test_waiting_time_schedule_follows_every_tw_on_one_trajectory():
    sysm = _Clock()
    t_ws = [100, 0, 10, 500]
    res = analysis.waiting_time_msd(sysm, t_ws, n_md=1000, advance=sysm.advance, kmax=20)
    grid = analysis.log_time_grid(1000, 1.0, 20)
    steps = [c[0] for c in sysm.calls]
    assert steps == sorted(steps)  # one trajectory, never rewound
    assert sysm.step == 500 + grid[-1]
    resets = {slot: st for st, slot, r in sysm.calls if r}
    assert sorted(resets.values()) == [0, 10, 100, 500] and 0 not in resets  # slot 0 stays md_msd's
    for tw in t_ws:
        t, m = res[tw]
        assert list(t) == grid
        assert np.array_equal(m[:, 0], np.array(grid, dtype=float))  # measured exactly t after t_w
        assert np.array_equal(m[:, 1], 2.0 * np.array(grid, dtype=float))
    with pytest.raises(ValueError):
        analysis.waiting_time_msd(_Clock(), list(range(8)), 100, advance=lambda n: None)
    with pytest.raises(ValueError):
        analysis.waiting_time_msd(_Clock(), [5, 5], 100, advance=lambda n: None)


class _Recorder:
    nrep = 2

    def __init__(self):
        self.calls = []

    def step_nvt(self, dt, n, T, kind, param, seed, log_every):
        self.calls.append(("nvt", n, T, kind, param, seed))
        return "bath"

    def step_nve(self, dt, n, log_every=0):
        self.calls.append(("nve", n))
        return "nve"


def test_cooling_ladder_runs_bath_nve_production_per_temperature():
    from paper_2001_07089_gb300 import kamd
    rec = _Recorder()
    temps = [5.0, 4.0, 3.0, 2.0, 1.0, 0.8, 0.6, 0.55, 0.5, 0.475, 0.466]
    out = analysis.cooling_ladder(rec, temps, 0.005, n_bath=200, n_nve=200, n_prod=400, nstep_boltz=50, seed=9)
    assert [s["T"] for s in out] == temps
    expect = []
    for k, T in enumerate(temps):
        expect += [("nvt", 200, T, kamd.MD_NVT_RESAMPLE, 50, 9 + k), ("nve", 200), ("nve", 400)]
    assert rec.calls == expect
    seen = []
    analysis.cooling_ladder(_Recorder(), [2.0, 1.0], 0.005, 10, 10, 10, production=lambda s, T: seen.append(T) or T)
    assert seen == [2.0, 1.0]
