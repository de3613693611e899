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


# ------------------------------------------------------------------ long-run statistics

def _ar1(n, phi, sigma, rng):
    x = np.zeros(n)
    z = rng.normal(0.0, sigma, size=n)
    for k in range(1, n):
        x[k] = phi * x[k - 1] + z[k]
    return x


def test_drift_fit_error_bar_is_calibrated_on_correlated_noise():
    """A known slope under strongly correlated (AR(1), phi = 0.95) noise: over many independent
    series the bootstrap error bar matches the actual scatter of the fitted slopes (within 35 %),
    and about 95 % of fits lie within 2 error bars of the true slope. A bar that ignored the
    correlation (plain least squares) would be several times too small and fail both."""
    rng = np.random.default_rng(3)
    t = np.arange(1000) * 0.05
    slope = 2e-5
    fits = []
    for _ in range(200):
        e = -5.0 + slope * t + _ar1(len(t), 0.95, 1e-5, rng)
        fits.append(analysis.drift_fit(t, e, nboot=200, seed=int(rng.integers(1 << 30))))
    s = np.array([f["slope"] for f in fits])
    err = np.array([f["err"] for f in fits])
    assert 0.65 < np.median(err) / np.std(s) < 1.35
    inside = np.mean(np.abs(s - slope) <= 2 * err)
    assert 0.85 <= inside <= 0.995
    # no trend: zero within the bar; too short a series: no fit
    f0 = analysis.drift_fit(t, -5.0 + _ar1(len(t), 0.9, 1e-5, rng))
    assert abs(f0["slope"]) < 4 * f0["err"]
    assert analysis.drift_fit(t[:3], t[:3])["slope"] is None


def test_block_mean_error_of_independent_samples():
    rng = np.random.default_rng(5)
    x = rng.normal(2.0, 0.5, size=(20000, 3))
    m, e = analysis.block_mean(x, 20)
    assert np.allclose(m, 2.0, atol=4 * 0.5 / np.sqrt(20000))
    assert np.all((e > 0.5 * 0.5 / np.sqrt(20000)) & (e < 1.6 * 0.5 / np.sqrt(20000)))
    with pytest.raises(ValueError):
        analysis.block_mean(x[:1], 2)


def test_msd_over_time_origins_of_ballistic_particles():
    """Particles moving at constant velocity: MSD(lag) = <v^2> (lag dt)^2 per type, for any origin."""
    rng = np.random.default_rng(7)
    n, frames, dt = 50, 40, 0.1
    v = rng.normal(size=(n, 3))
    x0 = rng.uniform(0, 10, size=(n, 3))
    types = np.array([0] * 30 + [1] * 20)
    traj = x0[None] + v[None] * (np.arange(frames) * dt)[:, None, None]
    lags = [1, 5, 20]
    m = analysis.msd_time_origins(traj, types, 2, lags, origin_every=3)
    v2 = np.sum(v * v, axis=1)
    for k, lag in enumerate(lags):
        assert m[k, 0] == pytest.approx(v2[:30].mean() * (lag * dt) ** 2, rel=1e-12)
        assert m[k, 1] == pytest.approx(v2[30:].mean() * (lag * dt) ** 2, rel=1e-12)
