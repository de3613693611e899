"""Long chaotic runs: GPU paths against the FP64 oracle by their statistics.

Two MD trajectories that start from the same state part ways after a few
hundred steps (the dynamics is chaotic, and FP32 or even FP64 rounding in a
different order is enough), so long runs are compared by what they measure,
with statistical error bars (block averages), not step by step:

* the NVE energy drift per particle per tau (least-squares slope with a
  moving-block bootstrap error; Sec. "NVE molecular dynamics simulation");
* the time averages of the potential energy per particle and of T
  (Eqs. (EsysNpart), (equip3N));
* the partial g_AA, g_BB, g_AB (Eqs. (gAA), (gAB)), one histogram per frame;
* the per-type MSD (Eq. (msdwithi)) at several lags, averaged over time origins.

Workload: N = 1000 Kob-Andersen at density 1.2, melted by the oracle, then
2000 Nose-Hoover steps at T = 0.8 (tau = 0.5) by the oracle. From that
configuration, R = 8 replicas start with fresh Maxwell-Boltzmann velocities at
T = 0.8 (one seed each) and run 10 000 NVE steps at dt = 0.005 (50 tau) on the
mixed GPU path, the FP64 GPU path and the oracle (on all host threads,
per-thread force arrays added in a fixed order), with a frame every 100 steps.
Error bars are run-to-run: the drift of each replica (its least-squares slope)
gives a mean and a standard error over the 8 replicas; time averages (PE/N, T,
g(r), MSD over time origins) are taken over each half of each replica after
the first 1000 steps, 16 samples. Criteria, chosen so that a correct path
fails with a chance of about 1 % over all comparisons (Student t tails):
mean drift within 4.5 sigma of the oracle's; PE/N and T within 4.5 sigma; MSD
within 5 sigma at every lag and type; g(r): mean of z^2 over the bins <= 2 and
every |z| <= 6. The mixed path's drift is also checked to be no worse than the
FP64 path's (|d_mixed| <= |d_fp64| + 4.5 sigma): the metric's "equal or
better NVE energy drift". A single replica's drift is not used alone: over
50 tau the total energy wanders by several 10^-4 per particle (errors at
cutoff crossings add up like a random walk), so one run's slope scatters far
more than its own residuals suggest.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_2001_07089_gb300 import analysis
from paper_2001_07089_gb300 import kamd
from paper_2001_07089_gb300 import workloads as wl
from tests.helpers import ka_params, melted

pytestmark = pytest.mark.gpu

N, SEED, T_EQ, DT = 1000, 36, 0.8, 0.005
R, NVE_STEPS, FRAME, LOG_EVERY = 8, 10000, 100, 10
SKIP = 10  # frames left out of the time averages (velocities were just redrawn)
DR, NBINS = 0.05, 80
LAGS = [1, 2, 4, 8]  # frames


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kamd.load()


def _threads():
    return max(1, min(16, oracle.max_threads()))


@functools.lru_cache(maxsize=None)
def start_state():
    pos, vel, types, L = melted(N, SEED, nsteps=300, T0=T_EQ)
    oracle.set_threads(_threads())
    try:
        eq = oracle.run(pos, vel, types, ka_params(), L, DT, 2000, kind=oracle.NOSE_HOOVER, T_target=T_EQ,
                        Q=3 * N * T_EQ * 0.5 ** 2, log_every=0)
    finally:
        oracle.set_threads(1)
    vels = [oracle.maxwell_boltzmann(N, T_EQ, seed=9000 + r) for r in range(R)]
    return eq["pos"], vels, types, L


def _summarise(thermo, frames, gs):
    """thermo [R, samples, (step, etot, pe, T)], frames [R, F, N, 3], gs [R, F, 3, NBINS] -> statistics."""
    th = np.asarray(thermo)
    frames, gs = np.asarray(frames), np.asarray(gs)
    _, _, types, _ = start_state()
    drift = np.array([analysis.drift_fit(th[r, :, 0] * DT, th[r, :, 1])["slope"] for r in range(R)])
    per_sample = FRAME // LOG_EVERY
    halves = []
    for r in range(R):
        fr = np.arange(SKIP, frames.shape[1])
        for h in np.array_split(fr, 2):
            rows = slice(h[0] * per_sample, (h[-1] + 1) * per_sample)
            halves.append({"pe": th[r, rows, 2].mean(), "T": th[r, rows, 3].mean(), "g": gs[r, h].mean(axis=0),
                           "msd": analysis.msd_time_origins(frames[r, h], types, 2, LAGS)})
    out = {"drift": (drift.mean(), drift.std(ddof=1) / np.sqrt(R), drift)}
    for key in ("pe", "T", "g", "msd"):
        v = np.array([hh[key] for hh in halves])
        out[key] = (v.mean(axis=0), v.std(axis=0, ddof=1) / np.sqrt(len(v)))
    return out


@functools.lru_cache(maxsize=None)
def oracle_run():
    pos, vels, types, L = start_state()
    thermo, frames, gs = [], [], []
    oracle.set_threads(_threads())
    try:
        for r in range(R):
            f, _, _ = oracle.forces(pos, types, ka_params(), L)
            x, v, img = pos, vels[r], np.zeros((N, 3), np.int32)
            rows, fr, g = [], [], []
            for k in range(NVE_STEPS // FRAME):
                out = oracle.run(x, v, types, ka_params(), L, DT, FRAME, forces_in=f, img=img, step0=k * FRAME,
                                 log_every=LOG_EVERY)
                x, v, f, img = out["pos"], out["vel"], out["forces"], out["img"]
                t = out["thermo"]
                rows.append(np.stack([t[:, 0], t[:, 4], t[:, 2], t[:, 1]], axis=1))
                fr.append(x + L * img)
                g.append(oracle.rdf(x, types, L, DR, NBINS))
            thermo.append(np.concatenate(rows))
            frames.append(fr)
            gs.append(g)
    finally:
        oracle.set_threads(1)
    return _summarise(thermo, frames, gs)


@functools.lru_cache(maxsize=None)
def gpu_run(prec):
    pos, vels, types, L = start_state()
    thermo, frames, gs = [], [], []
    for r in range(R):
        rows, fr, g = [], [], []
        with kamd.System(N, L, types, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, wl.KA_MASS, wl.SKIN, prec) as s:
            s.set_state(pos, vels[r])
            for _ in range(NVE_STEPS // FRAME):
                log = s.step_nve(DT, FRAME, log_every=LOG_EVERY)
                rows.append(np.stack([log["step"][:, 0], log["etot_per_n"][:, 0], log["pe_per_n"][:, 0],
                                      log["T"][:, 0]], axis=1).astype(np.float64))
                p, _, img = s.get_state()
                fr.append(p + L * img)
                g.append(s.rdf(DR, NBINS, reset=True))
        thermo.append(np.concatenate(rows))
        frames.append(fr)
        gs.append(g)
    return _summarise(thermo, frames, gs)


def _z(a, b):
    """Welch z of two (mean, standard error) pairs."""
    return (a[0] - b[0]) / np.sqrt(a[1] ** 2 + b[1] ** 2)


def _compare(gpu, ref):
    out = {"drift": _z(gpu["drift"], ref["drift"]), "pe": _z(gpu["pe"], ref["pe"]), "T": _z(gpu["T"], ref["T"]),
           "msd": _z(gpu["msd"], ref["msd"])}
    (mg, eg), (mo, eo) = gpu["g"], ref["g"]
    e = np.sqrt(eg * eg + eo * eo)
    seen = (mg > 0) | (mo > 0)
    # bins that neither side's samples scatter in must agree exactly (e.g. both empty)
    assert np.all(mg[seen & (e == 0)] == mo[seen & (e == 0)])
    out["g"] = (mg - mo)[seen & (e > 0)] / e[seen & (e > 0)]
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_long_run_statistics_match_oracle(prec):
    g, o = gpu_run(prec), oracle_run()
    c = _compare(g, o)
    summary = (f"{prec}: drift {g['drift'][0]:.2e}+-{g['drift'][1]:.1e} vs oracle {o['drift'][0]:.2e}"
               f"+-{o['drift'][1]:.1e} (z {c['drift']:.2f}); PE/N {g['pe'][0]:.5f} vs {o['pe'][0]:.5f} "
               f"(z {c['pe']:.2f}); T z {c['T']:.2f}; g(r) mean z^2 {np.mean(c['g'] ** 2):.2f} "
               f"max |z| {np.max(np.abs(c['g'])):.2f} over {c['g'].size} bins; MSD max |z| "
               f"{np.max(np.abs(c['msd'])):.2f}")
    print(summary)
    assert abs(c["drift"]) <= 4.5, summary
    assert abs(c["pe"]) <= 4.5 and abs(c["T"]) <= 4.5, summary
    assert np.mean(c["g"] ** 2) <= 2.0 and np.max(np.abs(c["g"])) <= 6.0, summary
    assert np.max(np.abs(c["msd"])) <= 5.0, summary
    # the runs resolve the MSD beyond the cage and the first g(r) peaks
    msd = g["msd"][0]
    assert msd[-1, 0] > 3 * msd[0, 0]
    assert 2.0 < np.max(g["g"][0][0]) < 5.0


def test_mixed_drift_equal_or_better_than_fp64():
    """The metric's condition: the mixed path's NVE drift is not worse than the all-FP64 path's
    beyond the error bars (|d_mixed| <= |d_fp64| + 4.5 sigma of the difference)."""
    dm, d64 = gpu_run("mixed")["drift"], gpu_run("fp64")["drift"]
    sig = np.hypot(dm[1], d64[1])
    assert abs(dm[0]) <= abs(d64[0]) + 4.5 * sig, (dm, d64)
