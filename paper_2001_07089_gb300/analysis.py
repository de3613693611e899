"""Measurement schedules around the library's analysis kernels.

The arithmetic (g(r) histograms, mean square displacements) runs in
md_rdf / md_msd; this module only decides *when* to measure and collects the
results, as Sec. "Mean square displacement with Python" and Sec. "Radial
distribution function with Python" describe.
"""
from __future__ import annotations

import numpy as np

from . import kamd


def log_time_grid(n_md: int, t0: float = 1.0, kmax: int = 60) -> list[int]:
    """Measurement steps evenly spaced in log time, Eqs. (logtimessteps) and (A).

    t_k/dt = t0 * A^k with A = (n_md / t0)^(1/kmax); the step of the k-th
    point is round(t_k/dt) (half to even), and points that round to the same
    step are measured once (the paper's while loop over k).
    """
    if n_md < 1 or t0 <= 0 or kmax < 1:
        raise ValueError("n_md >= 1, t0 > 0, kmax >= 1 required")
    A = (float(n_md) / t0) ** (1.0 / float(kmax))
    steps = []
    t = t0
    nxt = int(round(t))
    while nxt <= n_md:
        steps.append(nxt)
        while int(round(t)) == nxt:
            t *= A
            if t > 10.0 * n_md + 10:
                break
        nxt = int(round(t))
        if steps and nxt <= steps[-1]:
            break
    return steps


def msd_on_grid(system: "kamd.System", dt: float, steps: list[int], advance=None) -> np.ndarray:
    """Advance `system` to each step of `steps` and record the per-type MSD there.

    The reference is the configuration at call time (step 0). `advance(n)`
    advances n steps (default: NVE). Returns an array [len(steps), ntypes].
    """
    advance = advance or (lambda n: system.step_nve(dt, n))
    system.msd(reset_reference=True)
    out = np.zeros((len(steps), system.ntypes))
    done = 0
    for k, s in enumerate(steps):
        if s > done:
            advance(s - done)
            done = s
        out[k] = system.msd()
    return out


def rdf_time_average(system: "kamd.System", dr: float, nbins: int, every: int, count: int, advance) -> np.ndarray:
    """Time-averaged partial g(r) (AA, BB, AB): `count` measurements `every` steps apart."""
    g = None
    for k in range(count):
        advance(every)
        g = system.rdf(dr, nbins, reset=(k == 0))
    return g


def waiting_time_msd(system: "kamd.System", t_ws: list[int], n_md: int, advance, t0: float = 1.0,
                     kmax: int = 60) -> dict:
    """Per-type <|r(t_w + t) - r(t_w)|^2> (Eq. (msdtw)) for several waiting times along one trajectory.

    t_ws are waiting times in steps counted from the call (each gets its own
    reference slot, 1 .. MD_MSD_SLOTS - 1); t runs over the log grid of
    `log_time_grid(n_md, t0, kmax)`. `advance(n)` moves the system n steps
    (NVE for an equilibrium run, NVT after a quench). Returns
    {t_w: (t_steps, msd[len(t_steps), ntypes])}.
    """
    t_ws = [int(t) for t in t_ws]
    if len(set(t_ws)) != len(t_ws) or min(t_ws, default=0) < 0:
        raise ValueError("waiting times must be distinct and >= 0")
    if len(t_ws) > kamd.MD_MSD_SLOTS - 1:
        raise ValueError(f"at most {kamd.MD_MSD_SLOTS - 1} waiting times")
    grid = log_time_grid(n_md, t0, kmax)
    slot = {tw: k + 1 for k, tw in enumerate(sorted(t_ws))}
    # events at each step: references first (order 0), then measurements (order 1)
    events = sorted([(tw, 0, tw, -1) for tw in t_ws] +
                    [(tw + s, 1, tw, k) for tw in t_ws for k, s in enumerate(grid)])
    out = {tw: (np.array(grid, dtype=np.int64), np.zeros((len(grid), system.ntypes))) for tw in t_ws}
    done = 0
    for step, kind, tw, k in events:
        if step > done:
            advance(step - done)
            done = step
        if kind == 0:
            system.msd_tw(slot[tw], reset_reference=True)
        else:
            out[tw][1][k] = system.msd_tw(slot[tw])
    return out


def cooling_ladder(system: "kamd.System", temperatures, dt: float, n_bath: int, n_nve: int, n_prod: int,
                   nstep_boltz: int = 50, seed: int = 0, log_every: int = 0, production=None) -> list:
    """The cooling sequence of Sec. "Simulation Run Sequence", applied to every replica at once.

    For each temperature in turn: the stochastic bath for n_bath steps, NVE for
    n_nve steps, then the production run: `production(system, T)` if given
    (it advances the system itself and its result is kept), else n_prod NVE
    steps. Each stage starts from the configuration the previous one left.
    Returns one dict per temperature with the stages' thermo logs.
    """
    stages = []
    for k, T in enumerate(temperatures):
        bath = system.step_nvt(dt, n_bath, T, kind=kamd.MD_NVT_RESAMPLE, param=nstep_boltz, seed=seed + k,
                               log_every=log_every)
        nve = system.step_nve(dt, n_nve, log_every=log_every)
        prod = production(system, T) if production is not None else system.step_nve(dt, n_prod, log_every=log_every)
        stages.append({"T": T, "bath": bath, "nve": nve, "production": prod})
    return stages


# ------------------------------------------------------------------ statistics of long runs

def drift_fit(t, e, block=None, nboot=400, seed=12345) -> dict:
    """Energy drift of an NVE run: least-squares slope of e(t) with a moving-block bootstrap error.

    The residuals about the fitted line are correlated in time, so the error
    bar resamples them in overlapping blocks of `block` consecutive samples
    (default: 1/10 of the series, at least 2; Kunsch's moving-block
    bootstrap), adds them back to the fitted line and refits; the error is the
    standard deviation of the refitted slopes. Also returned: the RMS residual
    (the size of the energy fluctuations about the trend).
    """
    t = np.asarray(t, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    n = len(e)
    if n < 4 or len(t) != n:
        return {"slope": None, "err": None, "rms": None, "n": n}
    A = np.vstack([t, np.ones_like(t)]).T
    coef, *_ = np.linalg.lstsq(A, e, rcond=None)
    fit = A @ coef
    res = e - fit
    b = int(block) if block else max(2, n // 10)
    b = min(max(b, 1), n)
    rng = np.random.default_rng(seed)
    nblk = -(-n // b)
    starts = rng.integers(0, n - b + 1, size=(nboot, nblk))
    idx = (starts[:, :, None] + np.arange(b)[None, None, :]).reshape(nboot, -1)[:, :n]
    boot = fit[None, :] + res[idx]
    # slope of each resampled series (closed-form least squares against the same t)
    tc = t - t.mean()
    slopes = (boot - boot.mean(axis=1, keepdims=True)) @ tc / np.dot(tc, tc)
    return {"slope": float(coef[0]), "err": float(np.std(slopes, ddof=1)), "rms": float(np.std(res)), "n": n}


def block_mean(samples, nblocks: int):
    """Mean over axis 0 and its standard error from `nblocks` contiguous blocks (block averaging).

    Block means of a correlated series are nearly independent once a block is
    longer than the correlation time; the error is std(block means)/sqrt(nblocks).
    """
    x = np.asarray(samples, dtype=np.float64)
    m = (x.shape[0] // nblocks) * nblocks
    if nblocks < 2 or m == 0:
        raise ValueError("need at least 2 blocks of one sample")
    blocks = x[:m].reshape((nblocks, m // nblocks) + x.shape[1:]).mean(axis=1)
    return blocks.mean(axis=0), blocks.std(axis=0, ddof=1) / np.sqrt(nblocks)


def msd_time_origins(unwrapped, types, ntypes: int, lags, origin_every: int = 1) -> np.ndarray:
    """Per-type MSD (Eq. (msdwithi)) at the frame lags `lags`, averaged over time origins.

    unwrapped: [frames, n, 3] unwrapped positions; origins every `origin_every`
    frames, each lag averaged over the origins that fit. Returns [len(lags), ntypes].
    """
    x = np.asarray(unwrapped, dtype=np.float64)
    types = np.asarray(types)
    out = np.zeros((len(lags), ntypes))
    for k, lag in enumerate(lags):
        orig = np.arange(0, x.shape[0] - lag, origin_every)
        d2 = np.sum((x[orig + lag] - x[orig]) ** 2, axis=2)  # [origins, n]
        for a in range(ntypes):
            out[k, a] = d2[:, types == a].mean()
    return out
