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
