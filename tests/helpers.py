"""Shared test helpers: seeded configurations built with the oracle only."""
from __future__ import annotations

import functools

import numpy as np

import oracle
from paper_2001_07089_gb300 import workloads as wl


def ka_params():
    return oracle.Params(wl.KA_EPS, wl.KA_SIG, wl.KA_RC, wl.KA_MASS)


@functools.lru_cache(maxsize=None)
def melted(n: int, seed: int, nsteps: int = 200, T0: float = 2.0, density: float = wl.DENSITY):
    """A KA configuration melted by the oracle: lattice start at T0, then nsteps
    of the stochastic bath at T0 (resampling every 10 steps) to drain the
    lattice's excess potential energy.

    Returns (pos, vel, types, L); cached per arguments (arrays are read-only).
    """
    L = wl.box_length(n, density)
    types = wl.ka_types(n, seed).astype(np.int32)
    pos, vel = oracle.init_lattice(n, L, T0, seed)
    if nsteps:
        out = oracle.run(pos, vel, types, ka_params(), L, wl.DT, nsteps, kind=oracle.RESAMPLE,
                         T_target=T0, nstep_boltz=10, seed=seed, log_every=0)
        pos, vel = out["pos"], out["vel"]
    for a in (pos, vel, types):
        a.setflags(write=False)
    return pos, vel, types, L


def force_errors(f_test, f_ref):
    """(max_i |dF_i| / F_rms, ||dF||_2 / ||F_ref||_2) -- the force parity metric."""
    f_test = np.asarray(f_test, dtype=np.float64).reshape(-1, 3)
    f_ref = np.asarray(f_ref, dtype=np.float64).reshape(-1, 3)
    d = np.linalg.norm(f_test - f_ref, axis=1)
    frms = np.sqrt(np.mean(np.sum(f_ref * f_ref, axis=1)))
    return float(d.max() / frms), float(np.linalg.norm(f_test - f_ref) / np.linalg.norm(f_ref))


def min_image_diff(a, b, L):
    d = np.asarray(a) - np.asarray(b)
    return d - L * np.rint(d / L)


@functools.lru_cache(maxsize=None)
def melted_2d(n: int, seed: int, nsteps: int = 200, T0: float = 1.0):
    """The two-dimensional KA mixture (A:B = 65:35, N/L^2 = 1.204) melted by the oracle: square
    lattice at T0 in the plane z = L/2, then nsteps of the stochastic bath at T0 (resampling every
    10 steps). Returns (pos, vel, types, L); cached per arguments (arrays are read-only)."""
    L = wl.box_length_2d(n)
    types = wl.ka_types(n, seed, frac_b=wl.FRAC_B_2D).astype(np.int32)
    pos, vel = oracle.init_lattice(n, L, T0, seed, ndim=2)
    if nsteps:
        out = oracle.run(pos, vel, types, ka_params(), L, wl.DT, nsteps, kind=oracle.RESAMPLE, T_target=T0,
                         nstep_boltz=10, seed=seed, log_every=0, ndim=2)
        pos, vel = out["pos"], out["vel"]
    for a in (pos, vel, types):
        a.setflags(write=False)
    return pos, vel, types, L
