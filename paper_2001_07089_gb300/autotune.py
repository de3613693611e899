"""Cached launch-configuration choices for md_autotune.

md_autotune (C ABI) times short NVE probes over lanes per particle, CTA size
and the two list skins, and keeps the fastest. This module remembers the
choice per (GPU name, precision, replica count, particle-count bucket,
density bucket) in a JSON file so that later runs on the same kind of
system reuse it without probing.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "kamd", "tuning.json")


def cache_key(gpu_name: str, precision: str, n_per, L_per) -> str:
    """Key: GPU, precision, replica count, log2 bucket of particles per replica, density to 0.05."""
    n_per = [int(n) for n in n_per]
    L_per = [float(L) for L in L_per]
    nbar = sum(n_per) / len(n_per)
    rho = sum(n / (L ** 3) for n, L in zip(n_per, L_per)) / len(n_per)
    return f"{gpu_name}|{precision}|r{len(n_per)}|n2^{round(math.log2(max(nbar, 1.0)))}|rho{round(rho / 0.05) * 0.05:.2f}"


def load(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(key: str, tuning: dict, seconds_per_step: float, path: str = DEFAULT_CACHE) -> None:
    """Atomically add or replace one entry."""
    data = load(path)
    data[key] = {"tuning": tuning, "seconds_per_step": seconds_per_step}
    d = os.path.dirname(path)
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".tuning.")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(system, dt: float, gpu_name: str, probe_steps: int = 200, path: str = DEFAULT_CACHE,
         refresh: bool = False, skin=None) -> dict:
    """Apply the cached tuning for this kind of system, or run md_autotune (md_autotune_skin when
    `skin` fixes the force list's skin) and cache it."""
    key = cache_key(gpu_name, system.precision, system.n_per, system.L_per)
    if skin is not None:
        key += f"|skin{skin:g}"
    entry = None if refresh else load(path).get(key)
    if entry is not None:
        t = entry["tuning"]
        system.set_tuning(threads_per_atom=t["threads_per_atom"], block_size=t["block_size"], skin=t["skin"],
                          skin_outer=t["skin_outer"])
        return t
    t, sec = system.autotune(dt, probe_steps) if skin is None else system.autotune(dt, probe_steps, skin=skin)
    store(key, t, sec, path)
    return t
