"""FP64 CPU oracle for the Kob-Andersen Lennard-Jones MD method.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path
(the CUDA library and its Python binding) never imports, links or executes it.

The arithmetic lives in ``ka_oracle.c`` (plain C, compiled with
``-ffp-contract=off`` so every machine evaluates the same expressions). This
module only compiles it and marshals numpy arrays through ctypes. Each
function cites the passage of the paper it restates:

* ``forces`` -- Eq. (KAFix) with Eq. (VshiftedKALJ), all pairs, half loop
  (Sec. "Accelerations"), minimum image by the branch rule (Sec. "Periodic
  boundary conditions").
* ``forces_threads`` -- the same sum spread over host threads (per-thread
  force arrays added in thread order), for timing on all cores and for long
  runs; ``set_threads`` makes ``run`` use it.
* ``force_on`` -- Eq. (KAFix) for one particle against every other particle.
* ``run`` -- velocity Verlet (Eqs. (velVerletPos)/(velVerletVel)) in the order
  of Sec. "NVE molecular dynamics simulation"; the stochastic bath of Sec.
  "NVT molecular dynamics simulation"; Nose-Hoover by the Fox-Andersen rules
  of Appendix B (Eqs. (Noseupdate_ri)-(Noseupdate_xiapprox), (ridotKVLRoman)
  or (ridotsolved), (FoxAndersen_ydottplush)).
* ``maxwell_boltzmann`` / ``init_lattice`` -- Sec. "Statistical temperature
  bath" steps 1-4 and Sec. "Initialization of positions".
* ``ndim=2`` (``maxwell_boltzmann``, ``init_lattice``, ``run``, ``rdf``) -- the
  two-dimensional problem of Sec. "Suggested problems": particles in the plane
  z = L/2 with v_z = 0, 2 instead of 3 in Eq. (equip3N) (T, the velocity
  rescale, X of the Nose-Hoover bath) and the shell area in g(r).
* ``rdf`` / ``msd`` -- Eqs. (gAA)/(gAB) with the histogram normalisation of
  Sec. "Radial distribution function with Python"; Eqs. (msd)/(msdwithi).
* ``philox4x32_10`` -- the counter-based generator of Salmon et al. (SC'11).

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or published test vectors; the
long-run statistics (energy drift, g(r), MSD of an equilibrated glass) have no
published value to pin to ("parity unpinned" for those quantities).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ka_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libka_oracle.so")
_lock = threading.Lock()
_lib = None

NVE, NOSE_HOOVER, RESAMPLE, NOSE_HOOVER_EXACT = 0, 1, 2, 3
THERMO_FIELDS = ("step", "T", "pe_per_n", "ke_per_n", "etot_per_n", "virial", "h_nh", "xi")


def build(force: bool = False) -> str:
    """Compile ka_oracle.c into a shared library (gcc, -O2, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    # OpenMP for the threaded force sum; without it that routine runs on one thread
    if subprocess.run(cmd[:-1] + ["-fopenmp", "-lm"], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        i32 = ctypes.POINTER(ctypes.c_int32)
        u32 = ctypes.POINTER(ctypes.c_uint32)
        i64, c_int, dbl, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        lib.ora_philox4x32_10.argtypes = [u32, u32, u32]
        lib.ora_philox4x32_10.restype = None
        lib.ora_draw_gauss3.argtypes = [u64, u64, ctypes.c_uint32, d]
        lib.ora_draw_gauss3.restype = None
        lib.ora_draw_jitter3.argtypes = [u64, ctypes.c_uint32, d]
        lib.ora_draw_jitter3.restype = None
        lib.ora_forces.argtypes = [i64, d, i32, c_int, d, d, d, dbl, d, d, d]
        lib.ora_force_on.argtypes = [i64, i64, d, i32, c_int, d, d, d, dbl, d, d]
        lib.ora_forces_threads.argtypes = [i64, d, i32, c_int, d, d, d, dbl, d, d, d, c_int]
        lib.ora_set_threads.argtypes = [c_int]
        lib.ora_max_threads.argtypes = []
        lib.ora_maxwell_boltzmann.argtypes = [i64, c_int, dbl, dbl, u64, u64, i32, d]
        lib.ora_init_lattice.argtypes = [i64, c_int, dbl, dbl, dbl, dbl, u64, d, d]
        lib.ora_run.argtypes = [i64, c_int, d, d, d, i32, i32, c_int, d, d, d, dbl, dbl, dbl, i64, i64,
                                c_int, dbl, dbl, i64, u64, d, d, i64]
        lib.ora_rdf.argtypes = [i64, c_int, d, i32, dbl, dbl, i64, d]
        lib.ora_msd.argtypes = [i64, d, i32, d, i32, c_int, dbl, d]
        for name in ("ora_forces", "ora_force_on", "ora_maxwell_boltzmann", "ora_init_lattice",
                     "ora_run", "ora_rdf", "ora_msd", "ora_forces_threads", "ora_set_threads", "ora_max_threads"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(rc, name):
    if rc != 0:
        raise ValueError(f"oracle {name} rejected its arguments (code {rc})")


class Params:
    """Interaction table: eps, sig, rc are (ntypes, ntypes) symmetric arrays."""

    def __init__(self, eps, sig, rc, mass=1.0):
        self.eps = _f64(eps)
        self.sig = _f64(sig)
        self.rc = _f64(rc)
        self.ntypes = int(self.eps.shape[0])
        self.mass = float(mass)


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.ora_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def gauss3(seed, draw, p):
    out = np.zeros(3)
    _load().ora_draw_gauss3(int(seed), int(draw), int(p), _dp(out))
    return out


def jitter3(seed, p):
    out = np.zeros(3)
    _load().ora_draw_jitter3(int(seed), int(p), _dp(out))
    return out


def forces(pos, types, params: Params, L):
    """Return (F (n,3), V, W) for all pairs."""
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    t = _i32(types)
    f = np.zeros((n, 3))
    pe = ctypes.c_double()
    vir = ctypes.c_double()
    rc = _load().ora_forces(n, _dp(pos), _ip(t), params.ntypes, _dp(params.eps), _dp(params.sig),
                            _dp(params.rc), float(L), _dp(f), ctypes.byref(pe), ctypes.byref(vir))
    _check(rc, "forces")
    return f, pe.value, vir.value


def forces_threads(pos, types, params: Params, L, nthreads):
    """The all-pairs sum of ``forces`` over nthreads host threads (per-thread force arrays added
    in thread order: reproducible for a fixed thread count; one thread is ``forces`` bitwise)."""
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    t = _i32(types)
    f = np.zeros((n, 3))
    pe = ctypes.c_double()
    vir = ctypes.c_double()
    rc = _load().ora_forces_threads(n, _dp(pos), _ip(t), params.ntypes, _dp(params.eps), _dp(params.sig),
                                    _dp(params.rc), float(L), _dp(f), ctypes.byref(pe), ctypes.byref(vir),
                                    int(nthreads))
    _check(rc, "forces_threads")
    return f, pe.value, vir.value


def set_threads(nthreads):
    """Host threads for the force sums inside ``run`` (1 = the single-thread oracle)."""
    _check(_load().ora_set_threads(int(nthreads)), "set_threads")


def max_threads():
    """Threads OpenMP would use by default (1 when the oracle was built without OpenMP)."""
    return int(_load().ora_max_threads())


def force_on(pos, types, params: Params, L, i):
    """Force on particle i from every other particle, and half its pair energy."""
    pos = _f64(pos, (-1, 3))
    t = _i32(types)
    f = np.zeros(3)
    pe = ctypes.c_double()
    rc = _load().ora_force_on(pos.shape[0], int(i), _dp(pos), _ip(t), params.ntypes, _dp(params.eps),
                              _dp(params.sig), _dp(params.rc), float(L), _dp(f), ctypes.byref(pe))
    _check(rc, "force_on")
    return f, pe.value


def maxwell_boltzmann(n, T, seed, draw=0, mass=1.0, ids=None, ndim=3):
    vel = np.zeros((n, 3))
    keep = _i32(ids) if ids is not None else None
    idp = _ip(keep) if keep is not None else ctypes.POINTER(ctypes.c_int32)()
    rc = _load().ora_maxwell_boltzmann(int(n), int(ndim), float(T), float(mass), int(seed), int(draw), idp, _dp(vel))
    _check(rc, "maxwell_boltzmann")
    return vel


def init_lattice(n, L, T0, seed, jitter=0.05, mass=1.0, ndim=3):
    pos = np.zeros((n, 3))
    vel = np.zeros((n, 3))
    rc = _load().ora_init_lattice(int(n), int(ndim), float(L), float(T0), float(mass), float(jitter), int(seed),
                                  _dp(pos), _dp(vel))
    _check(rc, "init_lattice")
    return pos, vel


def run(pos, vel, types, params: Params, L, dt, nsteps, kind=NVE, T_target=0.0, Q=0.0,
        nstep_boltz=50, seed=0, state=None, forces_in=None, img=None, step0=0, log_every=1, ndim=3):
    """Advance (pos, vel) by nsteps; returns a dict with the new state and the thermo log.

    The inputs are copied, never modified. ``state`` = [xi, ln s] for Nose-Hoover.
    """
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    n = pos.shape[0]
    t = _i32(types)
    if forces_in is None:
        f, _, _ = forces(pos, t, params, L)
    else:
        f = _f64(forces_in, (-1, 3)).copy()
    img = np.zeros((n, 3), dtype=np.int32) if img is None else _i32(img).reshape(n, 3).copy()
    st = np.array([0.0, 0.0] if state is None else state, dtype=np.float64)
    nlog = (nsteps // log_every) if log_every > 0 else 0
    thermo = np.zeros((max(nlog, 1), 8))
    rc = _load().ora_run(n, int(ndim), _dp(pos), _dp(vel), _dp(f), _ip(img), _ip(t), params.ntypes,
                         _dp(params.eps), _dp(params.sig), _dp(params.rc), float(L), params.mass,
                         float(dt), int(step0), int(nsteps), int(kind), float(T_target), float(Q),
                         int(nstep_boltz), int(seed), _dp(st), _dp(thermo), int(log_every))
    _check(rc, "run")
    return {"pos": pos, "vel": vel, "forces": f, "img": img, "state": st, "thermo": thermo[:nlog]}


def log_time_grid(n_md, t0=1.0, kmax=60):
    """Steps of the log-spaced MSD grid (Sec. "Mean square displacement with
    Python", Eqs. (logtimessteps), (A)), following the paper's loop: walk the
    time steps, and at each measured step advance t_k by factors of A until
    round(t_k) moves past it."""
    A = (float(n_md) / t0) ** (1.0 / float(kmax))
    t = t0
    target = int(round(t))
    out = []
    for step in range(1, n_md + 1):
        if target == step:
            while target == step:
                t = A * t
                target = int(round(t))
            out.append(step)
    return out


def rdf(pos, types, L, dr, nbins, ndim=3):
    pos = _f64(pos, (-1, 3))
    g = np.zeros(3 * nbins)
    rc = _load().ora_rdf(pos.shape[0], int(ndim), _dp(pos), _ip(_i32(types)), float(L), float(dr), int(nbins),
                         _dp(g))
    _check(rc, "rdf")
    return g.reshape(3, nbins)


def msd(pos, img, ref, types, ntypes, L):
    pos = _f64(pos, (-1, 3))
    out = np.zeros(ntypes)
    rc = _load().ora_msd(pos.shape[0], _dp(pos), _ip(_i32(img)), _dp(_f64(ref, (-1, 3))),
                         _ip(_i32(types)), int(ntypes), float(L), _dp(out))
    _check(rc, "msd")
    return out
