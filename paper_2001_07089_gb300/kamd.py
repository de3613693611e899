"""Python binding of libkamd (include/kamd.h): argument marshalling only.

Every computation runs in the library's sm_103a kernels. The functions
``md_create`` ... ``md_destroy`` mirror the C entry points one to one; the
``System`` class wraps them for convenience. Arrays may be numpy arrays (host)
or CUDA torch tensors (device, passed as pointers on the system's stream).

There is no fallback: if the shared library cannot be built or loaded, or the
GPU is not an sm_103a part, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MD_OK, MD_ERR_INVALID_ARG, MD_ERR_CUDA, MD_ERR_OOM, MD_ERR_UNSTABLE = 0, 1, 2, 3, 4
MD_ERR_NLIST_OVERFLOW, MD_ERR_TIMEOUT, MD_ERR_NOT_SUPPORTED = 5, 6, 7
MD_PREC_FP64, MD_PREC_MIXED = 0, 1
MD_NVT_NOSE_HOOVER, MD_NVT_RESAMPLE, MD_NVT_NOSE_HOOVER_EXACT = 0, 1, 2
MD_MSD_SLOTS = 8

STATUS_NAMES = {0: "MD_OK", 1: "MD_ERR_INVALID_ARG", 2: "MD_ERR_CUDA", 3: "MD_ERR_OOM", 4: "MD_ERR_UNSTABLE",
                5: "MD_ERR_NLIST_OVERFLOW", 6: "MD_ERR_TIMEOUT", 7: "MD_ERR_NOT_SUPPORTED"}

THERMO_DTYPE = np.dtype([("step", np.int64), ("T", np.float64), ("pe_per_n", np.float64),
                         ("ke_per_n", np.float64), ("etot_per_n", np.float64), ("virial", np.float64),
                         ("h_nh", np.float64), ("xi", np.float64)])

EXPORTED = ("md_create", "md_create_batch", "md_create_batch_dim", "md_set_state", "md_get_state", "md_init_lattice", "md_forces",
            "md_step_nve", "md_step_nvt", "md_rdf", "md_msd", "md_msd_tw", "md_set_tuning", "md_get_tuning", "md_autotune",
            "md_autotune_skin",
            "md_get_info", "md_count_pairs", "md_selftest_barrier", "md_time_forces", "md_time_lists", "md_forces_noalloc", "md_last_error",
            "md_destroy")


class md_tuning(ctypes.Structure):
    _fields_ = [("threads_per_atom", ctypes.c_int), ("block_size", ctypes.c_int), ("skin", ctypes.c_double),
                ("skin_outer", ctypes.c_double)]


class md_info(ctypes.Structure):
    _fields_ = [("n_total", ctypes.c_int64), ("n_replicas", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
                ("steps_done", ctypes.c_int64), ("rebuilds", ctypes.c_int64), ("list_entries", ctypes.c_int64),
                ("list_capacity", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("all_pairs_replicas", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("graph_launches", ctypes.c_int64), ("prunes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64)]


class KamdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libkamd.so (compiling it in-tree with nvcc when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"libkamd.so not found at {path}; run paper_2001_07089_gb300/build.py")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, dbl, c_int, u64 = ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_uint64
        sig = {
            "md_create": [i64, P, c_int, dbl, P, P, P, dbl, dbl, c_int, P, ctypes.POINTER(P)],
            "md_create_batch": [c_int, P, P, P, c_int, P, P, P, dbl, dbl, c_int, P, ctypes.POINTER(P)],
            "md_create_batch_dim": [c_int, c_int, P, P, P, c_int, P, P, P, dbl, dbl, c_int, P, ctypes.POINTER(P)],
            "md_set_state": [P, P, P, c_int],
            "md_get_state": [P, P, P, P, c_int],
            "md_init_lattice": [P, P, dbl, u64],
            "md_forces": [P, P, P, P, c_int],
            "md_step_nve": [P, dbl, i64, P, i64],
            "md_step_nvt": [P, dbl, i64, P, c_int, dbl, u64, P, i64],
            "md_rdf": [P, dbl, i64, P, c_int],
            "md_msd": [P, P, c_int],
            "md_msd_tw": [P, c_int, P, c_int],
            "md_set_tuning": [P, ctypes.POINTER(md_tuning)],
            "md_get_tuning": [P, ctypes.POINTER(md_tuning)],
            "md_autotune": [P, dbl, i64, ctypes.POINTER(md_tuning), ctypes.POINTER(dbl)],
            "md_autotune_skin": [P, dbl, i64, dbl, ctypes.POINTER(md_tuning), ctypes.POINTER(dbl)],
            "md_get_info": [P, ctypes.POINTER(md_info)],
            "md_count_pairs": [P, ctypes.POINTER(i64)],
            "md_selftest_barrier": [P, dbl],
            "md_time_forces": [P, i64, ctypes.POINTER(dbl)],
            "md_time_lists": [P, i64, ctypes.POINTER(dbl)],
            "md_forces_noalloc": [i64, P, P, c_int, dbl, P, P, P, P, P, P, P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.md_last_error.argtypes = [P]
        lib.md_last_error.restype = ctypes.c_char_p
        lib.md_destroy.argtypes = [P]
        lib.md_destroy.restype = None
        _lib = lib
        return lib


def _check(st, handle=None):
    if st != MD_OK:
        msg = load().md_last_error(handle).decode(errors="replace")
        raise KamdError(st, msg)


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype=np.float64):
    """(pointer, keepalive, on_device) for a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, None, 0
    if _is_torch(a):
        if not a.is_cuda or not a.is_contiguous():
            raise ValueError("torch tensors must be contiguous CUDA tensors")
        return a.data_ptr(), a, 1
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, arr, 0


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- C mirrors

def md_create(n, types, ntypes, L, eps, sigma, rc, mass, skin, prec, stream=None):
    t = np.ascontiguousarray(types, dtype=np.uint8)
    e, s, r = _f64(eps), _f64(sigma), _f64(rc)
    h = ctypes.c_void_p()
    _check(load().md_create(int(n), t.ctypes.data, int(ntypes), float(L), e.ctypes.data, s.ctypes.data,
                            r.ctypes.data, float(mass), float(skin), int(prec), stream, ctypes.byref(h)))
    return h


def md_create_batch(n_per, L_per, types, ntypes, eps, sigma, rc, mass, skin, prec, stream=None):
    n = np.ascontiguousarray(n_per, dtype=np.int64)
    Lp = _f64(L_per)
    t = np.ascontiguousarray(types, dtype=np.uint8)
    e, s, r = _f64(eps), _f64(sigma), _f64(rc)
    h = ctypes.c_void_p()
    _check(load().md_create_batch(len(n), n.ctypes.data, Lp.ctypes.data, t.ctypes.data, int(ntypes), e.ctypes.data,
                                  s.ctypes.data, r.ctypes.data, float(mass), float(skin), int(prec), stream,
                                  ctypes.byref(h)))
    return h


def md_create_batch_dim(ndim, n_per, L_per, types, ntypes, eps, sigma, rc, mass, skin, prec, stream=None):
    n = np.ascontiguousarray(n_per, dtype=np.int64)
    Lp = _f64(L_per)
    t = np.ascontiguousarray(types, dtype=np.uint8)
    e, s, r = _f64(eps), _f64(sigma), _f64(rc)
    h = ctypes.c_void_p()
    _check(load().md_create_batch_dim(int(ndim), len(n), n.ctypes.data, Lp.ctypes.data, t.ctypes.data, int(ntypes),
                                      e.ctypes.data, s.ctypes.data, r.ctypes.data, float(mass), float(skin), int(prec),
                                      stream, ctypes.byref(h)))
    return h


def md_set_state(h, pos, vel=None):
    pp, kp, dev = _ptr(pos)
    vp, kv, dev2 = _ptr(vel)
    if vel is not None and dev2 != dev:
        raise ValueError("pos and vel must both be host or both be device arrays")
    _check(load().md_set_state(h, pp, vp, dev), h)


def md_get_state(h, pos=None, vel=None, images=None, on_device=0):
    pp = pos.data_ptr() if on_device and pos is not None else (pos.ctypes.data if pos is not None else None)
    vp = vel.data_ptr() if on_device and vel is not None else (vel.ctypes.data if vel is not None else None)
    ip = images.data_ptr() if on_device and images is not None else (images.ctypes.data if images is not None else None)
    _check(load().md_get_state(h, pp, vp, ip, int(on_device)), h)


def md_init_lattice(h, T0, jitter, seed):
    t = _f64(np.atleast_1d(T0))
    _check(load().md_init_lattice(h, t.ctypes.data, float(jitter), int(seed)), h)


def md_forces(h, f=None, pe=None, virial=None, on_device=0):
    fp = (f.data_ptr() if on_device else f.ctypes.data) if f is not None else None
    _check(load().md_forces(h, fp, pe.ctypes.data if pe is not None else None,
                            virial.ctypes.data if virial is not None else None, int(on_device)), h)


def md_step_nve(h, dt, nsteps, log=None, log_every=0):
    _check(load().md_step_nve(h, float(dt), int(nsteps), log.ctypes.data if log is not None else None,
                              int(log_every)), h)


def md_step_nvt(h, dt, nsteps, T_target, kind, param, seed, log=None, log_every=0):
    t = _f64(np.atleast_1d(T_target))
    _check(load().md_step_nvt(h, float(dt), int(nsteps), t.ctypes.data, int(kind), float(param), int(seed),
                              log.ctypes.data if log is not None else None, int(log_every)), h)


def md_rdf(h, dr, nbins, g, reset):
    _check(load().md_rdf(h, float(dr), int(nbins), g.ctypes.data if g is not None else None, int(reset)), h)


def md_msd(h, out, reset_reference):
    _check(load().md_msd(h, out.ctypes.data if out is not None else None, int(reset_reference)), h)


def md_msd_tw(h, slot, out, reset_reference):
    _check(load().md_msd_tw(h, int(slot), out.ctypes.data if out is not None else None, int(reset_reference)), h)


def md_set_tuning(h, tpa, block, skin, skin_outer):
    t = md_tuning(int(tpa), int(block), float(skin), float(skin_outer))
    _check(load().md_set_tuning(h, ctypes.byref(t)), h)


def md_get_tuning(h):
    t = md_tuning()
    _check(load().md_get_tuning(h, ctypes.byref(t)), h)
    return t


def md_autotune(h, dt, probe_steps):
    t = md_tuning()
    sec = ctypes.c_double()
    _check(load().md_autotune(h, float(dt), int(probe_steps), ctypes.byref(t), ctypes.byref(sec)), h)
    return t, sec.value


def md_autotune_skin(h, dt, probe_steps, skin):
    t = md_tuning()
    sec = ctypes.c_double()
    _check(load().md_autotune_skin(h, float(dt), int(probe_steps), float(skin), ctypes.byref(t), ctypes.byref(sec)),
           h)
    return t, sec.value


def md_get_info(h):
    i = md_info()
    _check(load().md_get_info(h, ctypes.byref(i)), h)
    return i


def md_count_pairs(h):
    c = ctypes.c_int64()
    _check(load().md_count_pairs(h, ctypes.byref(c)), h)
    return c.value


def md_time_forces(h, repeats):
    """Seconds per force evaluation (the force phase alone, measured inside one launch)."""
    sec = ctypes.c_double()
    _check(load().md_time_forces(h, int(repeats), ctypes.byref(sec)), h)
    return sec.value


def md_time_lists(h, repeats):
    """Seconds per Verlet-list build (the list build alone, measured inside one launch)."""
    sec = ctypes.c_double()
    _check(load().md_time_lists(h, int(repeats), ctypes.byref(sec)), h)
    return sec.value


def md_selftest_barrier(h, timeout_s):
    """Returns the status code (MD_ERR_TIMEOUT expected) instead of raising."""
    return load().md_selftest_barrier(h, float(timeout_s))


def md_forces_noalloc(n, pos, types, ntypes, L, eps, sigma, rc, f, pe=None, virial=None, stream=None):
    """Device tensors in and out (pos, types, f, pe, virial); host tables. Allocates nothing."""
    e, s, r = _f64(eps), _f64(sigma), _f64(rc)
    dp = lambda t: t.data_ptr() if t is not None else None  # noqa: E731
    _check(load().md_forces_noalloc(int(n), dp(pos), dp(types), int(ntypes), float(L), e.ctypes.data, s.ctypes.data,
                                    r.ctypes.data, dp(f), dp(pe), dp(virial), stream))


def md_last_error(h=None):
    return load().md_last_error(h).decode(errors="replace")


def md_destroy(h):
    if h:
        load().md_destroy(h)


# ---------------------------------------------------------------- convenience

class System:
    """One system (or a batch of replicas when ``n`` is a sequence); ``ndim=2`` for the
    two-dimensional model (particles in the plane z = L/2)."""

    def __init__(self, n, L, types, eps, sigma, rc, mass=1.0, skin=0.3, precision="mixed", stream=None, ndim=3):
        prec = MD_PREC_MIXED if precision == "mixed" else MD_PREC_FP64
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        self.ntypes = int(np.asarray(eps).shape[0])
        self.ndim = int(ndim)
        if self.ndim != 3:
            self.n_per = np.atleast_1d(np.asarray(n, dtype=np.int64))
            self.L_per = np.broadcast_to(np.asarray(L, dtype=np.float64), self.n_per.shape).copy()
            self._h = md_create_batch_dim(self.ndim, self.n_per, self.L_per, types, self.ntypes, eps, sigma, rc, mass,
                                          skin, prec, stream)
        elif np.ndim(n) == 0:
            self.n_per = np.array([int(n)], dtype=np.int64)
            self.L_per = np.array([float(L)])
            self._h = md_create(int(n), types, self.ntypes, float(L), eps, sigma, rc, mass, skin, prec, stream)
        else:
            self.n_per = np.asarray(n, dtype=np.int64)
            self.L_per = np.asarray(L, dtype=np.float64)
            self._h = md_create_batch(self.n_per, self.L_per, types, self.ntypes, eps, sigma, rc, mass, skin, prec,
                                      stream)
        self.n_total = int(self.n_per.sum())
        self.nrep = len(self.n_per)
        self.precision = precision

    # context management
    def close(self):
        if self._h:
            md_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_state(self, pos, vel=None):
        md_set_state(self._h, pos, vel)

    def get_state(self):
        n = self.n_total
        pos, vel, img = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3), dtype=np.int32)
        md_get_state(self._h, pos, vel, img, 0)
        return pos, vel, img

    def get_state_device(self, pos, vel=None, images=None):
        md_get_state(self._h, pos, vel, images, 1)

    def init_lattice(self, T0, jitter=0.05, seed=1):
        md_init_lattice(self._h, np.broadcast_to(np.asarray(T0, dtype=np.float64), (self.nrep,)), jitter, seed)

    def forces(self):
        f = np.zeros((self.n_total, 3))
        pe, vir = np.zeros(self.nrep), np.zeros(self.nrep)
        md_forces(self._h, f, pe, vir, 0)
        return f, pe, vir

    def step_nve(self, dt, nsteps, log_every=0):
        nlog = nsteps // log_every if log_every > 0 else 0
        log = np.zeros(max(nlog, 1) * self.nrep, dtype=THERMO_DTYPE)
        md_step_nve(self._h, dt, nsteps, log if nlog else None, log_every if nlog else 0)
        return log[:nlog * self.nrep].reshape(nlog, self.nrep)

    def step_nvt(self, dt, nsteps, T_target, kind=MD_NVT_NOSE_HOOVER, param=None, seed=0, log_every=0):
        if param is None:
            param = 100.0 * dt if kind != MD_NVT_RESAMPLE else 50
        T = np.broadcast_to(np.asarray(T_target, dtype=np.float64), (self.nrep,))
        nlog = nsteps // log_every if log_every > 0 else 0
        log = np.zeros(max(nlog, 1) * self.nrep, dtype=THERMO_DTYPE)
        md_step_nvt(self._h, dt, nsteps, T, kind, param, seed, log if nlog else None, log_every if nlog else 0)
        return log[:nlog * self.nrep].reshape(nlog, self.nrep)

    def rdf(self, dr, nbins, reset=False):
        g = np.zeros(3 * nbins)
        md_rdf(self._h, dr, nbins, g, 1 if reset else 0)
        return g.reshape(3, nbins)

    def msd(self, reset_reference=False):
        out = np.zeros(self.ntypes)
        md_msd(self._h, out, 1 if reset_reference else 0)
        return out

    def msd_tw(self, slot, reset_reference=False):
        """Per-type MSD against reference slot `slot` (Eq. (msdtw)); reset = take r(t_w) now."""
        out = np.zeros(self.ntypes)
        md_msd_tw(self._h, slot, out, 1 if reset_reference else 0)
        return out

    @property
    def tuning(self):
        t = md_get_tuning(self._h)
        return {"threads_per_atom": t.threads_per_atom, "block_size": t.block_size, "skin": t.skin,
                "skin_outer": t.skin_outer}

    def set_tuning(self, threads_per_atom=None, block_size=None, skin=None, skin_outer=None):
        cur = self.tuning
        sk = cur["skin"] if skin is None else skin
        so = skin_outer if skin_outer is not None else max(cur["skin_outer"], sk + 0.4)
        md_set_tuning(self._h, threads_per_atom or cur["threads_per_atom"], block_size or cur["block_size"], sk, so)

    def autotune(self, dt, probe_steps=100, skin=None):
        """Search the launch configuration; with `skin`, the force list's skin stays fixed."""
        if skin is None:
            t, sec = md_autotune(self._h, dt, probe_steps)
        else:
            t, sec = md_autotune_skin(self._h, dt, probe_steps, skin)
        return {"threads_per_atom": t.threads_per_atom, "block_size": t.block_size, "skin": t.skin,
                "skin_outer": t.skin_outer}, sec

    def info(self):
        i = md_get_info(self._h)
        return {k: getattr(i, k) for k, _ in md_info._fields_}

    def count_pairs(self):
        return md_count_pairs(self._h)

    def time_forces(self, repeats=100):
        """Seconds per evaluation of the force phase alone (md_time_forces)."""
        return md_time_forces(self._h, repeats)

    def time_lists(self, repeats=20):
        """Seconds per Verlet-list build alone (md_time_lists); leaves the state as a rebuild does."""
        return md_time_lists(self._h, repeats)
