"""GPU path (through the C ABI) against the FP64 oracle on identical seeded inputs.

Tolerances (force metric = max_i |dF_i| / F_rms and ||dF||_2 / ||F||_2; energy
metric = |dE| / (|KE| + |PE|), the scale of the terms that make up E, because
E_tot itself can sit near zero):
  FP64 path   forces <= 1e-12, energies <= 1e-12 (single evaluation), 1e-10 over a trajectory
  mixed path  forces <= 1e-5, energies per step <= 1e-6
"""
import numpy as np
import pytest

import oracle
from paper_2001_07089_gb300 import kamd
from paper_2001_07089_gb300 import workloads as wl
from tests.helpers import force_errors, ka_params, melted, min_image_diff

pytestmark = pytest.mark.gpu

TOL_F = {"fp64": 1e-12, "mixed": 1e-5}
TOL_E = {"fp64": 1e-12, "mixed": 1e-6}
PRECS = ["fp64", "mixed"]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kamd.load()


def make_system(n, L, types, prec, skin=0.3, tpa=None):
    s = kamd.System(n, L, types, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, wl.KA_MASS, skin, prec)
    if tpa is not None:
        s.set_tuning(threads_per_atom=tpa)
    return s


def check_forces(f_gpu, f_ref, prec):
    emax, e2 = force_errors(f_gpu, f_ref)
    assert emax <= TOL_F[prec] and e2 <= TOL_F[prec], (emax, e2)


# ------------------------------------------------------------------ forces

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,seed", [(250, 21), (1000, 22), (4000, 23)])
def test_forces_match_oracle_melted(prec, n, seed):
    pos, vel, types, L = melted(n, seed, nsteps=200)
    f_ref, v_ref, w_ref = oracle.forces(pos, types, ka_params(), L)
    with make_system(n, L, types, prec) as s:
        s.set_state(pos, vel)
        f, pe, vir = s.forces()
    check_forces(f, f_ref, prec)
    assert abs(pe[0] - v_ref) <= TOL_E[prec] * abs(v_ref)
    assert abs(vir[0] - w_ref) <= TOL_E[prec] * abs(w_ref) * 10


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("tpa", [1, 2, 4, 8])
def test_forces_every_lane_split(prec, tpa):
    pos, vel, types, L = melted(1000, 24, nsteps=200)
    f_ref, v_ref, _ = oracle.forces(pos, types, ka_params(), L)
    with make_system(1000, L, types, prec, tpa=tpa) as s:
        s.set_state(pos, vel)
        f, pe, _ = s.forces()
    check_forces(f, f_ref, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_forces_32k_tiled_melt(prec):
    """N = 32 000 at rho = 1.2: an oracle-melted N = 4000 liquid tiled 2x2x2 (every particle keeps
    its environment because r_c < L_4000/2, so the oracle also checks replication invariance)."""
    pos4, vel4, types4, L4 = melted(4000, 23, nsteps=200)
    shifts = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=float) * L4
    pos = np.concatenate([pos4 + sh for sh in shifts])
    vel = np.concatenate([vel4] * 8)
    types = np.concatenate([types4] * 8)
    L = 2 * L4
    f_ref, v_ref, _ = oracle.forces(pos, types, ka_params(), L)
    f4, v4, _ = oracle.forces(pos4, types4, ka_params(), L4)
    assert np.max(np.abs(f_ref - np.concatenate([f4] * 8))) < 1e-9 * np.abs(f4).max()
    with make_system(32000, L, types, prec) as s:
        s.set_state(pos, vel)
        f, pe, _ = s.forces()
    check_forces(f, f_ref, prec)
    assert abs(pe[0] - v_ref) <= TOL_E[prec] * abs(v_ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("reach,group", [("1", "1"), ("1", "2"), ("1", "4"), ("1", "8"), ("2", "1"), ("2", "8"),
                                         ("2", "16"), ("2", "64")])
@pytest.mark.parametrize("n,tile", [(1000, 1), (4000, 1), (4000, 2)], ids=["1000", "4000", "32000-tiled"])
def test_list_build_every_group_shape(prec, reach, group, n, tile, monkeypatch):
    """The list build works on groups of 1 to 64 cells (1x1x1 ... 4x4x4) of full-width cells
    (3x3x3 stencil, KAMD_CELL_REACH=1) or half-width cells (5x5x5 stencil, corners culled). Every
    shape gives the oracle's forces with every lane split: N = 1000 is scanned whole (too small for
    cells at the default outer skin), N = 4000 has 4 full-width or 9 half-width cells per edge, the
    tiled N = 32 000 box 9 or 18 (staged fixed-point words where the group's neighbourhood spans
    more than half the box, FP32 relative coordinates elsewhere)."""
    pos, vel, types, L = melted(n, 23 if n == 4000 else 22, nsteps=200)
    if tile > 1:
        shifts = np.array([[i, j, k] for i in range(tile) for j in range(tile) for k in range(tile)], dtype=float) * L
        pos = np.concatenate([pos + sh for sh in shifts])
        vel = np.concatenate([vel] * tile ** 3)
        types = np.concatenate([types] * tile ** 3)
        L = tile * L
    f_ref, v_ref, _ = oracle.forces(pos, types, ka_params(), L)
    monkeypatch.setenv("KAMD_LIST_GROUP", group)
    monkeypatch.setenv("KAMD_CELL_REACH", reach)
    for tpa in (1, 4):
        with make_system(len(pos), L, types, prec, tpa=tpa) as s:
            s.set_state(pos, vel)
            f, pe, _ = s.forces()
        check_forces(f, f_ref, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_forces_32k_lattice_start(prec):
    """The 32k configuration's own start: 32^3 lattice sites (32 000 occupied), jitter 0.05."""
    n = 32000
    L = wl.box_length(n)
    types = wl.ka_types(n, 25).astype(np.int32)
    pos, vel = oracle.init_lattice(n, L, 2.0, seed=25, jitter=0.05)
    f_ref, v_ref, _ = oracle.forces(pos, types, ka_params(), L)
    with make_system(n, L, types, prec) as s:
        s.set_state(pos, vel)
        f, pe, _ = s.forces()
    check_forces(f, f_ref, prec)
    assert abs(pe[0] - v_ref) <= TOL_E[prec] * abs(v_ref)


@pytest.mark.parametrize("prec", PRECS)
def test_tiny_systems_and_ragged_tiles(prec):
    """N = 2 and 3 in a large box, and N = 33 (one full tile plus one particle)."""
    L = 10.0
    for pos, types in [
        (np.array([[1.0, 1.0, 1.0], [2.05, 1.2, 0.9]]), np.array([0, 1])),
        (np.array([[1.0, 1.0, 1.0], [2.05, 1.2, 0.9], [9.6, 1.1, 1.3]]), np.array([0, 1, 0])),
    ]:
        f_ref, v_ref, _ = oracle.forces(pos, types.astype(np.int32), ka_params(), L)
        with make_system(len(pos), L, types, prec) as s:
            s.set_state(pos, np.zeros_like(pos))
            f, pe, _ = s.forces()
        check_forces(f, f_ref, prec)
        assert abs(pe[0] - v_ref) <= TOL_E[prec] * abs(v_ref)
    n = 33
    L = wl.box_length(n, 0.2)
    types = wl.ka_types(n, 26).astype(np.int32)
    pos = wl.uniform_positions(n, L, 26)
    f_ref, v_ref, _ = oracle.forces(pos, types, ka_params(), L)
    with make_system(n, L, types, prec) as s:
        s.set_state(pos, np.zeros_like(pos))
        f, pe, _ = s.forces()
    check_forces(f, f_ref, prec)


# ------------------------------------------------------------------ dynamics

def thermo_rel(gpu_log, ref_thermo, field_gpu, col, n=1):
    """Largest per-step error of one thermo field, relative to |KE| + |PE| (times n for totals)."""
    a = gpu_log[field_gpu][:, 0]
    b = ref_thermo[:, col]
    scale = n * (np.abs(ref_thermo[:, 2]) + np.abs(ref_thermo[:, 3]))
    return np.max(np.abs(a - b) / scale)


@pytest.mark.parametrize("prec", PRECS)
def test_nve_100_steps_energies(prec):
    pos, vel, types, L = melted(1000, 31, nsteps=200)
    ref = oracle.run(pos, vel, types, ka_params(), L, 0.005, 100, log_every=1)
    with make_system(1000, L, types, prec) as s:
        s.set_state(pos, vel)
        log = s.step_nve(0.005, 100, log_every=1)
        p, v, img = s.get_state()
    assert list(log["step"][:, 0]) == list(range(1, 101))
    tol = 1e-10 if prec == "fp64" else TOL_E["mixed"]
    assert thermo_rel(log, ref["thermo"], "etot_per_n", 4) <= tol
    assert thermo_rel(log, ref["thermo"], "pe_per_n", 2) <= tol
    assert thermo_rel(log, ref["thermo"], "ke_per_n", 3) <= tol
    # PE and KE each against their own magnitude
    assert own_rel(log, ref["thermo"], "pe_per_n", 2) <= tol
    assert own_rel(log, ref["thermo"], "ke_per_n", 3) <= tol
    d = np.abs(min_image_diff(p, ref["pos"], L))
    assert d.max() < (1e-9 if prec == "fp64" else 1e-3)


def own_rel(gpu_log, ref_thermo, field_gpu, col):
    """Largest per-step error of one thermo field relative to that field's own magnitude."""
    a = gpu_log[field_gpu][:, 0]
    b = ref_thermo[:, col]
    return np.max(np.abs(a - b) / np.abs(b))


@pytest.mark.parametrize("prec", PRECS)
def test_nve_100_steps_at_T08_plain_relative_energies(prec):
    """The 32k configuration's temperature, T = 0.8, where E_tot/N (about -5.4) is far from zero:
    E_tot, PE and KE per step each within the plain relative tolerance |dE|/|E| over 100 steps."""
    pos, vel, types, L = melted(1000, 34, nsteps=300, T0=0.8)
    ref = oracle.run(pos, vel, types, ka_params(), L, 0.005, 100, log_every=1)
    th = ref["thermo"]
    assert np.all(np.abs(th[:, 4]) > 3.0)
    with make_system(1000, L, types, prec) as s:
        s.set_state(pos, vel)
        log = s.step_nve(0.005, 100, log_every=1)
    tol = 1e-10 if prec == "fp64" else TOL_E["mixed"]
    for field, col in (("etot_per_n", 4), ("pe_per_n", 2), ("ke_per_n", 3)):
        assert own_rel(log, th, field, col) <= tol, field


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", [kamd.MD_NVT_NOSE_HOOVER, kamd.MD_NVT_NOSE_HOOVER_EXACT])
def test_nose_hoover_100_steps(prec, kind):
    pos, vel, types, L = melted(1000, 32, nsteps=200)
    T, tau = 0.8, 0.5
    n = 1000
    okind = oracle.NOSE_HOOVER if kind == kamd.MD_NVT_NOSE_HOOVER else oracle.NOSE_HOOVER_EXACT
    ref = oracle.run(pos, vel, types, ka_params(), L, 0.005, 100, kind=okind, T_target=T, Q=3 * n * T * tau * tau,
                     log_every=1)
    with make_system(n, L, types, prec) as s:
        s.set_state(pos, vel)
        log = s.step_nvt(0.005, 100, T, kind=kind, param=tau, log_every=1)
    tol = 1e-10 if prec == "fp64" else TOL_E["mixed"]
    assert thermo_rel(log, ref["thermo"], "etot_per_n", 4) <= tol
    assert thermo_rel(log, ref["thermo"], "h_nh", 6, n=n) <= tol
    assert thermo_rel(log, ref["thermo"], "T", 1) <= (1e-10 if prec == "fp64" else 1e-5)
    xi_g, xi_r = log["xi"][:, 0], ref["thermo"][:, 7]
    assert np.max(np.abs(xi_g - xi_r)) <= (1e-10 if prec == "fp64" else 1e-4) * np.max(np.abs(xi_r))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("red_tiles", ["3", "16"])
def test_two_level_reductions(prec, red_tiles, monkeypatch):
    """Replicas larger than one reduction chunk are reduced in two levels (chunk sums by separate CTAs,
    then one CTA per replica). Shrinking the chunk to 3 or 16 tiles puts an N = 1000 system (32 tiles)
    on that path: Nose-Hoover (a reduction every step, xi fed back into the dynamics) and the
    resampling bath follow the oracle as closely as on the one-level path, and the trajectory is
    reproducible bitwise."""
    monkeypatch.setenv("KAMD_RED_TILES", red_tiles)
    pos, vel, types, L = melted(1000, 32, nsteps=200)
    T, tau, n = 0.8, 0.5, 1000
    ref = oracle.run(pos, vel, types, ka_params(), L, 0.005, 60, kind=oracle.NOSE_HOOVER, T_target=T,
                     Q=3 * n * T * tau * tau, log_every=1)
    runs = []
    for _ in range(2):
        with make_system(n, L, types, prec) as s:
            s.set_state(pos, vel)
            log = s.step_nvt(0.005, 60, T, kind=kamd.MD_NVT_NOSE_HOOVER, param=tau, log_every=1)
            runs.append((log, s.get_state()[0]))
    log = runs[0][0]
    tol = 1e-10 if prec == "fp64" else TOL_E["mixed"]
    assert thermo_rel(log, ref["thermo"], "etot_per_n", 4) <= tol
    assert thermo_rel(log, ref["thermo"], "h_nh", 6, n=n) <= tol
    xi_g, xi_r = log["xi"][:, 0], ref["thermo"][:, 7]
    assert np.max(np.abs(xi_g - xi_r)) <= (1e-10 if prec == "fp64" else 1e-4) * np.max(np.abs(xi_r))
    assert np.array_equal(runs[0][1], runs[1][1])
    ref_rs = oracle.run(pos, vel, types, ka_params(), L, 0.005, 20, kind=oracle.RESAMPLE, T_target=0.5,
                        nstep_boltz=10, seed=78, log_every=1)
    with make_system(n, L, types, prec) as s:
        s.set_state(pos, vel)
        log = s.step_nvt(0.005, 20, 0.5, kind=kamd.MD_NVT_RESAMPLE, param=10, seed=78, log_every=1)
    assert abs(log["T"][9, 0] - 0.5) < 1e-12 and abs(log["T"][19, 0] - 0.5) < 1e-12
    assert thermo_rel(log, ref_rs["thermo"], "etot_per_n", 4) <= tol


@pytest.mark.parametrize("prec", PRECS)
def test_resample_bath(prec):
    pos, vel, types, L = melted(1000, 33, nsteps=100)
    ref = oracle.run(pos, vel, types, ka_params(), L, 0.005, 40, kind=oracle.RESAMPLE, T_target=0.5, nstep_boltz=10,
                     seed=77, log_every=1)
    with make_system(1000, L, types, prec) as s:
        s.set_state(pos, vel)
        log = s.step_nvt(0.005, 40, 0.5, kind=kamd.MD_NVT_RESAMPLE, param=10, seed=77, log_every=1)
        p, v, _ = s.get_state()
    for k in (9, 19, 29, 39):
        assert abs(log["T"][k, 0] - 0.5) < 1e-12
    tol = 1e-10 if prec == "fp64" else TOL_E["mixed"]
    assert thermo_rel(log, ref["thermo"], "etot_per_n", 4) <= tol
    # the step-40 velocities are a fresh draw: identical up to rounding
    assert np.max(np.abs(v - ref["vel"])) < (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", PRECS)
def test_init_lattice_matches_oracle(prec):
    for n in (1000, 4000):
        L = wl.box_length(n)
        types = wl.ka_types(n, 41)
        pos_r, vel_r = oracle.init_lattice(n, L, 2.0, seed=41, jitter=0.05)
        with make_system(n, L, types, prec) as s:
            s.init_lattice(2.0, 0.05, 41)
            p, v, _ = s.get_state()
        assert np.max(np.abs(min_image_diff(p, pos_r, L))) < (1e-12 if prec == "fp64" else 1e-8)
        assert np.max(np.abs(v - vel_r)) < (1e-12 if prec == "fp64" else 1e-6)
        assert np.sum(v * v) / (3 * n) == pytest.approx(2.0, rel=1e-12 if prec == "fp64" else 1e-6)


# ------------------------------------------------------------------ structure

@pytest.mark.parametrize("prec", PRECS)
def test_deterministic_bitwise(prec):
    pos, vel, types, L = melted(1000, 51, nsteps=100)
    out = []
    for _ in range(2):
        with make_system(1000, L, types, prec) as s:
            s.set_state(pos, vel)
            log = s.step_nvt(0.005, 60, 1.0, kind=kamd.MD_NVT_NOSE_HOOVER, param=0.5, log_every=10)
            out.append((s.get_state(), log))
    (a, la), (b, lb) = out
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(la, lb)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("red_tiles", [None, "16"], ids=["one-level", "two-level"])
def test_batch_replicas_equal_standalone_runs(prec, red_tiles, monkeypatch):
    """Every replica of a batch is bitwise equal to its stand-alone run, also when the batch reduces in
    two levels (chunks of 16 tiles: the 1000- and 2000-particle replicas span several chunks, the
    others one) while a small stand-alone replica reduces in one."""
    if red_tiles is not None:
        monkeypatch.setenv("KAMD_RED_TILES", red_tiles)
    ns = [250, 1000, 500, 2000]
    Ts = [0.6, 1.2, 0.9, 2.0]
    cfg = [melted(n, 60 + k, nsteps=50) for k, n in enumerate(ns)]
    Ls = [c[3] for c in cfg]
    types = np.concatenate([c[2] for c in cfg])
    with kamd.System(ns, Ls, types, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, 1.0, 0.3, prec) as b:
        b.set_state(np.concatenate([c[0] for c in cfg]), np.concatenate([c[1] for c in cfg]))
        blog = b.step_nvt(0.005, 80, Ts, kind=kamd.MD_NVT_NOSE_HOOVER, param=0.5, log_every=20)
        bp, bv, bi = b.get_state()
    off = 0
    for k, n in enumerate(ns):
        with make_system(n, Ls[k], cfg[k][2], prec) as s:
            s.set_state(cfg[k][0], cfg[k][1])
            log = s.step_nvt(0.005, 80, Ts[k], kind=kamd.MD_NVT_NOSE_HOOVER, param=0.5, log_every=20)
            p, v, i = s.get_state()
        assert np.array_equal(p, bp[off:off + n]) and np.array_equal(v, bv[off:off + n])
        assert np.array_equal(log[:, 0], blog[:, k])
        off += n


@pytest.mark.parametrize("prec", PRECS)
def test_batch_nve_log_records_and_time_lists(prec):
    """NVE on a batch: the log records formed after the launch, one (slot, replica) pair per CTA,
    equal every replica's stand-alone records bitwise; md_time_lists then rebuilds every replica,
    and each replica's forces are the oracle's at its positions."""
    ns = [500, 2000, 1000]
    cfg = [melted(n, 70 + k, nsteps=50) for k, n in enumerate(ns)]
    Ls = [c[3] for c in cfg]
    types = np.concatenate([c[2] for c in cfg])
    with kamd.System(ns, Ls, types, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, 1.0, 0.3, prec) as b:
        b.set_state(np.concatenate([c[0] for c in cfg]), np.concatenate([c[1] for c in cfg]))
        blog = b.step_nve(0.005, 120, log_every=10)
        assert 0.0 < b.time_lists(5) < 1e-2
        bp, _, _ = b.get_state()
        bf, _, _ = b.forces()
    off = 0
    for k, n in enumerate(ns):
        with make_system(n, Ls[k], cfg[k][2], prec) as s:
            s.set_state(cfg[k][0], cfg[k][1])
            log = s.step_nve(0.005, 120, log_every=10)
        assert np.array_equal(log[:, 0], blog[:, k])
        f_ref, _, _ = oracle.forces(bp[off:off + n], cfg[k][2], ka_params(), Ls[k])
        check_forces(bf[off:off + n], f_ref, prec)
        off += n


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("skins", [None, (0.3, 0.3), (0.2, 0.5)], ids=["default", "one-list", "dual-0.2-0.5"])
def test_rebuilds_keep_parity_over_long_nve(prec, skins):
    """400 NVE steps at T=2 cross many list rebuilds (and inner-list prunes, for two lists).
    FP64 follows the oracle step by step over all 400 steps; the mixed path does for the first
    100 steps, after which chaos amplifies FP32 rounding until the trajectories part. From there
    on the mixed run is compared by its statistics in tests/test_gpu_longrun.py (drift, PE, T,
    g(r) and MSD with run-to-run error bars); here it only has to stay a finite, bounded NVE run:
    its energy may not wander further than the oracle's own largest excursion plus four times
    the excursion of a random walk with the larger of the two runs' RMS step-to-step changes of
    E_tot/N (sigma * sqrt(steps)): a bound that rounding noise of either size stays within."""
    pos, vel, types, L = melted(1000, 71, nsteps=100)
    ref = oracle.run(pos, vel, types, ka_params(), L, 0.005, 400, log_every=1)
    with make_system(1000, L, types, prec) as s:
        if skins is not None:
            s.set_tuning(skin=skins[0], skin_outer=skins[1])
        s.set_state(pos, vel)
        log = s.step_nve(0.005, 400, log_every=1)
        info = s.info()
    assert info["rebuilds"] >= 5
    if skins is not None and skins[0] == skins[1]:
        assert info["prunes"] == 0
    else:
        assert info["prunes"] >= info["rebuilds"]
    if prec == "fp64":
        assert thermo_rel(log, ref["thermo"], "etot_per_n", 4) <= 1e-9
    else:
        assert thermo_rel(log[:100], ref["thermo"][:100], "etot_per_n", 4) <= TOL_E["mixed"]
        e_g = log["etot_per_n"][:, 0]
        e_r = ref["thermo"][:, 4]
        assert np.all(np.isfinite(e_g))
        exc_g = np.max(np.abs(e_g - e_g[0]))
        exc_r = np.max(np.abs(e_r - e_r[0]))
        # step-to-step fluctuation of E_tot/N (integrator noise, the same physics on both sides)
        noise = max(np.std(np.diff(e_g)), np.std(np.diff(e_r)))
        assert exc_g <= exc_r + 4.0 * noise * np.sqrt(len(e_g)), (exc_g, exc_r, noise)


def test_sampled_forces_one_million():
    """N = 10^6 mixed: 200 sampled particles against O(N) oracle sums."""
    n = 1_000_000
    L = wl.box_length(n)
    types = wl.ka_types(n, 81)
    with make_system(n, L, types, "mixed") as s:
        s.init_lattice(0.5, 0.05, 81)
        s.step_nvt(0.005, 20, 0.5, kind=kamd.MD_NVT_NOSE_HOOVER, param=0.5)
        f, pe, _ = s.forces()
        p, _, _ = s.get_state()
    rng = np.random.default_rng(81)
    idx = rng.choice(n, size=200, replace=False)
    t32 = types.astype(np.int32)
    ref = np.array([oracle.force_on(p, t32, ka_params(), L, i)[0] for i in idx])
    frms = np.sqrt(np.mean(np.sum(f * f, axis=1)))
    err = np.linalg.norm(f[idx] - ref, axis=1) / frms
    assert err.max() <= TOL_F["mixed"], err.max()


# Launch configurations the benchmark's autotuner settled on for each workload
# (lanes per particle, CTA size, force-list skin, outer-list skin); the lists
# are built and pruned by the timed-style launches before the forces are read.
BENCH_LAUNCH = {
    "ka32k": (4, 512, 0.3, 1.2),
    "ka1m": (1, 512, 0.4, 0.4),
    "ka8m": (1, 512, 0.4, 0.4),
    "ensemble": (4, 256, 0.4, 0.4),
}


def sampled_force_errors(f, p, types, L, idx):
    """|dF_i| / F_rms for the sampled particles, against O(N) oracle sums."""
    t32 = types.astype(np.int32)
    ref = np.array([oracle.force_on(p, t32, ka_params(), L, i)[0] for i in idx])
    frms = np.sqrt(np.mean(np.sum(f * f, axis=1)))
    return np.linalg.norm(f[idx] - ref, axis=1) / frms, frms


@pytest.mark.parametrize("name,n,prec,nsamp", [
    ("ka32k", 32000, "mixed", 300), ("ka32k", 32000, "fp64", 300),
    ("ka1m", 1_000_000, "mixed", 200), ("ka8m", 8_000_000, "mixed", 48)])
def test_sampled_forces_full_size_in_bench_launch(name, n, prec, nsamp):
    """Full-size systems in the benchmark's launch configuration: a bath stage, then NVE launches
    of 100 steps that rebuild (and, for two lists, prune) the lists, then sampled forces against
    O(N) oracle sums, and the sum of all forces (zero by Newton's third law) against F_rms."""
    L = wl.box_length(n)
    types = wl.ka_types(n, 90 + len(name))
    tpa, bs, skin, skin_out = BENCH_LAUNCH[name]
    with make_system(n, L, types, prec) as s:
        s.set_tuning(threads_per_atom=tpa, block_size=bs, skin=skin, skin_outer=skin_out)
        s.init_lattice(2.0, 0.05, 90)
        s.step_nvt(0.005, 60, 0.8, kind=kamd.MD_NVT_NOSE_HOOVER, param=0.5)
        s.step_nve(0.005, 100)
        s.step_nve(0.005, 100)
        info = s.info()
        f, pe, _ = s.forces()
        p, _, _ = s.get_state()
    assert info["rebuilds"] >= 2
    if skin_out > skin:
        assert info["prunes"] >= info["rebuilds"]
    idx = np.random.default_rng(n).choice(n, size=nsamp, replace=False)
    err, frms = sampled_force_errors(f, p, types, L, idx)
    assert err.max() <= TOL_F[prec], err.max()
    assert np.linalg.norm(f.sum(axis=0)) <= TOL_F[prec] * frms * np.sqrt(n)
    assert np.isfinite(pe).all() and np.all((p >= 0) & (p < L))


def test_sampled_forces_ensemble_in_bench_launch():
    """The 512-replica mix (N in {250, ..., 8000}, about 1.3 million particles) in the benchmark's
    launch configuration, after a Nose-Hoover stage at each replica's own temperature: one sampled
    particle in every fourth replica against the O(N) oracle sum over its own box."""
    spec = wl.ensemble(512, 4)
    tpa, bs, skin, skin_out = BENCH_LAUNCH["ensemble"]
    types = np.concatenate(spec.types)
    with kamd.System(spec.n, spec.L, types, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, wl.KA_MASS, 0.3, "mixed") as s:
        s.set_tuning(threads_per_atom=tpa, block_size=bs, skin=skin, skin_outer=skin_out)
        s.init_lattice(2.0, 0.05, 4)
        s.step_nvt(0.005, 100, spec.T, kind=kamd.MD_NVT_NOSE_HOOVER, param=0.5)
        f, pe, _ = s.forces()
        p, _, _ = s.get_state()
    assert pe.shape[0] == 512 and np.isfinite(pe).all()
    off = np.concatenate([[0], np.cumsum(spec.n)])
    rng = np.random.default_rng(4)
    worst = 0.0
    for r in range(0, 512, 4):
        a, b = off[r], off[r + 1]
        i = int(rng.integers(0, b - a))
        err, _ = sampled_force_errors(f[a:b], p[a:b], spec.types[r], spec.L[r], [i])
        worst = max(worst, float(err[0]))
    assert worst <= TOL_F["mixed"], worst


class _MsdAgainstOracle:
    """Wraps a system for the waiting-time schedule: at each reset the caller-order positions and
    images are read back and kept as r(t_w); at each measurement the oracle's Eq. (msdwithi) is
    evaluated on the same read-back state against that reference."""

    def __init__(self, s, types, L):
        self.s, self.types, self.L = s, types, L
        self.ntypes = s.ntypes
        self.ref, self.pairs = {}, []

    def msd_tw(self, slot, reset_reference=False):
        out = self.s.msd_tw(slot, reset_reference)
        p, _, img = self.s.get_state()
        if reset_reference:
            self.ref[slot] = p + self.L * img
        else:
            self.pairs.append((out, oracle.msd(p, img, self.ref[slot], self.types, 2, self.L)))
        return out


@pytest.mark.parametrize("prec", PRECS)
def test_waiting_time_msd_matches_oracle(prec):
    """Eq. (msdtw) for t_w = 0, 10, 100 steps along one NVE trajectory (slots 1-3), every point
    against the oracle on the read-back state; slot 0 (md_msd) keeps its own reference."""
    from paper_2001_07089_gb300 import analysis
    pos, vel, types, L = melted(1000, 95, nsteps=100)
    with make_system(1000, L, types, prec) as s:
        s.set_state(pos, vel)
        chk = _MsdAgainstOracle(s, types, L)
        res = analysis.waiting_time_msd(chk, [0, 10, 100], 200, advance=lambda n: s.step_nve(0.005, n), kmax=12)
        p, _, img = s.get_state()
        m0 = s.msd()
    assert len(chk.pairs) == 3 * len(res[0][0])
    for got, ref in chk.pairs:
        assert np.allclose(got, ref, rtol=1e-9 if prec == "fp64" else 1e-5, atol=1e-14)
    assert np.allclose(m0, oracle.msd(p, img, pos, types, 2, L), rtol=1e-9 if prec == "fp64" else 1e-5)
    for tw in (0, 10, 100):
        assert res[tw][1][-1, 0] > 10 * res[tw][1][0, 0] > 0.0  # particles move away from r(t_w)


def test_msd_slots_reject_bad_use():
    pos, vel, types, L = melted(250, 96, nsteps=50)
    with make_system(250, L, types, "mixed") as s:
        s.set_state(pos, vel)
        with pytest.raises(kamd.KamdError):
            s.msd_tw(kamd.MD_MSD_SLOTS, reset_reference=True)
        with pytest.raises(kamd.KamdError):
            s.msd_tw(-1)
        with pytest.raises(kamd.KamdError):
            s.msd_tw(3)  # never reset
        s.msd_tw(3, reset_reference=True)
        s.step_nve(0.005, 20)
        assert np.all(s.msd_tw(3) > 0)
        s.set_state(pos, vel)  # a new state: slots other than 0 lose their reference
        with pytest.raises(kamd.KamdError):
            s.msd_tw(3)
        assert np.all(s.msd_tw(0) == 0.0)


def test_cooling_ladder_batch_matches_standalone_and_oracle():
    """The cooling sequence (stochastic bath, NVE, production at each temperature) on a batch of
    two replicas: every replica bitwise equal to its stand-alone ladder, T exactly at target after
    each bath, and the FP64 stand-alone run against the oracle stage by stage."""
    from paper_2001_07089_gb300 import analysis
    temps, nb, dt = [2.0, 1.0, 0.6], 10, 0.005
    ns = [250, 500]
    cfg = [melted(n, 97 + k, nsteps=50) for k, n in enumerate(ns)]
    Ls = [c[3] for c in cfg]
    with kamd.System(ns, Ls, np.concatenate([c[2] for c in cfg]), wl.KA_EPS, wl.KA_SIG, wl.KA_RC, 1.0, 0.3,
                     "fp64") as b:
        b.set_state(np.concatenate([c[0] for c in cfg]), np.concatenate([c[1] for c in cfg]))
        bl = analysis.cooling_ladder(b, temps, dt, 20, 20, 20, nstep_boltz=nb, seed=5, log_every=10)
        bp, bv, _ = b.get_state()
    off = 0
    for k, n in enumerate(ns):
        pos, vel, types, L = cfg[k]
        with make_system(n, L, types, "fp64") as s:
            s.set_state(pos, vel)
            sl = analysis.cooling_ladder(s, temps, dt, 20, 20, 20, nstep_boltz=nb, seed=5, log_every=10)
            p, v, _ = s.get_state()
        assert np.array_equal(p, bp[off:off + n]) and np.array_equal(v, bv[off:off + n])
        for st_b, st_s in zip(bl, sl):
            assert abs(st_s["bath"]["T"][-1, 0] - st_s["T"]) < 1e-12
            for key in ("bath", "nve", "production"):
                assert np.array_equal(st_b[key]["etot_per_n"][:, k], st_s[key]["etot_per_n"][:, 0])
        if k == 0:
            step, img = 0, np.zeros((n, 3), np.int32)
            x, u = pos, vel
            for j, st in enumerate(sl):
                r = oracle.run(x, u, types, ka_params(), L, dt, 20, kind=oracle.RESAMPLE, T_target=st["T"],
                               nstep_boltz=nb, seed=5 + j, img=img, step0=step, log_every=10)
                assert thermo_rel(st["bath"], r["thermo"], "etot_per_n", 4) <= 1e-10
                r2 = oracle.run(r["pos"], r["vel"], types, ka_params(), L, dt, 20, img=r["img"], step0=step + 20,
                                log_every=10)
                assert thermo_rel(st["nve"], r2["thermo"], "etot_per_n", 4) <= 1e-10
                r3 = oracle.run(r2["pos"], r2["vel"], types, ka_params(), L, dt, 20, img=r2["img"],
                                step0=step + 40, log_every=10)
                assert thermo_rel(st["production"], r3["thermo"], "etot_per_n", 4) <= 1e-10
                x, u, img, step = r3["pos"], r3["vel"], r3["img"], step + 60
        off += n


def rdf_counts(g, types, L, dr, nbins):
    """Pair counts per bin behind normalised partial g(r) rows (AA, BB, AB): the inverse of the
    normalisation of Sec. "Radial distribution function with Python" (like pairs counted twice)."""
    na = int(np.sum(np.asarray(types) == 0))
    nb = len(types) - na
    k = np.arange(nbins)
    shell = 4.0 / 3.0 * np.pi * ((k + 1) ** 3 - k ** 3) * dr ** 3
    V = L ** 3
    h = np.stack([g[0] * shell * na * (na - 1) / V, g[1] * shell * nb * (nb - 1) / V, g[2] * shell * na * nb / V])
    c = np.rint(h)
    assert np.max(np.abs(h - c)) < 1e-6 * max(1.0, c.max())
    return c.astype(np.int64)


def bin_edge_allowance(pos, types, L, dr, nbins, tol):
    """Per-bin count difference allowed for pairs whose distance lies within tol of a bin edge
    (either side may bin them on either side of it), and the number of such pairs."""
    pos = np.asarray(pos)
    t = np.asarray(types)
    allow = np.zeros((3, nbins), dtype=np.int64)
    nedge = 0
    for i in range(len(pos) - 1):
        d = pos[i] - pos[i + 1:]
        d -= L * np.rint(d / L)
        r = np.sqrt(np.sum(d * d, axis=1))
        x = r / dr
        k = np.rint(x).astype(np.int64)
        near = (np.abs(x - k) * dr < tol) & (k >= 0) & (k <= nbins)
        for j in np.nonzero(near)[0]:
            ti, tj = t[i], t[i + 1 + j]
            row = 0 if ti == tj == 0 else (1 if ti == tj == 1 else 2)
            w = 2 if ti == tj else 1
            for kk in (k[j] - 1, k[j]):
                if 0 <= kk < nbins:
                    allow[row, kk] += w
            nedge += 1
    return allow, nedge


@pytest.mark.parametrize("prec", PRECS)
def test_rdf_and_msd_match_oracle(prec):
    """g(r) bin by bin: both sides bin the same pair distances (the GPU's mixed path from the exact
    64-bit fixed-point differences, the oracle from the read-back doubles), so the pair counts behind
    every bin agree exactly except for pairs within 1e-12 L of a bin edge, which the test counts."""
    pos, vel, types, L = melted(1000, 91, nsteps=100)
    dr, nbins = 0.05, 80
    with make_system(1000, L, types, prec) as s:
        s.set_state(pos, vel)
        s.step_nve(0.005, 100)
        g = s.rdf(dr, nbins, reset=True)
        p, v, img = s.get_state()
        msd = s.msd()
    g_ref = oracle.rdf(p, types, L, dr, nbins)
    if prec == "fp64":
        assert np.allclose(g, g_ref, rtol=1e-12, atol=1e-12)
    cg, cr = rdf_counts(g, types, L, dr, nbins), rdf_counts(g_ref, types, L, dr, nbins)
    allow, nedge = bin_edge_allowance(p, types, L, dr, nbins, 1e-12 * L)
    assert np.all(np.abs(cg - cr) <= allow), (np.abs(cg - cr).max(), nedge)
    assert cg.sum() == cr.sum() or nedge > 0
    m_ref = oracle.msd(p, img, pos, types, 2, L)
    assert np.allclose(msd, m_ref, rtol=1e-9 if prec == "fp64" else 1e-5)


def test_count_pairs_matches_oracle():
    pos, vel, types, L = melted(1000, 92, nsteps=100)
    with make_system(1000, L, types, "fp64") as s:
        s.set_state(pos, vel)
        c = s.count_pairs()
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.rint(d / L)
    r2 = np.sum(d * d, axis=2)
    rc2 = (wl.KA_RC ** 2)[types[:, None], types[None, :]]
    ref = (np.sum(r2 < rc2) - len(pos)) // 2
    assert c == ref


def test_graph_launch_matches_direct_launch(monkeypatch):
    """The persistent kernel launched through its CUDA graph and launched directly give
    bitwise identical trajectories; the graph path is the one taken by default."""
    pos, vel, types, L = melted(1000, 95, nsteps=50)
    runs = []
    for no_graph in ("0", "1"):
        monkeypatch.setenv("KAMD_NO_GRAPH", no_graph)
        with make_system(1000, L, types, "mixed") as s:
            s.set_state(pos, vel)
            log = s.step_nvt(0.005, 60, 0.9, kind=kamd.MD_NVT_NOSE_HOOVER, param=0.5, log_every=10)
            log2 = s.step_nve(0.005, 40, log_every=10)
            st = s.get_state()
            info = s.info()
        runs.append((st, log, log2, info))
    monkeypatch.delenv("KAMD_NO_GRAPH", raising=False)
    assert runs[0][3]["graph_launches"] >= 2 and runs[1][3]["graph_launches"] == 0
    for a, b in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(runs[0][1], runs[1][1]) and np.array_equal(runs[0][2], runs[1][2])


@pytest.mark.parametrize("fixed_skin", [None, 0.3], ids=["free", "skin-0.3"])
def test_autotune_restores_state_and_keeps_parity(fixed_skin):
    """The autotuner (lanes per particle x CTA size x skins, or with the force-list skin fixed) times
    short NVE probes on a copy of the state: afterwards the state is the one it started from, the
    chosen tuning is valid, and the run continues with the oracle's energies."""
    pos, vel, types, L = melted(4000, 41, nsteps=100)
    ref = oracle.run(pos, vel, types, ka_params(), L, 0.005, 40, log_every=1)
    with make_system(4000, L, types, "mixed") as s:
        s.set_state(pos, vel)
        p0, v0, i0 = s.get_state()
        tun, sec = s.autotune(0.005, probe_steps=10, skin=fixed_skin)
        p1, v1, i1 = s.get_state()
        # velocities and images come back exactly; positions pass once more through the 64-bit
        # fixed-point form, which can move the last bits of a double
        assert np.array_equal(v0, v1) and np.array_equal(i0, i1)
        assert np.max(np.abs(p1 - p0)) <= 1e-12 * L
        assert tun == s.tuning and sec > 0
        assert tun["threads_per_atom"] in (1, 2, 4, 8) and tun["block_size"] in (128, 256, 512)
        assert tun["skin_outer"] >= tun["skin"]
        if fixed_skin is not None:
            assert tun["skin"] == fixed_skin
        log = s.step_nve(0.005, 40, log_every=1)
    assert thermo_rel(log, ref["thermo"], "etot_per_n", 4) <= TOL_E["mixed"]


def test_device_footprint_counter_tracks_frees():
    """md_get_info's device_bytes follows allocations and frees: retuning (which reallocates the lists)
    and autotuning leave it at the footprint of the final tuning, not the sum of every allocation."""
    pos, vel, types, L = melted(4000, 42, nsteps=50)
    with make_system(4000, L, types, "mixed") as s:
        s.set_state(pos, vel)
        s.step_nve(0.005, 10)
        base = s.info()["device_bytes"]
        for tpa in (1, 2, 4, 8, 4):
            s.set_tuning(threads_per_atom=tpa)
            s.step_nve(0.005, 10)
        again = s.info()["device_bytes"]
        s.autotune(0.005, probe_steps=5)
        s.set_tuning(threads_per_atom=4, block_size=256, skin=0.3, skin_outer=0.7)
        s.step_nve(0.005, 10)
        after = s.info()["device_bytes"]
    assert 0 < base < 2 ** 31
    assert abs(again - base) <= 0.5 * base and abs(after - base) <= 0.5 * base


@pytest.mark.parametrize("prec", PRECS)
def test_time_forces_leaves_the_trajectory_unchanged(prec):
    """md_time_forces (the force phase alone, repeated inside one launch) reports a positive time,
    leaves the stored forces at the oracle's, and the trajectory that follows is bitwise the one
    without the measurement."""
    pos, vel, types, L = melted(1000, 93, nsteps=100)
    f_ref, _, _ = oracle.forces(pos, types, ka_params(), L)
    runs = []
    for measure in (False, True):
        with make_system(1000, L, types, prec) as s:
            s.set_state(pos, vel)
            s.step_nve(0.005, 10)
            if measure:
                t = s.time_forces(20)
                assert 0.0 < t < 1e-2
            log = s.step_nve(0.005, 40, log_every=10)
            runs.append((s.get_state(), log))
    (a, la), (b, lb) = runs
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(la, lb)
    with make_system(1000, L, types, prec) as s:
        s.set_state(pos, vel)
        s.time_forces(5)
        f, _, _ = s.forces()
    check_forces(f, f_ref, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,log_every", [(4000, 10), (4000, 1), (1000, 7)])
def test_log_records_reduced_after_the_launch_equal_those_at_the_step(prec, n, log_every, monkeypatch):
    """NVE log records whose sums are formed after the launch's last step (the default) are bitwise
    those formed at their steps (KAMD_LOG_NOW=1), and the trajectory is the same; log_every = 1 has
    more log steps than the 64 slots of a launch, so both kinds of record occur in one call."""
    pos, vel, types, L = melted(n, 96, nsteps=100)
    runs = []
    for now in ("1", "0"):
        monkeypatch.setenv("KAMD_LOG_NOW", now)
        with make_system(n, L, types, prec) as s:
            s.set_state(pos, vel)
            log = s.step_nve(0.005, 150, log_every=log_every)
            runs.append((log, s.get_state()))
    (la, a), (lb, b) = runs
    assert len(la) == 150 // log_every and np.all(np.diff(la["step"][:, 0]) == log_every)
    assert np.array_equal(la, lb)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("ntypes", [3, 4])
def test_forces_with_three_and_four_species(prec, ntypes):
    """More than two species (the list build's general radius selection, the type tables): a melted
    N = 4000 liquid relabelled at random into 3 or 4 species with their own symmetric eps/sigma
    (Lorentz-like mixing, r_c = 2.5 sigma_ab), one and four lanes per particle, against the oracle."""
    pos, vel, _, L = melted(4000, 23, nsteps=200)
    rng = np.random.default_rng(40 + ntypes)
    types = rng.integers(0, ntypes, size=len(pos)).astype(np.int32)
    sig1 = np.array([1.0, 0.88, 0.94, 0.82])[:ntypes]
    eps1 = np.array([1.0, 0.5, 0.8, 1.2])[:ntypes]
    sig = 0.5 * (sig1[:, None] + sig1[None, :])
    eps = np.sqrt(eps1[:, None] * eps1[None, :])
    rc = 2.5 * sig
    f_ref, v_ref, _ = oracle.forces(pos, types, oracle.Params(eps, sig, rc, 1.0), L)
    for tpa in (1, 4):
        with kamd.System(len(pos), L, types, eps, sig, rc, 1.0, 0.3, prec) as s:
            s.set_tuning(threads_per_atom=tpa)
            s.set_state(pos, vel)
            f, pe, _ = s.forces()
        check_forces(f, f_ref, prec)
        assert abs(pe[0] - v_ref) <= TOL_E[prec] * abs(v_ref)


def test_log_records_after_the_launch_with_the_stochastic_bath(monkeypatch):
    """The stochastic bath (Maxwell-Boltzmann redraw every 50 steps): records of redraw steps are
    formed at their steps, those of the NVE steps between after the launch; the log is bitwise the
    one with every record formed at its step (KAMD_LOG_NOW=1)."""
    pos, vel, types, L = melted(2000, 97, nsteps=100)
    logs = []
    for now in ("1", "0"):
        monkeypatch.setenv("KAMD_LOG_NOW", now)
        with make_system(2000, L, types, "mixed") as s:
            s.set_state(pos, vel)
            logs.append(s.step_nvt(0.005, 150, 1.2, kind=kamd.MD_NVT_RESAMPLE, param=50, seed=7, log_every=10))
    a, b = logs
    assert len(a) == 15 and np.all(np.isfinite(a["T"]))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", PRECS)
def test_time_lists_leaves_a_rebuilt_state(prec):
    """md_time_lists (the list build alone, repeated inside one launch after a full rebuild)
    reports a positive time and leaves the state of a rebuild at unchanged positions: the forces
    there are the oracle's, and the 40 steps that follow keep the energy of the run without the
    measurement (the re-sort may change the summation order, so not bitwise). N = 4000: half-width
    cells and several list-build groups."""
    pos, vel, types, L = melted(4000, 94, nsteps=100)
    logs = []
    for measure in (False, True):
        with make_system(4000, L, types, prec) as s:
            s.set_state(pos, vel)
            s.step_nve(0.005, 10)
            if measure:
                t = s.time_lists(5)
                assert 0.0 < t < 1e-2
                p, _, _ = s.get_state()
                f, _, _ = s.forces()
                f_ref, _, _ = oracle.forces(p, types, ka_params(), L)
                check_forces(f, f_ref, prec)
            logs.append(s.step_nve(0.005, 40, log_every=10))
    a, b = logs
    scale = np.abs(a["pe_per_n"]) + 1.5 * a["T"]
    tol = 1e-5 if prec == "mixed" else 1e-10
    assert np.all(np.abs(a["etot_per_n"] - b["etot_per_n"]) <= tol * scale)
