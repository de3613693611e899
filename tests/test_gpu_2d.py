"""The two-dimensional Kob-Andersen model (Sec. "Suggested problems": N = 1000 at N/L^2 = 1.204,
L = 28.82, A:B = 65:35) on both GPU paths, through the C ABI, against the FP64 oracle run with
ndim = 2 on identical seeded inputs. Tolerances as in the three-dimensional parity tests."""
import numpy as np
import pytest

import oracle
from paper_2001_07089_gb300 import kamd
from paper_2001_07089_gb300 import workloads as wl
from tests.helpers import force_errors, ka_params, melted_2d, min_image_diff

pytestmark = pytest.mark.gpu

TOL_F = {"fp64": 1e-12, "mixed": 1e-5}
PRECS = ["fp64", "mixed"]
N = 1000


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kamd.load()


def system(L, types, prec):
    return kamd.System(N, L, types, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, wl.KA_MASS, wl.SKIN, prec, ndim=2)


def own_rel(log, th, field, col):
    return np.max(np.abs(log[field][:, 0] - th[:, col]) / np.abs(th[:, col]))


@pytest.mark.parametrize("prec", PRECS)
def test_2d_forces_match_oracle(prec):
    pos, vel, types, L = melted_2d(N, 81)
    f_ref, v_ref, w_ref = oracle.forces(pos, types, ka_params(), L)
    assert np.all(f_ref[:, 2] == 0.0)
    with system(L, types, prec) as s:
        s.set_state(pos, vel)
        f, pe, vir = s.forces()
    emax, e2 = force_errors(f, f_ref)
    assert emax <= TOL_F[prec] and e2 <= TOL_F[prec], (emax, e2)
    assert np.all(f[:, 2] == 0.0)
    assert abs(pe[0] - v_ref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(v_ref)


@pytest.mark.parametrize("prec", PRECS)
def test_2d_nve_100_steps(prec):
    pos, vel, types, L = melted_2d(N, 82)
    ref = oracle.run(pos, vel, types, ka_params(), L, 0.005, 100, log_every=1, ndim=2)
    th = ref["thermo"]
    with system(L, types, prec) as s:
        s.set_state(pos, vel)
        log = s.step_nve(0.005, 100, log_every=1)
        p, v, _ = s.get_state()
    tol = 1e-10 if prec == "fp64" else 1e-6
    for field, col in (("etot_per_n", 4), ("pe_per_n", 2), ("ke_per_n", 3), ("T", 1)):
        assert own_rel(log, th, field, col) <= tol, field
    assert np.all(p[:, 2] == 0.5 * L) and np.all(v[:, 2] == 0.0)
    assert np.max(np.abs(min_image_diff(p, ref["pos"], L))) < (1e-9 if prec == "fp64" else 1e-3)


@pytest.mark.parametrize("prec", PRECS)
def test_2d_nose_hoover_and_resampling_bath(prec):
    """Nose-Hoover with X = 2N and Q = 2N T tau^2, and the stochastic bath rescaled to exactly
    2N T, against the oracle with ndim = 2."""
    pos, vel, types, L = melted_2d(N, 83)
    T, tau = 0.45, 0.5
    ref = oracle.run(pos, vel, types, ka_params(), L, 0.005, 100, kind=oracle.NOSE_HOOVER, T_target=T,
                     Q=2 * N * T * tau * tau, log_every=1, ndim=2)
    with system(L, types, prec) as s:
        s.set_state(pos, vel)
        log = s.step_nvt(0.005, 100, T, kind=kamd.MD_NVT_NOSE_HOOVER, param=tau, log_every=1)
    tol = 1e-10 if prec == "fp64" else 1e-6
    assert own_rel(log, ref["thermo"], "etot_per_n", 4) <= tol
    assert own_rel(log, ref["thermo"], "h_nh", 6) <= tol
    assert np.max(np.abs(log["xi"][:, 0] - ref["thermo"][:, 7])) <= (1e-10 if prec == "fp64" else 1e-4) * np.max(
        np.abs(ref["thermo"][:, 7]))
    rs = oracle.run(pos, vel, types, ka_params(), L, 0.005, 20, kind=oracle.RESAMPLE, T_target=0.3, nstep_boltz=10,
                    seed=5, log_every=1, ndim=2)
    with system(L, types, prec) as s:
        s.set_state(pos, vel)
        log = s.step_nvt(0.005, 20, 0.3, kind=kamd.MD_NVT_RESAMPLE, param=10, seed=5, log_every=1)
        _, v, _ = s.get_state()
    assert abs(log["T"][9, 0] - 0.3) < 1e-12 and abs(log["T"][19, 0] - 0.3) < 1e-12
    assert np.all(v[:, 2] == 0.0)
    assert np.max(np.abs(v - rs["vel"])) < (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", PRECS)
def test_2d_lattice_start_matches_oracle(prec):
    L = wl.box_length_2d(N)
    types = wl.ka_types(N, 84, frac_b=wl.FRAC_B_2D)
    pos_r, vel_r = oracle.init_lattice(N, L, 0.4, seed=84, jitter=0.05, ndim=2)
    with system(L, types, prec) as s:
        s.init_lattice(0.4, 0.05, 84)
        p, v, _ = s.get_state()
    assert np.max(np.abs(min_image_diff(p, pos_r, L))) < (1e-12 if prec == "fp64" else 1e-8)
    assert np.max(np.abs(v - vel_r)) < (1e-12 if prec == "fp64" else 1e-6)
    assert np.sum(v * v) / (2 * N) == pytest.approx(0.4, rel=1e-12 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec", PRECS)
def test_2d_rdf_and_msd(prec):
    """g(r) with the ring normalisation, bin counts exactly equal to the oracle's (the 2-D
    problem's shell-volume adjustment), and the per-type MSD from unwrapped positions."""
    pos, vel, types, L = melted_2d(N, 85)
    dr, nbins = 0.05, 120
    with system(L, types, prec) as s:
        s.set_state(pos, vel)
        s.step_nve(0.005, 200)
        g = s.rdf(dr, nbins, reset=True)
        p, _, img = s.get_state()
        msd = s.msd()
    g_ref = oracle.rdf(p, types, L, dr, nbins, ndim=2)
    na = int(np.sum(types == 0))
    nb = N - na
    k = np.arange(nbins)
    ring = np.pi * ((k + 1) ** 2 - k ** 2) * dr * dr
    norm = np.stack([ring * na * (na - 1), ring * nb * (nb - 1), ring * na * nb]) / L ** 2
    cg, cr = np.rint(g * norm), np.rint(g_ref * norm)
    assert np.max(np.abs(g * norm - cg)) < 1e-6 and np.max(np.abs(g_ref * norm - cr)) < 1e-6
    assert np.array_equal(cg, cr)
    assert 2.0 < g_ref[0].max() < 8.0  # a liquid's first peak in the ring-normalised g_AA
    m_ref = oracle.msd(p, img, pos, types, 2, L)
    assert np.allclose(msd, m_ref, rtol=1e-9 if prec == "fp64" else 1e-5)
