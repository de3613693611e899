"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these tests retypes the oracle's formulas: each checks a closed form,
an invariant, a special case, brute force, or a published vector, chosen so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2001_07089_gb300 import workloads as wl
from tests.helpers import ka_params, melted

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- inputs

def test_philox_known_answers():
    """Philox4x32-10 reproduces the published known-answer vectors (SC'11 / Random123)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_ka_parameters_match_paper():
    """The parameter table used everywhere equals the paper's (Sec. "Model")."""
    rows = {l.split()[0]: [float(x) for x in l.split()[1:]]
            for l in open(os.path.join(GOLDEN, "ka_parameters.txt")) if l.strip() and not l.startswith("#")}
    idx = {"AA": (0, 0), "AB": (0, 1), "BB": (1, 1)}
    for k, (a, b) in idx.items():
        eps, sig, rc = rows[k]
        assert wl.KA_EPS[a, b] == eps and wl.KA_EPS[b, a] == eps
        assert wl.KA_SIG[a, b] == sig and wl.KA_SIG[b, a] == sig
        assert abs(wl.KA_RC[a, b] - rc) < 1e-15


# -------------------------------------------------------------- pair term

def _two(r, a, b, L=20.0, axis=np.array([1.0, 0.0, 0.0])):
    pos = np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.0]]) + 0.0
    pos[1] += r * axis / np.linalg.norm(axis)
    f, v, w = oracle.forces(pos, np.array([a, b]), ka_params(), L)
    return pos, f, v, w


@pytest.mark.parametrize("a,b", [(0, 0), (0, 1), (1, 1)])
def test_pair_minimum_and_depth(a, b):
    """F = 0 at r = 2^(1/6) sigma and V there = -eps - V(r_c) with V(r_c) = 4 eps (2.5^-12 - 2.5^-6)."""
    eps, sig = wl.KA_EPS[a, b], wl.KA_SIG[a, b]
    rmin = 2.0 ** (1.0 / 6.0) * sig
    _, f, v, w = _two(rmin, a, b)
    assert np.all(np.abs(f) < 1e-12 * eps / sig)
    vc = 4.0 * eps * (2.5 ** -12 - 2.5 ** -6)
    assert abs(vc / eps - (-0.016316891136)) < 1e-11
    assert abs(v - (-eps - vc)) < 1e-13
    assert abs(w) < 1e-12 * eps


@pytest.mark.parametrize("a,b", [(0, 0), (0, 1), (1, 1)])
def test_pair_cutoff_truncation(a, b):
    """Beyond r_c (strict test) force and energy vanish; just inside, V -> 0+ continuously."""
    sig = wl.KA_SIG[a, b]
    rc = 2.5 * sig
    for r in (rc * (1 + 1e-9), rc * 1.01, rc * 1.5):
        _, f, v, w = _two(r, a, b)
        assert np.all(f == 0.0) and v == 0.0 and w == 0.0
    _, f, v, _ = _two(rc * (1 - 1e-7), a, b)
    assert 0.0 < abs(v) < 1e-6
    assert np.linalg.norm(f[0]) > 0.0


@pytest.mark.parametrize("a,b", [(0, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("rfac", [0.9, 1.05, 1.5, 2.3])
def test_pair_force_is_minus_gradient(a, b, rfac):
    """F_i = -dV/dr_i by central differences along an oblique direction."""
    sig = wl.KA_SIG[a, b]
    axis = np.array([0.3, -0.5, 0.8])
    pos, f, v, _ = _two(rfac * sig, a, b, axis=axis)
    h = 1e-6
    for c in range(3):
        p1 = pos.copy(); p1[0, c] += h
        p2 = pos.copy(); p2[0, c] -= h
        v1 = oracle.forces(p1, np.array([a, b]), ka_params(), 20.0)[1]
        v2 = oracle.forces(p2, np.array([a, b]), ka_params(), 20.0)[1]
        g = -(v1 - v2) / (2 * h)
        assert abs(f[0, c] - g) <= 1e-7 * max(1.0, abs(f[0]).max())
    assert np.allclose(f[0], -f[1], rtol=0, atol=1e-12 * max(1.0, abs(f).max()))
    assert np.dot(f[0], pos[0] - pos[1]) * 1 == pytest.approx(_two(rfac * sig, a, b, axis=axis)[3], rel=1e-12)


def test_pair_repulsive_attractive_sign():
    """Repulsive inside the minimum (F_0 points away from particle 1), attractive outside."""
    for a, b in [(0, 0), (0, 1), (1, 1)]:
        sig = wl.KA_SIG[a, b]
        _, f, _, _ = _two(0.95 * sig, a, b)
        assert f[0, 0] < 0 < f[1, 0]
        _, f, _, _ = _two(1.4 * sig, a, b)
        assert f[0, 0] > 0 > f[1, 0]


def test_type_table_is_used_per_pair():
    """Swapping the two particles' types leaves an AB pair unchanged; AA and BB differ from AB."""
    r = 1.0
    vs = {}
    for a, b in [(0, 0), (0, 1), (1, 0), (1, 1)]:
        vs[(a, b)] = _two(r, a, b)[2]
    assert vs[(0, 1)] == vs[(1, 0)]
    assert len({vs[(0, 0)], vs[(0, 1)], vs[(1, 1)]}) == 3


# --------------------------------------------------------- many particles

def _numgrad(pos, types, L, h=1e-6):
    g = np.zeros_like(pos)
    for i in range(pos.shape[0]):
        for c in range(3):
            p1 = pos.copy(); p1[i, c] += h
            p2 = pos.copy(); p2[i, c] -= h
            g[i, c] = -(oracle.forces(p1, types, ka_params(), L)[1]
                        - oracle.forces(p2, types, ka_params(), L)[1]) / (2 * h)
    return g


def test_forces_equal_numerical_gradient_melted():
    """On a melted 64-particle KA configuration (rho = 0.4, L > 2 r_c), F = -grad V."""
    pos, vel, types, L = melted(64, 11, nsteps=100, density=0.4)
    f, v, w = oracle.forces(pos, types, ka_params(), L)
    g = _numgrad(pos, types, L)
    frms = np.sqrt(np.mean(np.sum(f * f, axis=1)))
    assert np.max(np.abs(f - g)) < 1e-6 * max(frms, 1.0)


def test_newton_third_law_and_translation_invariance():
    """Sum of forces is zero; a rigid periodic shift leaves forces, V and W unchanged."""
    pos, vel, types, L = melted(500, 12, nsteps=50)
    f, v, w = oracle.forces(pos, types, ka_params(), L)
    frms = np.sqrt(np.mean(np.sum(f * f, axis=1)))
    assert np.all(np.abs(f.sum(axis=0)) < 1e-11 * frms * len(pos))
    shifted = np.mod(pos + np.array([L / 3, L / 7, L / 11]), L)
    f2, v2, w2 = oracle.forces(shifted, types, ka_params(), L)
    assert np.max(np.abs(f2 - f)) < 1e-9 * frms
    assert abs(v2 - v) < 1e-10 * abs(v)
    assert abs(w2 - w) < 1e-10 * abs(w)


def test_force_on_is_row_of_all_pairs_sum_and_gradient():
    """ora_force_on (particle i against every other particle, O(N)) is what the large-N GPU
    checks compare against. On a melted N = 500 liquid it gives row i of the all-pairs forces for
    every i, its half pair energies add up to V, and for sampled particles it equals the
    central-difference gradient -dV/dr_i of the total energy (Eq. (KAFix) as the gradient of
    Eq. (VshiftedKALJ)), so a dropped 1/2, a swapped i/j in the minimum image or a skipped j
    fails here."""
    pos, vel, types, L = melted(500, 19, nsteps=100)
    f, v, w = oracle.forces(pos, types, ka_params(), L)
    frms = np.sqrt(np.mean(np.sum(f * f, axis=1)))
    fo = np.zeros_like(f)
    vhalf = np.zeros(len(pos))
    for i in range(len(pos)):
        fo[i], vhalf[i] = oracle.force_on(pos, types, ka_params(), L, i)
    assert np.max(np.linalg.norm(fo - f, axis=1)) <= 1e-13 * frms
    assert vhalf.sum() == pytest.approx(v, rel=1e-13)
    h = 1e-6
    for i in (0, 137, 499):
        for c in range(3):
            p1 = pos.copy(); p1[i, c] += h
            p2 = pos.copy(); p2[i, c] -= h
            g = -(oracle.forces(p1, types, ka_params(), L)[1] - oracle.forces(p2, types, ka_params(), L)[1]) / (2 * h)
            assert abs(fo[i, c] - g) <= 1e-6 * frms


@pytest.mark.parametrize("a,b", [(0, 0), (0, 1), (1, 1)])
def test_force_on_pair_minimum_and_far_image(a, b):
    """Two particles at 2^(1/6) sigma_ab: force_on gives F = 0 on both and half the shifted
    depth -eps - V(r_c) each; placed across the periodic boundary the pair is found through its
    minimum image; beyond r_c it gives exactly nothing."""
    eps, sig = wl.KA_EPS[a, b], wl.KA_SIG[a, b]
    rmin = 2.0 ** (1.0 / 6.0) * sig
    vc = 4.0 * eps * (2.5 ** -12 - 2.5 ** -6)
    L = 20.0
    types = np.array([a, b], dtype=np.int32)
    for x0 in (5.0, L - 0.5 * rmin):  # second case: the pair straddles x = L
        pos = np.array([[x0, 3.0, 4.0], [np.mod(x0 + rmin, L), 3.0, 4.0]])
        for i in (0, 1):
            fi, vh = oracle.force_on(pos, types, ka_params(), L, i)
            assert np.all(np.abs(fi) < 1e-12 * eps / sig)
            assert vh == pytest.approx(0.5 * (-eps - vc), rel=1e-13)
    pos = np.array([[5.0, 3.0, 4.0], [5.0, 3.0 + 2.5 * sig * (1 + 1e-9), 4.0]])
    fi, vh = oracle.force_on(pos, types, ka_params(), L, 0)
    assert np.all(fi == 0.0) and vh == 0.0
    # inside the cutoff but off the minimum: F on i points along r_i - r_j with Eq. (KAFix)'s sign
    pos = np.array([[5.0, 3.0, 4.0], [5.0 + 1.3 * sig, 3.0, 4.0]])
    fi, _ = oracle.force_on(pos, types, ka_params(), L, 0)
    r = 1.3 * sig
    fmag = 48 * eps * (sig ** 12 / r ** 13 - 0.5 * sig ** 6 / r ** 7)
    assert fi[0] == pytest.approx(-fmag, rel=1e-13) and fi[1] == 0.0 and fi[2] == 0.0


def test_perfect_lattice_zero_force_and_lattice_sum():
    """A perfect simple-cubic A lattice: F_i = 0 by symmetry; V/N = half the lattice sum over shells."""
    m = 8
    rho = 1.2
    L = (m ** 3 / rho) ** (1 / 3)
    a = L / m
    k = np.arange(m)
    gx, gy, gz = np.meshgrid(k, k, k, indexing="ij")
    pos = (np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1) + 0.5) * a
    types = np.zeros(m ** 3, dtype=np.int32)
    f, v, w = oracle.forces(pos, types, ka_params(), L)
    assert np.max(np.abs(f)) < 1e-11
    # brute-force lattice sum: all integer vectors with |n| a < 2.5 (one image each, L/2 > 2.5)
    rng = np.arange(-3, 4)
    vsum = 0.0
    vc = 4.0 * (2.5 ** -12 - 2.5 ** -6)
    for nx in rng:
        for ny in rng:
            for nz in rng:
                if nx == ny == nz == 0:
                    continue
                r = a * np.sqrt(nx * nx + ny * ny + nz * nz)
                if r < 2.5:
                    vsum += 4.0 * (r ** -12 - r ** -6) - vc
    assert v / m ** 3 == pytest.approx(0.5 * vsum, rel=1e-12)


# -------------------------------------------------------------- integrator

def test_two_body_matches_rk4_and_is_second_order():
    """Two bound particles (no cutoff crossing): velocity Verlet converges to an RK4
    reference with dt/100 at second order (error ratio ~4 per halving of dt)."""
    L = 20.0
    types = np.array([0, 1], dtype=np.int32)
    p0 = np.array([[5.0, 5.0, 5.0], [5.95, 5.1, 5.0]])
    v0 = np.array([[0.1, 0.3, 0.0], [-0.1, -0.3, 0.05]])
    T_end = 0.8

    def acc(p):
        return oracle.forces(p, types, ka_params(), L)[0]

    def rk4(p, v, h, n):
        for _ in range(n):
            k1p, k1v = v, acc(p)
            k2p, k2v = v + 0.5 * h * k1v, acc(p + 0.5 * h * k1p)
            k3p, k3v = v + 0.5 * h * k2v, acc(p + 0.5 * h * k2p)
            k4p, k4v = v + h * k3v, acc(p + h * k3p)
            p = p + h / 6 * (k1p + 2 * k2p + 2 * k3p + k4p)
            v = v + h / 6 * (k1v + 2 * k2v + 2 * k3v + k4v)
        return p, v

    pr, vr = rk4(p0.copy(), v0.copy(), 0.005 / 100, int(round(T_end / (0.005 / 100))))
    errs = []
    for dt in (0.01, 0.005, 0.0025):
        out = oracle.run(p0, v0, types, ka_params(), L, dt, int(round(T_end / dt)), log_every=0)
        errs.append(np.max(np.abs(out["pos"] - pr)))
    assert errs[0] < 1e-3
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7


def test_energy_error_scales_as_dt_squared():
    """NVE energy fluctuation amplitude of a bound 3-particle cluster scales as dt^2."""
    L = 20.0
    types = np.array([0, 0, 1], dtype=np.int32)
    p0 = np.array([[5.0, 5.0, 5.0], [6.1, 5.05, 5.0], [5.5, 5.9, 5.1]])
    v0 = np.array([[0.2, -0.1, 0.05], [-0.1, 0.25, 0.0], [-0.1, -0.15, -0.05]])
    amps = []
    for dt in (0.004, 0.002, 0.001):
        nst = int(round(2.0 / dt))
        out = oracle.run(p0, v0, types, ka_params(), L, dt, nst, log_every=1)
        e = out["thermo"][:, 4] * 3
        f0, pe0, _ = oracle.forces(p0, types, ka_params(), L)
        e0 = pe0 + 0.5 * np.sum(v0 * v0)
        amps.append(np.max(np.abs(e - e0)))
    assert 3.5 < amps[0] / amps[1] < 4.5 and 3.5 < amps[1] / amps[2] < 4.5


def test_time_reversibility_and_momentum():
    """n steps forward, reverse velocities, n steps: back to the start; momentum stays zero."""
    pos, vel, types, L = melted(256, 13, nsteps=0)
    out = oracle.run(pos, vel, types, ka_params(), L, 0.005, 100, log_every=0)
    assert np.all(np.abs(out["vel"].sum(axis=0)) < 1e-10)
    back = oracle.run(out["pos"], -out["vel"], types, ka_params(), L, 0.005, 100, log_every=0,
                      forces_in=out["forces"])
    d = back["pos"] - pos
    d -= L * np.rint(d / L)
    assert np.max(np.abs(d)) < 1e-8
    assert np.max(np.abs(back["vel"] + vel)) < 1e-8


def test_nve_energy_conserved_on_melt():
    """1000 NVE steps of a melted N=256 KA liquid: |E(t) - E(0)|/N stays small and bounded."""
    pos, vel, types, L = melted(256, 14, nsteps=100)
    out = oracle.run(pos, vel, types, ka_params(), L, 0.005, 1000, log_every=10)
    e = out["thermo"][:, 4]
    assert np.max(np.abs(e - e[0])) < 5e-3
    assert np.ptp(e) < 5e-3


# --------------------------------------------------------------- thermostats

def test_maxwell_boltzmann_exact_temperature_zero_momentum():
    n, T = 4000, 0.73
    v = oracle.maxwell_boltzmann(n, T, seed=5, draw=3)
    assert np.all(np.abs(v.sum(axis=0)) < 1e-10)
    assert np.sum(v * v) / (3 * n) == pytest.approx(T, rel=1e-13)
    # Gaussian shape: kurtosis of components near 3
    z = v.ravel() / np.sqrt(T)
    assert abs(np.mean(z ** 4) / np.mean(z ** 2) ** 2 - 3.0) < 0.15


def test_box_muller_normals_statistics():
    g = np.array([oracle.gauss3(77, 0, p) for p in range(20000)]).ravel()
    assert abs(g.mean()) < 4 / np.sqrt(g.size)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2 / g.size)
    assert abs(np.mean(np.abs(g) < 1.0) - 0.682689492) < 0.01


def test_resample_bath_sets_exact_temperature():
    """After each resampling step T equals the bath temperature and the momentum is zero."""
    pos, vel, types, L = melted(256, 15, nsteps=50)
    out = oracle.run(pos, vel, types, ka_params(), L, 0.005, 40, kind=oracle.RESAMPLE, T_target=0.4,
                     nstep_boltz=10, seed=9, log_every=1)
    th = out["thermo"]
    for rec in th:
        if int(rec[0]) % 10 == 0:
            assert rec[1] == pytest.approx(0.4, rel=1e-13)
        else:
            assert abs(rec[1] - 0.4) > 1e-6
    assert np.all(np.abs(out["vel"].sum(axis=0)) < 1e-10)


@pytest.mark.parametrize("kind", [oracle.NOSE_HOOVER, oracle.NOSE_HOOVER_EXACT])
def test_nose_hoover_conserves_extended_hamiltonian(kind):
    """Eq. (HNosetilde) is a constant of the Fox-Andersen Nose-Hoover dynamics; its drift is
    far below the drift of the physical energy, which the bath changes on purpose."""
    pos, vel, types, L = melted(256, 16, nsteps=100)
    T = 0.8
    n = len(pos)
    Q = 3 * n * T * 0.5 ** 2
    out = oracle.run(pos, vel, types, ka_params(), L, 0.0025, 2000, kind=kind, T_target=T, Q=Q,
                     log_every=10)
    th = out["thermo"]
    h = th[:, 6] / n
    e = th[:, 4]
    assert np.ptp(e) > 0.05
    assert np.ptp(h) < 2e-3 * np.ptp(e) + 2e-4


def test_nose_hoover_infinite_mass_reduces_to_nve():
    """Q -> infinity freezes xi at 0: the Nose-Hoover path reproduces plain NVE."""
    pos, vel, types, L = melted(256, 17, nsteps=20)
    nve = oracle.run(pos, vel, types, ka_params(), L, 0.005, 50, log_every=0)
    nh = oracle.run(pos, vel, types, ka_params(), L, 0.005, 50, kind=oracle.NOSE_HOOVER, T_target=1.0,
                    Q=1e30, log_every=0)
    d = nh["pos"] - nve["pos"]
    d -= L * np.rint(d / L)
    assert np.max(np.abs(d)) < 1e-9
    assert np.max(np.abs(nh["vel"] - nve["vel"])) < 1e-9


def test_nose_hoover_reaches_target_temperature():
    pos, vel, types, L = melted(256, 18, nsteps=0, T0=2.0)
    T = 0.8
    n = len(pos)
    Q = 3 * n * T * 0.5 ** 2
    out = oracle.run(pos, vel, types, ka_params(), L, 0.005, 6000, kind=oracle.NOSE_HOOVER, T_target=T,
                     Q=Q, log_every=10)
    Tm = out["thermo"][300:, 1]
    assert abs(Tm.mean() - T) < 0.06


# --------------------------------------------------------------- init

def test_lattice_start_sites_and_jitter():
    n = 1000
    L = wl.box_length(n)
    pos0, vel0 = oracle.init_lattice(n, L, 2.0, seed=3, jitter=0.0)
    a = L / 10
    k = np.rint(pos0 / a - 0.5)
    assert np.allclose(pos0, (k + 0.5) * a, atol=1e-12)
    assert len({tuple(r) for r in k.astype(int)}) == n
    pos, vel = oracle.init_lattice(n, L, 2.0, seed=3, jitter=0.05)
    d = pos - pos0
    d -= L * np.rint(d / L)
    assert np.max(np.abs(d)) <= 0.05 + 1e-12 and np.max(np.abs(d)) > 0.045
    assert np.allclose(vel, vel0)
    assert np.sum(vel * vel) / (3 * n) == pytest.approx(2.0, rel=1e-13)


def test_lattice_start_partial_fill_spreads_sites():
    n = 32000
    L = wl.box_length(n)
    pos, _ = oracle.init_lattice(n, L, 1.0, seed=4, jitter=0.0)
    a = L / 32
    k = np.rint(pos / a - 0.5).astype(int)
    assert len({tuple(r) for r in k}) == n
    assert k.min() == 0 and k.max() == 31


# ---------------------------------------------------------------- analysis

def test_rdf_ideal_gas_is_one():
    n, L = 3000, 14.0
    pos = wl.uniform_positions(n, L, 8)
    types = wl.ka_types(n, 8).astype(np.int32)
    g = oracle.rdf(pos, types, L, 0.25, 24)
    for row in g:
        assert abs(row[4:].mean() - 1.0) < 0.05


def test_rdf_two_particles_brute_force():
    """One AB pair at r = 1.234: a single bin holds exactly V/(N_A N_B shell)."""
    L, dr = 10.0, 0.1
    pos = np.array([[1.0, 1.0, 1.0], [1.0 + 1.234, 1.0, 1.0]])
    g = oracle.rdf(pos, np.array([0, 1]), L, dr, 40)
    k = 12
    shell = 4 / 3 * np.pi * ((k + 1) ** 3 - k ** 3) * dr ** 3
    assert g[2, k] == pytest.approx(L ** 3 / shell, rel=1e-13)
    assert np.count_nonzero(g[2]) == 1 and not g[0].any() and not g[1].any()


def test_msd_free_flight_and_unwrapping():
    """Non-interacting particles (all pair distances > r_c) fly freely: the MSD from
    unwrapped coordinates equals <v^2> t^2 even across the periodic boundary."""
    L = 40.0
    pos = np.array([[1.0, 1.0, 1.0], [15.0, 15.0, 15.0], [30.0, 5.0, 20.0], [10.0, 32.0, 36.0]])
    vel = np.array([[-2.0, 0.5, 0.0], [1.0, 1.0, -1.0], [0.0, 0.0, 3.0], [0.5, -1.5, 2.0]])
    types = np.array([0, 0, 1, 1], dtype=np.int32)
    out = oracle.run(pos, vel, types, ka_params(), L, 0.01, 200, log_every=0)
    t = 2.0
    msd = oracle.msd(out["pos"], out["img"], pos, types, 2, L)
    v2 = np.sum(vel * vel, axis=1)
    assert msd[0] == pytest.approx(v2[:2].mean() * t * t, rel=1e-12)
    assert msd[1] == pytest.approx(v2[2:].mean() * t * t, rel=1e-12)
    assert out["img"][0, 0] == -1 and out["img"][2, 2] == 0 and out["img"][3, 2] == 1
    still = oracle.msd(pos, np.zeros((4, 3), np.int32), pos, types, 2, L)
    assert np.all(still == 0.0)


def test_waiting_time_msd_free_flight():
    """Eq. (msdtw): with the reference taken at t_w (unwrapped positions then), free flight gives
    <v^2> t^2 for every t_w, also when particles cross the boundary before or after t_w; t_w = 0
    is Eq. (msd)."""
    L = 40.0
    pos = np.array([[1.0, 1.0, 1.0], [15.0, 15.0, 15.0], [30.0, 5.0, 20.0], [10.0, 32.0, 36.0]])
    vel = np.array([[-2.0, 0.5, 0.0], [1.0, 1.0, -1.0], [0.0, 0.0, 3.0], [0.5, -1.5, 2.0]])
    types = np.array([0, 0, 1, 1], dtype=np.int32)
    v2 = np.sum(vel * vel, axis=1)
    dt = 0.01
    for tw in (0, 50, 120):
        a = oracle.run(pos, vel, types, ka_params(), L, dt, tw, log_every=0) if tw else {
            "pos": pos, "vel": vel, "img": np.zeros((4, 3), np.int32)}
        ref = a["pos"] + L * a["img"]
        b = oracle.run(a["pos"], a["vel"], types, ka_params(), L, dt, 100, img=a["img"], log_every=0)
        msd = oracle.msd(b["pos"], b["img"], ref, types, 2, L)
        t = 100 * dt
        assert msd[0] == pytest.approx(v2[:2].mean() * t * t, rel=1e-12)
        assert msd[1] == pytest.approx(v2[2:].mean() * t * t, rel=1e-12)


# ------------------------------------------------------------- threaded sum

def test_threaded_force_sum_reproducible_and_equal_to_serial():
    """The threaded all-pairs sum (per-thread force arrays added in thread order): one thread is the
    serial oracle bitwise; a fixed thread count gives bitwise identical results on every call; any
    thread count agrees with the serial sum to rounding; a run with threads follows the serial run."""
    pos, vel, types, L = melted(1000, 35, nsteps=50)
    f, v, w = oracle.forces(pos, types, ka_params(), L)
    f1, v1, w1 = oracle.forces_threads(pos, types, ka_params(), L, 1)
    assert np.array_equal(f, f1) and v == v1 and w == w1
    frms = np.sqrt(np.mean(np.sum(f * f, axis=1)))
    for nt in (2, 3, 8):
        fa, va, wa = oracle.forces_threads(pos, types, ka_params(), L, nt)
        fb, vb, wb = oracle.forces_threads(pos, types, ka_params(), L, nt)
        assert np.array_equal(fa, fb) and va == vb and wa == wb
        assert np.max(np.abs(fa - f)) < 1e-13 * frms
        assert abs(va - v) < 1e-13 * abs(v) and abs(wa - w) < 1e-13 * abs(w)
    serial = oracle.run(pos, vel, types, ka_params(), L, 0.005, 20, log_every=1)
    try:
        oracle.set_threads(4)
        par = oracle.run(pos, vel, types, ka_params(), L, 0.005, 20, log_every=1)
        oracle.set_threads(1)
        again = oracle.run(pos, vel, types, ka_params(), L, 0.005, 20, log_every=1)
    finally:
        oracle.set_threads(1)
    scale = np.maximum(np.abs(serial["thermo"]), 1.0)
    assert np.max(np.abs(par["thermo"] - serial["thermo"]) / scale) < 1e-12
    assert np.array_equal(again["thermo"], serial["thermo"])


# ------------------------------------------------------------- two dimensions
# The 2-D Kob-Andersen problem of Sec. "Suggested problems": N = 1000 in a
# square box at N/L^2 = 1.204 (L = 28.82), A:B = 65:35, 2 instead of 3 in
# Eq. (equip3N), and the shell volume of g(r) adjusted to two dimensions.

def test_2d_maxwell_boltzmann_exact_temperature_in_plane():
    n, T = 1000, 0.4
    v = oracle.maxwell_boltzmann(n, T, seed=5, draw=0, ndim=2)
    assert np.all(v[:, 2] == 0.0)
    assert np.all(np.abs(v.sum(axis=0)) < 1e-12)
    assert np.sum(v * v) / (2 * n) == pytest.approx(T, rel=1e-13)
    # x and y are the three-dimensional draws (same Philox stream), recentred and rescaled
    v3 = np.array([oracle.gauss3(5, 0, p) for p in range(n)])[:, :2]
    v3 -= v3.mean(axis=0)
    v3 *= np.sqrt(2 * n * T / np.sum(v3 * v3))
    assert np.allclose(v[:, :2], v3, rtol=1e-12, atol=1e-14)


def test_2d_lattice_start_square_sites_in_one_plane():
    n, L = 1000, wl.box_length_2d(1000)
    assert L == pytest.approx(28.82, abs=5e-3)
    pos, vel = oracle.init_lattice(n, L, 0.4, seed=3, jitter=0.0, ndim=2)
    assert np.all(pos[:, 2] == 0.5 * L)
    a = L / 32
    k = np.rint(pos[:, :2] / a - 0.5).astype(int)
    assert len({tuple(r) for r in k}) == n and k.min() == 0 and k.max() == 31
    assert np.allclose(pos[:, :2], (k + 0.5) * a, atol=1e-12)
    assert np.sum(vel * vel) / (2 * n) == pytest.approx(0.4, rel=1e-13)


def test_2d_square_lattice_zero_force_and_lattice_sum():
    """A perfect square A lattice at density 1.204: F_i = 0 by symmetry, F_z = 0, and V/N is half
    the brute-force sum over the 2-D integer vectors inside the cutoff."""
    m = 16
    L = np.sqrt(m * m / 1.204)
    a = L / m
    k = np.arange(m)
    gx, gy = np.meshgrid(k, k, indexing="ij")
    pos = np.stack([(gx.ravel() + 0.5) * a, (gy.ravel() + 0.5) * a, np.full(m * m, 0.5 * L)], axis=1)
    types = np.zeros(m * m, dtype=np.int32)
    f, v, w = oracle.forces(pos, types, ka_params(), L)
    assert np.max(np.abs(f)) < 1e-11
    vc = 4.0 * (2.5 ** -12 - 2.5 ** -6)
    vsum = 0.0
    for nx in range(-3, 4):
        for ny in range(-3, 4):
            if nx == ny == 0:
                continue
            r = a * np.hypot(nx, ny)
            if r < 2.5:
                vsum += 4.0 * (r ** -12 - r ** -6) - vc
    assert v / (m * m) == pytest.approx(0.5 * vsum, rel=1e-12)


def test_2d_ideal_gas_rdf_is_one_with_shell_areas():
    n, L = 4000, 40.0
    rng = np.random.default_rng(11)
    pos = np.zeros((n, 3))
    pos[:, :2] = rng.uniform(0, L, size=(n, 2))
    pos[:, 2] = 0.5 * L
    types = wl.ka_types(n, 11, frac_b=0.35).astype(np.int32)
    g = oracle.rdf(pos, types, L, 0.5, 30, ndim=2)
    for row in g:
        assert abs(row[6:].mean() - 1.0) < 0.05
    # the 3-D normalisation is not flat for a planar gas (it falls off like L / r)
    g3 = oracle.rdf(pos, types, L, 0.5, 30, ndim=3)
    assert g3[0, 6] > 1.8 * g3[0, 29] > 1.8


def test_2d_nve_stays_in_plane_and_conserves_energy():
    """2-D NVE from the melted square lattice: z and v_z stay exactly fixed, momentum stays zero,
    the energy is conserved, and T = sum m v^2 / (2N)."""
    n = 256
    L = wl.box_length_2d(n)
    types = wl.ka_types(n, 14, frac_b=0.35).astype(np.int32)
    pos, vel = oracle.init_lattice(n, L, 1.0, seed=14, ndim=2)
    melt = oracle.run(pos, vel, types, ka_params(), L, 0.005, 200, kind=oracle.RESAMPLE, T_target=1.0,
                      nstep_boltz=10, seed=14, log_every=0, ndim=2)
    out = oracle.run(melt["pos"], melt["vel"], types, ka_params(), L, 0.005, 1000, log_every=10, ndim=2)
    assert np.all(out["pos"][:, 2] == 0.5 * L) and np.all(out["vel"][:, 2] == 0.0)
    assert np.all(np.abs(out["vel"].sum(axis=0)) < 1e-10)
    e = out["thermo"][:, 4]
    assert np.ptp(e) < 5e-3
    th = out["thermo"][-1]
    assert th[1] == pytest.approx(np.sum(out["vel"] ** 2) / (2 * n), rel=1e-12)
    # the resampling bath sets T exactly with 2N degrees of freedom
    assert abs(np.sum(melt["vel"] ** 2) / (2 * n) - 1.0) < 1e-12


def test_2d_nose_hoover_reaches_target_with_2n_degrees_of_freedom():
    n = 256
    L = wl.box_length_2d(n)
    types = wl.ka_types(n, 15, frac_b=0.35).astype(np.int32)
    pos, vel = oracle.init_lattice(n, L, 1.0, seed=15, ndim=2)
    T = 0.45
    out = oracle.run(pos, vel, types, ka_params(), L, 0.005, 6000, kind=oracle.NOSE_HOOVER, T_target=T,
                     Q=2 * n * T * 0.5 ** 2, log_every=10, ndim=2)
    assert abs(out["thermo"][300:, 1].mean() - T) < 0.04
    h = out["thermo"][:, 6] / n
    assert np.ptp(h[100:]) < 0.05 * np.ptp(out["thermo"][:, 4])
