/*
 * ka_oracle.c -- plain, slow FP64 reference for the Kob-Andersen binary
 * Lennard-Jones MD method (test infrastructure only).
 *
 * This file is the ORACLE. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table
 * or helper with the CUDA library; neither side includes or links the other.
 *
 * Everything is the textbook definition, written in the paper's order:
 *   - pair potential and force: Eq. (VKALJ), Eq. (VshiftedKALJ), Eq. (KAFix)
 *     (Sec. "Model");
 *   - all-pairs half loop j > i with Newton's third law (Sec. "Accelerations");
 *   - minimum image by the branch rule of Sec. "Periodic boundary conditions"
 *     and its Python form in Sec. "Accelerations";
 *   - velocity Verlet, Eqs. (velVerletPos)/(velVerletVel), in the update order
 *     of Sec. "NVE molecular dynamics simulation" (wrap into (0, L]);
 *   - Maxwell-Boltzmann velocities with centre-of-mass removal and an exact
 *     rescale (Sec. "Statistical temperature bath", Eqs. (vxocitydistribution),
 *     (sigmavx), (equip3N); Sec. "Initialization of velocities");
 *   - the stochastic bath: resample after every nstepBoltz-th step
 *     (Sec. "NVT molecular dynamics simulation");
 *   - Nose-Hoover integrated by Fox-Andersen, Eqs. (Noseupdate_ri),
 *     (Noseupdate_lns), (Noseupdate_xiapprox), (ridotKVLRoman) or
 *     (ridotsolved), and (FoxAndersen_ydottplush); conserved quantity
 *     Eq. (HNosetilde) (Appendices A and B);
 *   - simple-cubic lattice start (Sec. "Initialization of positions");
 *   - partial g(r), Eqs. (gAA)/(gAB), and the MSD, Eqs. (msd)/(msdwithi).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel
 * random numbers: as easy as 1, 2, 3") written here from its published
 * definition, and the Box-Muller transform (Box & Muller 1958).
 *
 * Layouts: positions, velocities and forces are AoS xyz, n*3 doubles.
 * Types are int32 in [0, ntypes). Tables eps, sig, rc are ntypes*ntypes,
 * row-major, symmetric; rc holds absolute cutoff radii.
 * Every function returns 0 on success and a negative code on a bad argument.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds (SC'11, Sec. 3 and Table 2): the round multipliers
 * and Weyl key increments are the constants published there. */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A uniform double in (0, 1) from two 32-bit words: the top 53 bits,
 * offset by half a step so that 0 and 1 never occur. */
static double ora_u01(uint32_t a, uint32_t b)
{
    uint64_t m = ((uint64_t)a << 21) ^ (uint64_t)(b >> 11);
    m &= ((uint64_t)1 << 53) - 1;
    return ((double)m + 0.5) * (1.0 / 9007199254740992.0);
}

/* Stream tags of the counter-based draws (counter word 2 carries the tag
 * and the block index within a particle). */
enum { ORA_TAG_JITTER = 1, ORA_TAG_GAUSS = 2 };

/* Three standard normals for particle p (its index in the caller's order),
 * draw number d, key = seed: two Philox blocks, Box-Muller on each pair. */
static void ora_gauss3(uint64_t seed, uint64_t d, uint32_t p, double g[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    double z[4];
    for (uint32_t blk = 0; blk < 2; ++blk) {
        uint32_t ctr[4] = {p, (uint32_t)d, (ORA_TAG_GAUSS << 16) | blk, (uint32_t)(d >> 32)};
        ora_philox4x32_10(ctr, key, out);
        double u1 = ora_u01(out[0], out[1]);
        double u2 = ora_u01(out[2], out[3]);
        double rad = sqrt(-2.0 * log(u1));
        double ang = 2.0 * M_PI * u2;
        z[2 * blk] = rad * cos(ang);
        z[2 * blk + 1] = rad * sin(ang);
    }
    g[0] = z[0]; g[1] = z[1]; g[2] = z[2];
}

/* Three uniforms in (-1, 1) for the lattice jitter of particle p. */
static void ora_jitter3(uint64_t seed, uint32_t p, double u[3])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4], out2[4];
    uint32_t ctr[4] = {p, 0u, (ORA_TAG_JITTER << 16) | 0u, 0u};
    uint32_t ctr2[4] = {p, 0u, (ORA_TAG_JITTER << 16) | 1u, 0u};
    ora_philox4x32_10(ctr, key, out);
    ora_philox4x32_10(ctr2, key, out2);
    u[0] = 2.0 * ora_u01(out[0], out[1]) - 1.0;
    u[1] = 2.0 * ora_u01(out[2], out[3]) - 1.0;
    u[2] = 2.0 * ora_u01(out2[0], out2[1]) - 1.0;
}

/* Exposed for the tests: the standard normals and jitter uniforms above. */
void ora_draw_gauss3(uint64_t seed, uint64_t d, uint32_t p, double g[3]) { ora_gauss3(seed, d, p, g); }
void ora_draw_jitter3(uint64_t seed, uint32_t p, double u[3]) { ora_jitter3(seed, p, u); }

/* ------------------------------------------------------------ pair terms */

/* Minimum image by the branch rule of Sec. "Periodic boundary conditions":
 * if d > L/2 subtract L, else if d < -L/2 add L. Positions lie in the box,
 * so |d| < L and one branch suffices. */
static double ora_min_image(double d, double L)
{
    double half = 0.5 * L;
    if (d > half) d -= L;
    else if (d < -half) d += L;
    return d;
}

/* Eq. (VKALJ): the unshifted pair potential at squared distance r2. */
static double ora_v_lj(double eps, double sig, double r2)
{
    double s2 = sig * sig / r2;
    double s6 = s2 * s2 * s2;
    return 4.0 * eps * (s6 * s6 - s6);
}

/* Eq. (KAFix) without the leading 48: eps*(sig^12/r^14 - 0.5*sig^6/r^8),
 * the scalar that multiplies (x_i - x_j). */
static double ora_f_over_r(double eps, double sig, double r2)
{
    double inv2 = 1.0 / r2;
    double sig6 = pow(sig, 6.0);
    double sig12 = sig6 * sig6;
    double inv8 = inv2 * inv2 * inv2 * inv2;
    double inv14 = inv8 * inv2 * inv2 * inv2;
    return eps * (sig12 * inv14 - 0.5 * sig6 * inv8);
}

/* Pair energy (Eq. (VshiftedKALJ)) and the scalar 48*eps*(...) of
 * Eq. (KAFix) for one pair at squared distance r2 (inside the cutoff). */
static void ora_pair(int a, int b, int ntypes, const double *eps, const double *sig,
                     const double *rc, double r2, double *v, double *fscal)
{
    int t = a * ntypes + b;
    double vcut = ora_v_lj(eps[t], sig[t], rc[t] * rc[t]);
    *v = ora_v_lj(eps[t], sig[t], r2) - vcut;
    *fscal = 48.0 * ora_f_over_r(eps[t], sig[t], r2);
}

static int ora_check_tables(int ntypes, const double *eps, const double *sig, const double *rc, double L)
{
    if (ntypes < 1 || ntypes > 8) return -1;
    for (int a = 0; a < ntypes; ++a)
        for (int b = 0; b < ntypes; ++b) {
            int t = a * ntypes + b, u = b * ntypes + a;
            if (!(eps[t] > 0.0) || !(sig[t] > 0.0) || !(rc[t] > 0.0)) return -2;
            if (eps[t] != eps[u] || sig[t] != sig[u] || rc[t] != rc[u]) return -3;
            if (!(rc[t] < 0.5 * L)) return -4; /* minimum image must be unique */
        }
    return 0;
}

/* ---------------------------------------------------------------- forces */

/* All-pairs forces, potential energy (Eq. (Vij) with the shifted pair term)
 * and virial W = sum_{i<j} r_ij . F_ij. Half loop j > i; each pair adds to i
 * and subtracts from j (Sec. "Accelerations"). Cutoff test is strict: r < rc. */
int ora_forces(int64_t n, const double *pos, const int32_t *types, int ntypes,
               const double *eps, const double *sig, const double *rc, double L,
               double *f, double *pe, double *virial)
{
    if (n < 0 || !pos || !types || !f) return -1;
    int e = ora_check_tables(ntypes, eps, sig, rc, L);
    if (e) return e;
    for (int64_t i = 0; i < 3 * n; ++i) f[i] = 0.0;
    double V = 0.0, W = 0.0;
    for (int64_t i = 0; i + 1 < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = ora_min_image(pos[3 * i + 0] - pos[3 * j + 0], L);
            double dy = ora_min_image(pos[3 * i + 1] - pos[3 * j + 1], L);
            double dz = ora_min_image(pos[3 * i + 2] - pos[3 * j + 2], L);
            double r2 = dx * dx + dy * dy + dz * dz;
            int t = types[i] * ntypes + types[j];
            if (r2 < rc[t] * rc[t]) {
                double v, fs;
                ora_pair(types[i], types[j], ntypes, eps, sig, rc, r2, &v, &fs);
                V += v;
                W += fs * r2;
                f[3 * i + 0] += fs * dx; f[3 * j + 0] -= fs * dx;
                f[3 * i + 1] += fs * dy; f[3 * j + 1] -= fs * dy;
                f[3 * i + 2] += fs * dz; f[3 * j + 2] -= fs * dz;
            }
        }
    }
    if (pe) *pe = V;
    if (virial) *virial = W;
    return 0;
}

/* The same all-pairs sum spread over nthreads host threads (OpenMP): thread
 * t takes the rows i = t, t + nthreads, ... of the half loop and adds its
 * pair terms to a force array of its own; the arrays, energies and virials
 * are then added in thread order 0, 1, ..., so the result is the same on
 * every run with the same thread count. With one thread every sum is formed
 * in the order of ora_forces, bitwise. Without OpenMP the pragmas are
 * ignored and the loop runs on one thread (the result for nthreads > 1 is
 * then the one-thread result). */
int ora_forces_threads(int64_t n, const double *pos, const int32_t *types, int ntypes,
                       const double *eps, const double *sig, const double *rc, double L,
                       double *f, double *pe, double *virial, int nthreads)
{
    if (n < 0 || !pos || !types || !f || nthreads < 1) return -1;
    int e = ora_check_tables(ntypes, eps, sig, rc, L);
    if (e) return e;
#ifndef _OPENMP
    nthreads = 1;
#endif
    double *ft = (double *)calloc((size_t)nthreads * 3 * (size_t)n + 1, sizeof(double));
    double *vt = (double *)calloc((size_t)nthreads * 2, sizeof(double));
    if (!ft || !vt) { free(ft); free(vt); return -5; }
#pragma omp parallel num_threads(nthreads)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *fl = ft + (size_t)t * 3 * (size_t)n;
        double V = 0.0, W = 0.0;
        for (int64_t i = t; i + 1 < n; i += nthreads) {
            for (int64_t j = i + 1; j < n; ++j) {
                double dx = ora_min_image(pos[3 * i + 0] - pos[3 * j + 0], L);
                double dy = ora_min_image(pos[3 * i + 1] - pos[3 * j + 1], L);
                double dz = ora_min_image(pos[3 * i + 2] - pos[3 * j + 2], L);
                double r2 = dx * dx + dy * dy + dz * dz;
                int tt = types[i] * ntypes + types[j];
                if (r2 < rc[tt] * rc[tt]) {
                    double v, fs;
                    ora_pair(types[i], types[j], ntypes, eps, sig, rc, r2, &v, &fs);
                    V += v;
                    W += fs * r2;
                    fl[3 * i + 0] += fs * dx; fl[3 * j + 0] -= fs * dx;
                    fl[3 * i + 1] += fs * dy; fl[3 * j + 1] -= fs * dy;
                    fl[3 * i + 2] += fs * dz; fl[3 * j + 2] -= fs * dz;
                }
            }
        }
        vt[2 * t] = V;
        vt[2 * t + 1] = W;
    }
    double V = 0.0, W = 0.0;
    for (int64_t k = 0; k < 3 * n; ++k) {
        double s = 0.0;
        for (int t = 0; t < nthreads; ++t) s += ft[(size_t)t * 3 * (size_t)n + (size_t)k];
        f[k] = s;
    }
    for (int t = 0; t < nthreads; ++t) { V += vt[2 * t]; W += vt[2 * t + 1]; }
    free(ft);
    free(vt);
    if (pe) *pe = V;
    if (virial) *virial = W;
    return 0;
}

/* Host threads used by the force sums of ora_run (1: ora_forces itself). */
static int ora_run_threads = 1;
int ora_set_threads(int nthreads)
{
    if (nthreads < 1) return -1;
    ora_run_threads = nthreads;
    return 0;
}
int ora_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Forces of ora_run: the single-thread oracle, or its threaded form. */
static int ora_run_forces(int64_t n, const double *pos, const int32_t *types, int ntypes,
                          const double *eps, const double *sig, const double *rc, double L,
                          double *f, double *pe, double *virial)
{
    if (ora_run_threads <= 1) return ora_forces(n, pos, types, ntypes, eps, sig, rc, L, f, pe, virial);
    return ora_forces_threads(n, pos, types, ntypes, eps, sig, rc, L, f, pe, virial, ora_run_threads);
}

/* Force on one particle i from all j != i (Eq. (KAFix) summed over every
 * other particle), plus its half share of the pair energies. O(n) per call:
 * used to check sampled particles of systems too large for ora_forces. */
int ora_force_on(int64_t n, int64_t i, const double *pos, const int32_t *types, int ntypes,
                 const double *eps, const double *sig, const double *rc, double L,
                 double *f3, double *pe_half)
{
    if (n < 1 || i < 0 || i >= n || !f3) return -1;
    int e = ora_check_tables(ntypes, eps, sig, rc, L);
    if (e) return e;
    double fx = 0, fy = 0, fz = 0, V = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double dx = ora_min_image(pos[3 * i + 0] - pos[3 * j + 0], L);
        double dy = ora_min_image(pos[3 * i + 1] - pos[3 * j + 1], L);
        double dz = ora_min_image(pos[3 * i + 2] - pos[3 * j + 2], L);
        double r2 = dx * dx + dy * dy + dz * dz;
        int t = types[i] * ntypes + types[j];
        if (r2 < rc[t] * rc[t]) {
            double v, fs;
            ora_pair(types[i], types[j], ntypes, eps, sig, rc, r2, &v, &fs);
            V += 0.5 * v;
            fx += fs * dx; fy += fs * dy; fz += fs * dz;
        }
    }
    f3[0] = fx; f3[1] = fy; f3[2] = fz;
    if (pe_half) *pe_half = V;
    return 0;
}

/* ------------------------------------------------------------ velocities */

/* Maxwell-Boltzmann velocities at temperature T (k_B = 1, mass m) for the
 * particles [0, n) in ndim = 3 or 2 dimensions: step 1 draw each component
 * from a Gaussian of standard deviation sqrt(T/m) (Eqs. (vxocitydistribution),
 * (sigmavx)); in two dimensions v_z = 0 (the z draw is discarded, so x and y
 * are the draws of the three-dimensional case); step 3 subtract the mean
 * velocity; step 4 rescale so that sum m v^2 = ndim n T (Eq. (equip3N) with
 * ndim N degrees of freedom; the 2-D problem of Sec. "Suggested problems"
 * replaces 3 by 2 there). Draw number d selects the random stream (0 at
 * initialisation, k for the k-th resampling). ids gives each particle's index
 * for the counter (NULL: its position in the array). */
int ora_maxwell_boltzmann(int64_t n, int ndim, double T, double mass, uint64_t seed, uint64_t d,
                          const int32_t *ids, double *vel)
{
    if (n < 1 || (ndim != 2 && ndim != 3) || !(T >= 0.0) || !(mass > 0.0) || !vel) return -1;
    double sd = sqrt(T / mass);
    for (int64_t i = 0; i < n; ++i) {
        double g[3];
        ora_gauss3(seed, d, ids ? (uint32_t)ids[i] : (uint32_t)i, g);
        vel[3 * i + 0] = sd * g[0];
        vel[3 * i + 1] = sd * g[1];
        vel[3 * i + 2] = ndim == 3 ? sd * g[2] : 0.0;
    }
    double mx = 0, my = 0, mz = 0;
    for (int64_t i = 0; i < n; ++i) { mx += vel[3 * i]; my += vel[3 * i + 1]; mz += vel[3 * i + 2]; }
    mx /= (double)n; my /= (double)n; mz /= (double)n;
    for (int64_t i = 0; i < n; ++i) { vel[3 * i] -= mx; vel[3 * i + 1] -= my; vel[3 * i + 2] -= mz; }
    double s2 = 0;
    for (int64_t i = 0; i < n; ++i)
        s2 += mass * (vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] + vel[3 * i + 2] * vel[3 * i + 2]);
    double scale = (s2 > 0.0) ? sqrt((double)ndim * (double)n * T / s2) : 0.0;
    for (int64_t i = 0; i < 3 * n; ++i) vel[i] *= scale;
    return 0;
}

/* Simple-cubic lattice start (Sec. "Initialization of positions"):
 * m = ceil(n^(1/3)) sites per edge, site (kx, ky, kz) at ((0.5+k) L/m),
 * kx fastest. When n < m^3, particle p takes site floor(p m^3 / n) (sites
 * spread evenly; for n = m^3 this is the paper's assignment). Each coordinate
 * is then moved by jitter * u with u uniform in (-1, 1) and wrapped into
 * [0, L). Velocities are Maxwell-Boltzmann at T0 (draw number 0).
 * ndim = 2 (the 2-D problem of Sec. "Suggested problems"): the same on a
 * square lattice of m = ceil(n^(1/2)) sites per edge in the plane z = L/2,
 * which no particle leaves (z_i = v_iz = 0 relative to it); no z jitter. */
int ora_init_lattice(int64_t n, int ndim, double L, double T0, double mass, double jitter, uint64_t seed,
                     double *pos, double *vel)
{
    if (n < 1 || (ndim != 2 && ndim != 3) || !(L > 0.0) || !pos || !vel) return -1;
    int64_t m = 1;
    if (ndim == 3) while (m * m * m < n) ++m;
    else while (m * m < n) ++m;
    double a = L / (double)m;
    int64_t sites = ndim == 3 ? m * m * m : m * m;
    for (int64_t p = 0; p < n; ++p) {
        int64_t s = (int64_t)(((__int128)p * sites) / n);
        int64_t kx = s % m, ky = (s / m) % m, kz = s / (m * m);
        double u[3];
        ora_jitter3(seed, (uint32_t)p, u);
        double r[3] = {(0.5 + (double)kx) * a + jitter * u[0],
                       (0.5 + (double)ky) * a + jitter * u[1],
                       ndim == 3 ? (0.5 + (double)kz) * a + jitter * u[2] : 0.5 * L};
        for (int c = 0; c < 3; ++c) {
            double x = r[c];
            if (x >= L) x -= L;
            else if (x < 0.0) x += L;
            pos[3 * p + c] = x;
        }
    }
    return ora_maxwell_boltzmann(n, ndim, T0, mass, seed, 0, NULL, vel);
}

/* ------------------------------------------------------------- dynamics */

typedef struct {
    double step, T, pe_per_n, ke_per_n, etot_per_n, virial, h_nh, xi;
} ora_thermo; /* one log record; step stored as a double for a flat layout */

static double ora_sum_mv2(int64_t n, const double *vel, double mass)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        s += mass * (vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] + vel[3 * i + 2] * vel[3 * i + 2]);
    return s;
}

/* Wrap into (0, L] by the rule of Sec. "NVE molecular dynamics simulation":
 * if x > L subtract L, else if x <= 0 add L (one move per step is < L). The
 * image counter records each crossing so unwrapped coordinates survive. */
static void ora_wrap(double *x, int32_t *img, double L)
{
    if (*x > L) { *x -= L; if (img) ++*img; }
    else if (*x <= 0.0) { *x += L; if (img) --*img; }
}

/* Thermostat kinds for ora_run. */
enum { ORA_NVE = 0, ORA_NOSE_HOOVER = 1, ORA_RESAMPLE = 2, ORA_NOSE_HOOVER_EXACT = 3 };

/*
 * Run nsteps of MD from (pos, vel) at time t; pos, vel, img are updated in
 * place. ndim = 3, or 2 for the 2-D problem of Sec. "Suggested problems"
 * (particles in one plane with v_z = 0, which the dynamics keeps: every pair
 * has dz = 0, so F_z = 0; ndim N degrees of freedom in T, X and the bath). f (n*3) must hold F(x(t)) on entry and holds F at the end.
 *
 *  kind = ORA_NVE: velocity Verlet, order of Sec. "NVE molecular dynamics
 *    simulation": x += v dt + a dt^2/2; wrap; v += a dt/2; a = F(x)/m;
 *    v += a dt/2.
 *  kind = ORA_RESAMPLE: NVE steps, and after every step whose number is a
 *    multiple of nstep_boltz the velocities are redrawn by
 *    ora_maxwell_boltzmann at T_target with draw number step/nstep_boltz
 *    (Sec. "NVT molecular dynamics simulation").
 *  kind = ORA_NOSE_HOOVER(_EXACT): Fox-Andersen update of Appendix B, with
 *    X = ndim n and g = (sum m v^2 - X T)/Q:
 *      x(t+dt)   = x + v dt + (F/m - xi v) dt^2/2          Eq. (Noseupdate_ri)
 *      ln s(t+dt)= ln s + xi dt + g dt^2/2                  Eq. (Noseupdate_lns)
 *      xi_a      = xi + g dt                                Eq. (Noseupdate_xiapprox)
 *      v(t+dt)   = v + (dt/2){(F+F')/m - (xi+xi_a) v}(1 - xi_a dt/2)
 *                                                           Eq. (ridotKVLRoman)
 *        or, EXACT: {v + (dt/2)[F/m - xi v + F'/m]} / (1 + xi_a dt/2)
 *                                                           Eq. (ridotsolved)
 *      xi(t+dt)  = xi + (dt/2)(g + g')                      Eq. (FoxAndersen_ydottplush)
 *    state[0] = xi, state[1] = ln s carry the bath across calls.
 *
 * Steps are numbered step0+1 .. step0+nsteps. Every log_every steps (if
 * log_every > 0) one ora_thermo record is written after the thermostat has
 * acted: T = sum m v^2 / (ndim n), PE/N, KE/N, Etot/N, W, and
 * H = KE + PE + Q xi^2/2 + X T ln s (Eq. (HNosetilde); NVE: H = Etot).
 */
int ora_run(int64_t n, int ndim, double *pos, double *vel, double *f, int32_t *img,
            const int32_t *types, int ntypes, const double *eps, const double *sig, const double *rc,
            double L, double mass, double dt, int64_t step0, int64_t nsteps,
            int kind, double T_target, double Q, int64_t nstep_boltz, uint64_t seed,
            double *state, double *thermo, int64_t log_every)
{
    if (n < 1 || !pos || !vel || !f || !(dt > 0.0) || !(mass > 0.0) || nsteps < 0) return -1;
    if (ndim != 2 && ndim != 3) return -1;
    if (kind < 0 || kind > 3) return -1;
    if ((kind == ORA_NOSE_HOOVER || kind == ORA_NOSE_HOOVER_EXACT) && (!(Q > 0.0) || !state)) return -1;
    if (kind == ORA_RESAMPLE && nstep_boltz < 1) return -1;
    int e = ora_check_tables(ntypes, eps, sig, rc, L);
    if (e) return e;
    const double X = (double)ndim * (double)n;
    double *fn = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!fn) return -5;
    double xi = state ? state[0] : 0.0, lns = state ? state[1] : 0.0;
    double pe = 0.0, W = 0.0;
    int64_t nlog = 0;
    for (int64_t s = 1; s <= nsteps; ++s) {
        int64_t step = step0 + s;
        if (kind == ORA_NOSE_HOOVER || kind == ORA_NOSE_HOOVER_EXACT) {
            double g = (ora_sum_mv2(n, vel, mass) - X * T_target) / Q;
            for (int64_t i = 0; i < n; ++i)
                for (int c = 0; c < 3; ++c) {
                    double x = pos[3 * i + c] + vel[3 * i + c] * dt
                             + 0.5 * (f[3 * i + c] / mass - xi * vel[3 * i + c]) * dt * dt;
                    ora_wrap(&x, img ? &img[3 * i + c] : NULL, L);
                    pos[3 * i + c] = x;
                }
            double lns_new = lns + xi * dt + 0.5 * g * dt * dt;
            double xi_a = xi + dt * g;
            e = ora_run_forces(n, pos, types, ntypes, eps, sig, rc, L, fn, &pe, &W);
            if (e) { free(fn); return e; }
            for (int64_t i = 0; i < n; ++i)
                for (int c = 0; c < 3; ++c) {
                    double v = vel[3 * i + c], F0 = f[3 * i + c], F1 = fn[3 * i + c];
                    double vn;
                    if (kind == ORA_NOSE_HOOVER)
                        vn = v + 0.5 * dt * ((F0 + F1) / mass - (xi + xi_a) * v) * (1.0 - 0.5 * dt * xi_a);
                    else
                        vn = (v + 0.5 * dt * (F0 / mass - xi * v + F1 / mass)) / (1.0 + 0.5 * dt * xi_a);
                    vel[3 * i + c] = vn;
                }
            memcpy(f, fn, sizeof(double) * 3 * (size_t)n);
            double g_new = (ora_sum_mv2(n, vel, mass) - X * T_target) / Q;
            xi = xi + 0.5 * dt * (g + g_new);
            lns = lns_new;
        } else {
            for (int64_t i = 0; i < n; ++i)
                for (int c = 0; c < 3; ++c) {
                    double a = f[3 * i + c] / mass;
                    double x = pos[3 * i + c] + vel[3 * i + c] * dt + 0.5 * a * dt * dt;
                    ora_wrap(&x, img ? &img[3 * i + c] : NULL, L);
                    pos[3 * i + c] = x;
                }
            for (int64_t i = 0; i < 3 * n; ++i) vel[i] += 0.5 * (f[i] / mass) * dt;
            e = ora_run_forces(n, pos, types, ntypes, eps, sig, rc, L, f, &pe, &W);
            if (e) { free(fn); return e; }
            for (int64_t i = 0; i < 3 * n; ++i) vel[i] += 0.5 * (f[i] / mass) * dt;
            if (kind == ORA_RESAMPLE && step % nstep_boltz == 0) {
                e = ora_maxwell_boltzmann(n, ndim, T_target, mass, seed, (uint64_t)(step / nstep_boltz), NULL, vel);
                if (e) { free(fn); return e; }
            }
        }
        if (log_every > 0 && thermo && s % log_every == 0) {
            double mv2 = ora_sum_mv2(n, vel, mass);
            double ke = 0.5 * mv2;
            double h = ke + pe;
            if (kind == ORA_NOSE_HOOVER || kind == ORA_NOSE_HOOVER_EXACT)
                h += 0.5 * Q * xi * xi + X * T_target * lns;
            double *rec = thermo + 8 * nlog;
            rec[0] = (double)step;
            rec[1] = mv2 / X;
            rec[2] = pe / (double)n;
            rec[3] = ke / (double)n;
            rec[4] = (ke + pe) / (double)n;
            rec[5] = W;
            rec[6] = h;
            rec[7] = xi;
            ++nlog;
        }
    }
    if (state) { state[0] = xi; state[1] = lns; }
    free(fn);
    return 0;
}

/* ------------------------------------------------------------- analysis */

/* Partial radial distribution functions (Sec. "Radial distribution function
 * with Python", Eqs. (gAA), (gAB)) for one configuration of a 2-type system.
 * Every pair j > i with r < rmax adds to bin floor(r/dr); like pairs count
 * twice (once per ordered pair), unlike pairs once. Normalisation divides by
 * the shell volume 4/3 pi ((k+1)^3 - k^3) dr^3 and by N_a(N_a - 1)/V
 * (like) or N_A N_B / V (unlike), V = L^3. ndim = 2 (the 2-D problem of Sec.
 * "Suggested problems", which asks for the shell volume to be adjusted): the
 * shell area pi ((k+1)^2 - k^2) dr^2 and V = L^2. g holds 3*nbins: AA, BB, AB. */
int ora_rdf(int64_t n, int ndim, const double *pos, const int32_t *types, double L, double dr, int64_t nbins,
            double *g)
{
    if (n < 2 || (ndim != 2 && ndim != 3) || !(dr > 0.0) || nbins < 1 || !g) return -1;
    double rmax = dr * (double)nbins;
    if (rmax > 0.5 * L * (1.0 + 1e-12)) return -2;
    int64_t na = 0, nb = 0;
    for (int64_t i = 0; i < n; ++i) { if (types[i] == 0) ++na; else if (types[i] == 1) ++nb; else return -3; }
    double *h = (double *)calloc(3 * (size_t)nbins, sizeof(double));
    if (!h) return -5;
    for (int64_t i = 0; i + 1 < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = ora_min_image(pos[3 * i] - pos[3 * j], L);
            double dy = ora_min_image(pos[3 * i + 1] - pos[3 * j + 1], L);
            double dz = ora_min_image(pos[3 * i + 2] - pos[3 * j + 2], L);
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (!(r < rmax)) continue;
            int64_t k = (int64_t)(r / dr);
            if (k >= nbins) continue;
            if (types[i] == 0 && types[j] == 0) h[k] += 2.0;
            else if (types[i] == 1 && types[j] == 1) h[nbins + k] += 2.0;
            else h[2 * nbins + k] += 1.0;
        }
    double V = ndim == 3 ? L * L * L : L * L;
    for (int64_t k = 0; k < nbins; ++k) {
        double shell = ndim == 3 ? (4.0 / 3.0) * M_PI * (pow((double)(k + 1), 3) - pow((double)k, 3)) * dr * dr * dr
                                 : M_PI * (pow((double)(k + 1), 2) - pow((double)k, 2)) * dr * dr;
        g[k] = (na > 1) ? h[k] / shell * V / ((double)na * (double)(na - 1)) : 0.0;
        g[nbins + k] = (nb > 1) ? h[nbins + k] / shell * V / ((double)nb * (double)(nb - 1)) : 0.0;
        g[2 * nbins + k] = (na > 0 && nb > 0) ? h[2 * nbins + k] / shell * V / ((double)na * (double)nb) : 0.0;
    }
    free(h);
    return 0;
}

/* Mean square displacement per type (Eqs. (msd), (msdwithi)) from unwrapped
 * coordinates x + L*img against reference unwrapped coordinates ref (n*3).
 * out[a] = (1/N_a) sum_{i of type a} |r_i - r_i^ref|^2 for a < ntypes. */
int ora_msd(int64_t n, const double *pos, const int32_t *img, const double *ref, const int32_t *types,
            int ntypes, double L, double *out)
{
    if (n < 1 || !pos || !img || !ref || !out || ntypes < 1) return -1;
    for (int a = 0; a < ntypes; ++a) {
        double s = 0.0;
        int64_t cnt = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (types[i] != a) continue;
            double d2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                double u = pos[3 * i + c] + L * (double)img[3 * i + c];
                double d = u - ref[3 * i + c];
                d2 += d * d;
            }
            s += d2;
            ++cnt;
        }
        out[a] = cnt ? s / (double)cnt : 0.0;
    }
    return 0;
}
