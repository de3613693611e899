/*
 * kamd.h -- C ABI of the GB300 (sm_103a) Kob-Andersen Lennard-Jones MD library.
 *
 * The library advances one system, or a packed batch of independent
 * replicas, of particles interacting by the truncated-and-shifted binary
 * Lennard-Jones potential of the Kob-Andersen model, with velocity-Verlet
 * NVE and two NVT baths, on one GPU. Every step of the method runs in the
 * library's own CUDA kernels; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *  - The return value is an md_status; no C++ exception crosses the ABI.
 *    On failure md_last_error() describes the cause.
 *  - Arrays passed in are borrowed for the duration of the call only. Where
 *    a call takes `on_device`, 1 means the array pointers are device
 *    pointers usable on the system's stream, 0 means host memory.
 *  - Particle order: the API speaks in the caller's order (replica 0's
 *    particles first, then replica 1's, ...). The internal cell-sorted order
 *    is hidden.
 *  - Positions are xyz triples (AoS, n*3 doubles). On output they lie in
 *    [0, L); on input any real value is accepted and wrapped.
 *  - All work is enqueued on the stream given to md_create (NULL = the
 *    legacy default stream). Calls that return values to the host
 *    synchronise that stream before returning.
 *  - Results are deterministic: the same inputs and the same tuning give
 *    bitwise identical results (no floating-point atomics anywhere).
 *  - Units: sigma_AA = eps_AA = m = k_B = 1 in the Kob-Andersen setting; the
 *    library itself is unit-free.
 *  - A system handle must not be used from two host threads at once.
 */
#ifndef KAMD_H
#define KAMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_system md_system; /* opaque; owns all device memory it allocates */

typedef enum {
    MD_OK = 0,
    MD_ERR_INVALID_ARG = 1,    /* an argument failed validation (see md_last_error) */
    MD_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    MD_ERR_OOM = 3,            /* device allocation failed */
    MD_ERR_UNSTABLE = 4,       /* NaN/Inf state, or a particle moved >= L/4 in one step */
    MD_ERR_NLIST_OVERFLOW = 5, /* neighbour-list capacity could not be grown */
    MD_ERR_TIMEOUT = 6,        /* a grid barrier waited past its limit; the state is undefined */
    MD_ERR_NOT_SUPPORTED = 7   /* the device cannot run the library (needs sm_103a) */
} md_status;

typedef enum {
    MD_PREC_FP64 = 0,  /* positions, velocities, forces and pair arithmetic in FP64 */
    MD_PREC_MIXED = 1  /* 64-bit fixed-point positions, FP32 velocities, forces and pair
                          arithmetic, FP64 energy/virial/momentum reductions */
} md_precision;

typedef enum {
    MD_NVT_NOSE_HOOVER = 0,       /* Fox-Andersen integration, Taylor velocity rule */
    MD_NVT_RESAMPLE = 1,          /* Maxwell-Boltzmann redraw every nstep_boltz steps */
    MD_NVT_NOSE_HOOVER_EXACT = 2  /* Fox-Andersen integration, solved velocity rule */
} md_thermostat;

/* One thermodynamic record (per replica, per logged step).
 * Source: Sec. "NVT simulations" (thermo_style step temp pe ke etotal),
 * Eq. (equip3N) for T, Eq. (HNosetilde) for h_nh. PE is the SHIFTED energy of
 * Eq. (VshiftedKALJ). virial = sum_{i<j} r_ij . F_ij. For NVE and the
 * resampling bath h_nh = KE + PE. */
typedef struct {
    int64_t step;
    double T, pe_per_n, ke_per_n, etot_per_n, virial, h_nh, xi;
} md_thermo;

/* Tuning knobs (chosen by md_autotune or set by hand). Changing them never
 * changes the physics except through the order of floating-point sums. */
typedef struct {
    int threads_per_atom; /* 1, 2, 4 or 8 lanes share one particle's neighbour loop */
    int block_size;       /* 128, 256 or 512 threads per CTA of the persistent kernel */
    double skin;          /* inner list: radius r_c,ab + skin, pruned from the outer list
                             once any particle moved skin/2 since the last prune */
    double skin_outer;    /* outer list (>= skin): radius r_c,ab + skin_outer, rebuilt with the
                             cell sort once a particle moved (skin_outer - skin)/2 since;
                             skin_outer == skin: one list of radius r_c,ab + skin, rebuilt
                             once a particle moved skin/2, never pruned */
} md_tuning;

/* Counters and sizes, for measurement. */
typedef struct {
    int64_t n_total;          /* particles over all replicas */
    int32_t n_replicas;
    int32_t grid_blocks;      /* CTAs of the persistent kernel (co-resident) */
    int64_t steps_done;       /* steps advanced since md_create */
    int64_t rebuilds;         /* neighbour-list rebuilds (summed over replicas) */
    int64_t list_entries;     /* entries of the list the force phase reads (the inner list when
                                 there are two; candidate pairs, full list) */
    int64_t list_capacity;    /* entries per particle the list can hold */
    int64_t device_bytes;     /* device memory held by the system */
    int32_t all_pairs_replicas; /* replicas too small for cells (list built by all-pairs scan) */
    int32_t precision;
    int64_t graph_launches;   /* persistent launches issued as CUDA-graph launches */
    int64_t prunes;           /* inner-list prune passes */
    int64_t kernel_launches;  /* kernels launched by the persistent-kernel operations: each
                                 launch of the persistent kernel, and of the kernel that forms
                                 the log records of a launch afterwards */
} md_info;

/*
 * md_create: one system of n particles in a cubic periodic box of edge L.
 *   types   host, n entries in [0, ntypes)     (Sec. "Model": types A, B)
 *   eps, sigma, rc  host, ntypes*ntypes row-major, symmetric, all > 0;
 *                   rc holds absolute cutoffs (2.5*sigma for Kob-Andersen),
 *                   each < L/2 so that the minimum image is unique
 *                   (Eqs. (VKALJ), (VshiftedKALJ), (KAFix); Sec. "Periodic
 *                   boundary conditions").
 *   mass    the particle mass (> 0).
 *   skin    Verlet-list skin (>= 0), e.g. 0.3 (LAMMPS "neighbor 0.3 bin"): the
 *           force list holds pairs within r_c,ab + skin. It is pruned from an
 *           outer list of skin + 0.4 (md_set_tuning changes both).
 *   prec    MD_PREC_FP64 or MD_PREC_MIXED.
 *   stream  cudaStream_t to enqueue on (NULL: legacy default stream).
 * Positions and velocities start at zero: call md_set_state or md_init_lattice.
 * On success *out receives the handle (release with md_destroy). ntypes <= 4.
 */
md_status md_create(int64_t n, const uint8_t* types, int ntypes, double L,
                    const double* eps, const double* sigma, const double* rc,
                    double mass, double skin, md_precision prec, void* stream,
                    md_system** out);

/*
 * md_create_batch: nrep independent replicas packed into one system
 * (replicas average independent runs, Sec. "Radial distribution function").
 *   n_per   host, nrep particle counts (each >= 2)
 *   L_per   host, nrep box edges
 *   types   host, sum(n_per) entries, replica 0's first
 * Other arguments as md_create; the interaction table is shared. Every
 * replica evolves exactly as it would alone (bitwise, for equal tuning).
 */
md_status md_create_batch(int nrep, const int64_t* n_per, const double* L_per,
                          const uint8_t* types, int ntypes,
                          const double* eps, const double* sigma, const double* rc,
                          double mass, double skin, md_precision prec, void* stream,
                          md_system** out);

/*
 * md_create_batch_dim: as md_create_batch, in ndim = 3 or 2 dimensions. The
 * two-dimensional model is the Kob-Andersen problem of Sec. "Suggested
 * problems" (e.g. N = 1000 at N/L^2 = 1.204, L = 28.82, A:B = 65:35): every
 * particle lies in the plane z = L/2 of the cubic box and keeps v_z = 0
 * (md_set_state ignores the z coordinates and z velocities it is given, and
 * md_get_state returns z = L/2, v_z = 0); every pair then has dz = 0, so the
 * forces stay in the plane. Wherever the three-dimensional model counts 3N
 * degrees of freedom the two-dimensional one counts 2N: the temperature of
 * Eq. (equip3N) (3 replaced by 2, as the problem says), the Maxwell-Boltzmann
 * rescale, X and the bath mass Q = X T tau^2 of Nose-Hoover. md_rdf
 * normalises by the ring area pi((k+1)^2 - k^2) dr^2 and V = L^2;
 * md_init_lattice uses a square lattice of m = ceil(n^(1/2)) sites per edge
 * in the plane (no z jitter). ndim = 3 is md_create_batch. MD_ERR_INVALID_ARG
 * for any other ndim.
 */
md_status md_create_batch_dim(int ndim, int nrep, const int64_t* n_per, const double* L_per,
                              const uint8_t* types, int ntypes,
                              const double* eps, const double* sigma, const double* rc,
                              double mass, double skin, md_precision prec, void* stream,
                              md_system** out);

/* md_set_state: overwrite positions and velocities (n_total*3 doubles each,
 * caller order; vel may be NULL for zero velocities). Clears image counters,
 * marks forces stale and forces a neighbour-list rebuild. */
md_status md_set_state(md_system* sys, const double* pos, const double* vel, int on_device);

/* md_get_state: copy out positions in [0, L), velocities and the periodic
 * image counters (n_total*3 int32; unwrapped x = x + L*image). Any pointer may
 * be NULL to skip that array. */
md_status md_get_state(md_system* sys, double* pos, double* vel, int32_t* images, int on_device);

/*
 * md_init_lattice: the simple-cubic lattice start of Sec. "Initialization of
 * positions" and the Maxwell-Boltzmann velocities of Sec. "Statistical
 * temperature bath" (steps 1-4), per replica:
 *   m = ceil(n^(1/3)) sites per edge, site (0.5+k)L/m (x fastest); particle p
 *   takes site floor(p m^3 / n); each coordinate moves by jitter*u, u uniform
 *   in (-1, 1); velocities are Gaussian with variance T0/m, centred, then
 *   scaled so that sum m v^2 = 3 n T0 exactly.
 * Random numbers: Philox4x32-10 keyed by seed, counter = (p, draw, tag|block,
 * 0), Box-Muller for normals. T0: host, one temperature per replica.
 */
md_status md_init_lattice(md_system* sys, const double* T0, double jitter, uint64_t seed);

/*
 * md_forces: forces (Eq. (KAFix) with the cutoff of Eq. (VshiftedKALJ) and
 * the minimum image) on the current positions, written to f (n_total*3
 * doubles, caller order); pe and virial (host, one double per replica) get
 * the shifted potential energy V = sum_{i<j} V_ij^cut and W = sum r.F. Any
 * output may be NULL. Rebuilds the neighbour list if it is stale.
 */
md_status md_forces(md_system* sys, double* f, double* pe, double* virial, int on_device);

/*
 * md_step_nve: nsteps velocity-Verlet steps (Eqs. (velVerletPos),
 * (velVerletVel)), all replicas in lockstep inside one persistent launch.
 * The neighbour list is rebuilt on the device whenever a particle has moved
 * more than skin/2 since the last build ("neigh_modify every 1 check yes").
 * log (host, may be NULL): nrep * floor(nsteps/log_every) records, record
 * k*nrep + r for replica r at the k-th logged step.
 */
md_status md_step_nve(md_system* sys, double dt, int64_t nsteps, md_thermo* log, int64_t log_every);

/*
 * md_step_nvt: nsteps at bath temperature T_target[r] (host, per replica).
 *   kind = MD_NVT_NOSE_HOOVER(_EXACT): Eqs. (nosehoover_rddot),
 *     (nosehoover_xidot) integrated by the Fox-Andersen rules of Appendix B
 *     (Eqs. (Noseupdate_ri)-(Noseupdate_xiapprox), then (ridotKVLRoman), or
 *     (ridotsolved) for _EXACT, and (FoxAndersen_ydottplush)), X = 3n, bath
 *     mass Q = X T_target tau^2 with tau = param (the LAMMPS damping time;
 *     100*dt is the paper's choice). xi and ln s persist across calls.
 *   kind = MD_NVT_RESAMPLE: velocity-Verlet steps; after every step whose
 *     global number is a multiple of nstep_boltz = (int)param all velocities
 *     are redrawn as in md_init_lattice's velocity part (Sec. "NVT molecular
 *     dynamics simulation"), draw number = step/nstep_boltz, key = seed.
 * log as in md_step_nve (records taken after the bath has acted).
 */
md_status md_step_nvt(md_system* sys, double dt, int64_t nsteps, const double* T_target,
                      md_thermostat kind, double param, uint64_t seed,
                      md_thermo* log, int64_t log_every);

/*
 * md_rdf: accumulate partial radial distribution functions (Eqs. (gAA),
 * (gAB); histogram of Sec. "Radial distribution function with Python") of the
 * current configuration, for 2-type systems: nbins bins of width dr from 0,
 * nbins*dr <= L/2 for every replica. g (host, 3*nbins: AA, BB, AB) receives
 * the average over all measurements since the last reset and over replicas.
 * reset = 1 clears the accumulated histogram first.
 */
md_status md_rdf(md_system* sys, double dr, int64_t nbins, double* g, int reset);

/*
 * md_msd: mean square displacement per type (Eqs. (msd), (msdwithi)) from
 * unwrapped coordinates against the reference taken at the last call with
 * reset_reference = 1 (or at md_set_state / md_init_lattice). msd_per_type
 * (host, ntypes doubles) receives the average over particles of each type
 * and over replicas.
 */
md_status md_msd(md_system* sys, double* msd_per_type, int reset_reference);

/*
 * md_msd_tw: waiting-time mean square displacement per type (Eq. (msdtw) and
 * its per-type form in the problems of Sec. "Mean square displacement"),
 * <|r_i(t_w + t) - r_i(t_w)|^2> over the particles of each type and over
 * replicas, against one of MD_MSD_SLOTS reference slots, so that several
 * waiting times t_w can be followed along one trajectory (ageing after a
 * quench, Sec. "Simulation Run Sequence"). reset_reference = 1 first takes
 * the current unwrapped positions as the slot's r(t_w) (t = 0). Slot 0 is the
 * reference of md_msd; the others get their device buffer (24 bytes per
 * particle) at their first reset. msd_per_type: host, ntypes doubles, or NULL
 * (reset only). Errors: MD_ERR_INVALID_ARG for a slot outside
 * [0, MD_MSD_SLOTS) or one that has no reference yet (slots other than 0 lose
 * theirs at md_set_state / md_init_lattice).
 */
#define MD_MSD_SLOTS 8
md_status md_msd_tw(md_system* sys, int slot, double* msd_per_type, int reset_reference);

/* md_set_tuning / md_get_tuning: change or read the launch configuration. */
md_status md_set_tuning(md_system* sys, const md_tuning* t);
md_status md_get_tuning(const md_system* sys, md_tuning* t);

/*
 * md_autotune: time short NVE probes (probe_steps each, dt) and keep the
 * fastest candidate. Coordinate search: threads_per_atom x block_size at the
 * current skins, then nine (skin, skin_outer) pairs (three of them one-list)
 * at the best of those, then threads_per_atom x block_size at the best pair.
 * The system's state is saved before and restored after, so the trajectory
 * is unaffected. best (may be NULL) receives the choice, seconds_per_step (may
 * be NULL) its measured cost.
 */
md_status md_autotune(md_system* sys, double dt, int64_t probe_steps, md_tuning* best,
                      double* seconds_per_step);

/*
 * md_autotune_skin: as md_autotune, but the force list's skin stays `skin`
 * (for a configuration that prescribes it); threads_per_atom, block_size and
 * the outer list's skin (skin, skin + 0.3, + 0.5, + 0.7, + 0.9, + 1.1) are searched.
 * MD_ERR_INVALID_ARG unless 0.05 <= skin < 2. (The paper has no counterpart.)
 */
md_status md_autotune_skin(md_system* sys, double dt, int64_t probe_steps, double skin, md_tuning* best,
                           double* seconds_per_step);

/*
 * md_time_forces: measurement of the force phase alone. One persistent launch
 * evaluates the forces of the current positions `repeats` times (the pair
 * sums over the force list and the force stores of a time step, without the
 * velocity update, the position update or energies), each evaluation closed
 * by a grid barrier; a launch with one evaluation is timed too, and
 * *seconds_per_eval = (t(repeats) - t(1)) / (repeats - 1), CUDA events on the
 * system's stream. Lists are brought up to date first (not timed). The state
 * is unchanged except for the stored forces, which are those of the current
 * positions either way. 1 <= repeats <= 100000. (The paper has no
 * counterpart: this is a measurement interface.)
 */
md_status md_time_forces(md_system* sys, int64_t repeats, double* seconds_per_eval);

/*
 * md_time_lists: measurement of the Verlet-list build alone (the step that
 * follows the cell sort of a rebuild). Every replica is marked for a rebuild;
 * one persistent launch then sorts the cells and builds the lists, and builds
 * the (outer) lists of the same cells `repeats` - 1 more times, each closed by
 * a grid barrier. A launch with a single rebuild is timed too, and
 * *seconds_per_build = (t(repeats) - t(1)) / (repeats - 1), CUDA events on
 * the system's stream. Needs 2 <= repeats <= 10000. The state afterwards is
 * that of a rebuild at the current positions: particles are re-sorted into
 * their cells (the same reordering a rebuild in a run makes), positions,
 * velocities and stored forces are unchanged as a set, and later force sums
 * may differ from those of an uninterrupted run in the last bits (summation
 * order). (The paper has no counterpart: this is a measurement interface.)
 */
md_status md_time_lists(md_system* sys, int64_t repeats, double* seconds_per_build);

/* md_get_info: counters and sizes (synchronises the stream). */
md_status md_get_info(md_system* sys, md_info* info);

/* md_count_pairs: number of particle pairs (i<j) currently inside their
 * cutoff r < rc_ab, summed over replicas (runs one extra pass). */
md_status md_count_pairs(md_system* sys, int64_t* pairs_within_cutoff);

/*
 * md_selftest_barrier: failure-detection self-test of the grid barrier. A
 * small kernel runs the barrier with one block that never arrives, so the
 * others' bounded wait runs out after timeout_s (0 < timeout_s <= 60) and they
 * return. Expected result: MD_ERR_TIMEOUT, with the system's state untouched
 * and the CUDA context still usable. Any other result means the time limit
 * does not work. No memory is read or written except the control block.
 */
md_status md_selftest_barrier(md_system* sys, double timeout_s);

/*
 * md_forces_noalloc: forces, shifted potential energy and virial of one
 * configuration, computed without allocating any memory. The paper has no
 * counterpart: this is an interface for callers that cannot allocate.
 *
 * Who needs it: code that enqueues work while a stream is being captured
 * into a CUDA graph (cudaMalloc is not allowed inside a capture), real-time
 * loops and plugins that must not pay for, or may not trigger, the device
 * allocator and its implicit synchronisation, and hosts that give the
 * library a fixed memory budget. Every other caller should use md_forces.
 *
 * All scratch lives in one static device array of 1.4 MiB that every GPU
 * which loads the library holds until the process exits. Hence the limits:
 * 2 <= n <= 131072 particles and at most 32 cells per box edge (larger boxes
 * use larger cells); larger n is rejected with MD_ERR_INVALID_ARG and a
 * message in md_last_error(NULL).
 *   pos     device, n*3 doubles (any real values; wrapped into [0, L))
 *   types   device, n uint8 in [0, ntypes). A value >= ntypes is never used
 *           as a table index: that particle's force, and the force of every
 *           particle that meets it in the cell search, comes out NaN, and so
 *           do pe and virial.
 *   eps, sigma, rc  host tables as in md_create (rc < L/2)
 *   f       device, n*3 doubles (output, caller order)
 *   pe, virial  device, one double each (outputs; may be NULL)
 *   stream  cudaStream_t for all work (NULL: legacy default stream)
 * The arithmetic is that of md_forces on the FP64 path, over a cell list of
 * cell edge >= the largest cutoff; results are deterministic.
 * The call only enqueues work and returns. The host-side name of the static
 * array is not a device address, so every call made outside a stream capture
 * looks up the array's device address in the current CUDA context; a call
 * made while its stream is being captured uses the address found by the last
 * uncaptured call in the same context. Hence: make one call in each context
 * (and again after cudaDeviceReset) before capturing a stream; a captured
 * call with no earlier one fails with MD_ERR_INVALID_ARG. Every call on a
 * device shares the one array, which keeps the previous call's contents
 * (each call clears what must start at zero): calls that overlap on the GPU
 * -- on different streams, or from different host threads -- race and give
 * wrong results; order them.
 */
md_status md_forces_noalloc(int64_t n, const double* pos, const uint8_t* types, int ntypes, double L,
                            const double* eps, const double* sigma, const double* rc,
                            double* f, double* pe, double* virial, void* stream);

/* Message for the last failure of this handle (or of md_create when sys is
 * NULL, per host thread). Never NULL. */
const char* md_last_error(const md_system* sys);

/* Release every resource of the handle. NULL is ignored. */
void md_destroy(md_system* sys);

#ifdef __cplusplus
}
#endif

#endif /* KAMD_H */
