// md_internal.cuh -- definitions shared by the library's translation units.
//
// Memory layout in HBM (all arrays packed over replicas; each replica owns
// a contiguous slot range starting at a multiple of 32 and padded to a
// multiple of 32, so every 32-slot tile belongs to exactly one replica):
//
//   mixed precision                       all-FP64
//   pfx   u64  [3][ntot]  fixed point     p4[2] double4_32a [ntot]  (x,y,z,type)
//   pq[2] uint4 [ntot] (x,y,z hi32,type)  -- gather copy = master, double-buffered
//   velf  f32  [3][ntot]                  veld f64 [3][ntot]
//   frcf  f32  [3][ntot]                  frcd f64 [3][ntot]
//   xbq   uint4 [ntot] (position at the   xbd  double4_32a [ntot]
//         last list build, hi32)
//   gid i32 [ntot] caller index; typ u8 [ntot]; img i32 [3][ntot] image counters
//   nbr i32 [ntiles][maxrows][32*T]: lane s of particle a of a tile owns
//       column a*T + s; its q-th neighbour sits in row q. nnb i32 [ntot*T]
//       holds each lane's count. The T lanes of a particle read consecutive
//       words, so a warp reads 128 contiguous bytes per row.
//   cells: ccount/ccursor [ncells], cstart [ncells + nrep], cellof/scat [ntot]
//
// Fixed-point positions: u = x/L * 2^64 (mod 2^64). Wrapping into the box is
// the natural overflow of the integer; the minimum-image difference of two
// particles is the signed 32-bit difference of their top words, exact.
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#define MD_TILE 32
#define MD_MAXTYPES 4
#define MD_SCAN_CHUNK 1024  // cells per chunk of the cell-count scan
#define MD_UNION_MAX 512    // staged cells of one list-build group: (GX+2nr)(GY+2nr)(GZ+2nr) <= 8*8*8
#define MD_LOG_SLOTS 64     // log steps per launch whose reductions wait for the launch end
#define MD_ROWS_MAX 16      // (y, z) rows of cells in one list-build group: GY*GZ <= 4*4
#define MD_RED_TILES 256    // tiles per chunk of the two-level per-replica reduction (default)
#define MD_NPART 8   // per-tile partial sums: pe, ke, vir, px, py, pz, (2 spare)

// pending/commit flag bits (grid-uniform decisions)
#define MD_FLAG_REBUILD 1
#define MD_FLAG_OVERFLOW 2
#define MD_FLAG_UNSTABLE 4
#define MD_FLAG_TIMEOUT 8
#define MD_FLAG_PRUNE 16

enum { MD_OP_FORCES = 0, MD_OP_STEPS = 1, MD_OP_REBUILD = 2, MD_OP_INITVEL = 3, MD_OP_FORCE_REPEAT = 4,
       MD_OP_LIST_REPEAT = 5 };
enum { MD_KIND_NVE = 0, MD_KIND_NH = 1, MD_KIND_RESAMPLE = 2, MD_KIND_NH_EXACT = 3 };

// Per-replica description and state (device resident, one per replica).
struct RepDev {
  int64_t off;      // first slot (multiple of 32)
  int64_t out0;     // offset of this replica in caller order
  int64_t cell0;    // first cell in the packed cell arrays
  int64_t cs0;      // first cstart entry (= cell0 + replica index)
  int32_t n;        // particles
  int32_t ntiles;   // slots / 32
  int32_t tile0;    // first tile
  int32_t nc;       // cells per edge (0: list built by an all-pairs scan)
  int32_t nr;       // cells on each side that the list build scans: 2 (cells >= r_list / 2 wide) or 1
  int32_t gx, gy, gz;  // cells per list-build group along x, y, z (1, 2 or 4 each; per replica)
  double L, invL;
  double fx64;      // 2^64 / L
  float Lf, fxs;    // L, L / 2^32
  float fx64f;      // 2^64 / L
  float fx32f;      // 2^32 / L
  float cellw;      // L / nc
  // bath
  double T_target, Q;
  double xi, g, lns, lns_next, xi_a;
  float xif, xiaf;  // FP32 copies of xi and xi_a for the mixed path
  // last reductions
  double pe, ke, vir, px, py, pz;
  // resampling
  double vmean[3], vscale;
  float vmeanf[3], vscalef;
  int32_t want_rebuild, doing_rebuild;
  int64_t rebuilds;
  int64_t prune_epoch;    // force step whose inner list must be pruned first (set by drifts)
  int64_t rebuild_epoch;  // force step before which the outer list was last rebuilt
  int64_t cell_base;      // particles in the cells of earlier replicas that rebuild with this one
  int64_t list_entries;
};

// Grid barrier and launch-wide control block.
struct CtlDev {
  unsigned int bar_gen;
  int pending;          // bits 0..15: flags raised during a phase (atomicOr); 16..31: barrier arrivals
  int snap[2];          // pending as seen by the last arriver, per barrier parity
  int cur;              // parity of the current gather buffer
  int drifted;          // 1: positions at t+dt while velocities/forces are at t
  int log_slots_used;   // log slots the last launch filled (their records still to form)
  int forces_valid;
  int64_t step;         // global step counter
  int64_t steps_done;   // steps completed by the current/last launch
  int64_t prunes;       // prune passes since creation
  int err_where;        // phase id where a barrier timed out
  int pad;
#ifdef KAMD_PHASE_TIMERS
  unsigned long long t_last;
  unsigned long long phase_ns[128];
  unsigned long long phase_cnt[128];
#endif
};

struct ThermoDev {  // layout identical to md_thermo
  int64_t step;
  double T, pe_per_n, ke_per_n, etot_per_n, virial, h_nh, xi;
};

// Verlet list layout. A tile of 32 particles owns maxrows * 32T entries
// (maxrows a multiple of 4). List column L = a*T + s belongs to lane s of the
// tile's particle a. Entries are grouped in quads: entry q of column L sits at
//   tile * maxrows * 32T  +  (q / 4) * 4 * 32T  +  4 L  +  q % 4,
// so the 32 lanes of a warp that read one quad each touch 512 contiguous
// bytes, and a writer stores four entries with one 16-byte store.
__host__ __device__ inline int64_t list_col(int64_t tile, int maxrows, int T, int col) {
  return tile * (int64_t)maxrows * 32 * T + 4 * (int64_t)col;
}
__host__ __device__ inline int64_t list_at(int64_t colbase, int q, int gsz) {
  return colbase + (int64_t)(q >> 2) * 4 * gsz + (q & 3);
}

struct KParams {
  // sizes
  int nrep;
  int ntypes;
  int ndim;            // 3, or 2: every particle in the plane z = L/2 with v_z = 0
  int64_t ntot;        // slots
  int ntiles;
  int T;               // lanes per particle
  int maxrows;         // list entries per column (capacity per particle = maxrows*T), a multiple of 4
  int dual;            // 1: inner list pruned from the outer one; 0: one list (skin_outer == skin)
  // interaction tables, index a*ntypes+b
  float tab_f[MD_MAXTYPES * MD_MAXTYPES][4];   // rc^2, sigma^2, 48 eps, 4 eps
  float vsh_f[MD_MAXTYPES * MD_MAXTYPES];      // V(rc)
  float rl2_f[MD_MAXTYPES * MD_MAXTYPES];      // outer list radius^2: (rc + skin_outer)^2
  float rli2_f[MD_MAXTYPES * MD_MAXTYPES];     // inner list radius^2: (rc + skin)^2
  double tab_d[MD_MAXTYPES * MD_MAXTYPES][4];
  double vsh_d[MD_MAXTYPES * MD_MAXTYPES];
  double rl2_d[MD_MAXTYPES * MD_MAXTYPES];
  double rli2_d[MD_MAXTYPES * MD_MAXTYPES];
  double mass, inv_mass;
  double skin_half2;   // ((skin_outer - skin)/2)^2, one list: (skin/2)^2: move since the build that forces a rebuild
  double prune_half2;  // (skin/2)^2, one list: infinite: move since the last prune that forces a prune
  float massf, inv_massf, skin_half2f, dtf, prune_half2f;
  // operation
  int op;
  int kind;
  double dt;
  int64_t nsteps;      // steps to run in this launch
  int64_t nstep_boltz;
  uint64_t seed;
  int64_t log_every;
  int64_t log_step0;   // steps completed in this call before this launch
  int64_t log_cap;     // records per replica the log can hold
  ThermoDev* thermo;
  unsigned long long timeout_ns;
  // state
  RepDev* reps;
  int32_t* tile_rep;
  CtlDev* ctl;
  uint64_t* pfx;
  uint4* pq[2];
  float* velf;
  float* frcf;
  uint4* xbq;          // positions at the last outer build
  uint4* xbq_in;       // positions at the last prune
  double4_32a* p4[2];
  double* veld;
  double* frcd;
  double4_32a* xbd;
  double4_32a* xbd_in;
  int32_t* gid;
  uint8_t* typ;
  int32_t* img;
  // permutation scratch
  uint64_t* t_pfx;
  double4_32a* t_p4;
  void* t_vel;
  void* t_frc;
  int32_t* t_gid;
  uint8_t* t_typ;
  int32_t* t_img;
  // cells and list
  int32_t* cellof;
  int32_t* cell_rep;   // replica of each packed cell
  int64_t ncells;
  int stage_cap;       // candidates the list build can stage in dynamic shared memory
  int32_t* ccount;
  int32_t* cstart;
  int32_t* ccursor;
  int32_t* chunk;      // per-chunk cell-count sums of the cell scan (MD_SCAN_CHUNK cells each)
  int32_t* cta_sm;     // SM id of each CTA of the current launch
  const int2* grp;     // list-build groups: (replica, group index inside the replica)
  int red2;            // 1: reductions in two levels (some replica has more than 4 chunks)
  int red_tiles;       // tiles per reduction chunk
  int64_t nred;        // reduction chunks over all replicas
  const int2* redmap;  // chunk -> (replica, chunk index inside the replica)
  const int2* redrep;  // replica -> (first chunk, number of chunks)
  double* redpart;     // chunk sums, MD_NPART doubles per chunk
  int64_t ngroups;
  int32_t* scat;
  int32_t* nbr;        // outer list
  int32_t* nnb;
  int32_t* nbr_in;     // inner (pruned) list, same layout; read by the force phase
  int32_t* nnb_in;
  // reductions
  double* part[2];     // [ntiles][MD_NPART]: doubles (FP64 path) or float (hi, lo) pairs (mixed path)
  // partial records of NVE steps that only log, reduced after the launch's
  // last step: plog_slots slots of plog_stride doubles each
  double* plog;
  longlong2* plog_rec;  // per slot: (step, log record index)
  int64_t plog_stride;
  int plog_slots;
};

// Host-side launchers (md_kernel.cu).
cudaError_t md_launch_persistent(bool mixed, const KParams& p, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t md_launch_log_records(bool mixed, const KParams& p, int nslots, int block, cudaStream_t s);
cudaError_t md_occupancy(bool mixed, int block, size_t smem, int* blocks_per_sm);
const void* md_persistent_fn(bool mixed);
cudaError_t md_launch_barrier_selftest(const KParams& p, int blocks, cudaStream_t s);
// Message returned by md_last_error(NULL) on this host thread (md_api.cu).
void kamd_set_global_error(const std::string& msg);
