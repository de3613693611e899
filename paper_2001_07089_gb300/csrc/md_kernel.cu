// md_kernel.cu -- the persistent sm_103a kernel that advances every replica.
//
// One cooperative launch runs a whole md_step call: all CTAs stay resident
// and meet at a bounded grid barrier between phases. Per time step:
//
//   force phase   F_i = sum_j 48 eps_ab (sigma^12/r^14 - sigma^6/(2 r^8)) r_ij
//                 (Eq. (KAFix), cutoff of Eq. (VshiftedKALJ), minimum image of
//                 Sec. "Periodic boundary conditions"), gathered over a full
//                 Verlet list by T lanes per particle (no atomics), then the
//                 velocity update (Eq. (velVerletVel), or Eq. (ridotKVLRoman) /
//                 (ridotsolved) under Nose-Hoover), per-tile FP64 partial sums
//                 of PE, KE, virial, momentum, and -- for NVE steps -- the next
//                 position update (Eq. (velVerletPos)) fused in.
//   barrier
//   reduce        per replica, fixed-order sum of tile partials; Nose-Hoover
//                 xi, ln s updates (Eqs. (Noseupdate_lns), (Noseupdate_xiapprox),
//                 (FoxAndersen_ydottplush)); thermo record.
//   [Nose-Hoover: barrier, position update Eq. (Noseupdate_ri), barrier]
//   [resampling step: Maxwell-Boltzmann draw, reduce, centre+rescale+drift]
//   [rebuild when any particle moved > skin/2: cell count, scan, scatter,
//    in-cell rank sort by caller index, permute, Verlet-list build]
//
// All decisions that change the phase sequence are read from a snapshot the
// barrier takes, so every CTA takes the same branch. Every barrier wait is
// bounded in time; on expiry the kernel raises MD_FLAG_TIMEOUT and returns.
#include "md_device.cuh"
#include "md_internal.cuh"

#ifndef KAMD_MIN_BLOCKS
#define KAMD_MIN_BLOCKS 2
#endif

namespace kamd {

enum { KICK_NONE = 0, KICK_VV = 1, KICK_NH = 2, KICK_NH_EXACT = 3 };
enum { RED_FORCES = 0, RED_KE = 1, RED_STEP = 2, RED_RESAMPLE = 3, RED_STEP_KE = 4, RED_LOG = 5 };

struct Shared {
  float4 tabf[MD_MAXTYPES * MD_MAXTYPES];
  float vshf[MD_MAXTYPES * MD_MAXTYPES];
  float rl2f[MD_MAXTYPES * MD_MAXTYPES];
  float rli2f[MD_MAXTYPES * MD_MAXTYPES];
  double4_32a tabd[MD_MAXTYPES * MD_MAXTYPES];
  double vshd[MD_MAXTYPES * MD_MAXTYPES];
  double rl2d[MD_MAXTYPES * MD_MAXTYPES];
  double rli2d[MD_MAXTYPES * MD_MAXTYPES];
  double red[16][MD_NPART];
  int scan[32];
  int snap;
  unsigned gen;  // grid barrier generation this CTA waits for next (thread 0)
  // SM-local work layout of this launch (see sm_layout)
  unsigned sm_bits[8];
  int sm_ok, sm_idx, sm_used, sm_cnt, sm_rank;
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int sm_id() {
  int v;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
  return v;
}

// Contiguous share [*b, *e) of n items for the SM this CTA runs on, taken by
// its `per` workers per CTA (warps or the CTA itself) with stride *st.
// Neighbouring tiles and cells then run on one SM and share its L1. Falls
// back to a grid-strided split when the layout is unknown.
__device__ __forceinline__ void sm_share(const Shared& sh, int64_t n, int per, int worker, int64_t* b, int64_t* e,
                                         int64_t* st) {
  if (sh.sm_ok) {
    const int64_t lo = n * sh.sm_idx / sh.sm_used, hi = n * (sh.sm_idx + 1) / sh.sm_used;
    *b = lo + (int64_t)sh.sm_rank * per + worker;
    *e = hi;
    *st = (int64_t)sh.sm_cnt * per;
  } else {
    *b = (int64_t)blockIdx.x * per + worker;
    *e = n;
    *st = (int64_t)gridDim.x * per;
  }
}

__device__ __forceinline__ unsigned vload_u32(const unsigned* p) { return *(volatile const unsigned*)p; }
__device__ __forceinline__ int vload_i32(const int* p) { return *(volatile const int*)p; }

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_acqrel_u32(unsigned* p, unsigned x) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(x) : "memory");
  return old;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned x) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}

// Grid barrier with a time limit (acquire/release on the generation word).
// The arrival count shares the control word `pending` with the flags (count
// in bits 16..31, flags in bits 0..15): a flag raised before a CTA arrives
// precedes that arrival in the word's modification order, so the atomic of
// the last CTA to arrive returns every flag of the phase, with no further
// read. Thread 0 of each CTA keeps the generation it waits for in shared
// memory (read once at launch). Returns the flags as seen by the last arriver
// (identical for every CTA), or -1 after a timeout.
__device__ int grid_sync(const KParams& p, Shared& sh, int where) {
  __syncthreads();
  if (threadIdx.x == 0) {
    CtlDev* c = p.ctl;
    const unsigned g = sh.gen;
    const unsigned old = atom_add_acqrel_u32(reinterpret_cast<unsigned*>(&c->pending), 1u << 16);
    int res = -1;
    if ((old >> 16) == gridDim.x - 1) {
      const int pend = (int)(old & 0xffffu);
      atomicAnd(&c->pending, 0xffff);  // clear the count before the release
      c->snap[(g + 1) & 1] = pend;
      st_release_u32(&c->bar_gen, g + 1);
      res = pend;
    } else {
      const unsigned long long t0 = globaltimer();
      unsigned it = 0;
      while (true) {
        if (ld_acquire_u32(&c->bar_gen) != g) {
          res = vload_i32(&c->snap[(g + 1) & 1]);
          break;
        }
        if (((++it) & 255u) == 0) {
          if (vload_i32(&c->pending) & MD_FLAG_TIMEOUT) break;
          if (globaltimer() - t0 > p.timeout_ns || it > (1u << 30)) {
            atomicOr(&c->pending, MD_FLAG_TIMEOUT);
            atomicExch(&c->err_where, where);
            break;
          }
        }
      }
    }
    sh.gen = g + 1;
    sh.snap = res;
#ifdef KAMD_PHASE_TIMERS
    // profiling builds only: time between consecutive barriers, charged to
    // the barrier that closes the phase (block 0's view)
    if (blockIdx.x == 0 && res >= 0) {
      const unsigned long long t = globaltimer();
      if (c->t_last) {
        c->phase_ns[where & 127] += t - c->t_last;
        c->phase_cnt[where & 127] += 1;
      }
      c->t_last = t;
    }
#endif
  }
  __syncthreads();
  return sh.snap;
}

// Float-float (compensated) addition: exact TwoSum of the high parts, low
// parts added with the rounding error, then renormalised. Commutative, so
// an xor-butterfly leaves the same value in every lane.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  const float lo = (a.lo + b.lo) + e;
  const float h = s + lo;
  return {h, lo - (h - s)};
}
__device__ __forceinline__ ff warp_sum_ff(ff v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const ff w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = ff_add(v, w);
  }
  return v;
}

__device__ __forceinline__ void raise_flag(const KParams& p, int f) {
  if (!(vload_i32(&p.ctl->pending) & f)) atomicOr(&p.ctl->pending, f);
}

// ------------------------------------------------------------------ drift

// Position update of one particle, mixed path: an FP32 increment is turned
// into a 64-bit fixed-point step with 32-bit conversions only (x = d 2^32/L,
// high word floor(x), low word from the fraction) and added to the integer
// coordinate; the wrap is the integer overflow and the image counter follows
// the carry. Also refreshes the gather copy and checks the half-skin trigger.
__device__ __forceinline__ void drift_mix(const KParams& p, const RepDev& R, int64_t i, int cur, const float v[3],
                                          const float a[3], float xi, uint32_t type, int64_t nstep) {
  const int64_t nt = p.ntot;
  const float dt = p.dtf, hdt2 = 0.5f * p.dtf * p.dtf;
  float d[3];
  bool bad = false;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    d[c] = fmaf(v[c], dt, (a[c] - xi * v[c]) * hdt2);
    bad |= !(fabsf(d[c]) < 0.25f * R.Lf);
  }
  if (bad) { raise_flag(p, MD_FLAG_UNSTABLE); return; }
  uint32_t hi[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float x = d[c] * R.fx32f;
    const float xh = floorf(x);
    const float fr = x - xh;  // exact, in [0, 1)
    const uint32_t lo = __float2uint_rn(fr * 4294967296.0f);
    const long long du = (long long)((uint64_t)(uint32_t)__float2int_rn(xh) << 32) + (long long)lo;
    const uint64_t u = p.pfx[c * nt + i];
    const uint64_t un = u + (uint64_t)du;
    if (du > 0 && un < u) p.img[c * nt + i] += 1;
    else if (du < 0 && un > u) p.img[c * nt + i] -= 1;
    p.pfx[c * nt + i] = un;
    hi[c] = (uint32_t)(un >> 32);
  }
  p.pq[cur ^ 1][i] = make_uint4(hi[0], hi[1], hi[2], type);
  // outer list: rebuild once a particle moved more than (skin_outer - skin)/2
  // since the build; inner list: prune once it moved more than skin/2 since
  // the last prune
  const uint4 xb = p.xbq[i];
  const float ex = (float)(int)(hi[0] - xb.x) * R.fxs;
  const float ey = (float)(int)(hi[1] - xb.y) * R.fxs;
  const float ez = (float)(int)(hi[2] - xb.z) * R.fxs;
  if (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) > p.skin_half2f) {
    p.reps[p.tile_rep[i >> 5]].want_rebuild = 1;
    raise_flag(p, MD_FLAG_REBUILD);
  }
  if (!p.dual) return;
  const uint4 xp = p.xbq_in[i];
  const float gx = (float)(int)(hi[0] - xp.x) * R.fxs;
  const float gy = (float)(int)(hi[1] - xp.y) * R.fxs;
  const float gz = (float)(int)(hi[2] - xp.z) * R.fxs;
  if (fmaf(gx, gx, fmaf(gy, gy, gz * gz)) > p.prune_half2f) {
    p.reps[p.tile_rep[i >> 5]].prune_epoch = nstep;
    raise_flag(p, MD_FLAG_PRUNE);
  }
}

// Position update of one particle, FP64 path: wrap into [0, L).
__device__ __forceinline__ void drift_f64(const KParams& p, const RepDev& R, int64_t i, int cur, const double v[3],
                                          const double a[3], double xi, int64_t nstep) {
  const int64_t nt = p.ntot;
  const double dt = p.dt, hdt2 = 0.5 * p.dt * p.dt;
  const double4_32a x = p.p4[cur][i];
  double d[3];
  bool bad = false;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    d[c] = v[c] * dt + (a[c] - xi * v[c]) * hdt2;
    bad |= !(fabs(d[c]) < 0.25 * R.L);
  }
  if (bad) { raise_flag(p, MD_FLAG_UNSTABLE); return; }
  double xs[3] = {x.x + d[0], x.y + d[1], x.z + d[2]};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (xs[c] >= R.L) { xs[c] -= R.L; p.img[c * nt + i] += 1; }
    else if (xs[c] < 0.0) {
      xs[c] += R.L; p.img[c * nt + i] -= 1;
      if (xs[c] >= R.L) { xs[c] -= R.L; p.img[c * nt + i] += 1; }
    }
  }
  p.p4[cur ^ 1][i] = make_double4_32a(xs[0], xs[1], xs[2], x.w);
  const double4_32a xb = p.xbd[i];
  double e[3] = {xs[0] - xb.x, xs[1] - xb.y, xs[2] - xb.z};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (e[c] > 0.5 * R.L) e[c] -= R.L;
    else if (e[c] < -0.5 * R.L) e[c] += R.L;
  }
  if (e[0] * e[0] + e[1] * e[1] + e[2] * e[2] > p.skin_half2) {
    p.reps[p.tile_rep[i >> 5]].want_rebuild = 1;
    raise_flag(p, MD_FLAG_REBUILD);
  }
  if (!p.dual) return;
  const double4_32a xp = p.xbd_in[i];
  double g[3] = {xs[0] - xp.x, xs[1] - xp.y, xs[2] - xp.z};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (g[c] > 0.5 * R.L) g[c] -= R.L;
    else if (g[c] < -0.5 * R.L) g[c] += R.L;
  }
  if (g[0] * g[0] + g[1] * g[1] + g[2] * g[2] > p.prune_half2) {
    p.reps[p.tile_rep[i >> 5]].prune_epoch = nstep;
    raise_flag(p, MD_FLAG_PRUNE);
  }
}

// Stand-alone position update for every particle (first step of a call,
// Nose-Hoover steps, and the step after a resampling). With `rescale` the
// velocities are first centred and scaled by the replica's resampling factors.
template <bool MIX>
__device__ void drift_phase(const KParams& p, int cur, bool nh, bool rescale, bool drift, int64_t nstep) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nt = p.ntot;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += stride) {
    const RepDev& R = p.reps[p.tile_rep[i >> 5]];
    if (i - R.off >= R.n) continue;
    if constexpr (MIX) {
      float v[3], a[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v[c] = p.velf[c * nt + i];
        a[c] = p.frcf[c * nt + i] * p.inv_massf;
      }
      if (rescale) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          v[c] = (v[c] - R.vmeanf[c]) * R.vscalef;
          p.velf[c * nt + i] = v[c];
        }
      }
      if (drift) drift_mix(p, R, i, cur, v, a, nh ? R.xif : 0.0f, p.pq[cur][i].w, nstep);
    } else {
      double v[3], a[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v[c] = p.veld[c * nt + i];
        a[c] = p.frcd[c * nt + i] * p.inv_mass;
      }
      if (rescale) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          v[c] = (v[c] - R.vmean[c]) * R.vscale;
          p.veld[c * nt + i] = v[c];
        }
      }
      if (drift) drift_f64(p, R, i, cur, v, a, nh ? R.xi : 0.0, nstep);
    }
  }
}

// ------------------------------------------------------------------ forces

// Pair term for one list entry (mixed path): minimum-image displacement from
// the signed 32-bit difference of fixed-point top words, then Eq. (KAFix)
// (force) and Eq. (VshiftedKALJ) (energy) inside the cutoff.
template <bool ENERGY>
__device__ __forceinline__ void pair_mix(const Shared& sh, const uint4& pi, const uint4& pj, int tb, float sc,
                                         float& fx, float& fy, float& fz, float& pe, float& vir) {
  const float dx = (float)(int)(pi.x - pj.x) * sc;
  const float dy = (float)(int)(pi.y - pj.y) * sc;
  const float dz = (float)(int)(pi.z - pj.z) * sc;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const int tt = tb + (int)pj.w;
  const float4 c = sh.tabf[tt];
  const float ir2 = __fdividef(1.0f, r2);
  const float s2 = c.y * ir2;
  const float s6 = s2 * s2 * s2;
  const float w = c.z * s6 * (s6 - 0.5f);
  const bool in = r2 < c.x;
  const float fr = in ? w * ir2 : 0.0f;
  fx = fmaf(fr, dx, fx);
  fy = fmaf(fr, dy, fy);
  fz = fmaf(fr, dz, fz);
  if (ENERGY) {
    pe += in ? fmaf(c.w * s6, s6 - 1.0f, -sh.vshf[tt]) : 0.0f;
    vir += in ? w : 0.0f;
  }
}

// Walk one lane's column of the list: each quad of indices is one 16-byte
// load, issued two quads ahead of the gathers it feeds, so that a list read
// from HBM has two rounds of pair terms to arrive. List words are read once
// per pass, so they are loaded with the evict-first (streaming) policy: once
// the list outgrows L2 it would otherwise push out the gather copy that every
// pass re-reads.
template <bool ENERGY>
__device__ __forceinline__ void lane_sum_mix(const Shared& sh, const uint4* __restrict__ pq, const int* lp, int gsz,
                                             int cnt, int4 jq, const uint4& pi, int tb, float sc, float& fx,
                                             float& fy, float& fz, float& pe, float& vir) {
  // jq: the column's first quad of indices, loaded by the caller; jn: the next
  const int64_t qstride = 4 * (int64_t)gsz;  // ints between consecutive quads of one column
  int4 jn = make_int4(0, 0, 0, 0);
  if (cnt > 4) jn = __ldcs(reinterpret_cast<const int4*>(lp + qstride));
  int q = 0;
  for (; q + 4 <= cnt; q += 4) {
    const uint4 p0 = pq[jq.x], p1 = pq[jq.y], p2 = pq[jq.z], p3 = pq[jq.w];
    jq = jn;
    if (q + 8 < cnt) jn = __ldcs(reinterpret_cast<const int4*>(lp + (int64_t)((q + 8) >> 2) * qstride));
    pair_mix<ENERGY>(sh, pi, p0, tb, sc, fx, fy, fz, pe, vir);
    pair_mix<ENERGY>(sh, pi, p1, tb, sc, fx, fy, fz, pe, vir);
    pair_mix<ENERGY>(sh, pi, p2, tb, sc, fx, fy, fz, pe, vir);
    pair_mix<ENERGY>(sh, pi, p3, tb, sc, fx, fy, fz, pe, vir);
  }
  // tail: 1 to 3 entries of the last quad, already in jq
  const int r = cnt - q;
  if (r > 0) pair_mix<ENERGY>(sh, pi, pq[jq.x], tb, sc, fx, fy, fz, pe, vir);
  if (r > 1) pair_mix<ENERGY>(sh, pi, pq[jq.y], tb, sc, fx, fy, fz, pe, vir);
  if (r > 2) pair_mix<ENERGY>(sh, pi, pq[jq.z], tb, sc, fx, fy, fz, pe, vir);
}

// Force phase. The work unit is one warp: 32/T particles of one tile with T
// lanes each (a tile of 32 particles is T units). Lane s of particle a walks
// its own column of the list; the T lanes are combined by a fixed xor tree;
// lane 0 then applies the velocity rule of `kick`, stores force and velocity
// and (if `fuse`) already performs the next position update into the other
// gather buffer. Without `pairs` only the kinetic partials are formed. Each
// unit writes its own partial sums, so no CTA-wide synchronisation is needed.
// `energy` = also form PE and virial (steps whose energies are reported).
template <bool MIX>
__device__ void force_phase(const KParams& p, Shared& sh, int cur, int kick, bool fuse, double* part, bool pairs,
                            bool energy, bool partials, int64_t nstep) {
  const int T = p.T;
  const int gsz = 32 * T;
  const int lane = threadIdx.x & 31;
  const int nunits = p.ntiles * T;
  const int64_t nt = p.ntot;
  int64_t ub, ue, us;
  sm_share(sh, nunits, (int)(blockDim.x >> 5), (int)(threadIdx.x >> 5), &ub, &ue, &us);
  for (int u = (int)ub; u < ue; u += (int)us) {
    const int tile = u / T;
    const int w = u - tile * T;
    const int rr = w * 32 + lane;
    const int a = rr / T, s = rr - a * T;
    const int64_t i = (int64_t)tile * 32 + a;
    const int* lp = p.nbr_in + list_col(tile, p.maxrows, T, a * T + s);
    if constexpr (MIX) {
      // the particle's own data does not depend on its replica: issue these
      // loads first so that they overlap the replica lookup
      const uint4 pi = p.pq[cur][i];
      const int cnt0 = pairs ? p.nnb_in[i * T + s] : 0;
      float v[3] = {0.f, 0.f, 0.f}, fo[3] = {0.f, 0.f, 0.f};
      if (s == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          v[c] = p.velf[c * nt + i];
          fo[c] = p.frcf[c * nt + i];
        }
      }
      // the first quad of list indices does not depend on the replica either
      // (slots past a replica's end have empty lists)
      int4 jq0 = make_int4(0, 0, 0, 0);
      if (cnt0 > 0) jq0 = __ldcs(reinterpret_cast<const int4*>(lp));
      const RepDev* R = &p.reps[p.tile_rep[tile]];
      const bool act = (tile - R->tile0) * 32 + a < R->n;
      const int cnt = act ? cnt0 : 0;
      float fx = 0.f, fy = 0.f, fz = 0.f, pe = 0.f, vir = 0.f;
      if (act) {
        const uint4* __restrict__ pq = p.pq[cur];
        if (energy)
          lane_sum_mix<true>(sh, pq, lp, gsz, cnt, jq0, pi, (int)pi.w * p.ntypes, R->fxs, fx, fy, fz, pe, vir);
        else
          lane_sum_mix<false>(sh, pq, lp, gsz, cnt, jq0, pi, (int)pi.w * p.ntypes, R->fxs, fx, fy, fz, pe, vir);
      }
      for (int o = T >> 1; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
        if (energy) {
          pe += __shfl_xor_sync(0xffffffffu, pe, o);
          vir += __shfl_xor_sync(0xffffffffu, vir, o);
        }
      }
      float e[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (act && s == 0) {
        const float im = p.inv_massf, hdt = 0.5f * p.dtf, m = p.massf;
        const float xi = R->xif, xia = R->xiaf;
        const float F[3] = {fx, fy, fz};
        float an[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float vf = v[c];
          const float ao = fo[c] * im;
          const float af = F[c] * im;
          an[c] = af;
          if (kick == KICK_VV) vf = fmaf(hdt, ao + af, vf);
          else if (kick == KICK_NH) vf = vf + hdt * ((ao + af) - (xi + xia) * vf) * (1.0f - hdt * xia);
          else if (kick == KICK_NH_EXACT) vf = (vf + hdt * (ao - xi * vf + af)) / (1.0f + hdt * xia);
          v[c] = vf;
          if (pairs) p.frcf[c * nt + i] = F[c];
          if (kick != KICK_NONE) p.velf[c * nt + i] = vf;
        }
        e[0] = 0.5f * pe;
        e[1] = 0.5f * m * fmaf(v[0], v[0], fmaf(v[1], v[1], v[2] * v[2]));
        e[2] = 0.5f * vir;
        e[3] = m * v[0];
        e[4] = m * v[1];
        e[5] = m * v[2];
        if (fuse) drift_mix(p, *R, i, cur, v, an, 0.0f, pi.w, nstep);
      }
      if (partials) {
        float2* out = reinterpret_cast<float2*>(part) + (int64_t)u * MD_NPART;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const ff t = warp_sum_ff(ff{e[k], 0.0f});
          if (lane == 0) out[k] = make_float2(t.hi, t.lo);
        }
      }
    } else {
      const RepDev* R = &p.reps[p.tile_rep[tile]];
      const bool act = (tile - R->tile0) * 32 + a < R->n;
      const int cnt = (act && pairs) ? p.nnb_in[i * T + s] : 0;
      double fx = 0, fy = 0, fz = 0, pe = 0, vir = 0;
      if (act) {
        const double4_32a* __restrict__ p4 = p.p4[cur];
        const double4_32a pi = p4[i];
        const int tb = (int)pi.w * p.ntypes;
        const double L = R->L, hL = 0.5 * R->L;
        for (int q = 0; q < cnt; ++q) {
          const int j = __ldcs(lp + list_at(0, q, gsz));
          const double4_32a pj = p4[j];
          double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
          if (dx > hL) dx -= L; else if (dx < -hL) dx += L;
          if (dy > hL) dy -= L; else if (dy < -hL) dy += L;
          if (dz > hL) dz -= L; else if (dz < -hL) dz += L;
          const double r2 = dx * dx + dy * dy + dz * dz;
          const int tt = tb + (int)pj.w;
          const double4_32a c = sh.tabd[tt];
          if (r2 < c.x) {
            const double ir2 = 1.0 / r2;
            const double s2 = c.y * ir2;
            const double s6 = s2 * s2 * s2;
            const double w = c.z * s6 * (s6 - 0.5);
            const double fr = w * ir2;
            fx += fr * dx; fy += fr * dy; fz += fr * dz;
            pe += c.w * s6 * (s6 - 1.0) - sh.vshd[tt];
            vir += w;
          }
        }
      }
      for (int o = T >> 1; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
        pe += __shfl_xor_sync(0xffffffffu, pe, o);
        vir += __shfl_xor_sync(0xffffffffu, vir, o);
      }
      double e[6] = {0, 0, 0, 0, 0, 0};
      if (act && s == 0) {
        const double im = p.inv_mass, hdt = 0.5 * p.dt, m = p.mass;
        const double xi = R->xi, xia = R->xi_a;
        const double F[3] = {fx, fy, fz};
        double v[3], an[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double vd = p.veld[c * nt + i];
          const double ao = p.frcd[c * nt + i] * im;
          const double ad = F[c] * im;
          an[c] = ad;
          if (kick == KICK_VV) vd = vd + hdt * (ao + ad);
          else if (kick == KICK_NH) vd = vd + hdt * ((ao + ad) - (xi + xia) * vd) * (1.0 - hdt * xia);
          else if (kick == KICK_NH_EXACT) vd = (vd + hdt * (ao - xi * vd + ad)) / (1.0 + hdt * xia);
          v[c] = vd;
          if (pairs) p.frcd[c * nt + i] = F[c];
          if (kick != KICK_NONE) p.veld[c * nt + i] = vd;
        }
        e[0] = 0.5 * pe;
        e[1] = 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        e[2] = 0.5 * vir;
        e[3] = m * v[0];
        e[4] = m * v[1];
        e[5] = m * v[2];
        if (fuse) drift_f64(p, *R, i, cur, v, an, 0.0, nstep);
      }
      if (partials) {
        double* out = part + (int64_t)u * MD_NPART;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const double t = warp_sum(e[k]);
          if (lane == 0) out[k] = t;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ prune

// Accepted entries pass through a 4-deep shift register (b1, b2, b3 plus the
// new one); every fourth entry completes a quad, stored with one 16-byte store.
__device__ __forceinline__ void list_push(int32_t* col, int gsz, int maxrows, int& k, int& b1, int& b2, int& b3,
                                          int j) {
  if ((k & 3) == 3 && k < maxrows)
    *reinterpret_cast<int4*>(col + (int64_t)(k >> 2) * 4 * gsz) = make_int4(b1, b2, b3, j);
  b1 = b2;
  b2 = b3;
  b3 = j;
  ++k;
}

// Store the last, partial quad of a column (k % 4 entries in b1..b3).
__device__ __forceinline__ void list_flush(int32_t* col, int gsz, int maxrows, int k, int b1, int b2, int b3) {
  const int r = k & 3;
  if (r == 0 || k - r >= maxrows) return;
  const int4 v = r == 1 ? make_int4(b3, 0, 0, 0) : (r == 2 ? make_int4(b2, b3, 0, 0) : make_int4(b1, b2, b3, 0));
  *reinterpret_cast<int4*>(col + (int64_t)(k >> 2) * 4 * gsz) = v;
}

// Inner list from the outer one: every lane keeps, in order, the entries of
// its outer column that now lie within r_c,ab + skin, and the particle's
// position becomes the reference of the next prune trigger. A replica is
// pruned before force step `epoch` if one of its particles asked for it
// during the drift to that step, or if its outer list was just rebuilt;
// epochs only grow, so no flag has to be cleared (no race between phases).
template <bool MIX>
__device__ void prune_phase(const KParams& p, Shared& sh, int cur, int64_t epoch) {
  const int T = p.T;
  const int gsz = 32 * T;
  const int lane = threadIdx.x & 31;
  const int nunits = p.ntiles * T;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAnd(&p.ctl->pending, ~MD_FLAG_PRUNE);
    p.ctl->prunes += 1;
  }
  // the force phase's SM-local layout: neighbouring tiles, whose gathers
  // overlap, are pruned on one SM and share its L1
  int64_t ub, ue, us;
  sm_share(sh, nunits, (int)(blockDim.x >> 5), (int)(threadIdx.x >> 5), &ub, &ue, &us);
  for (int u = (int)ub; u < ue; u += (int)us) {
    const int tile = u / T;
    const int w = u - tile * T;
    const int rr = w * 32 + lane;
    const int a = rr / T, s = rr - a * T;
    const int64_t i = (int64_t)tile * 32 + a;
    const RepDev& R = p.reps[p.tile_rep[tile]];
    if ((tile - R.tile0) * 32 + a >= R.n) continue;
    // only replicas with a particle past half the inner skin, or a new outer list
    if (R.prune_epoch != epoch && R.rebuild_epoch != epoch) continue;
    const int64_t off = list_col(tile, p.maxrows, T, a * T + s);
    const int* lo = p.nbr + off;
    int* li = p.nbr_in + off;
    const int cnt = p.nnb[i * T + s];
    int k = 0;
    int b1 = 0, b2 = 0, b3 = 0;  // quad shift register of the list writer
    if constexpr (MIX) {
      const uint4* __restrict__ pq = p.pq[cur];
      const uint4 pi = pq[i];
      const int tb = (int)pi.w * p.ntypes;
      const float sc = R.fxs;
      // a quad of outer entries per iteration: one 16-byte index load, issued
      // a quad ahead, and four position gathers in flight together
      const int64_t qstride = 4 * (int64_t)gsz;
      int4 jq = make_int4(0, 0, 0, 0);
      if (cnt > 0) jq = __ldcs(reinterpret_cast<const int4*>(lo));
      for (int q = 0; q < cnt; q += 4) {
        const int m = min(4, cnt - q);
        const int j[4] = {jq.x, jq.y, jq.z, jq.w};
        uint4 pj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) pj[u] = pq[u < m ? j[u] : j[0]];
        if (q + 4 < cnt) jq = __ldcs(reinterpret_cast<const int4*>(lo + (int64_t)((q + 4) >> 2) * qstride));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float dx = (float)(int)(pi.x - pj[u].x) * sc;
          const float dy = (float)(int)(pi.y - pj[u].y) * sc;
          const float dz = (float)(int)(pi.z - pj[u].z) * sc;
          if (u < m && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < sh.rli2f[tb + (int)pj[u].w])
            list_push(li, gsz, p.maxrows, k, b1, b2, b3, j[u]);
        }
      }
      if (s == 0) p.xbq_in[i] = pi;
    } else {
      const double4_32a* __restrict__ p4 = p.p4[cur];
      const double4_32a pi = p4[i];
      const int tb = (int)pi.w * p.ntypes;
      const double L = R.L, hL = 0.5 * R.L;
      for (int q = 0; q < cnt; ++q) {
        const int j = __ldcs(lo + list_at(0, q, gsz));
        const double4_32a pj = p4[j];
        double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        if (dx > hL) dx -= L; else if (dx < -hL) dx += L;
        if (dy > hL) dy -= L; else if (dy < -hL) dy += L;
        if (dz > hL) dz -= L; else if (dz < -hL) dz += L;
        if (dx * dx + dy * dy + dz * dz < sh.rli2d[tb + (int)pj.w])
          list_push(li, gsz, p.maxrows, k, b1, b2, b3, j);
      }
      if (s == 0) p.xbd_in[i] = pi;
    }
    list_flush(li, gsz, p.maxrows, k, b1, b2, b3);
    p.nnb_in[i * T + s] = k;
  }
}

// ------------------------------------------------------------------ resampling

// Draw Maxwell-Boltzmann velocities (step 1 of the flow chart in Sec.
// "Statistical temperature bath") and store per-tile sums of v and v^2.
// One warp per tile.
template <bool MIX>
__device__ void resample_draw_phase(const KParams& p, uint64_t draw, double* part) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nt = p.ntot;
  for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < p.ntiles; tile += nw) {
    const RepDev& R = p.reps[p.tile_rep[tile]];
    const int64_t i = tile * 32 + lane;
    const bool act = i - R.off < R.n;
    double g[3] = {0, 0, 0};
    if (act) gauss3(p.seed, draw, (uint32_t)(p.gid[i] - R.out0), g);
    if (p.ndim == 2) g[2] = 0.0;  // particles stay in their plane: v_z = 0
    if constexpr (MIX) {
      float e[4] = {0.f, 0.f, 0.f, 0.f};
      if (act) {
        const float sd = sqrtf((float)R.T_target * p.inv_massf);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float v = sd * (float)g[c];
          p.velf[c * nt + i] = v;
          e[c] = v;
          e[3] = fmaf(v, v, e[3]);
        }
      }
      float2* out = reinterpret_cast<float2*>(part) + tile * MD_NPART;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const ff w = warp_sum_ff(ff{e[k], 0.0f});
        if (lane == 0) out[k] = make_float2(w.hi, w.lo);
      }
    } else {
      double e[4] = {0, 0, 0, 0};
      if (act) {
        const double sd = sqrt(R.T_target * p.inv_mass);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double v = sd * g[c];
          p.veld[c * nt + i] = v;
          e[c] = v;
          e[3] += v * v;
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double w = warp_sum(e[k]);
        if (lane == 0) part[tile * MD_NPART + k] = w;
      }
    }
  }
}

// ------------------------------------------------------------------ reductions

__device__ __noinline__ void reduce_scalars(const KParams& p, RepDev& R, int64_t r, const double* acc, int mode,
                                            int64_t step, bool log_now, int64_t log_idx, bool nh);

// Sum of the partial records [u0, u0 + nu) (fixed order): thread-strided
// float-float (mixed) or double accumulation, warp trees, then the CTA's
// warps in order; the warps' sums are added by lanes 0..5 of warp 0, one
// quantity each (each sum in the same order as one thread adding them one
// after the other). Thread 0 receives the six totals in acc.
template <bool MIX>
__device__ void sum_records(Shared& sh, const double* part, int64_t u0, int64_t nu, double* acc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int64_t B = blockDim.x;
  double tot = 0.0;  // lane k < 6 of warp 0: total of quantity k
  if constexpr (MIX) {
    ff a[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = ff{0.f, 0.f};
    const float2* q0 = reinterpret_cast<const float2*>(part);
    for (int64_t t = threadIdx.x; t < nu; t += B) {
      const float2* q = q0 + (u0 + t) * MD_NPART;
#pragma unroll
      for (int k = 0; k < 6; ++k) a[k] = ff_add(a[k], ff{q[k].x, q[k].y});
    }
    float2* red = reinterpret_cast<float2*>(&sh.red[0][0]);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      a[k] = warp_sum_ff(a[k]);
      if (lane == 0) red[warp * MD_NPART + k] = make_float2(a[k].hi, a[k].lo);
    }
    __syncthreads();
    if (warp == 0 && lane < 6) {
      ff u = {red[lane].x, red[lane].y};
      for (int w = 1; w < nwarp; ++w) u = ff_add(u, ff{red[w * MD_NPART + lane].x, red[w * MD_NPART + lane].y});
      tot = (double)u.hi + (double)u.lo;
    }
  } else {
    double a[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = 0.0;
    for (int64_t t = threadIdx.x; t < nu; t += B) {
      const double* q = part + (u0 + t) * MD_NPART;
#pragma unroll
      for (int k = 0; k < 6; ++k) a[k] += q[k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      a[k] = warp_sum(a[k]);
      if (lane == 0) sh.red[warp][k] = a[k];
    }
    __syncthreads();
    if (warp == 0 && lane < 6) {
      double u = sh.red[0][lane];
      for (int w = 1; w < nwarp; ++w) u += sh.red[w][lane];
      tot = u;
    }
  }
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double v = __shfl_sync(0xffffffffu, tot, k);
      if (lane == 0) acc[k] = v;
    }
  }
  __syncthreads();
}

// Per-replica totals of the partial records (upt records per tile) and the
// scalar updates of `mode`. One CTA per replica, unless some replica spans
// more than four chunks (p.red2): then chunks of red_tiles tiles are summed
// by separate CTAs, then, after a grid barrier, one CTA per replica adds its
// chunk sums in chunk order. Both orders are fixed, so results are
// reproducible. Returns false after a barrier timeout.
template <bool MIX>
__device__ bool reduce_phase(const KParams& p, Shared& sh, const double* part, int upt, int mode, int64_t step,
                             bool log_now, int64_t log_idx) {
  const bool nh = (p.kind == MD_KIND_NH || p.kind == MD_KIND_NH_EXACT) && p.op == MD_OP_STEPS;
  double acc[6];
  if (!p.red2) {
    for (int r = blockIdx.x; r < p.nrep; r += gridDim.x) {
      RepDev& R = p.reps[r];
      sum_records<MIX>(sh, part, (int64_t)R.tile0 * upt, (int64_t)R.ntiles * upt, acc);
      if (threadIdx.x == 0) reduce_scalars(p, R, r, acc, mode, step, log_now, log_idx, nh);
      __syncthreads();
    }
    return true;
  }
  for (int64_t g = blockIdx.x; g < p.nred; g += gridDim.x) {
    const int2 rc = p.redmap[g];
    const RepDev& R = p.reps[rc.x];
    const int t0 = rc.y * p.red_tiles;
    const int nt = min(p.red_tiles, R.ntiles - t0);
    sum_records<MIX>(sh, part, (int64_t)(R.tile0 + t0) * upt, (int64_t)nt * upt, acc);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < 6; ++k) p.redpart[g * MD_NPART + k] = acc[k];
    }
  }
  if (grid_sync(p, sh, 17) < 0) return false;
  // level 2: one CTA per replica sums the replica's chunk sums as FP64
  // records (thread-strided, warp trees, warps in order: a fixed order)
  for (int r = blockIdx.x; r < p.nrep; r += gridDim.x) {
    const int2 rr = p.redrep[r];
    sum_records<false>(sh, p.redpart, rr.x, rr.y, acc);
    if (threadIdx.x == 0) reduce_scalars(p, p.reps[r], r, acc, mode, step, log_now, log_idx, nh);
  }
  __syncthreads();
  return true;
}

__device__ __noinline__ void reduce_scalars(const KParams& p, RepDev& R, int64_t r, const double* acc, int mode,
                                            int64_t step, bool log_now, int64_t log_idx, bool nh) {
  const double n = (double)R.n, X = (double)p.ndim * n, dt = p.dt;
  if (mode == RED_LOG) {
    // the log record of an NVE step reduced after the launch's last step: the
    // same values as the record written at the step, the replica untouched
    const double pe = acc[0], ke = acc[1];
    ThermoDev th;
    th.step = step;
    th.T = 2.0 * ke / X;
    th.pe_per_n = pe / n;
    th.ke_per_n = ke / n;
    th.etot_per_n = (ke + pe) / n;
    th.virial = acc[2];
    th.h_nh = ke + pe + 0.0;
    th.xi = 0.0;
    if (p.thermo) p.thermo[log_idx * p.nrep + r] = th;
    return;
  }
  if (mode == RED_RESAMPLE) {
    const double mx = acc[0] / n, my = acc[1] / n, mz = acc[2] / n;
    const double S = acc[3] - n * (mx * mx + my * my + mz * mz);
    const double sc = (S > 0.0) ? sqrt(X * R.T_target / (p.mass * S)) : 0.0;
    R.vmean[0] = mx; R.vmean[1] = my; R.vmean[2] = mz;
    R.vscale = sc;
    R.vmeanf[0] = (float)mx; R.vmeanf[1] = (float)my; R.vmeanf[2] = (float)mz;
    R.vscalef = (float)sc;
    R.ke = 0.5 * p.mass * sc * sc * S;
    R.px = R.py = R.pz = 0.0;
  } else {
    if (mode == RED_FORCES || mode == RED_STEP) { R.pe = acc[0]; R.vir = acc[2]; }
    R.ke = acc[1];
    R.px = acc[3]; R.py = acc[4]; R.pz = acc[5];
    if (nh) {
      const double gnew = (2.0 * R.ke - X * R.T_target) / R.Q;
      if (mode == RED_STEP || mode == RED_STEP_KE) {
        R.xi = R.xi + 0.5 * dt * (R.g + gnew);  // Eq. (FoxAndersen_ydottplush)
        R.lns = R.lns_next;
      }
      R.g = gnew;
      R.xi_a = R.xi + dt * R.g;                              // Eq. (Noseupdate_xiapprox)
      R.lns_next = R.lns + R.xi * dt + 0.5 * R.g * dt * dt;  // Eq. (Noseupdate_lns)
      R.xif = (float)R.xi;
      R.xiaf = (float)R.xi_a;
    }
  }
  if (log_now && p.thermo) {
    ThermoDev th;
    th.step = step;
    th.T = 2.0 * R.ke / X;
    th.pe_per_n = R.pe / n;
    th.ke_per_n = R.ke / n;
    th.etot_per_n = (R.ke + R.pe) / n;
    th.virial = R.vir;
    th.h_nh = R.ke + R.pe + (nh ? 0.5 * R.Q * R.xi * R.xi + X * R.T_target * R.lns : 0.0);
    th.xi = nh ? R.xi : 0.0;
    p.thermo[log_idx * p.nrep + r] = th;
  }
}

// ------------------------------------------------------------------ rebuild

template <bool MIX>
__device__ __forceinline__ void cell_of_pos(const KParams& p, const RepDev& R, int64_t i, int cur, int& cx, int& cy,
                                            int& cz) {
  const int nc = R.nc;
  if constexpr (MIX) {
    const uint4 q = p.pq[cur][i];
    cx = (int)(((uint64_t)q.x * (uint64_t)nc) >> 32);
    cy = (int)(((uint64_t)q.y * (uint64_t)nc) >> 32);
    cz = (int)(((uint64_t)q.z * (uint64_t)nc) >> 32);
  } else {
    const double4_32a x = p.p4[cur][i];
    const double s = (double)nc * R.invL;
    cx = min(max((int)(x.x * s), 0), nc - 1);
    cy = min(max((int)(x.y * s), 0), nc - 1);
    cz = min(max((int)(x.z * s), 0), nc - 1);
  }
}

// Block-wide exclusive scan of one int per thread.
__device__ int block_exclusive_scan(Shared& sh, int v, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh.scan[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nwarp ? sh.scan[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nwarp) sh.scan[lane] = w;
  }
  __syncthreads();
  const int before = (warp > 0 ? sh.scan[warp - 1] : 0) + x - v;
  *total = sh.scan[nwarp - 1];
  __syncthreads();
  return before;
}

// Pair list radius^2 of one particle's row for a candidate whose staged word
// carries its type in the top two bits (NT2: at most two types).
template <bool NT2>
__device__ __forceinline__ float lim_of(float l0, float l1, float l2, float l3, uint32_t w) {
  if constexpr (NT2) {
    return w >= (1u << 30) ? l1 : l0;
  } else {
    const uint32_t t = w >> 30;
    const float a = (t & 1u) ? l1 : l0, b = (t & 1u) ? l3 : l2;
    return (t & 2u) ? b : a;
  }
}

// First pass over one chunk of staged candidates q0, q0 + T, ..., nq of them
// (nq <= 32, T = 2^tsh), mixed path: each is tested against its own pair
// radius (selected by its type bits) and the hits are marked in a bit mask
// (bit u: candidate q0 + u T).
// REL: staged FP32 coordinates relative to the group's reference particle;
// otherwise staged fixed-point words and exact integer differences.
template <bool REL, bool NT2>
__device__ __forceinline__ unsigned chunk_mask(uint32_t st_s, int q0, int nq, int tsh, float x, float y, float z,
                                               const uint4& pq, float sc, float l0, float l1, float l2, float l3) {
  unsigned mask = 0u;
#pragma unroll 4
  for (int u = 0; u < nq; ++u) {
    uint32_t c0, c1, c2, c3;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(c0), "=r"(c1), "=r"(c2), "=r"(c3)
                 : "r"(st_s + 16u * (uint32_t)(q0 + (u << tsh))));
    float dx, dy, dz;
    if constexpr (REL) {
      dx = x - __uint_as_float(c0);
      dy = y - __uint_as_float(c1);
      dz = z - __uint_as_float(c2);
    } else {
      dx = (float)(int)(pq.x - c0) * sc;
      dy = (float)(int)(pq.y - c1) * sc;
      dz = (float)(int)(pq.z - c2) * sc;
    }
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    // hit: r2 - lim < 0 (the sign of a rounded difference is that of the
    // exact one, and equal values give +0), shifted in from the top
    const float d = r2 - lim_of<NT2>(l0, l1, l2, l3, c3);
    mask = (mask >> 1) | (__float_as_uint(d) & 0x80000000u);
  }
  return nq > 0 ? mask >> (32 - nq) : 0u;  // candidate u at bit u
}

// Scan of one run of staged candidates [qs, qe) for column `sl` of one
// particle, mixed path: the candidates qs + sl, qs + sl + T, ... (T = 2^tsh)
// in chunks of up to 32. The first pass (chunk_mask) marks the hits; the
// particle itself is then cleared by index, and a second pass stores the
// marked candidates in order, reading only their slot words.
template <bool REL, bool NT2>
__device__ __forceinline__ int scan_run_mix(uint32_t st_s, int qs, int qe, int tsh, float x, float y, float z,
                                            const uint4& pq, float sc, float l0, float l1, float l2, float l3,
                                            int own_q, int32_t* col, int gsz, int maxrows, int k, int& b1, int& b2,
                                            int& b3) {
  const int T = 1 << tsh;
  for (int q0 = qs; q0 < qe; q0 += 32 << tsh) {
    const int nq = min(32, (qe - q0 + T - 1) >> tsh);
    unsigned mask = chunk_mask<REL, NT2>(st_s, q0, nq, tsh, x, y, z, pq, sc, l0, l1, l2, l3);
    const int d = own_q - q0;
    if (d >= 0 && (d & (T - 1)) == 0 && (d >> tsh) < nq) mask &= ~(1u << (d >> tsh));
    while (mask) {
      const int u = __ffs(mask) - 1;
      mask &= mask - 1u;
      uint32_t w;
      asm volatile("ld.shared.b32 %0, [%1];" : "=r"(w) : "r"(st_s + 16u * (uint32_t)(q0 + (u << tsh)) + 12u));
      list_push(col, gsz, maxrows, k, b1, b2, b3, (int)(w & 0x3fffffffu));
    }
  }
  return k;
}

// Distance from a particle at fraction f of its cell's width (f in [0, w)) to
// the nearest face of the cell o cells away along one axis (0 for its own).
__device__ __forceinline__ float face_dist(int o, float f, float w) {
  return o < 0 ? f + (float)(-o - 1) * w : (o > 0 ? (w - f) + (float)(o - 1) * w : 0.0f);
}

// All runs of one particle, mixed path: each of the (2 nr + 1)^2 rows of its
// neighbourhood that comes within the largest list radius (lcut, with a
// rounding margin), trimmed at both ends to the cells that do; or, for a
// replica without cells (nc == 0), the whole staged replica. u_own: staged
// cell of the particle's own cell; (fx, fy, fz): its position inside that
// cell. Returns the entries found; b1..b3 hold the writer's partial quad.
template <bool REL, bool NT2>
__device__ __forceinline__ int scan_particle_mix(uint32_t st_s, const int* s_ub, int ncand, int nc, int nr, int UX,
                                                 int UY, int u_own, float fx, float fy, float fz, float wc,
                                                 float lcut, int sl, int tsh, float x, float y, float z,
                                                 const uint4& pq, float sc, float l0, float l1, float l2, float l3,
                                                 int own_q, int32_t* col, int gsz, int maxrows, int& b1, int& b2,
                                                 int& b3) {
  if (nc == 0)
    return scan_run_mix<REL, NT2>(st_s, sl, ncand, tsh, x, y, z, pq, sc, l0, l1, l2, l3, own_q, col, gsz, maxrows, 0,
                                  b1, b2, b3);
  // distances along x to the cells at the ends of a row (nr <= 2)
  const float em2 = fx + wc, em1 = fx, ep1 = wc - fx, ep2 = (wc - fx) + wc;
  int k = 0;
  for (int oz = -nr; oz <= nr; ++oz) {
    const float ez = face_dist(oz, fz, wc);
    for (int oy = -nr; oy <= nr; ++oy) {
      const float ey = face_dist(oy, fy, wc);
      const float d2 = fmaf(ey, ey, ez * ez);
      if (d2 >= lcut) continue;  // the whole row is out of reach
      int xl = -nr, xh = nr;
      if (xl == -2 && fmaf(em2, em2, d2) >= lcut) xl = -1;
      if (xl == -1 && fmaf(em1, em1, d2) >= lcut) xl = 0;
      if (xh == 2 && fmaf(ep2, ep2, d2) >= lcut) xh = 1;
      if (xh == 1 && fmaf(ep1, ep1, d2) >= lcut) xh = 0;
      const int us0 = u_own + (oz * UY + oy) * UX;  // the row's cell in the particle's own column
      k = scan_run_mix<REL, NT2>(st_s, s_ub[us0 + xl] + sl, s_ub[us0 + xh + 1], tsh, x, y, z, pq, sc, l0, l1, l2,
                                 l3, own_q, col, gsz, maxrows, k, b1, b2, b3);
    }
  }
  return k;
}

// One particle on two lanes (lane h of the pair, pmask the pair's lanes), T =
// 1, mixed path, a replica with cells: lane h takes the rows h, h + 2, ... of
// the particle's neighbourhood (row order as in scan_particle_mix, the same
// culling). In each round both lanes test one chunk of up to 32 candidates of
// their current row, trade their hit counts, and store their hits one after
// the other (lane 0's first) with 4-byte stores, so the column fills without
// gaps, in an order fixed by the data. Returns the column's length (the same
// on both lanes).
template <bool REL, bool NT2>
__device__ __forceinline__ int scan_particle_pair_mix(uint32_t st_s, const int* s_ub, int nr, int UX, int UY,
                                                      int u_own, float fx, float fy, float fz, float wc, float lcut,
                                                      int h, unsigned pmask, float x, float y, float z,
                                                      const uint4& pq, float sc, float l0, float l1, float l2,
                                                      float l3, int own_q, int32_t* col, int gsz, int maxrows) {
  const float em2 = fx + wc, em1 = fx, ep1 = wc - fx, ep2 = (wc - fx) + wc;
  int oy = -nr + h - 2, oz = -nr;  // row cursor: advanced by two rows before use
  int q0 = 0, qe = 0;
  // move to this lane's next row that has candidates within reach
  auto next_row = [&]() -> bool {
    while (true) {
      oy += 2;
      if (oy > nr) {
        oy -= 2 * nr + 1;
        ++oz;
      }
      if (oz > nr) return false;
      const float ez = face_dist(oz, fz, wc), ey = face_dist(oy, fy, wc);
      const float d2 = fmaf(ey, ey, ez * ez);
      if (d2 >= lcut) continue;
      int xl = -nr, xh = nr;
      if (xl == -2 && fmaf(em2, em2, d2) >= lcut) xl = -1;
      if (xl == -1 && fmaf(em1, em1, d2) >= lcut) xl = 0;
      if (xh == 2 && fmaf(ep2, ep2, d2) >= lcut) xh = 1;
      if (xh == 1 && fmaf(ep1, ep1, d2) >= lcut) xh = 0;
      const int us0 = u_own + (oz * UY + oy) * UX;
      q0 = s_ub[us0 + xl];
      qe = s_ub[us0 + xh + 1];
      if (q0 < qe) return true;
    }
  };
  bool have = next_row();
  int k = 0;
  while (true) {
    unsigned mask = 0u;
    const int base = q0;
    if (have) {
      const int nq = min(32, qe - q0);
      mask = chunk_mask<REL, NT2>(st_s, q0, nq, 0, x, y, z, pq, sc, l0, l1, l2, l3);
      const int d = own_q - q0;
      if (d >= 0 && d < nq) mask &= ~(1u << d);
      q0 += nq;
      if (q0 >= qe) have = next_row();
    }
    const int c = __popc(mask);
    const int other = __shfl_xor_sync(pmask, (c << 1) | (have ? 1 : 0), 1);
    int e = k + (h ? (other >> 1) : 0);
    while (mask) {
      const int u = __ffs(mask) - 1;
      mask &= mask - 1u;
      uint32_t w;
      asm volatile("ld.shared.b32 %0, [%1];" : "=r"(w) : "r"(st_s + 16u * (uint32_t)(base + u) + 12u));
      if (e < maxrows) col[list_at(0, e, gsz)] = (int)(w & 0x3fffffffu);
      ++e;
    }
    k += c + (other >> 1);
    if (!have && !(other & 1)) return k;
  }
}

// B6: Verlet lists, radius r_c,ab + skin, built per GROUP of up to GX x GY x
// GZ neighbouring cells (one CTA per group). Cells are at least r_list / nr
// wide (nr = 2: half-width cells, or nr = 1), so every partner of a particle
// lies in the (2 nr + 1)^3 cells around its own. The union of the cells
// around the group, (GX + 2nr) x (GY + 2nr) x (GZ + 2nr) cells with x fastest,
// is staged in shared memory once; each particle of the group then scans the
// (2 nr + 1)^2 rows of its own neighbourhood, each a run of (2 nr + 1)
// consecutive staged cells, leaving out rows, and cells at the ends of rows,
// that lie wholly beyond its largest list radius (with half-width cells that
// skips the corners of the 5 x 5 x 5 block, so far fewer candidates are tested
// than in 27 cells of full width). List column s takes the run entries s,
// s + T, s + 2T, ... of every row. A replica too small for cells is one group
// whose single staged "cell" is the whole replica.
template <bool MIX>
__device__ __forceinline__ void build_lists(const KParams& p, Shared& sh, int cur) {
  const int T = p.T, gsz = 32 * T;
  extern __shared__ __align__(32) unsigned char dyn[];
  const int stage_cap = p.stage_cap;
  double4_32a* st_d = reinterpret_cast<double4_32a*>(dyn);  // FP64: positions, then slots
  int32_t* st_j = reinterpret_cast<int32_t*>(dyn + (size_t)stage_cap * 32);
  float4* st_f = reinterpret_cast<float4*>(dyn);
  uint4* st_u = reinterpret_cast<uint4*>(dyn);
  // union cells: first slot, staged base; group rows (ly, lz): first slot,
  // particle count prefix
  __shared__ int s_ulo[MD_UNION_MAX], s_ub[MD_UNION_MAX + 1];
  __shared__ int s_plo[MD_ROWS_MAX], s_pb[MD_ROWS_MAX + 1];
  __shared__ int s_ref;
  // groups, then one pseudo-group per all-pairs replica; grid-strided, so
  // that a rebuild of a few replicas still spreads over every SM
  const int64_t ngrp_all = p.ngroups + p.nrep;
  for (int64_t g = blockIdx.x; g < ngrp_all; g += gridDim.x) {
    int r, lg = 0;
    if (g < p.ngroups) {
      const int2 gi = p.grp[g];
      r = gi.x;
      lg = gi.y;
    } else {
      r = (int)(g - p.ngroups);
    }
    const RepDev& R = p.reps[r];
    if (!R.doing_rebuild) continue;
    if (g >= p.ngroups && R.nc != 0) continue;
    const int nc = R.nc;
    const int nr = R.nr;  // cells of the stencil on each side
    const int GX = R.gx, GY = R.gy, GZ = R.gz;
    const int UX = GX + 2 * nr, UY = GY + 2 * nr, UZ = GZ + 2 * nr;
    int nu, nrows, cx = 0, cy = 0, cz = 0;
    if (nc > 0) {
      const int ngx = (nc + GX - 1) / GX, ngy = (nc + GY - 1) / GY;
      cx = (lg % ngx) * GX;
      cy = ((lg / ngx) % ngy) * GY;
      cz = (lg / (ngx * ngy)) * GZ;
      const int gxe = min(GX, nc - cx), gye = min(GY, nc - cy), gze = min(GZ, nc - cz);
      nu = UX * UY * UZ;
      nrows = GY * GZ;
      for (int t = threadIdx.x; t < nu; t += blockDim.x) {
        const int ux = t % UX, uy = (t / UX) % UY, uz = t / (UX * UY);
        const int q = (((cz - nr + uz + 4 * nc) % nc) * nc + (cy - nr + uy + 4 * nc) % nc) * nc +
                      (cx - nr + ux + 4 * nc) % nc;
        const int lo = p.cstart[R.cs0 + q];
        s_ulo[t] = lo;
        s_ub[t] = p.cstart[R.cs0 + q + 1] - lo;  // count for now, prefix below
      }
      for (int t = threadIdx.x; t < nrows; t += blockDim.x) {
        const int ly = t % GY, lz = t / GY;
        int lo = 0, n = 0;
        if (ly < gye && lz < gze) {
          const int c0 = ((cz + lz) * nc + (cy + ly)) * nc + cx;  // cells cx .. cx+gxe-1 are consecutive
          lo = p.cstart[R.cs0 + c0];
          n = p.cstart[R.cs0 + c0 + gxe] - lo;
        }
        s_plo[t] = lo;
        s_pb[t] = n;
      }
    } else {
      nu = 1;
      nrows = 1;
      if (threadIdx.x == 0) {
        s_ulo[0] = (int)R.off;
        s_ub[0] = R.n;
        s_plo[0] = (int)R.off;
        s_pb[0] = R.n;
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // exclusive prefix of the staged-cell counts: lane l sums its chunk of
      // per consecutive counts (nu <= 32 * per), a warp scan, then the chunk
      const int lane = threadIdx.x;
      const int per = (nu + 31) / 32;
      const int b0 = min(lane * per, nu), b1 = min(b0 + per, nu);
      int sum = 0;
      for (int t = b0; t < b1; ++t) sum += s_ub[t];
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      int run = incl - sum;
      for (int t = b0; t < b1; ++t) {
        const int c = s_ub[t];
        s_ub[t] = run;
        run += c;
      }
      if (lane == 31) s_ub[nu] = incl;
      if (lane == 0) {
        int m = 0, ref = -1;
        for (int t = 0; t < nrows; ++t) {
          const int k = s_pb[t];
          if (ref < 0 && k > 0) ref = s_plo[t];
          s_pb[t] = m;
          m += k;
        }
        s_pb[nrows] = m;
        s_ref = ref;
      }
    }
    __syncthreads();
    const int ncand = s_ub[nu];
    const int npart = s_pb[nrows];
    if (npart == 0) continue;  // empty group: no particle needs a list
    if (ncand > stage_cap) {
      // more candidates than the staging area holds: flag and skip (the host regrows it)
      if (threadIdx.x == 0) raise_flag(p, MD_FLAG_OVERFLOW);
      __syncthreads();
      continue;
    }
    // mixed path with enough cells per edge: stage coordinates relative to a
    // particle of the group as FP32 (exact integer differences, converted once
    // per candidate). Every staged candidate then lies within (G + nr) cells
    // of the reference along each axis, less than half the box, so
    // differences of relative coordinates are the minimum image; the list
    // test has a whole skin of margin, so FP32 is ample. Otherwise the
    // fixed-point words are staged and every test takes the exact integer
    // difference.
    const bool rel = MIX && nc >= 2 * (GX + nr) + 1 && nc >= 2 * (GY + nr) + 1 && nc >= 2 * (GZ + nr) + 1;
    uint4 ref = make_uint4(0u, 0u, 0u, 0u);
    if constexpr (MIX) ref = p.pq[cur][s_ref];
    {
      constexpr int STAGE_U = 2;
      const uint4* __restrict__ pqc = p.pq[cur];
      const double4_32a* __restrict__ p4c = p.p4[cur];
      for (int t0 = threadIdx.x; t0 < ncand; t0 += STAGE_U * blockDim.x) {
        int src[STAGE_U];
#pragma unroll
        for (int u = 0; u < STAGE_U; ++u) {
          const int t = t0 + u * (int)blockDim.x;
          src[u] = -1;
          if (t < ncand) {
            int lo = 0, hi = nu;  // s_ub[lo] <= t < s_ub[hi]
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (s_ub[mid] <= t) lo = mid; else hi = mid;
            }
            src[u] = s_ulo[lo] + (t - s_ub[lo]);
          }
        }
        if constexpr (MIX) {
          uint4 q[STAGE_U];
#pragma unroll
          for (int u = 0; u < STAGE_U; ++u)
            if (src[u] >= 0) q[u] = pqc[src[u]];
          const float sc = R.fxs;
#pragma unroll
          for (int u = 0; u < STAGE_U; ++u) {
            if (src[u] < 0) continue;
            const int t = t0 + u * (int)blockDim.x;
            const unsigned w = (q[u].w << 30) | (unsigned)src[u];
            if (rel)
              st_f[t] = make_float4((float)(int)(q[u].x - ref.x) * sc, (float)(int)(q[u].y - ref.y) * sc,
                                    (float)(int)(q[u].z - ref.z) * sc, __int_as_float((int)w));
            else
              st_u[t] = make_uint4(q[u].x, q[u].y, q[u].z, w);
          }
        } else {
          double4_32a q[STAGE_U];
#pragma unroll
          for (int u = 0; u < STAGE_U; ++u)
            if (src[u] >= 0) q[u] = p4c[src[u]];
#pragma unroll
          for (int u = 0; u < STAGE_U; ++u) {
            if (src[u] < 0) continue;
            const int t = t0 + u * (int)blockDim.x;
            st_d[t] = q[u];
            st_j[t] = src[u];
          }
        }
      }
    }
    __syncthreads();
    // scan: T threads per particle, particles of the group in row order; with
    // T = 1 and at most half as many particles as threads (mixed path, cells),
    // two lanes per particle (scan_particle_pair_mix)
    const bool pair = MIX && T == 1 && nc > 0 && 2 * npart <= (int)blockDim.x;
    const int lanes = pair ? 2 : T;
    const int per_pass = (int)blockDim.x / lanes;
    const int sl = pair ? 0 : (int)threadIdx.x % T;
    const int h = pair ? (int)(threadIdx.x & 1u) : 0;
    const int side = 2 * nr + 1;  // stencil cells per axis
    for (int pidx = (int)threadIdx.x / lanes; pidx < npart && (int)threadIdx.x < per_pass * lanes;
         pidx += per_pass) {
      int row = 0;
      while (pidx >= s_pb[row + 1]) ++row;
      const int64_t i = s_plo[row] + (pidx - s_pb[row]);
      const int ly = row % GY, lz = row / GY;
      // the particle's own cell (the binning of B1) and its position inside it
      int ccx = 0, ccy = 0, ccz = 0;
      if (nc > 0) cell_of_pos<MIX>(p, R, i, cur, ccx, ccy, ccz);
      const int lx = ccx - cx;
      // own staged position (each particle is a candidate of its own cell)
      const int own_u = nc > 0 ? ((lz + nr) * UY + (ly + nr)) * UX + (lx + nr) : 0;
      const int own_q = s_ub[own_u] + (int)(i - s_ulo[own_u]);
      int32_t* lb = p.nbr + list_col(i >> 5, p.maxrows, T, (int)(i & 31) * T + sl);
      int k = 0;
      int b1 = 0, b2 = 0, b3 = 0;  // quad shift register of the list writer
      const int nruns = nc > 0 ? side * side : 1;
      if constexpr (MIX) {
        const uint4 pq_i = p.pq[cur][i];
        const float sc = R.fxs;
        const float x = (float)(int)(pq_i.x - ref.x) * sc;
        const float y = (float)(int)(pq_i.y - ref.y) * sc;
        const float z = (float)(int)(pq_i.z - ref.z) * sc;
        // this particle's row of pair list radii^2, by partner type
        const float* rl = sh.rl2f + (int)pq_i.w * p.ntypes;
        const int nty = p.ntypes;
        const float l0 = rl[0], l1 = nty > 1 ? rl[1] : 0.0f, l2 = nty > 2 ? rl[2] : 0.0f, l3 = nty > 3 ? rl[3] : 0.0f;
        const float lmax = fmaxf(fmaxf(l0, l1), fmaxf(l2, l3));
        const uint32_t st_s = (uint32_t)__cvta_generic_to_shared(dyn);
        // position inside the own cell (the binning of B1: cell = (u * nc) >> 32,
        // so the low word of u * nc is the fraction), for culling the rows and
        // row ends that lie wholly beyond the largest list radius of this
        // particle's row
        const float wc = R.cellw;
        const float f2w = wc * 2.3283064365386963e-10f;  // cell width / 2^32
        const float fxl = (float)(uint32_t)((uint64_t)pq_i.x * (uint64_t)nc) * f2w;
        const float fyl = (float)(uint32_t)((uint64_t)pq_i.y * (uint64_t)nc) * f2w;
        const float fzl = (float)(uint32_t)((uint64_t)pq_i.z * (uint64_t)nc) * f2w;
        const float lcut = (sqrtf(lmax) + 1e-3f * wc) * (sqrtf(lmax) + 1e-3f * wc);  // rounding margin
        const int tsh = __ffs(T) - 1;
#define KAMD_SCAN(R_, N_)                                                                                         \
  scan_particle_mix<R_, N_>(st_s, s_ub, ncand, nc, nr, UX, UY, own_u, fxl, fyl, fzl, wc, lcut, sl, tsh, x, y, z, pq_i, \
                            sc, l0, l1, l2, l3, own_q, lb, gsz, p.maxrows, b1, b2, b3)
#define KAMD_SCAN2(R_, N_)                                                                                           \
  scan_particle_pair_mix<R_, N_>(st_s, s_ub, nr, UX, UY, own_u, fxl, fyl, fzl, wc, lcut, h,                         \
                                 3u << (threadIdx.x & 30u), x, y, z, pq_i, sc, l0, l1, l2, l3, own_q, lb, gsz,        \
                                 p.maxrows)
        if (pair) {
          if (rel)
            k = nty <= 2 ? KAMD_SCAN2(true, true) : KAMD_SCAN2(true, false);
          else
            k = nty <= 2 ? KAMD_SCAN2(false, true) : KAMD_SCAN2(false, false);
        } else {
          if (rel)
            k = nty <= 2 ? KAMD_SCAN(true, true) : KAMD_SCAN(true, false);
          else
            k = nty <= 2 ? KAMD_SCAN(false, true) : KAMD_SCAN(false, false);
        }
#undef KAMD_SCAN
#undef KAMD_SCAN2
        if (sl == 0 && h == 0) p.xbq[i] = pq_i;
      } else {
        const double4_32a pi = p.p4[cur][i];
        const int tb = (int)pi.w * p.ntypes;
        const double L = R.L, hL = 0.5 * R.L;
        double lmax = 0.0;
        for (int t = 0; t < p.ntypes; ++t) lmax = fmax(lmax, sh.rl2d[tb + t]);
        // position inside the own cell, for the same culling as the mixed path
        const double wc = R.L / (double)(nc > 0 ? nc : 1);
        const double fxl = pi.x - ccx * wc, fyl = pi.y - ccy * wc, fzl = pi.z - ccz * wc;
        const double lcut = (sqrt(lmax) + 1e-9 * wc) * (sqrt(lmax) + 1e-9 * wc);
        auto fd = [&](int o, double f) { return o < 0 ? f + (-o - 1) * wc : (o > 0 ? (wc - f) + (o - 1) * wc : 0.0); };
        for (int run = 0; run < nruns; ++run) {
          int qs = 0, qe = ncand;
          if (nc > 0) {
            const int oy = run % side - nr, oz = run / side - nr;
            const double ey = fd(oy, fyl), ez = fd(oz, fzl);
            const double d2 = ey * ey + ez * ez;
            if (d2 >= lcut) continue;
            int xl = -nr, xh = nr;
            while (xl < 0 && fd(xl, fxl) * fd(xl, fxl) + d2 >= lcut) ++xl;
            while (xh > 0 && fd(xh, fxl) * fd(xh, fxl) + d2 >= lcut) --xh;
            const int us0 = ((lz + nr + oz) * UY + (ly + nr + oy)) * UX + lx + nr;
            qs = s_ub[us0 + xl];
            qe = s_ub[us0 + xh + 1];
          }
          for (int q = qs + sl; q < qe; q += T) {
            const double4_32a pj = st_d[q];
            double dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            if (dx > hL) dx -= L; else if (dx < -hL) dx += L;
            if (dy > hL) dy -= L; else if (dy < -hL) dy += L;
            if (dz > hL) dz -= L; else if (dz < -hL) dz += L;
            if (q != own_q && dx * dx + dy * dy + dz * dz < sh.rl2d[tb + (int)pj.w]) {
              list_push(lb, gsz, p.maxrows, k, b1, b2, b3, st_j[q]);
            }
          }
        }
        if (sl == 0) p.xbd[i] = pi;
      }
      if (!pair) list_flush(lb, gsz, p.maxrows, k, b1, b2, b3);
      if (h == 0) {
        if (k > p.maxrows) raise_flag(p, MD_FLAG_OVERFLOW);
        p.nnb[i * T + sl] = min(k, p.maxrows);
      }
    }
    __syncthreads();
  }
}

// Cell sort + Verlet list build for every replica whose want_rebuild is set.
// Returns false after a barrier timeout. *fl receives the last snapshot.
template <bool MIX>
__device__ bool rebuild(const KParams& p, Shared& sh, int cur, int* fl, int64_t epoch) {
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nt = p.ntot;
  // B1: cell index and count per cell; owners copy want -> doing
  for (int64_t r = gtid; r < p.nrep; r += stride) p.reps[r].doing_rebuild = p.reps[r].want_rebuild;
  for (int64_t i = gtid; i < nt; i += stride) {
    const RepDev& R = p.reps[p.tile_rep[i >> 5]];
    if (i - R.off >= R.n || !R.want_rebuild || R.nc == 0) continue;
    int cx, cy, cz;
    cell_of_pos<MIX>(p, R, i, cur, cx, cy, cz);
    const int c = (cz * R.nc + cy) * R.nc + cx;
    p.cellof[i] = c;
    atomicAdd(&p.ccount[R.cell0 + c], 1);
  }
  int f = grid_sync(p, sh, 101);
  if (f < 0) return false;
  // B2: exclusive scan of the cell counts over all packed cells, in chunks of
  // MD_SCAN_CHUNK cells spread over the grid. B2a: chunk sums, and (last CTA)
  // each replica's base = particles in the cells of earlier rebuilding replicas.
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAnd(&p.ctl->pending, ~MD_FLAG_REBUILD);
  const int nchunks = (int)((p.ncells + MD_SCAN_CHUNK - 1) / MD_SCAN_CHUNK);
  const int cpt = MD_SCAN_CHUNK / (int)blockDim.x;  // cells per thread in a chunk (<= 8)
  // a single chunk (up to MD_SCAN_CHUNK cells): the last CTA computes the
  // replica bases and scans the chunk itself, with no barrier in between
  const bool one = nchunks <= 1;
  for (int k = one ? nchunks : (int)blockIdx.x; k < nchunks; k += gridDim.x) {
    const int64_t c0 = (int64_t)k * MD_SCAN_CHUNK;
    int sum = 0;
    for (int u = 0; u < cpt; ++u) {
      const int64_t gc = c0 + u * (int)blockDim.x + threadIdx.x;
      if (gc < p.ncells) sum += p.ccount[gc];
    }
    int total;
    block_exclusive_scan(sh, sum, &total);
    if (threadIdx.x == 0) p.chunk[k] = total;
  }
  if (blockIdx.x == gridDim.x - 1) {
    int64_t carry = 0;
    for (int r0 = 0; r0 < p.nrep; r0 += blockDim.x) {
      const int r = r0 + (int)threadIdx.x;
      int v = 0;
      if (r < p.nrep) {
        const RepDev& R = p.reps[r];
        v = (R.doing_rebuild && R.nc > 0) ? R.n : 0;
      }
      int total;
      const int pre = block_exclusive_scan(sh, v, &total);
      if (r < p.nrep) p.reps[r].cell_base = carry + pre;
      carry += total;
    }
  }
  if (!one) {
    f = grid_sync(p, sh, 109);
    if (f < 0) return false;
  }
  // B2b: chunk base (sum of the earlier chunks), scan inside the chunk, and
  // cell start = replica offset + (global prefix - replica base). Cells of
  // replicas that do not rebuild keep their ranges.
  for (int64_t r = gtid; r < p.nrep; r += stride) {
    RepDev& R = p.reps[r];
    if (!R.doing_rebuild) continue;
    R.want_rebuild = 0;
    R.rebuilds += 1;
    R.rebuild_epoch = epoch;
    if (R.nc > 0) p.cstart[R.cs0 + R.nc * R.nc * R.nc] = (int)(R.off + R.n);
  }
  for (int k = one ? (blockIdx.x == gridDim.x - 1 ? 0 : nchunks) : (int)blockIdx.x; k < nchunks; k += gridDim.x) {
    int part = 0;
    for (int t = threadIdx.x; t < k; t += blockDim.x) part += p.chunk[t];
    int base;
    block_exclusive_scan(sh, part, &base);
    // thread t owns cells c0 + t*cpt .. c0 + t*cpt + cpt - 1 (consecutive)
    const int64_t c0 = (int64_t)k * MD_SCAN_CHUNK + (int64_t)threadIdx.x * cpt;
    int v[8], rep[8];
    int sum = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool in = u < cpt && c0 + u < p.ncells;
      v[u] = in ? p.ccount[c0 + u] : 0;
      rep[u] = in ? p.cell_rep[c0 + u] : -1;
      sum += v[u];
    }
    int total;
    int run = base + block_exclusive_scan(sh, sum, &total);
    // replica fields are reloaded only when the replica changes
    int cur_r = -1;
    bool r_doing = false;
    int64_t r_off = 0, r_base = 0, r_cs0 = 0, r_cell0 = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (rep[u] < 0) break;
      if (rep[u] != cur_r) {
        const RepDev& R = p.reps[rep[u]];
        cur_r = rep[u];
        r_doing = R.doing_rebuild != 0;
        r_off = R.off;
        r_base = R.cell_base;
        r_cs0 = R.cs0;
        r_cell0 = R.cell0;
      }
      const int64_t gc = c0 + u;
      if (r_doing) {
        const int start = (int)(r_off + (run - r_base));
        p.cstart[r_cs0 + (gc - r_cell0)] = start;
        p.ccursor[gc] = start;
        p.ccount[gc] = 0;
      }
      run += v[u];
    }
  }
  f = grid_sync(p, sh, 102);
  if (f < 0) return false;
  // B3: scatter slot indices into their cells (order inside a cell arbitrary)
  for (int64_t i = gtid; i < nt; i += stride) {
    const RepDev& R = p.reps[p.tile_rep[i >> 5]];
    if (i - R.off >= R.n || !R.doing_rebuild || R.nc == 0) continue;
    const int slot = atomicAdd(&p.ccursor[R.cell0 + p.cellof[i]], 1);
    p.scat[slot] = (int)i;
  }
  f = grid_sync(p, sh, 103);
  if (f < 0) return false;
  // B4: rank inside the cell by (type, caller index) (deterministic order) and move
  // every per-particle array to its new slot in the scratch copy. One warp
  // per cell: each lane holds one member's caller index and counts, by
  // shuffles, the members with a smaller one.
  {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = stride >> 5;
    for (int64_t gc = gtid >> 5; gc < p.ncells; gc += nwarps) {
      const RepDev& R = p.reps[p.cell_rep[gc]];
      if (!R.doing_rebuild || R.nc == 0) continue;
      const int c = (int)(gc - R.cell0);
      const int lo = p.cstart[R.cs0 + c], hi = p.cstart[R.cs0 + c + 1];
      const int n = hi - lo;
      // key = (type, caller index): particles of one species sit together, so
      // the lanes of a warp walk lists of similar length
      for (int e0 = 0; e0 < n; e0 += 32) {
        int o = -1;
        unsigned my = 0xffffffffu;
        if (e0 + lane < n) {
          o = p.scat[lo + e0 + lane];
          my = ((unsigned)p.typ[o] << 30) | (unsigned)p.gid[o];
        }
        int rank = 0;
        for (int m0 = 0; m0 < n; m0 += 32) {
          unsigned other = 0xffffffffu;
          if (m0 == e0) {
            other = my;  // the lanes already hold this chunk's keys
          } else if (m0 + lane < n) {
            const int oo = p.scat[lo + m0 + lane];
            other = ((unsigned)p.typ[oo] << 30) | (unsigned)p.gid[oo];
          }
          const int lim = min(32, n - m0);
          for (int t = 0; t < lim; ++t) rank += (__shfl_sync(0xffffffffu, other, t) < my);
        }
        if (o < 0) continue;
        const int64_t d = lo + rank;
        // every load before any store (the arrays may not be assumed disjoint)
        const int gd = (int)(my & 0x3fffffffu);
        const uint8_t ty = (uint8_t)(my >> 30);
        int im[3];
        for (int cc = 0; cc < 3; ++cc) im[cc] = p.img[cc * nt + o];
        if constexpr (MIX) {
          uint64_t u[3];
          float v[3], fo[3];
          for (int cc = 0; cc < 3; ++cc) {
            u[cc] = p.pfx[cc * nt + o];
            v[cc] = p.velf[cc * nt + o];
            fo[cc] = p.frcf[cc * nt + o];
          }
          for (int cc = 0; cc < 3; ++cc) {
            p.t_pfx[cc * nt + d] = u[cc];
            ((float*)p.t_vel)[cc * nt + d] = v[cc];
            ((float*)p.t_frc)[cc * nt + d] = fo[cc];
            p.t_img[cc * nt + d] = im[cc];
          }
          // the gather copy goes straight to its new slot (nothing in this
          // phase reads it), so the list build need not wait for B5
          p.pq[cur][d] = make_uint4((uint32_t)(u[0] >> 32), (uint32_t)(u[1] >> 32), (uint32_t)(u[2] >> 32), ty);
        } else {
          const double4_32a x = p.p4[cur][o];
          double v[3], fo[3];
          for (int cc = 0; cc < 3; ++cc) {
            v[cc] = p.veld[cc * nt + o];
            fo[cc] = p.frcd[cc * nt + o];
          }
          p.t_p4[d] = x;
          for (int cc = 0; cc < 3; ++cc) {
            ((double*)p.t_vel)[cc * nt + d] = v[cc];
            ((double*)p.t_frc)[cc * nt + d] = fo[cc];
            p.t_img[cc * nt + d] = im[cc];
          }
        }
        p.t_gid[d] = gd;
        p.t_typ[d] = ty;
      }
    }
  }
  f = grid_sync(p, sh, 104);
  if (f < 0) return false;
  // B5: copy back (FP64: positions included, which are also the gather copy)
  for (int64_t i = gtid; i < nt; i += stride) {
    const RepDev& R = p.reps[p.tile_rep[i >> 5]];
    if (i - R.off >= R.n || !R.doing_rebuild || R.nc == 0) continue;
    const int gd = p.t_gid[i];
    const uint8_t ty = p.t_typ[i];
    int im[3];
    for (int cc = 0; cc < 3; ++cc) im[cc] = p.t_img[cc * nt + i];
    if constexpr (MIX) {
      uint64_t u[3];
      float v[3], fo[3];
      for (int cc = 0; cc < 3; ++cc) {
        u[cc] = p.t_pfx[cc * nt + i];
        v[cc] = ((const float*)p.t_vel)[cc * nt + i];
        fo[cc] = ((const float*)p.t_frc)[cc * nt + i];
      }
      for (int cc = 0; cc < 3; ++cc) {
        p.pfx[cc * nt + i] = u[cc];
        p.velf[cc * nt + i] = v[cc];
        p.frcf[cc * nt + i] = fo[cc];
        p.img[cc * nt + i] = im[cc];
      }
    } else {
      const double4_32a x = p.t_p4[i];
      double v[3], fo[3];
      for (int cc = 0; cc < 3; ++cc) {
        v[cc] = ((const double*)p.t_vel)[cc * nt + i];
        fo[cc] = ((const double*)p.t_frc)[cc * nt + i];
      }
      p.p4[cur][i] = x;
      for (int cc = 0; cc < 3; ++cc) {
        p.veld[cc * nt + i] = v[cc];
        p.frcd[cc * nt + i] = fo[cc];
        p.img[cc * nt + i] = im[cc];
      }
    }
    p.gid[i] = gd;
    p.typ[i] = ty;
  }
  // mixed path: B5 and B6 share a phase (B6 reads only the gather copy,
  // written in B4, and writes only the lists); FP64: B6 reads the positions
  // that B5 moves back, so a barrier separates them
  if constexpr (!MIX) {
    f = grid_sync(p, sh, 105);
    if (f < 0) return false;
  }
  // B6: Verlet lists (build_lists)
  build_lists<MIX>(p, sh, cur);
  f = grid_sync(p, sh, 106);
  if (f < 0) return false;
  *fl = f;
  return true;
}

// ------------------------------------------------------------------ kernel

// Which SM each CTA runs on (written before the launch's first barrier):
// CTA rank among the CTAs of its SM, their number, and the SM's index among
// the SMs in use. Any SM id past the 256-bit map leaves the grid-strided split.
__device__ void sm_layout(const KParams& p, Shared& sh) {
  const int mine = p.cta_sm[blockIdx.x];
  int cnt = 0, rank = 0, bad = 0;
  for (int j = threadIdx.x; j < (int)gridDim.x; j += blockDim.x) {
    const int sj = p.cta_sm[j];
    if (sj < 0 || sj >= 256) { bad = 1; continue; }
    atomicOr(&sh.sm_bits[sj >> 5], 1u << (sj & 31));
    if (sj == mine) {
      ++cnt;
      if (j < (int)blockIdx.x) ++rank;
    }
  }
  int tc, tr, tb;
  block_exclusive_scan(sh, cnt, &tc);
  block_exclusive_scan(sh, rank, &tr);
  block_exclusive_scan(sh, bad, &tb);
  if (threadIdx.x == 0) {
    int idx = 0, used = 0;
    if (tb == 0 && mine >= 0 && mine < 256) {
      for (int w = 0; w < 8; ++w) {
        const unsigned bits = sh.sm_bits[w];
        used += __popc(bits);
        if (w < (mine >> 5)) idx += __popc(bits);
        else if (w == (mine >> 5)) idx += __popc(bits & ((1u << (mine & 31)) - 1u));
      }
    }
    sh.sm_ok = (tb == 0 && mine >= 0 && mine < 256 && used > 0) ? 1 : 0;
    sh.sm_idx = idx;
    sh.sm_used = used;
    sh.sm_cnt = tc;
    sh.sm_rank = tr;
  }
  __syncthreads();
}

template <bool MIX>
__global__ void __launch_bounds__(512, KAMD_MIN_BLOCKS) md_persistent(KParams p) {
  __shared__ Shared sh;
  const int nt2 = p.ntypes * p.ntypes;
  for (int t = threadIdx.x; t < nt2; t += blockDim.x) {
    sh.tabf[t] = make_float4(p.tab_f[t][0], p.tab_f[t][1], p.tab_f[t][2], p.tab_f[t][3]);
    sh.vshf[t] = p.vsh_f[t];
    sh.rl2f[t] = p.rl2_f[t];
    sh.rli2f[t] = p.rli2_f[t];
    sh.tabd[t] = make_double4_32a(p.tab_d[t][0], p.tab_d[t][1], p.tab_d[t][2], p.tab_d[t][3]);
    sh.vshd[t] = p.vsh_d[t];
    sh.rl2d[t] = p.rl2_d[t];
    sh.rli2d[t] = p.rli2_d[t];
  }
  if (threadIdx.x < 8) sh.sm_bits[threadIdx.x] = 0u;
  if (threadIdx.x == 0) p.cta_sm[blockIdx.x] = sm_id();
  CtlDev* C = p.ctl;
  if (threadIdx.x == 0) sh.gen = ld_acquire_u32(&C->bar_gen);
  int cur = C->cur;
  const int drifted = C->drifted;
  const int fvalid = C->forces_valid;
  const int64_t step0 = C->step;
  int fl = grid_sync(p, sh, 1);
  if (fl < 0) return;
  sm_layout(p, sh);
  const bool nh = p.kind == MD_KIND_NH || p.kind == MD_KIND_NH_EXACT;
  const int kick = p.kind == MD_KIND_NH ? KICK_NH : (p.kind == MD_KIND_NH_EXACT ? KICK_NH_EXACT : KICK_VV);
  int64_t done = 0;
  bool now_drifted = drifted != 0;
  // NVE steps that only write a log record keep their partial sums in a slot
  // of p.plog (slot k: step and record index in p.plog_rec[k]); their records
  // are formed after the launch by k_log_records, so that no CTA starts the
  // next step late
  int ndef = 0;


  // record where this launch left the state: the gather-buffer parity, the
  // global step, whether positions are one drift ahead of velocities/forces,
  // and whether the stored forces belong to the stored positions
  auto finish = [&](bool is_drifted, int forces_valid) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      C->cur = cur;
      C->step = step0 + done;
      C->steps_done = done;
      C->drifted = is_drifted ? 1 : 0;
      C->forces_valid = forces_valid;
      C->log_slots_used = ndef;
    }
  };

  if (!drifted) {
    // list epochs: the force evaluation at the current positions is "step0"
    if (fl & MD_FLAG_REBUILD) {
      if (!rebuild<MIX>(p, sh, cur, &fl, step0)) return;
      if (fl & MD_FLAG_OVERFLOW) { finish(false, fvalid); return; }
      if (p.dual) {
        prune_phase<MIX>(p, sh, cur, step0);
        if ((fl = grid_sync(p, sh, 107)) < 0) return;
      }
    } else if (fl & MD_FLAG_PRUNE) {
      prune_phase<MIX>(p, sh, cur, step0);
      if ((fl = grid_sync(p, sh, 108)) < 0) return;
    }
    if (p.op == MD_OP_REBUILD) { finish(false, fvalid); return; }
    if (p.op == MD_OP_LIST_REPEAT) {
      // measurement: the launch began with a rebuild of every replica (the
      // host marks them all); nsteps - 1 more list builds of the same cells
      // follow, each closed by a grid barrier. Positions do not move, so each
      // build writes the same lists again.
      for (int64_t k = 1; k < p.nsteps; ++k) {
        build_lists<MIX>(p, sh, cur);
        if ((fl = grid_sync(p, sh, 19)) < 0) return;
      }
      finish(false, fvalid);
      return;
    }
    if (p.op == MD_OP_FORCE_REPEAT) {
      // measurement: nsteps force evaluations of the current positions, as the
      // step loop does them (pair sums and force stores, no energy, no
      // partials), each closed by a grid barrier
      for (int64_t k = 0; k < p.nsteps; ++k) {
        force_phase<MIX>(p, sh, cur, KICK_NONE, false, p.part[0], true, false, false, step0);
        if ((fl = grid_sync(p, sh, 18)) < 0) return;
      }
      finish(false, 1);
      return;
    }
    if (p.op == MD_OP_INITVEL) {
      // Maxwell-Boltzmann start: draw 0 at each replica's bath temperature,
      // then centre and rescale (steps 1-4 of Sec. "Statistical temperature bath")
      resample_draw_phase<MIX>(p, 0, p.part[0]);
      if ((fl = grid_sync(p, sh, 2)) < 0) return;
      if (!reduce_phase<MIX>(p, sh, p.part[0], 1, RED_RESAMPLE, step0, false, 0)) return;
      if ((fl = grid_sync(p, sh, 3)) < 0) return;
      drift_phase<MIX>(p, cur, false, true, false, step0);
      finish(false, fvalid);
      return;
    }
    const bool pairs = !fvalid || p.op == MD_OP_FORCES;
    force_phase<MIX>(p, sh, cur, KICK_NONE, false, p.part[0], pairs, true, true, step0);
    if ((fl = grid_sync(p, sh, 4)) < 0) return;
    if (!reduce_phase<MIX>(p, sh, p.part[0], p.T, pairs ? RED_FORCES : RED_KE, step0, false, 0)) return;
    if ((fl = grid_sync(p, sh, 5)) < 0) return;
    if (p.op == MD_OP_FORCES || p.nsteps == 0) { finish(false, 1); return; }
    drift_phase<MIX>(p, cur, nh, false, true, step0 + 1);
    cur ^= 1;
    now_drifted = true;
    if ((fl = grid_sync(p, sh, 6)) < 0) return;
  }
  for (int64_t s = 0; s < p.nsteps; ++s) {
    if (fl & MD_FLAG_UNSTABLE) break;
    const int64_t step = step0 + s + 1;
    if (fl & MD_FLAG_REBUILD) {
      if (!rebuild<MIX>(p, sh, cur, &fl, step)) return;
      if (fl & MD_FLAG_OVERFLOW) { finish(true, 1); return; }
      if (p.dual) {
        prune_phase<MIX>(p, sh, cur, step);
        if ((fl = grid_sync(p, sh, 107)) < 0) return;
      }
    } else if (fl & MD_FLAG_PRUNE) {
      prune_phase<MIX>(p, sh, cur, step);
      if ((fl = grid_sync(p, sh, 108)) < 0) return;
    }
    const bool last = s == p.nsteps - 1;
    const bool rs = p.kind == MD_KIND_RESAMPLE && (step % p.nstep_boltz == 0);
    const bool fuse = !nh && !rs && !last;
    double* part = p.part[step & 1];  // (replaced by a log slot below when deferred)
    const int64_t li = p.log_step0 + s + 1;
    const bool log_now = p.log_every > 0 && (li % p.log_every) == 0 && (li / p.log_every - 1) < p.log_cap;
    const int64_t lidx = p.log_every > 0 ? li / p.log_every - 1 : 0;
    const bool energy = log_now || last;
    const bool need_red = log_now || nh || last || rs;
    const bool defer = log_now && !nh && !rs && !last && ndef < p.plog_slots;
    if (defer) part = p.plog + (int64_t)ndef * p.plog_stride;
    force_phase<MIX>(p, sh, cur, kick, fuse, part, true, energy, need_red, step + 1);
    if ((fl = grid_sync(p, sh, 10)) < 0) return;
    if (fuse) cur ^= 1;
    now_drifted = fuse;
    if (defer) {
      if (blockIdx.x == 0 && threadIdx.x == 0) p.plog_rec[ndef] = make_longlong2(step, lidx);
      ++ndef;
    } else if (need_red &&
               !reduce_phase<MIX>(p, sh, part, p.T, energy ? RED_STEP : RED_STEP_KE, step, log_now && !rs, lidx)) {
      return;
    }
    if (nh) {
      if ((fl = grid_sync(p, sh, 11)) < 0) return;
      if (!last) {
        drift_phase<MIX>(p, cur, true, false, true, step + 1);
        cur ^= 1;
        now_drifted = true;
        if ((fl = grid_sync(p, sh, 12)) < 0) return;
      }
    } else if (rs) {
      if ((fl = grid_sync(p, sh, 13)) < 0) return;
      double* part2 = p.part[(step & 1) ^ 1];
      resample_draw_phase<MIX>(p, (uint64_t)(step / p.nstep_boltz), part2);
      if ((fl = grid_sync(p, sh, 14)) < 0) return;
      if (!reduce_phase<MIX>(p, sh, part2, 1, RED_RESAMPLE, step, log_now, lidx)) return;
      if ((fl = grid_sync(p, sh, 15)) < 0) return;
      drift_phase<MIX>(p, cur, false, true, !last, step + 1);
      if (!last) { cur ^= 1; now_drifted = true; }
      if ((fl = grid_sync(p, sh, 16)) < 0) return;
    }
    done = s + 1;
  }
  finish(now_drifted && done < p.nsteps, 1);
}

// Barrier self-test: block 0 leaves without arriving, so the other blocks'
// wait runs out after timeout_ns and they raise MD_FLAG_TIMEOUT. Nothing is
// read or written but the control block.
// The log records of the NVE steps whose partial sums a launch of
// md_persistent left in slots of p.plog (slot k: step and record index in
// p.plog_rec[k]; nslots used): one (slot, replica) pair per CTA, the same sums
// as reduce_phase forms at a step for a replica reduced by one CTA, so the
// records are those that step would have written. Launched after the
// persistent kernel on the same stream.
template <bool MIX>
__global__ void __launch_bounds__(512) k_log_records(KParams p, int nslots) {
  __shared__ Shared sh;
  for (int64_t w = blockIdx.x; w < (int64_t)nslots * p.nrep; w += gridDim.x) {
    const int k = (int)(w / p.nrep), r = (int)(w - (int64_t)k * p.nrep);
    RepDev& R = p.reps[r];
    double acc[6];
    sum_records<MIX>(sh, p.plog + (int64_t)k * p.plog_stride, (int64_t)R.tile0 * p.T, (int64_t)R.ntiles * p.T, acc);
    if (threadIdx.x == 0) {
      const longlong2 rec = p.plog_rec[k];
      reduce_scalars(p, R, r, acc, RED_LOG, rec.x, true, rec.y, false);
    }
    __syncthreads();
  }
}

__global__ void k_barrier_selftest(KParams p) {
  __shared__ Shared sh;
  if (blockIdx.x == 0) return;
  if (threadIdx.x == 0) sh.gen = ld_acquire_u32(&p.ctl->bar_gen);
  (void)grid_sync(p, sh, 200);
}

}  // namespace kamd

cudaError_t md_launch_log_records(bool mixed, const KParams& p, int nslots, int block, cudaStream_t s) {
  // the persistent kernel's block size: sum_records strides by it, so the
  // sums come out in the order the step itself would have used
  const int64_t pairs = (int64_t)nslots * p.nrep;
  const int blocks = (int)(pairs < 1024 ? pairs : 1024);
  if (mixed) kamd::k_log_records<true><<<blocks, block, 0, s>>>(p, nslots);
  else kamd::k_log_records<false><<<blocks, block, 0, s>>>(p, nslots);
  return cudaGetLastError();
}

cudaError_t md_launch_barrier_selftest(const KParams& p, int blocks, cudaStream_t s) {
  kamd::k_barrier_selftest<<<blocks, 32, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t md_launch_persistent(bool mixed, const KParams& p, int grid, int block, size_t smem, cudaStream_t s) {
  void* args[] = {(void*)&p};
  const void* fn = mixed ? (const void*)kamd::md_persistent<true> : (const void*)kamd::md_persistent<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, s);
}

const void* md_persistent_fn(bool mixed) {
  return mixed ? (const void*)kamd::md_persistent<true> : (const void*)kamd::md_persistent<false>;
}

cudaError_t md_occupancy(bool mixed, int block, size_t smem, int* blocks_per_sm) {
  const void* fn = mixed ? (const void*)kamd::md_persistent<true> : (const void*)kamd::md_persistent<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}
