// md_api.cu -- the C ABI declared in include/kamd.h: system set-up, device
// memory, state transfer, and the launches of the persistent step kernel.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "kamd.h"
#include "md_device.cuh"
#include "md_internal.cuh"

struct md_system {
  // configuration
  int nrep = 0, ntypes = 0;
  int ndim = 3;         // 2: particles in the plane z = L/2, v_z = 0 (two-dimensional model)
  int64_t n_total = 0;  // particles, caller order
  int64_t ntot = 0;     // slots (padded)
  int ntiles = 0;
  bool mixed = true;
  std::vector<int64_t> n_per, out0;
  std::vector<double> L_per;
  double eps[16] = {0}, sig[16] = {0}, rc[16] = {0};
  double mass = 1.0;
  md_tuning tun{4, 256, 0.3, 0.7};
  cudaStream_t stream = nullptr;
  int device = 0, nsm = 0;
  int grid = 0;
  int maxrows = 0;
  int stage_cap = 0;  // candidates the list build stages per group (dynamic shared memory)
  int64_t ncells = 0;
  bool have_state = false;
  // host mirrors
  std::vector<RepDev> reps;
  CtlDev ctl{};
  // device memory
  RepDev* d_reps = nullptr;
  int32_t* d_tile_rep = nullptr;
  CtlDev* d_ctl = nullptr;
  uint64_t* d_pfx = nullptr;
  uint4* d_pq[2] = {nullptr, nullptr};
  float* d_velf = nullptr;
  float* d_frcf = nullptr;
  uint4* d_xbq = nullptr;
  uint4* d_xbq_in = nullptr;
  double4_32a* d_p4[2] = {nullptr, nullptr};
  double* d_veld = nullptr;
  double* d_frcd = nullptr;
  double4_32a* d_xbd = nullptr;
  double4_32a* d_xbd_in = nullptr;
  int32_t* d_gid = nullptr;
  uint8_t* d_typ = nullptr;
  int32_t* d_img = nullptr;
  uint64_t* d_tpfx = nullptr;
  double4_32a* d_tp4 = nullptr;
  void* d_tvel = nullptr;
  void* d_tfrc = nullptr;
  int32_t* d_tgid = nullptr;
  uint8_t* d_ttyp = nullptr;
  int32_t* d_timg = nullptr;
  int32_t* d_cellof = nullptr;
  int32_t* d_cell_rep = nullptr;
  int32_t* d_ccount = nullptr;
  int32_t* d_cstart = nullptr;
  int32_t* d_ccursor = nullptr;
  int32_t* d_chunk = nullptr;
  int32_t* d_cta_sm = nullptr;  // SM id per CTA of the persistent grid
  int2* d_grp = nullptr;        // list-build groups (replica, index in replica)
  int2* d_redmap = nullptr;     // reduction chunks (replica, chunk index)
  int2* d_redrep = nullptr;     // per replica (first chunk, chunks)
  double* d_redpart = nullptr;  // chunk sums
  int64_t nred = 0;
  int red2 = 0;
  int red_tiles = MD_RED_TILES;
  int64_t ngroups = 0;
  int cta_sm_cap = 0;
  int32_t* d_scat = nullptr;
  int32_t* d_nbr = nullptr;
  int32_t* d_nbr_in = nullptr;
  int32_t* d_nnb_in = nullptr;
  int32_t* d_nnb = nullptr;
  double* d_part[2] = {nullptr, nullptr};
  uint8_t* d_typ_caller = nullptr;
  int32_t* d_rep_of_caller = nullptr;
  double* d_msd_ref[MD_MSD_SLOTS] = {};  // unwrapped reference positions r(t_w), caller order; [0] always held
  bool msd_valid[MD_MSD_SLOTS] = {};
  ThermoDev* d_thermo = nullptr;
  int64_t thermo_cap = 0;
  double* d_io = nullptr;  // caller-order staging (n_total*3 doubles)
  int32_t* d_io_i = nullptr;
  unsigned long long* d_rdf = nullptr;
  int64_t rdf_nbins = 0;
  double rdf_dr = 0.0;
  int64_t rdf_meas = 0;
  double* d_msd_part = nullptr;
  unsigned long long* d_count = nullptr;
  size_t bytes = 0;  // device bytes currently held (dalloc/dfree)
  std::unordered_map<const void*, size_t> alloc_sizes;
  size_t list_bytes = 0;
  unsigned long long timeout_ns = 10ull * 1000 * 1000 * 1000;
  // the persistent launch as an instantiated CUDA graph (one cooperative
  // kernel node whose parameters are updated per call)
  bool use_graph = true;
  // partial records of NVE log steps reduced after the launch (size in doubles)
  double* d_plog = nullptr;
  longlong2* d_plog_rec = nullptr;
  size_t plog_cap = 0;
  int plog_slots = 0;
  bool log_now = false;  // KAMD_LOG_NOW=1: every log record reduced at its step
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphNode_t gnode = nullptr;
  int g_grid = 0, g_block = 0;
  size_t g_smem = 0;
  int64_t graph_launches = 0;
  int64_t kernel_launches = 0;  // persistent launches and log-record launches
  std::string err;
};

namespace {

thread_local std::string g_create_err;

md_status fail(md_system* s, md_status code, const std::string& msg) {
  if (s) s->err = msg;
  else g_create_err = msg;
  return code;
}

md_status cuda_fail(md_system* s, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(s, e == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA, m);
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(s, e_, #call); \
  } while (0)

template <typename T>
md_status dalloc(md_system* s, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(s, e, "cudaMalloc");
  s->bytes += count * sizeof(T);
  s->alloc_sizes[(const void*)*p] = count * sizeof(T);
  e = cudaMemsetAsync(*p, 0, count * sizeof(T), s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "cudaMemsetAsync");
  return MD_OK;
}

// Free a device array allocated by dalloc and take its size off the
// footprint counter (md_get_info's device_bytes).
template <typename T>
void dfree(md_system* s, T*& p) {
  if (p) {
    auto it = s->alloc_sizes.find((const void*)p);
    if (it != s->alloc_sizes.end()) {
      s->bytes -= it->second;
      s->alloc_sizes.erase(it);
    }
    cudaFree((void*)p);
  }
  p = nullptr;
}

#define CKS(call)                 \
  do {                            \
    md_status st_ = (call);       \
    if (st_ != MD_OK) return st_; \
  } while (0)

// ------------------------------------------------------------------ kernels

// Map caller-order particle g to its slot: identity order inside a replica.
__global__ void k_set_state(bool mixed, int ndim, int64_t n_total, int64_t ntot, const RepDev* reps,
                            const int32_t* rep_of, const uint8_t* typ_caller, const double* pos, const double* vel,
                            int cur, uint64_t* pfx, uint4* pq, float* velf, float* frcf, uint4* xbq, double4_32a* p4,
                            double* veld, double* frcd, double4_32a* xbd, int32_t* gid, uint8_t* typ, int32_t* img) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_total) return;
  const RepDev& R = reps[rep_of[g]];
  const int64_t i = R.off + (g - R.out0);
  const uint32_t t = typ_caller[g];
  double x[3];
  for (int c = 0; c < 3; ++c) x[c] = kamd::wrap_box(pos[3 * g + c], R.L);
  if (ndim == 2) x[2] = 0.5 * R.L;  // two dimensions: the plane z = L/2
  if (mixed) {
    uint32_t hi[3];
    for (int c = 0; c < 3; ++c) {
      const uint64_t u = kamd::to_fixed(x[c], R.invL);
      pfx[c * ntot + i] = u;
      hi[c] = (uint32_t)(u >> 32);
      velf[c * ntot + i] = (vel && (ndim == 3 || c < 2)) ? (float)vel[3 * g + c] : 0.0f;
      frcf[c * ntot + i] = 0.0f;
    }
    pq[i] = make_uint4(hi[0], hi[1], hi[2], t);
    xbq[i] = pq[i];
  } else {
    p4[i] = make_double4_32a(x[0], x[1], x[2], (double)t);
    xbd[i] = p4[i];
    for (int c = 0; c < 3; ++c) {
      veld[c * ntot + i] = (vel && (ndim == 3 || c < 2)) ? vel[3 * g + c] : 0.0;
      frcd[c * ntot + i] = 0.0;
    }
  }
  for (int c = 0; c < 3; ++c) img[c * ntot + i] = 0;
  gid[i] = (int32_t)g;
  typ[i] = (uint8_t)t;
}

// Simple-cubic lattice with jitter (Sec. "Initialization of positions"); in
// two dimensions a square lattice in the plane z = L/2.
__global__ void k_lattice(int ndim, int64_t n_total, const RepDev* reps, const int32_t* rep_of, double jitter,
                          uint64_t seed, double* pos) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_total) return;
  const RepDev& R = reps[rep_of[g]];
  const int64_t p = g - R.out0, n = R.n;
  int64_t m = 1;
  if (ndim == 3) while (m * m * m < n) ++m;
  else while (m * m < n) ++m;
  const double a = R.L / (double)m;
  const int64_t sites = ndim == 3 ? m * m * m : m * m;
  const int64_t site = (int64_t)(((unsigned __int128)p * (unsigned __int128)sites) / (unsigned __int128)n);
  const int64_t k[3] = {site % m, (site / m) % m, site / (m * m)};
  double u[3];
  kamd::jitter3(seed, (uint32_t)p, u);
  for (int c = 0; c < 3; ++c) {
    double x = (ndim == 2 && c == 2) ? 0.5 * R.L : (0.5 + (double)k[c]) * a + jitter * u[c];
    if (x >= R.L) x -= R.L;
    else if (x < 0.0) x += R.L;
    pos[3 * g + c] = x;
  }
}

__global__ void k_get_state(bool mixed, int64_t ntot, const RepDev* reps, const int32_t* tile_rep, int cur,
                            const uint64_t* pfx, const float* velf, const double4_32a* p4, const double* veld,
                            const int32_t* gid, const int32_t* img, double* pos, double* vel, int32_t* imgo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntot) return;
  const RepDev& R = reps[tile_rep[i >> 5]];
  if (i - R.off >= R.n) return;
  const int64_t g = gid[i];
  for (int c = 0; c < 3; ++c) {
    if (pos) pos[3 * g + c] = mixed ? kamd::from_fixed(pfx[c * ntot + i], R.L) : (c == 0 ? p4[i].x : c == 1 ? p4[i].y : p4[i].z);
    if (vel) vel[3 * g + c] = mixed ? (double)velf[c * ntot + i] : veld[c * ntot + i];
    if (imgo) imgo[3 * g + c] = img[c * ntot + i];
  }
}

__global__ void k_get_forces(bool mixed, int64_t ntot, const RepDev* reps, const int32_t* tile_rep, const float* frcf,
                             const double* frcd, const int32_t* gid, double* f) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntot) return;
  const RepDev& R = reps[tile_rep[i >> 5]];
  if (i - R.off >= R.n) return;
  const int64_t g = gid[i];
  for (int c = 0; c < 3; ++c) f[3 * g + c] = mixed ? (double)frcf[c * ntot + i] : frcd[c * ntot + i];
}

__global__ void k_set_images(int64_t n_total, int64_t ntot, const RepDev* reps, const int32_t* rep_of,
                             const int32_t* imgs, int32_t* img) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_total) return;
  const RepDev& R = reps[rep_of[g]];
  const int64_t i = R.off + (g - R.out0);
  for (int c = 0; c < 3; ++c) img[c * ntot + i] = imgs[3 * g + c];
}

// Unwrapped caller-order positions x + L*image (MSD reference / current).
__global__ void k_unwrapped(bool mixed, int64_t ntot, const RepDev* reps, const int32_t* tile_rep, const uint64_t* pfx,
                            const double4_32a* p4, const int32_t* gid, const int32_t* img, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntot) return;
  const RepDev& R = reps[tile_rep[i >> 5]];
  if (i - R.off >= R.n) return;
  const int64_t g = gid[i];
  for (int c = 0; c < 3; ++c) {
    const double x = mixed ? kamd::from_fixed(pfx[c * ntot + i], R.L) : (c == 0 ? p4[i].x : c == 1 ? p4[i].y : p4[i].z);
    out[3 * g + c] = x + R.L * (double)img[c * ntot + i];
  }
}

// Per-tile sums of squared displacement per type (Eq. (msdwithi)); counts in
// the second half of the partial row.
__global__ void k_msd_tiles(bool mixed, int ntiles, int ntypes, int64_t ntot, const RepDev* reps, const int32_t* tile_rep,
                            const uint64_t* pfx, const double4_32a* p4, const int32_t* gid, const uint8_t* typ,
                            const int32_t* img, const double* ref, double* part) {
  const int lane = threadIdx.x & 31;
  const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (tile >= ntiles) return;
  const RepDev& R = reps[tile_rep[tile]];
  const int64_t i = tile * 32 + lane;
  double d2 = 0.0;
  int t = -1;
  if (i - R.off < R.n) {
    const int64_t g = gid[i];
    t = typ[i];
    for (int c = 0; c < 3; ++c) {
      const double x = mixed ? kamd::from_fixed(pfx[c * ntot + i], R.L) : (c == 0 ? p4[i].x : c == 1 ? p4[i].y : p4[i].z);
      const double d = x + R.L * (double)img[c * ntot + i] - ref[3 * g + c];
      d2 += d * d;
    }
  }
  for (int a = 0; a < ntypes; ++a) {
    const double v = kamd::warp_sum(t == a ? d2 : 0.0);
    const double cnt = kamd::warp_sum(t == a ? 1.0 : 0.0);
    if (lane == 0) {
      part[tile * MD_NPART + a] = v;
      part[tile * MD_NPART + MD_MAXTYPES + a] = cnt;
    }
  }
}

// One thread per type: fixed-order sum over all tiles.
__global__ void k_msd_final(int ntiles, int ntypes, const double* part, double* out) {
  const int a = threadIdx.x;
  if (a >= ntypes) return;
  double s = 0.0, c = 0.0;
  for (int t = 0; t < ntiles; ++t) {
    s += part[(int64_t)t * MD_NPART + a];
    c += part[(int64_t)t * MD_NPART + MD_MAXTYPES + a];
  }
  out[a] = c > 0 ? s / c : 0.0;
}

// Pair-distance histogram of Sec. "Radial distribution function with
// Python": every unordered pair with r < nbins*dr adds 2 (like) or 1 (unlike)
// to bin floor(r/dr) of its replica (integer counts; exact, order-free).
// Mixed path: a conservative FP32 test on the 32-bit gather words rejects the
// pairs beyond r_max (most candidates); the bin of the others comes from the
// exact 64-bit positions in FP64, as before. A block whose particles all
// belong to one replica (and nbins <= RDF_SMEM_BINS) counts into a shared-
// memory histogram and adds it to the replica's histogram once.
#define RDF_SMEM_BINS 1024
__global__ void k_rdf(bool mixed, int64_t ntot, int nbins, double dr, double skin, const RepDev* reps,
                      const int32_t* tile_rep, int cur, const uint4* pq, const uint64_t* pfx, const double4_32a* p4,
                      const uint8_t* typ, const int32_t* cstart, unsigned long long* hist) {
  __shared__ unsigned int sh_h[3 * RDF_SMEM_BINS];
  __shared__ int sh_rep;
  const int64_t b0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t i = b0 + threadIdx.x;
  if (threadIdx.x == 0) {
    const int64_t last = min(b0 + (int64_t)blockDim.x, ntot) - 1;
    const int r0 = tile_rep[b0 >> 5];
    sh_rep = (nbins <= RDF_SMEM_BINS && tile_rep[last >> 5] == r0) ? r0 : -1;
  }
  __syncthreads();
  const bool priv = sh_rep >= 0;
  if (priv)
    for (int t = threadIdx.x; t < 3 * nbins; t += blockDim.x) sh_h[t] = 0u;
  __syncthreads();
  bool act = i < ntot;
  const int r = act ? tile_rep[i >> 5] : 0;
  const RepDev& R = reps[r];
  if (act && i - R.off >= R.n) act = false;
  if (act) {
    const double rmax = dr * nbins, rmax2 = rmax * rmax;
    const float rmax2f = (float)(rmax2 * (1.0 + 1e-4)) + 1e-6f;  // FP32 pre-test, widened
    const float scf = R.fxs;
    const int ti = typ[i];
    double xi[3];
    uint64_t ui[3];
    for (int c = 0; c < 3; ++c) {
      if (mixed) ui[c] = pfx[c * ntot + i];
      else xi[c] = c == 0 ? p4[i].x : c == 1 ? p4[i].y : p4[i].z;
    }
    const uint4 qi = mixed ? pq[i] : make_uint4(0u, 0u, 0u, 0u);
    const int nc = R.nc;
    const int layers = nc > 0 ? (int)ceil((rmax + skin) * (1.0 + 1e-6) / (double)R.cellw) : 0;
    const bool all = nc == 0 || 2 * layers + 1 > nc;
    int cx = 0, cy = 0, cz = 0;
    if (!all) {
      if (mixed) {
        cx = (int)(((uint64_t)(uint32_t)(ui[0] >> 32) * (uint64_t)nc) >> 32);
        cy = (int)(((uint64_t)(uint32_t)(ui[1] >> 32) * (uint64_t)nc) >> 32);
        cz = (int)(((uint64_t)(uint32_t)(ui[2] >> 32) * (uint64_t)nc) >> 32);
      } else {
        const double sc = (double)nc * R.invL;
        cx = min(max((int)(xi[0] * sc), 0), nc - 1);
        cy = min(max((int)(xi[1] * sc), 0), nc - 1);
        cz = min(max((int)(xi[2] * sc), 0), nc - 1);
      }
    }
    unsigned long long* h = hist + (int64_t)r * 3 * nbins;
    auto visit = [&](int64_t j) {
      if (j <= i) return;
      if (mixed) {
        const uint4 qj = pq[j];
        const float fx = (float)(int)(qi.x - qj.x) * scf, fy = (float)(int)(qi.y - qj.y) * scf,
                    fz = (float)(int)(qi.z - qj.z) * scf;
        if (!(fmaf(fx, fx, fmaf(fy, fy, fz * fz)) < rmax2f)) return;
      }
      double d[3];
      for (int c = 0; c < 3; ++c) {
        if (mixed) {
          d[c] = (double)(int64_t)(ui[c] - pfx[c * ntot + j]) * (R.L * (1.0 / 18446744073709551616.0));
        } else {
          const double xj = c == 0 ? p4[j].x : c == 1 ? p4[j].y : p4[j].z;
          double e = xi[c] - xj;
          if (e > 0.5 * R.L) e -= R.L;
          else if (e < -0.5 * R.L) e += R.L;
          d[c] = e;
        }
      }
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (!(r2 < rmax2)) return;
      const int k = (int)(sqrt(r2) / dr);
      if (k >= nbins) return;
      const int tj = typ[j];
      const int slot = (ti == 0 && tj == 0) ? k : ((ti == 1 && tj == 1) ? nbins + k : 2 * nbins + k);
      const unsigned w = (ti == tj) ? 2u : 1u;
      if (priv) atomicAdd(&sh_h[slot], w);
      else atomicAdd(&h[slot], (unsigned long long)w);
    };
    if (all) {
      for (int64_t j = R.off; j < R.off + R.n; ++j) visit(j);
    } else {
      // cells are those of the last list build; every particle has moved less
      // than half a skin since, so layers computed with rmax + skin cover all pairs
      for (int oz = -layers; oz <= layers; ++oz)
        for (int oy = -layers; oy <= layers; ++oy)
          for (int ox = -layers; ox <= layers; ++ox) {
            const int c = (((cz + oz + 8 * nc) % nc) * nc + (cy + oy + 8 * nc) % nc) * nc + (cx + ox + 8 * nc) % nc;
            const int lo = cstart[R.cs0 + c], hi = cstart[R.cs0 + c + 1];
            for (int j = lo; j < hi; ++j) visit(j);
          }
    }
  }
  if (priv) {
    __syncthreads();
    unsigned long long* h = hist + (int64_t)sh_rep * 3 * nbins;
    for (int t = threadIdx.x; t < 3 * nbins; t += blockDim.x)
      if (sh_h[t]) atomicAdd(&h[t], (unsigned long long)sh_h[t]);
  }
}

// Pairs (i < j) inside their cutoff r < r_c,ab, from exact distances (mixed:
// 64-bit fixed-point differences; FP64: the minimum-image branch rule), found
// through the cells of the last list build. Every particle has moved less
// than half the outer skin since, so the cells within (r_c,max + skin_outer)
// of its current position hold every partner; a replica with too few cells
// for that is scanned whole.
__global__ void k_count_pairs(bool mixed, int64_t ntot, int ntypes, double reach, const RepDev* reps,
                              const int32_t* tile_rep, const uint64_t* pfx, const double4_32a* p4, const uint8_t* typ,
                              const int32_t* cstart, const double* rc2d, unsigned long long* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntot) return;
  const RepDev& R = reps[tile_rep[i >> 5]];
  if (i - R.off >= R.n) return;
  const int ti = typ[i];
  double xi[3];
  uint64_t ui[3];
  for (int c = 0; c < 3; ++c) {
    if (mixed) ui[c] = pfx[c * ntot + i];
    else xi[c] = c == 0 ? p4[i].x : c == 1 ? p4[i].y : p4[i].z;
  }
  unsigned long long cnt = 0;
  auto visit = [&](int64_t j) {
    if (j <= i) return;
    double d2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      double d;
      if (mixed) {
        d = (double)(int64_t)(ui[c] - pfx[c * ntot + j]) * (R.L * (1.0 / 18446744073709551616.0));
      } else {
        const double xj = c == 0 ? p4[j].x : c == 1 ? p4[j].y : p4[j].z;
        d = xi[c] - xj;
        if (d > 0.5 * R.L) d -= R.L;
        else if (d < -0.5 * R.L) d += R.L;
      }
      d2 += d * d;
    }
    cnt += d2 < rc2d[ti * ntypes + typ[j]];
  };
  const int nc = R.nc;
  const int layers = nc > 0 ? (int)ceil(reach * (1.0 + 1e-6) / (double)R.cellw) : 0;
  if (nc == 0 || 2 * layers + 1 > nc) {
    for (int64_t j = R.off; j < R.off + R.n; ++j) visit(j);
  } else {
    int cc[3];
    for (int c = 0; c < 3; ++c) {
      if (mixed) cc[c] = (int)(((uint64_t)(uint32_t)(ui[c] >> 32) * (uint64_t)nc) >> 32);
      else cc[c] = min(max((int)(xi[c] * (double)nc * R.invL), 0), nc - 1);
    }
    for (int oz = -layers; oz <= layers; ++oz)
      for (int oy = -layers; oy <= layers; ++oy)
        for (int ox = -layers; ox <= layers; ++ox) {
          const int c = (((cc[2] + oz + 8 * nc) % nc) * nc + (cc[1] + oy + 8 * nc) % nc) * nc + (cc[0] + ox + 8 * nc) % nc;
          for (int j = cstart[R.cs0 + c]; j < cstart[R.cs0 + c + 1]; ++j) visit(j);
        }
  }
  if (cnt) atomicAdd(out, cnt);
}

// Sum of n non-negative ints (warp sums, one atomic per warp).
__global__ void k_sum_i32(int64_t n, const int32_t* v, unsigned long long* out) {
  unsigned long long acc = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    acc += (unsigned long long)v[k];
  acc = kamd::warp_sum(acc);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

int blocks_for(int64_t n, int b) { return (int)((n + b - 1) / b); }

// ------------------------------------------------------------------ host helpers

md_status upload_reps(md_system* s) {
  CK(cudaMemcpyAsync(s->d_reps, s->reps.data(), sizeof(RepDev) * s->nrep, cudaMemcpyHostToDevice, s->stream));
  return MD_OK;
}
md_status download_reps(md_system* s) {
  CK(cudaMemcpyAsync(s->reps.data(), s->d_reps, sizeof(RepDev) * s->nrep, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return MD_OK;
}
md_status upload_ctl(md_system* s) {
  CK(cudaMemcpyAsync(s->d_ctl, &s->ctl, sizeof(CtlDev), cudaMemcpyHostToDevice, s->stream));
  return MD_OK;
}
md_status download_ctl(md_system* s) {
  CK(cudaMemcpyAsync(&s->ctl, s->d_ctl, sizeof(CtlDev), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return MD_OK;
}

double rc_max(const md_system* s) {
  double m = 0;
  for (int t = 0; t < s->ntypes * s->ntypes; ++t) m = std::max(m, s->rc[t]);
  return m;
}

// Cells per edge and list capacity follow from the skin; both are recomputed
// whenever the tuning changes. Cells are at least half the outer list radius
// wide, so the list build scans the 5 x 5 x 5 cells around a particle's own
// (less volume than 27 cells of the full radius, and the corners are culled);
// a box with fewer than 8 such cells per edge uses cells of the full radius
// (3 x 3 x 3), and one with fewer than 3 of those an all-pairs scan.
// KAMD_CELL_REACH=1 keeps cells of the full radius (for tests of that path).
void layout_cells(md_system* s) {
  const double rl = rc_max(s) + s->tun.skin_outer;
  int reach = 2;
  if (const char* e = std::getenv("KAMD_CELL_REACH")) reach = std::atoi(e) == 1 ? 1 : 2;
  int64_t cell0 = 0;
  for (int r = 0; r < s->nrep; ++r) {
    RepDev& R = s->reps[r];
    int nr = reach;
    int nc = (int)std::min(std::floor(R.L / (rl / nr)), 1024.0);
    const int nc1 = (int)std::floor(R.L / rl);
    // full-width cells where they fit 3 per edge and half-width cells fewer
    // than 8 (measured on 8 replicas of N = 1000, L = 9.41: 6 half-width
    // cells per edge were 13 % slower than 3 full-width ones), and where the
    // box is too small for 5 half-width cells; half-width cells otherwise
    // (N = 1000 with an outer radius of 3.7: 5 half-width cells per edge were
    // twice as fast as an all-pairs scan)
    if (nr == 2 && ((nc < 8 && nc1 >= 3) || nc < 5)) {
      nr = 1;
      nc = nc1;
    }
    if (nc < 3) nc = 0;
    R.nc = nc;
    R.nr = nc > 0 ? nr : 1;
    R.cellw = nc > 0 ? (float)(R.L / nc) : 0.0f;
    R.cell0 = cell0;
    R.cs0 = cell0 + r;
    cell0 += (int64_t)nc * nc * nc;
  }
  s->ncells = cell0;
}

int list_capacity(const md_system* s) {
  const double rl = rc_max(s) + s->tun.skin_outer;
  double dens = 0;
  int64_t nmax = 0;
  for (int r = 0; r < s->nrep; ++r) {
    const double Lr = s->L_per[r];
    dens = std::max(dens, (double)s->n_per[r] / (s->ndim == 3 ? Lr * Lr * Lr : Lr * Lr));
    nmax = std::max(nmax, s->n_per[r]);
  }
  // particles within the list radius: a sphere, or in two dimensions a disc
  double est = s->ndim == 3 ? 4.0 / 3.0 * M_PI * rl * rl * rl * dens : M_PI * rl * rl * dens;
  int cap = (int)std::ceil(1.5 * est + 32);
  // KAMD_LIST_CAPACITY: start from a given capacity (the list still grows on overflow)
  if (const char* e = std::getenv("KAMD_LIST_CAPACITY")) cap = std::max(1, std::atoi(e));
  if (cap > nmax - 1) cap = (int)std::max<int64_t>(nmax - 1, 1);
  return cap;
}

// List-build groups, per replica: as many neighbouring cells per CTA (powers
// of two up to 4 x 4 x 4, 4 x 4 in a plane) as T threads per particle fill to
// at most 90 % of the CTA, from the replica's own cells (a batch can mix
// half-width, full-width and no cells). KAMD_LIST_GROUP forces one size.
void choose_groups(md_system* s) {
  const int gmax = s->ndim == 3 ? 64 : 16;
  int forced = 0;
  if (const char* e = std::getenv("KAMD_LIST_GROUP")) {
    const int v = std::atoi(e);
    if (v >= 1 && v <= gmax && (v & (v - 1)) == 0) forced = v;
  }
  for (int r = 0; r < s->nrep; ++r) {
    RepDev& R = s->reps[r];
    int g = 1;
    if (R.nc > 0) {
      // particles per occupied cell (two dimensions: only the cells of the plane hold particles)
      const double w = (double)R.cellw;
      const double occ = s->ndim == 3 ? (double)s->n_per[r] / (R.L * R.L * R.L) * w * w * w
                                      : (double)s->n_per[r] / (R.L * R.L) * w * w;
      // 10 % headroom: a group whose particles overflow the CTA needs a second,
      // mostly idle pass (measured: 1.7x slower list build at N = 32 000, T = 2).
      // Groups stop at 64 cells: the staging area of 128-cell groups (57 KB per
      // CTA at N = 10^6) takes shared memory from the L1 cache that the force
      // phase's gathers use (list build 20 % faster, force phase 8 % slower)
      const double fit = 0.9 * (double)s->tun.block_size / ((double)s->tun.threads_per_atom * occ);
      while (2 * g <= gmax && 2 * g <= fit) g *= 2;
    }
    if (forced) g = forced;
    // x doubles first, then y, then z (a plane: x and y only)
    int gx = 1, gy = 1, gz = 1;
    for (int k = 1; k < g; k *= 2) {
      if (gx <= gy && (s->ndim == 2 || gx <= gz) && gx < 4) gx *= 2;
      else if (gy <= gz || s->ndim == 2) gy *= 2;
      else gz *= 2;
    }
    R.gx = gx;
    R.gy = gy;
    R.gz = gz;
  }
}

// Staging area of the list build: the candidates of the cells around one
// group, (gx+2)(gy+2)(gz+2) cells (or a whole replica too small for cells),
// with headroom over the mean (overflow regrows it).
int stage_capacity(md_system* s) {
  choose_groups(s);
  int cap = 64;
  for (int r = 0; r < s->nrep; ++r) {
    const RepDev& R = s->reps[r];
    // occupied union cells (two dimensions: one plane of cells)
    const int e = 2 * R.nr;
    const double nu = s->ndim == 3 ? (double)(R.gx + e) * (R.gy + e) * (R.gz + e) : (double)(R.gx + e) * (R.gy + e);
    const double w = (double)R.cellw;
    const double occ = s->ndim == 3 ? (double)s->n_per[r] / (R.L * R.L * R.L) * w * w * w
                                    : (double)s->n_per[r] / (R.L * R.L) * w * w;
    int need;
    if (R.nc > 0) {
      const double mean = nu * occ;
      need = (int)std::ceil(1.1 * mean + 6.0 * std::sqrt(mean) + 32.0);
    } else {
      need = (int)s->n_per[r];
    }
    cap = std::max(cap, need);
  }
  return cap;
}

size_t stage_bytes(const md_system* s) { return (size_t)s->stage_cap * (s->mixed ? 16 : 36); }

md_status alloc_cells_and_list(md_system* s, int cap_entries) {
  const int T = s->tun.threads_per_atom;
  dfree(s, s->d_ccount);
  dfree(s, s->d_cstart);
  dfree(s, s->d_ccursor);
  dfree(s, s->d_chunk);
  dfree(s, s->d_nbr);
  dfree(s, s->d_nbr_in);
  dfree(s, s->d_cell_rep);
  s->maxrows = ((cap_entries + T - 1) / T + 3) / 4 * 4;  // list layout: whole quads per column
  CKS(dalloc(s, &s->d_cell_rep, (size_t)s->ncells));
  {
    std::vector<int32_t> cr((size_t)std::max<int64_t>(s->ncells, 1), 0);
    for (int r = 0; r < s->nrep; ++r) {
      const int64_t nc3 = (int64_t)s->reps[r].nc * s->reps[r].nc * s->reps[r].nc;
      for (int64_t c = 0; c < nc3; ++c) cr[s->reps[r].cell0 + c] = r;
    }
    // on the system's stream, after dalloc's clearing memset; cr is a local vector
    CK(cudaMemcpyAsync(s->d_cell_rep, cr.data(), 4 * cr.size(), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  CKS(dalloc(s, &s->d_ccount, (size_t)s->ncells));
  CKS(dalloc(s, &s->d_cstart, (size_t)(s->ncells + s->nrep)));
  CKS(dalloc(s, &s->d_ccursor, (size_t)s->ncells));
  CKS(dalloc(s, &s->d_chunk, (size_t)(s->ncells / MD_SCAN_CHUNK + 1)));
  {
    std::vector<int2> grp;
    for (int r = 0; r < s->nrep; ++r) {
      const int nc = s->reps[r].nc;
      if (nc == 0) continue;
      const RepDev& R = s->reps[r];
      const int ng = ((nc + R.gx - 1) / R.gx) * ((nc + R.gy - 1) / R.gy) * ((nc + R.gz - 1) / R.gz);
      for (int k = 0; k < ng; ++k) grp.push_back(make_int2(r, k));
    }
    s->ngroups = (int64_t)grp.size();
    // two-level reductions (chunks of red_tiles tiles) once a replica spans
    // more than 4 chunks: below that, one CTA per replica is as fast and, in
    // NVE, its reduction overlaps the next step instead of adding a barrier.
    // KAMD_RED_TILES sets the chunk and the threshold to the same value, for
    // tests of that path.
    s->red_tiles = MD_RED_TILES;
    int threshold = 4 * MD_RED_TILES;
    if (const char* e = std::getenv("KAMD_RED_TILES")) {
      const int v = std::atoi(e);
      if (v >= 1) s->red_tiles = threshold = v;
    }
    std::vector<int2> rmap, rrep;
    int maxtiles = 0;
    for (int r = 0; r < s->nrep; ++r) {
      const int nch = (s->reps[r].ntiles + s->red_tiles - 1) / s->red_tiles;
      rrep.push_back(make_int2((int)rmap.size(), nch));
      for (int c = 0; c < nch; ++c) rmap.push_back(make_int2(r, c));
      maxtiles = std::max(maxtiles, s->reps[r].ntiles);
    }
    s->red2 = maxtiles > threshold ? 1 : 0;
    s->nred = (int64_t)rmap.size();
    dfree(s, s->d_redmap);
    dfree(s, s->d_redrep);
    dfree(s, s->d_redpart);
    s->d_redmap = nullptr;
    s->d_redrep = nullptr;
    s->d_redpart = nullptr;
    CKS(dalloc(s, &s->d_redmap, std::max<size_t>(rmap.size(), 1)));
    CKS(dalloc(s, &s->d_redrep, std::max<size_t>(rrep.size(), 1)));
    CKS(dalloc(s, &s->d_redpart, std::max<size_t>(rmap.size(), 1) * MD_NPART));
    if (!rmap.empty()) {
      CK(cudaMemcpyAsync(s->d_redmap, rmap.data(), sizeof(int2) * rmap.size(), cudaMemcpyHostToDevice, s->stream));
      CK(cudaMemcpyAsync(s->d_redrep, rrep.data(), sizeof(int2) * rrep.size(), cudaMemcpyHostToDevice, s->stream));
      CK(cudaStreamSynchronize(s->stream));  // local vectors
    }
    dfree(s, s->d_grp);
    s->d_grp = nullptr;
    CKS(dalloc(s, &s->d_grp, std::max<size_t>(grp.size(), 1)));
    if (!grp.empty()) {
      CK(cudaMemcpyAsync(s->d_grp, grp.data(), sizeof(int2) * grp.size(), cudaMemcpyHostToDevice, s->stream));
      CK(cudaStreamSynchronize(s->stream));  // grp is a local vector
    }
  }
  const size_t entries = (size_t)s->ntiles * s->maxrows * 32 * T;
  CKS(dalloc(s, &s->d_nbr, entries));
  CKS(dalloc(s, &s->d_nbr_in, entries));
  s->list_bytes = entries * 8;
  return MD_OK;
}

md_status mark_rebuild_all(md_system* s) {
  CKS(download_reps(s));
  for (auto& R : s->reps) R.want_rebuild = 1;
  CKS(upload_reps(s));
  CKS(download_ctl(s));
  s->ctl.pending |= MD_FLAG_REBUILD;
  return upload_ctl(s);
}

md_status configure_grid(md_system* s) {
  const int b = s->tun.block_size;
  int per_sm = 0;
  if (stage_bytes(s) > 200 * 1024) return fail(s, MD_ERR_NLIST_OVERFLOW, "list-build staging exceeds shared memory");
  CK(md_occupancy(s->mixed, b, stage_bytes(s), &per_sm));
  if (per_sm < 1) return fail(s, MD_ERR_INVALID_ARG, "block size too large for the persistent kernel");
  s->grid = per_sm * s->nsm;
  if (s->grid > s->cta_sm_cap) {
    dfree(s, s->d_cta_sm);
    s->d_cta_sm = nullptr;
    s->cta_sm_cap = 0;
    CKS(dalloc(s, &s->d_cta_sm, (size_t)s->grid));
    s->cta_sm_cap = s->grid;
  }
  return MD_OK;
}

void fill_tables(const md_system* s, KParams& p) {
  const int nt = s->ntypes;
  for (int t = 0; t < nt * nt; ++t) {
    const double e = s->eps[t], sg = s->sig[t], rc = s->rc[t];
    const double sr6 = std::pow(sg / rc, 6.0);
    const double vc = 4.0 * e * (sr6 * sr6 - sr6);
    const double rl = rc + s->tun.skin_outer, rli = rc + s->tun.skin;
    p.tab_d[t][0] = rc * rc;
    p.tab_d[t][1] = sg * sg;
    p.tab_d[t][2] = 48.0 * e;
    p.tab_d[t][3] = 4.0 * e;
    p.vsh_d[t] = vc;
    p.rl2_d[t] = rl * rl;
    p.rli2_d[t] = rli * rli;
    p.rli2_f[t] = (float)(rli * rli * (1.0 + 1e-5));
    for (int k = 0; k < 4; ++k) p.tab_f[t][k] = (float)p.tab_d[t][k];
    p.vsh_f[t] = (float)vc;
    // the mixed list test runs in FP32 on cell-relative coordinates: widen the
    // radius by a relative 1e-5 so rounding can never drop a pair at the edge
    p.rl2_f[t] = (float)(rl * rl * (1.0 + 1e-5));
  }
}

KParams make_params(const md_system* s) {
  KParams p;
  std::memset(&p, 0, sizeof(p));
  p.nrep = s->nrep;
  p.ntypes = s->ntypes;
  p.ndim = s->ndim;
  p.ntot = s->ntot;
  p.ntiles = s->ntiles;
  p.T = s->tun.threads_per_atom;
  p.maxrows = s->maxrows;
  fill_tables(s, p);
  p.mass = s->mass;
  p.inv_mass = 1.0 / s->mass;
  // rebuild the outer list once a particle moved (skin_outer - skin)/2 since
  // its build (every pair within r_c + skin is then still in it); prune the
  // inner list once a particle moved skin/2 since the last prune. With
  // skin_outer == skin there is one list: rebuilt at skin/2, never pruned,
  // and the force phase reads it directly
  const double so = s->tun.skin_outer, si = s->tun.skin;
  p.dual = so > si ? 1 : 0;
  p.skin_half2 = p.dual ? 0.25 * (so - si) * (so - si) : 0.25 * si * si;
  p.prune_half2 = p.dual ? 0.25 * si * si : HUGE_VAL;
  p.massf = (float)s->mass;
  p.inv_massf = (float)(1.0 / s->mass);
  p.skin_half2f = (float)p.skin_half2;
  p.prune_half2f = (float)p.prune_half2;
  p.timeout_ns = s->timeout_ns;
  p.reps = s->d_reps;
  p.tile_rep = s->d_tile_rep;
  p.ctl = s->d_ctl;
  p.pfx = s->d_pfx;
  p.pq[0] = s->d_pq[0];
  p.pq[1] = s->d_pq[1];
  p.velf = s->d_velf;
  p.frcf = s->d_frcf;
  p.xbq = s->d_xbq;
  p.xbq_in = s->d_xbq_in;
  p.p4[0] = s->d_p4[0];
  p.p4[1] = s->d_p4[1];
  p.veld = s->d_veld;
  p.frcd = s->d_frcd;
  p.xbd = s->d_xbd;
  p.xbd_in = s->d_xbd_in;
  p.gid = s->d_gid;
  p.typ = s->d_typ;
  p.img = s->d_img;
  p.t_pfx = s->d_tpfx;
  p.t_p4 = s->d_tp4;
  p.t_vel = s->d_tvel;
  p.t_frc = s->d_tfrc;
  p.t_gid = s->d_tgid;
  p.t_typ = s->d_ttyp;
  p.t_img = s->d_timg;
  p.cellof = s->d_cellof;
  p.cell_rep = s->d_cell_rep;
  p.ncells = s->ncells;
  p.stage_cap = s->stage_cap;
  p.ccount = s->d_ccount;
  p.cstart = s->d_cstart;
  p.ccursor = s->d_ccursor;
  p.chunk = s->d_chunk;
  p.cta_sm = s->d_cta_sm;
  p.grp = s->d_grp;
  p.ngroups = s->ngroups;
  p.red2 = s->red2;
  p.red_tiles = s->red_tiles;
  p.nred = s->nred;
  p.redmap = s->d_redmap;
  p.redrep = s->d_redrep;
  p.redpart = s->d_redpart;
  p.scat = s->d_scat;
  p.nbr = s->d_nbr;
  p.nnb = s->d_nnb;
  p.nbr_in = p.dual ? s->d_nbr_in : s->d_nbr;
  p.nnb_in = p.dual ? s->d_nnb_in : s->d_nnb;
  p.part[0] = s->d_part[0];
  p.part[1] = s->d_part[1];
  p.plog = s->d_plog;
  p.plog_rec = s->d_plog_rec;
  p.plog_stride = (int64_t)s->ntiles * s->tun.threads_per_atom * MD_NPART;
  p.plog_slots = (s->plog_slots > 0 && (size_t)s->plog_slots * (size_t)p.plog_stride <= s->plog_cap) ? s->plog_slots : 0;
  return p;
}

void drop_graph(md_system* s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->graph) cudaGraphDestroy(s->graph);
  s->gexec = nullptr;
  s->graph = nullptr;
  s->gnode = nullptr;
}

// Launch the persistent kernel. By default through an instantiated CUDA graph
// holding one cooperative kernel node (built once per launch shape, its
// parameters updated per call); a direct cooperative launch if the graph
// cannot be built or KAMD_NO_GRAPH is set.
cudaError_t launch_persistent(md_system* s, const KParams& p) {
  const size_t smem = stage_bytes(s);
  const int block = s->tun.block_size;
  if (s->use_graph) {
    KParams pc = p;
    void* args[] = {(void*)&pc};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)md_persistent_fn(s->mixed);
    kp.gridDim = dim3(s->grid);
    kp.blockDim = dim3(block);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    cudaError_t e = cudaSuccess;
    if (!s->gexec || s->g_grid != s->grid || s->g_block != block || s->g_smem != smem) {
      drop_graph(s);
      e = cudaFuncSetAttribute(kp.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) e = cudaGraphCreate(&s->graph, 0);
      if (e == cudaSuccess) e = cudaGraphAddKernelNode(&s->gnode, s->graph, nullptr, 0, &kp);
      if (e == cudaSuccess) {
        cudaKernelNodeAttrValue v = {};
        v.cooperative = 1;
        e = cudaGraphKernelNodeSetAttribute(s->gnode, cudaKernelNodeAttributeCooperative, &v);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&s->gexec, s->graph, 0);
      if (e == cudaSuccess) {
        s->g_grid = s->grid;
        s->g_block = block;
        s->g_smem = smem;
      }
    } else {
      e = cudaGraphExecKernelNodeSetParams(s->gexec, s->gnode, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(s->gexec, s->stream);
    if (e == cudaSuccess) {
      ++s->graph_launches;
      return cudaSuccess;
    }
    // the driver refused the graph: clear the error and launch directly from now on
    cudaGetLastError();
    drop_graph(s);
    s->use_graph = false;
  }
  return md_launch_persistent(s->mixed, p, s->grid, block, smem, s->stream);
}

// Run the persistent kernel for one operation, growing the neighbour list
// and relaunching when it overflows. *steps_out receives completed steps.
md_status run_op(md_system* s, int op, int kind, double dt, int64_t nsteps, int64_t nstep_boltz, uint64_t seed,
                 int64_t log_every, int64_t log_cap, int64_t* steps_out) {
  int64_t done = 0;
  for (int attempt = 0; attempt < 8; ++attempt) {
    // clear the barrier counter and any error flag of an earlier launch (the
    // host mirror is current: every launch ends with a download of it)
    s->ctl.pending &= MD_FLAG_REBUILD;
    s->ctl.err_where = 0;
    CKS(upload_ctl(s));
    KParams p = make_params(s);
    p.op = op;
    p.kind = kind;
    p.dt = dt;
    p.dtf = (float)dt;
    p.nsteps = nsteps - done;
    p.nstep_boltz = nstep_boltz;
    p.seed = seed;
    p.log_every = log_every;
    p.log_step0 = done;
    p.log_cap = log_cap;
    p.thermo = s->d_thermo;
    CK(launch_persistent(s, p));
    ++s->kernel_launches;
    CKS(download_ctl(s));
    if (op == MD_OP_STEPS) done += s->ctl.steps_done;
    const int pend = s->ctl.pending;
    // log records whose sums the launch left in slots (before a relaunch reuses them)
    if (!(pend & MD_FLAG_TIMEOUT) && s->ctl.log_slots_used > 0) {
      CK(md_launch_log_records(s->mixed, p, s->ctl.log_slots_used, s->tun.block_size, s->stream));
      ++s->kernel_launches;
    }
    if (pend & MD_FLAG_TIMEOUT) {
      s->have_state = false;
      char buf[160];
      std::snprintf(buf, sizeof buf, "grid barrier timed out (phase %d); state is undefined, call md_set_state",
                    s->ctl.err_where);
      return fail(s, MD_ERR_TIMEOUT, buf);
    }
    if (pend & MD_FLAG_UNSTABLE) {
      if (steps_out) *steps_out = done;
      return fail(s, MD_ERR_UNSTABLE, "NaN/Inf state or a particle moved >= L/4 in one step");
    }
    if (pend & MD_FLAG_OVERFLOW) {
      // a list column or the build's staging area was too small: grow both
      const int cap = s->maxrows * s->tun.threads_per_atom;
      CKS(alloc_cells_and_list(s, cap + cap / 2 + 16));
      s->stage_cap = std::min(s->stage_cap + s->stage_cap / 2, (int)(200 * 1024 / (s->mixed ? 16 : 36)));
      CKS(configure_grid(s));
      CKS(mark_rebuild_all(s));
      continue;
    }
    if (steps_out) *steps_out = done;
    return MD_OK;
  }
  return fail(s, MD_ERR_NLIST_OVERFLOW, "neighbour list kept overflowing after growing it 8 times");
}

md_status ensure_thermo(md_system* s, int64_t records) {
  if (records <= s->thermo_cap) return MD_OK;
  dfree(s, s->d_thermo);
  CKS(dalloc(s, &s->d_thermo, (size_t)records));
  s->thermo_cap = records;
  return MD_OK;
}

// Take the current unwrapped positions as the reference r(t_w) of one MSD
// slot (Eq. (msdtw)); slots other than 0 get their buffer on first use.
md_status reset_msd_ref(md_system* s, int slot = 0) {
  if (!s->d_msd_ref[slot]) CKS(dalloc(s, &s->d_msd_ref[slot], 3 * (size_t)s->n_total));
  const int b = 256;
  k_unwrapped<<<blocks_for(s->ntot, b), b, 0, s->stream>>>(s->mixed, s->ntot, s->d_reps, s->d_tile_rep, s->d_pfx,
                                                           s->d_p4[s->ctl.cur], s->d_gid, s->d_img,
                                                           s->d_msd_ref[slot]);
  CK(cudaGetLastError());
  s->msd_valid[slot] = true;
  return MD_OK;
}

md_status after_new_state(md_system* s) {
  s->ctl = CtlDev{};
  s->ctl.pending = MD_FLAG_REBUILD;
  s->ctl.cur = 0;
  s->ctl.step = 0;
  CKS(download_reps(s));
  for (auto& R : s->reps) {
    R.want_rebuild = 1;
    R.xi = R.g = R.lns = R.lns_next = R.xi_a = 0.0;
    R.xif = R.xiaf = 0.0f;
    R.prune_epoch = R.rebuild_epoch = -1;
  }
  CKS(upload_reps(s));
  CKS(upload_ctl(s));
  s->have_state = true;
  for (int k = 1; k < MD_MSD_SLOTS; ++k) s->msd_valid[k] = false;  // references of the old state
  CKS(reset_msd_ref(s));
  s->rdf_meas = 0;
  return MD_OK;
}

md_status set_state_impl(md_system* s, const double* pos, const double* vel, int on_device) {
  const double* dpos = pos;
  const double* dvel = vel;
  const size_t bytes = sizeof(double) * 3 * (size_t)s->n_total;
  if (!on_device) {
    CK(cudaMemcpyAsync(s->d_io, pos, bytes, cudaMemcpyHostToDevice, s->stream));
    dpos = s->d_io;
    if (vel) {
      CK(cudaMemcpyAsync(s->d_io + 3 * s->n_total, vel, bytes, cudaMemcpyHostToDevice, s->stream));
      dvel = s->d_io + 3 * s->n_total;
    }
  }
  const int b = 256;
  k_set_state<<<blocks_for(s->n_total, b), b, 0, s->stream>>>(
      s->mixed, s->ndim, s->n_total, s->ntot, s->d_reps, s->d_rep_of_caller, s->d_typ_caller, dpos, dvel, 0, s->d_pfx,
      s->d_pq[0], s->d_velf, s->d_frcf, s->d_xbq, s->d_p4[0], s->d_veld, s->d_frcd, s->d_xbd, s->d_gid, s->d_typ,
      s->d_img);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(s->d_nnb, 0, sizeof(int32_t) * 8 * (size_t)s->ntot, s->stream));
  CK(cudaMemsetAsync(s->d_nnb_in, 0, sizeof(int32_t) * 8 * (size_t)s->ntot, s->stream));
  return after_new_state(s);
}

md_status validate_table(int ntypes, const double* eps, const double* sigma, const double* rc, const double* L, int nrep,
                         double skin) {
  if (ntypes < 1 || ntypes > MD_MAXTYPES) return fail(nullptr, MD_ERR_INVALID_ARG, "ntypes must be in [1, 4]");
  if (!eps || !sigma || !rc) return fail(nullptr, MD_ERR_INVALID_ARG, "eps, sigma and rc tables are required");
  for (int a = 0; a < ntypes; ++a)
    for (int b = 0; b < ntypes; ++b) {
      const int t = a * ntypes + b, u = b * ntypes + a;
      if (!(eps[t] > 0) || !(sigma[t] > 0) || !(rc[t] > 0))
        return fail(nullptr, MD_ERR_INVALID_ARG, "eps, sigma and rc must be > 0");
      if (eps[t] != eps[u] || sigma[t] != sigma[u] || rc[t] != rc[u])
        return fail(nullptr, MD_ERR_INVALID_ARG, "eps, sigma and rc tables must be symmetric");
      for (int r = 0; r < nrep; ++r)
        if (!(rc[t] < 0.5 * L[r]))
          return fail(nullptr, MD_ERR_INVALID_ARG, "every cutoff must be < L/2 (unique minimum image)");
    }
  if (!(skin >= 0)) return fail(nullptr, MD_ERR_INVALID_ARG, "skin must be >= 0");
  return MD_OK;
}

md_status destroy_fail(md_system* s, md_status st) {
  g_create_err = s->err;
  md_destroy(s);
  return st;
}

md_status tuning_ok(md_system* s, const md_tuning* t) {
  const int T = t->threads_per_atom, b = t->block_size;
  if (!(T == 1 || T == 2 || T == 4 || T == 8)) return fail(s, MD_ERR_INVALID_ARG, "threads_per_atom must be 1, 2, 4 or 8");
  if (!(b == 128 || b == 256 || b == 512)) return fail(s, MD_ERR_INVALID_ARG, "block_size must be 128, 256 or 512");
  if (b < 32 * T) return fail(s, MD_ERR_INVALID_ARG, "block_size must hold at least one 32-particle tile");
  if (!(t->skin >= 0) || !(t->skin < 2.0)) return fail(s, MD_ERR_INVALID_ARG, "skin must be in [0, 2)");
  if (!(t->skin_outer >= t->skin) || !(t->skin_outer < 3.0))
    return fail(s, MD_ERR_INVALID_ARG, "skin_outer must be in [skin, 3)");
  for (int r = 0; r < s->nrep; ++r)
    if (!(rc_max(s) < 0.5 * s->L_per[r])) return fail(s, MD_ERR_INVALID_ARG, "cutoff must be < L/2");
  return MD_OK;
}

}  // namespace

void kamd_set_global_error(const std::string& msg) { g_create_err = msg; }

// ====================================================================== ABI

extern "C" {

md_status md_create_batch_dim(int ndim, int nrep, const int64_t* n_per, const double* L_per, const uint8_t* types,
                              int ntypes, const double* eps, const double* sigma, const double* rc, double mass,
                              double skin, md_precision prec, void* stream, md_system** out) {
  if (!out) return fail(nullptr, MD_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  if (ndim != 2 && ndim != 3) return fail(nullptr, MD_ERR_INVALID_ARG, "ndim must be 2 or 3");
  if (nrep < 1 || !n_per || !L_per || !types) return fail(nullptr, MD_ERR_INVALID_ARG, "nrep >= 1 and arrays required");
  if (prec != MD_PREC_FP64 && prec != MD_PREC_MIXED) return fail(nullptr, MD_ERR_INVALID_ARG, "unknown precision");
  if (!(mass > 0)) return fail(nullptr, MD_ERR_INVALID_ARG, "mass must be > 0");
  int64_t ntotal = 0, nslots = 0;
  for (int r = 0; r < nrep; ++r) {
    if (n_per[r] < 2) return fail(nullptr, MD_ERR_INVALID_ARG, "every replica needs n >= 2");
    if (!(L_per[r] > 0) || !std::isfinite(L_per[r])) return fail(nullptr, MD_ERR_INVALID_ARG, "box edge must be > 0");
    if (n_per[r] >= (int64_t)1 << 30) return fail(nullptr, MD_ERR_INVALID_ARG, "too many particles");
    ntotal += n_per[r];
    nslots += (n_per[r] + 31) / 32 * 32;
  }
  // slot indices share a 32-bit word with a 2-bit type in the list build
  if (nslots >= (int64_t)1 << 30) return fail(nullptr, MD_ERR_INVALID_ARG, "at most 2^30 - 1 slots (particles padded to tiles of 32 per replica)");
  CKS(validate_table(ntypes, eps, sigma, rc, L_per, nrep, skin));
  for (int64_t g = 0; g < ntotal; ++g)
    if (types[g] >= ntypes) return fail(nullptr, MD_ERR_INVALID_ARG, "type index out of range");

  md_system* s = new md_system();
  s->ndim = ndim;
  s->stream = (cudaStream_t)stream;
  s->nrep = nrep;
  s->ntypes = ntypes;
  s->n_total = ntotal;
  s->mixed = prec == MD_PREC_MIXED;
  s->mass = mass;
  s->tun.skin = skin;
  s->tun.skin_outer = skin + 0.4;
  for (int t = 0; t < ntypes * ntypes; ++t) {
    s->eps[t] = eps[t];
    s->sig[t] = sigma[t];
    s->rc[t] = rc[t];
  }
  if (const char* e = std::getenv("KAMD_BARRIER_TIMEOUT_MS")) s->timeout_ns = (unsigned long long)std::atoll(e) * 1000000ull;
  if (const char* e = std::getenv("KAMD_NO_GRAPH")) s->use_graph = !(e[0] == '1');
  if (const char* e = std::getenv("KAMD_LOG_NOW")) s->log_now = e[0] == '1';
  cudaError_t ce = cudaGetDevice(&s->device);
  if (ce != cudaSuccess) return destroy_fail(s, cuda_fail(s, ce, "cudaGetDevice"));
  int major = 0, minor = 0, coop = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, s->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, s->device);
  cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->device);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
  if (major != 10 || minor != 3 || !coop) {
    s->err = "this library is built for sm_103a (GB300) with cooperative launch";
    return destroy_fail(s, MD_ERR_NOT_SUPPORTED);
  }
  // replicas: slot ranges padded to whole 32-particle tiles
  s->n_per.assign(n_per, n_per + nrep);
  s->L_per.assign(L_per, L_per + nrep);
  s->reps.resize(nrep);
  std::vector<int32_t> tile_rep;
  std::vector<int32_t> rep_of(ntotal);
  int64_t off = 0, o0 = 0;
  for (int r = 0; r < nrep; ++r) {
    RepDev R;
    std::memset(&R, 0, sizeof(R));
    R.off = off;
    R.out0 = o0;
    R.n = (int32_t)n_per[r];
    R.ntiles = (int32_t)((n_per[r] + 31) / 32);
    R.tile0 = (int32_t)(off / 32);
    R.L = L_per[r];
    R.invL = 1.0 / L_per[r];
    R.fx64 = 18446744073709551616.0 / L_per[r];
    R.Lf = (float)L_per[r];
    R.fxs = (float)(L_per[r] / 4294967296.0);
    R.fx64f = (float)R.fx64;
    R.fx32f = (float)(4294967296.0 / L_per[r]);
    s->reps[r] = R;
    s->out0.push_back(o0);
    for (int t = 0; t < R.ntiles; ++t) tile_rep.push_back(r);
    for (int64_t k = 0; k < n_per[r]; ++k) rep_of[o0 + k] = r;
    off += (int64_t)R.ntiles * 32;
    o0 += n_per[r];
  }
  s->ntot = off;
  s->ntiles = (int)(off / 32);
  layout_cells(s);
  md_status st;
  const size_t nt = (size_t)s->ntot;
#define AL(ptr, cnt)                                   \
  do {                                                 \
    st = dalloc(s, &(ptr), (cnt));                     \
    if (st != MD_OK) return destroy_fail(s, st);       \
  } while (0)
  AL(s->d_reps, (size_t)nrep);
  AL(s->d_plog_rec, (size_t)MD_LOG_SLOTS);
  AL(s->d_tile_rep, (size_t)s->ntiles);
  AL(s->d_ctl, 1);
  if (s->mixed) {
    AL(s->d_pfx, 3 * nt);
    AL(s->d_pq[0], nt);
    AL(s->d_pq[1], nt);
    AL(s->d_velf, 3 * nt);
    AL(s->d_frcf, 3 * nt);
    AL(s->d_xbq, nt);
    AL(s->d_xbq_in, nt);
    AL(s->d_tpfx, 3 * nt);
    float* tv = nullptr;
    float* tf = nullptr;
    AL(tv, 3 * nt);
    AL(tf, 3 * nt);
    s->d_tvel = tv;
    s->d_tfrc = tf;
  } else {
    AL(s->d_p4[0], nt);
    AL(s->d_p4[1], nt);
    AL(s->d_veld, 3 * nt);
    AL(s->d_frcd, 3 * nt);
    AL(s->d_xbd, nt);
    AL(s->d_xbd_in, nt);
    AL(s->d_tp4, nt);
    double* tv = nullptr;
    double* tf = nullptr;
    AL(tv, 3 * nt);
    AL(tf, 3 * nt);
    s->d_tvel = tv;
    s->d_tfrc = tf;
  }
  AL(s->d_gid, nt);
  AL(s->d_typ, nt);
  AL(s->d_img, 3 * nt);
  AL(s->d_tgid, nt);
  AL(s->d_ttyp, nt);
  AL(s->d_timg, 3 * nt);
  AL(s->d_cellof, nt);
  AL(s->d_scat, nt);
  AL(s->d_nnb, 8 * nt);
  AL(s->d_nnb_in, 8 * nt);
  AL(s->d_part[0], (size_t)s->ntiles * 8 * MD_NPART);
  AL(s->d_part[1], (size_t)s->ntiles * 8 * MD_NPART);
  AL(s->d_typ_caller, (size_t)ntotal);
  AL(s->d_rep_of_caller, (size_t)ntotal);
  AL(s->d_msd_ref[0], 3 * (size_t)ntotal);
  AL(s->d_io, 6 * (size_t)ntotal);
  AL(s->d_io_i, 3 * (size_t)ntotal);
  AL(s->d_msd_part, (size_t)s->ntiles * MD_NPART);
  AL(s->d_count, 1);
#undef AL
  s->stage_cap = stage_capacity(s);
  st = alloc_cells_and_list(s, list_capacity(s));
  if (st != MD_OK) return destroy_fail(s, st);
  ce = cudaMemcpyAsync(s->d_tile_rep, tile_rep.data(), 4 * tile_rep.size(), cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(s->d_rep_of_caller, rep_of.data(), 4 * rep_of.size(), cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_typ_caller, types, (size_t)ntotal, cudaMemcpyHostToDevice, s->stream);
  if (ce != cudaSuccess) return destroy_fail(s, cuda_fail(s, ce, "cudaMemcpyAsync"));
  st = upload_reps(s);
  if (st == MD_OK) st = upload_ctl(s);
  if (st == MD_OK) st = configure_grid(s);
  if (st != MD_OK) return destroy_fail(s, st);
  ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return destroy_fail(s, cuda_fail(s, ce, "cudaStreamSynchronize"));
  *out = s;
  return MD_OK;
}

md_status md_create_batch(int nrep, const int64_t* n_per, const double* L_per, const uint8_t* types, int ntypes,
                          const double* eps, const double* sigma, const double* rc, double mass, double skin,
                          md_precision prec, void* stream, md_system** out) {
  return md_create_batch_dim(3, nrep, n_per, L_per, types, ntypes, eps, sigma, rc, mass, skin, prec, stream, out);
}

md_status md_create(int64_t n, const uint8_t* types, int ntypes, double L, const double* eps, const double* sigma,
                    const double* rc, double mass, double skin, md_precision prec, void* stream, md_system** out) {
  return md_create_batch_dim(3, 1, &n, &L, types, ntypes, eps, sigma, rc, mass, skin, prec, stream, out);
}

md_status md_set_state(md_system* s, const double* pos, const double* vel, int on_device) {
  if (!s) return fail(nullptr, MD_ERR_INVALID_ARG, "NULL system");
  if (!pos) return fail(s, MD_ERR_INVALID_ARG, "pos must not be NULL");
  return set_state_impl(s, pos, vel, on_device);
}

md_status md_get_state(md_system* s, double* pos, double* vel, int32_t* images, int on_device) {
  if (!s) return fail(nullptr, MD_ERR_INVALID_ARG, "NULL system");
  if (!s->have_state) return fail(s, MD_ERR_INVALID_ARG, "no state: call md_set_state or md_init_lattice first");
  const size_t n3 = 3 * (size_t)s->n_total;
  double* dp = on_device ? pos : (pos ? s->d_io : nullptr);
  double* dv = on_device ? vel : (vel ? s->d_io + n3 : nullptr);
  int32_t* di = on_device ? images : (images ? s->d_io_i : nullptr);
  CKS(download_ctl(s));
  const int b = 256;
  k_get_state<<<blocks_for(s->ntot, b), b, 0, s->stream>>>(s->mixed, s->ntot, s->d_reps, s->d_tile_rep, s->ctl.cur,
                                                           s->d_pfx, s->d_velf, s->d_p4[s->ctl.cur], s->d_veld,
                                                           s->d_gid, s->d_img, dp, dv, di);
  CK(cudaGetLastError());
  if (!on_device) {
    if (pos) CK(cudaMemcpyAsync(pos, dp, 8 * n3, cudaMemcpyDeviceToHost, s->stream));
    if (vel) CK(cudaMemcpyAsync(vel, dv, 8 * n3, cudaMemcpyDeviceToHost, s->stream));
    if (images) CK(cudaMemcpyAsync(images, di, 4 * n3, cudaMemcpyDeviceToHost, s->stream));
  }
  CK(cudaStreamSynchronize(s->stream));
  return MD_OK;
}

md_status md_init_lattice(md_system* s, const double* T0, double jitter, uint64_t seed) {
  if (!s) return fail(nullptr, MD_ERR_INVALID_ARG, "NULL system");
  if (!T0) return fail(s, MD_ERR_INVALID_ARG, "T0 must not be NULL");
  if (!(jitter >= 0)) return fail(s, MD_ERR_INVALID_ARG, "jitter must be >= 0");
  for (int r = 0; r < s->nrep; ++r)
    if (!(T0[r] >= 0)) return fail(s, MD_ERR_INVALID_ARG, "T0 must be >= 0");
  const int b = 256;
  k_lattice<<<blocks_for(s->n_total, b), b, 0, s->stream>>>(s->ndim, s->n_total, s->d_reps, s->d_rep_of_caller,
                                                            jitter, seed, s->d_io);
  CK(cudaGetLastError());
  CKS(set_state_impl(s, s->d_io, nullptr, 1));
  CKS(download_reps(s));
  for (int r = 0; r < s->nrep; ++r) s->reps[r].T_target = T0[r];
  CKS(upload_reps(s));
  CKS(run_op(s, MD_OP_INITVEL, MD_KIND_NVE, 0.0, 0, 0, seed, 0, 0, nullptr));
  return MD_OK;
}

md_status md_forces(md_system* s, double* f, double* pe, double* virial, int on_device) {
  if (!s) return fail(nullptr, MD_ERR_INVALID_ARG, "NULL system");
  if (!s->have_state) return fail(s, MD_ERR_INVALID_ARG, "no state: call md_set_state or md_init_lattice first");
  CKS(run_op(s, MD_OP_FORCES, MD_KIND_NVE, 0.0, 0, 0, 0, 0, 0, nullptr));
  if (f) {
    double* df = on_device ? f : s->d_io;
    const int b = 256;
    k_get_forces<<<blocks_for(s->ntot, b), b, 0, s->stream>>>(s->mixed, s->ntot, s->d_reps, s->d_tile_rep, s->d_frcf,
                                                              s->d_frcd, s->d_gid, df);
    CK(cudaGetLastError());
    if (!on_device) CK(cudaMemcpyAsync(f, df, 24 * (size_t)s->n_total, cudaMemcpyDeviceToHost, s->stream));
  }
  CKS(download_reps(s));
  for (int r = 0; r < s->nrep; ++r) {
    if (pe) pe[r] = s->reps[r].pe;
    if (virial) virial[r] = s->reps[r].vir;
  }
  return MD_OK;
}

static md_status step_common(md_system* s, int kind, double dt, int64_t nsteps, int64_t nstep_boltz, uint64_t seed,
                             md_thermo* log, int64_t log_every) {
  if (!s->have_state) return fail(s, MD_ERR_INVALID_ARG, "no state: call md_set_state or md_init_lattice first");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(s, MD_ERR_INVALID_ARG, "dt must be > 0");
  if (nsteps < 0) return fail(s, MD_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (log && log_every <= 0) return fail(s, MD_ERR_INVALID_ARG, "log_every must be > 0 when log is given");
  const int64_t nlog = (log && log_every > 0) ? nsteps / log_every : 0;
  CKS(ensure_thermo(s, nlog * s->nrep));
  // room for the partial records of up to MD_LOG_SLOTS NVE log steps per
  // launch (at most 256 MB), reduced after the launch's last step; the
  // Nose-Hoover kinds reduce every step anyway
  int slots = 0;
  if (nlog > 0 && kind != MD_KIND_NH && kind != MD_KIND_NH_EXACT && !s->log_now) {
    const size_t stride = (size_t)s->ntiles * s->tun.threads_per_atom * MD_NPART;
    const size_t most = ((size_t)256 << 20) / sizeof(double) / stride;
    slots = (int)std::min<int64_t>(std::min<int64_t>(nlog, MD_LOG_SLOTS), (int64_t)most);
    if (slots > 0 && (size_t)slots * stride > s->plog_cap) {
      dfree(s, s->d_plog);
      s->d_plog = nullptr;
      s->plog_cap = 0;
      CKS(dalloc(s, &s->d_plog, (size_t)slots * stride));
      s->plog_cap = (size_t)slots * stride;
    }
  }
  s->plog_slots = slots;
  int64_t done = 0;
  md_status st = run_op(s, MD_OP_STEPS, kind, dt, nsteps, nstep_boltz, seed, log ? log_every : 0, nlog, &done);
  s->plog_slots = 0;
  if (st != MD_OK) return st;
  if (nlog > 0) {
    CK(cudaMemcpyAsync(log, s->d_thermo, sizeof(ThermoDev) * nlog * s->nrep, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  return MD_OK;
}

md_status md_step_nve(md_system* s, double dt, int64_t nsteps, md_thermo* log, int64_t log_every) {
  if (!s) return fail(nullptr, MD_ERR_INVALID_ARG, "NULL system");
  return step_common(s, MD_KIND_NVE, dt, nsteps, 0, 0, log, log_every);
}

md_status md_step_nvt(md_system* s, double dt, int64_t nsteps, const double* T_target, md_thermostat kind, double param,
                      uint64_t seed, md_thermo* log, int64_t log_every) {
  if (!s) return fail(nullptr, MD_ERR_INVALID_ARG, "NULL system");
  if (!T_target) return fail(s, MD_ERR_INVALID_ARG, "T_target must not be NULL");
  for (int r = 0; r < s->nrep; ++r)
    if (!(T_target[r] >= 0) || !std::isfinite(T_target[r])) return fail(s, MD_ERR_INVALID_ARG, "T_target must be >= 0");
  int k;
  int64_t nb = 0;
  if (kind == MD_NVT_NOSE_HOOVER || kind == MD_NVT_NOSE_HOOVER_EXACT) {
    if (!(param > 0)) return fail(s, MD_ERR_INVALID_ARG, "Nose-Hoover needs tau > 0");
    for (int r = 0; r < s->nrep; ++r)
      if (!(T_target[r] > 0)) return fail(s, MD_ERR_INVALID_ARG, "Nose-Hoover needs T_target > 0");
    k = kind == MD_NVT_NOSE_HOOVER ? MD_KIND_NH : MD_KIND_NH_EXACT;
  } else if (kind == MD_NVT_RESAMPLE) {
    nb = (int64_t)param;
    if (nb < 1) return fail(s, MD_ERR_INVALID_ARG, "resampling needs nstep_boltz >= 1");
    k = MD_KIND_RESAMPLE;
  } else {
    return fail(s, MD_ERR_INVALID_ARG, "unknown thermostat");
  }
  CKS(download_reps(s));
  for (int r = 0; r < s->nrep; ++r) {
    RepDev& R = s->reps[r];
    R.T_target = T_target[r];
    if (k != MD_KIND_RESAMPLE) R.Q = (double)s->ndim * R.n * T_target[r] * param * param;
  }
  CKS(upload_reps(s));
  return step_common(s, k, dt, nsteps, nb, seed, log, log_every);
}

md_status md_rdf(md_system* s, double dr, int64_t nbins, double* g, int reset) {
  if (!s) return fail(nullptr, MD_ERR_INVALID_ARG, "NULL system");
  if (!s->have_state) return fail(s, MD_ERR_INVALID_ARG, "no state");
  if (s->ntypes != 2) return fail(s, MD_ERR_INVALID_ARG, "md_rdf needs a 2-type system");
  if (!(dr > 0) || nbins < 1) return fail(s, MD_ERR_INVALID_ARG, "dr > 0 and nbins >= 1 required");
  for (int r = 0; r < s->nrep; ++r)
    if (dr * nbins > 0.5 * s->L_per[r] * (1 + 1e-12)) return fail(s, MD_ERR_INVALID_ARG, "nbins*dr must be <= L/2");
  if (reset || !s->d_rdf || nbins != s->rdf_nbins || dr != s->rdf_dr) {
    dfree(s, s->d_rdf);
    CKS(dalloc(s, &s->d_rdf, (size_t)s->nrep * 3 * nbins));
    s->rdf_nbins = nbins;
    s->rdf_dr = dr;
    s->rdf_meas = 0;
  }
  // the histogram walks the cell lists of the last build: make them current
  CKS(download_ctl(s));
  if (s->ctl.pending & MD_FLAG_REBUILD) CKS(run_op(s, MD_OP_REBUILD, MD_KIND_NVE, 0, 0, 0, 0, 0, 0, nullptr));
  CKS(download_ctl(s));
  const int b = 128;
  k_rdf<<<blocks_for(s->ntot, b), b, 0, s->stream>>>(s->mixed, s->ntot, (int)nbins, dr, s->tun.skin_outer, s->d_reps, s->d_tile_rep,
                                                     s->ctl.cur, s->d_pq[s->ctl.cur], s->d_pfx, s->d_p4[s->ctl.cur],
                                                     s->d_typ, s->d_cstart, s->d_rdf);
  CK(cudaGetLastError());
  s->rdf_meas += 1;
  if (g) {
    std::vector<unsigned long long> h((size_t)s->nrep * 3 * nbins);
    CK(cudaMemcpyAsync(h.data(), s->d_rdf, 8 * h.size(), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    std::vector<uint8_t> types(s->n_total);
    CK(cudaMemcpy(types.data(), s->d_typ_caller, s->n_total, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < 3 * nbins; ++k) g[k] = 0.0;
    for (int r = 0; r < s->nrep; ++r) {
      int64_t na = 0, nb = 0;
      for (int64_t q = 0; q < s->n_per[r]; ++q) (types[s->out0[r] + q] == 0 ? na : nb) += 1;
      // V and the shell volume of bin k; in two dimensions the area L^2 and the ring pi((k+1)^2 - k^2)dr^2
      const double Lr = s->L_per[r];
      const double V = s->ndim == 3 ? Lr * Lr * Lr : Lr * Lr;
      for (int64_t k = 0; k < nbins; ++k) {
        const double shell =
            s->ndim == 3 ? 4.0 / 3.0 * M_PI * (std::pow((double)(k + 1), 3) - std::pow((double)k, 3)) * dr * dr * dr
                         : M_PI * (std::pow((double)(k + 1), 2) - std::pow((double)k, 2)) * dr * dr;
        const unsigned long long* hr = h.data() + (size_t)r * 3 * nbins;
        const double m = (double)s->rdf_meas * s->nrep;
        if (na > 1) g[k] += hr[k] / shell * V / ((double)na * (na - 1)) / m;
        if (nb > 1) g[nbins + k] += hr[nbins + k] / shell * V / ((double)nb * (nb - 1)) / m;
        if (na > 0 && nb > 0) g[2 * nbins + k] += hr[2 * nbins + k] / shell * V / ((double)na * nb) / m;
      }
    }
  }
  return MD_OK;
}

md_status md_msd_tw(md_system* s, int slot, double* msd_per_type, int reset_reference) {
  if (!s) return fail(nullptr, MD_ERR_INVALID_ARG, "NULL system");
  if (!s->have_state) return fail(s, MD_ERR_INVALID_ARG, "no state");
  if (slot < 0 || slot >= MD_MSD_SLOTS) return fail(s, MD_ERR_INVALID_ARG, "MSD slot out of range");
  CKS(download_ctl(s));
  if (reset_reference) CKS(reset_msd_ref(s, slot));
  if (!s->msd_valid[slot]) return fail(s, MD_ERR_INVALID_ARG, "MSD slot has no reference (reset it first)");
  const int b = 256;
  k_msd_tiles<<<blocks_for((int64_t)s->ntiles * 32, b), b, 0, s->stream>>>(
      s->mixed, s->ntiles, s->ntypes, s->ntot, s->d_reps, s->d_tile_rep, s->d_pfx, s->d_p4[s->ctl.cur], s->d_gid,
      s->d_typ, s->d_img, s->d_msd_ref[slot], s->d_msd_part);
  CK(cudaGetLastError());
  k_msd_final<<<1, 32, 0, s->stream>>>(s->ntiles, s->ntypes, s->d_msd_part, s->d_io);
  CK(cudaGetLastError());
  if (msd_per_type) CK(cudaMemcpyAsync(msd_per_type, s->d_io, 8 * s->ntypes, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return MD_OK;
}

md_status md_msd(md_system* s, double* msd_per_type, int reset_reference) {
  return md_msd_tw(s, 0, msd_per_type, reset_reference);
}

md_status md_set_tuning(md_system* s, const md_tuning* t) {
  if (!s || !t) return fail(s, MD_ERR_INVALID_ARG, "NULL argument");
  CKS(tuning_ok(s, t));
  CKS(download_reps(s));
  s->tun = *t;
  layout_cells(s);
  for (auto& R : s->reps) R.want_rebuild = 1;
  s->stage_cap = stage_capacity(s);  // also picks each replica's group shape
  CKS(upload_reps(s));
  CKS(alloc_cells_and_list(s, list_capacity(s)));
  CKS(configure_grid(s));
  CKS(download_ctl(s));
  s->ctl.pending |= MD_FLAG_REBUILD;
  CKS(upload_ctl(s));
  return MD_OK;
}

// fixed_skin > 0: the force list's skin stays fixed_skin and only the outer
// skin is searched; otherwise both are.
static md_status autotune_impl(md_system* s, double dt, int64_t probe_steps, double fixed_skin, md_tuning* best,
                               double* seconds_per_step) {
  if (!s) return fail(nullptr, MD_ERR_INVALID_ARG, "NULL system");
  if (!s->have_state) return fail(s, MD_ERR_INVALID_ARG, "no state");
  if (!(dt > 0) || probe_steps < 1) return fail(s, MD_ERR_INVALID_ARG, "dt > 0 and probe_steps >= 1 required");
  // save the state (caller order, device) and the per-replica bath state
  const size_t n3 = 3 * (size_t)s->n_total;
  double* saved = nullptr;
  int32_t* saved_img = nullptr;
  CKS(dalloc(s, &saved, 2 * n3));
  CKS(dalloc(s, &saved_img, n3));
  md_status st = md_get_state(s, saved, saved + n3, saved_img, 1);
  if (st != MD_OK) { dfree(s, saved); dfree(s, saved_img); return st; }
  CKS(download_reps(s));
  const std::vector<RepDev> saved_reps = s->reps;
  const int64_t saved_step = s->ctl.step;
  const md_tuning start = s->tun;
  md_tuning bt = start;
  // starting skins of the first search stage
  const double s0 = fixed_skin > 0 ? fixed_skin : start.skin;
  const double so0 = fixed_skin > 0 ? fixed_skin : start.skin_outer;
  float bms = 1e30f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // one probe: set the candidate, restart from the saved state, warm up,
  // then time probe_steps NVE steps
  auto probe = [&](const md_tuning& c) {
    if (st != MD_OK) return;
    if (c.block_size < 32 * c.threads_per_atom) return;
    if (tuning_ok(s, &c) != MD_OK) return;
    st = md_set_tuning(s, &c);
    if (st == MD_OK) st = set_state_impl(s, saved, saved + n3, 1);
    if (st == MD_OK) st = md_step_nve(s, dt, std::max<int64_t>(probe_steps / 4, 1), nullptr, 0);
    if (st != MD_OK) return;
    cudaEventRecord(e0, s->stream);
    st = md_step_nve(s, dt, probe_steps, nullptr, 0);
    cudaEventRecord(e1, s->stream);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (st == MD_OK && ms < bms) { bms = ms; bt = c; }
  };
  const int Ts[4] = {1, 2, 4, 8};
  const int Bs[3] = {128, 256, 512};
  // (skin, skin_outer); equal values mean one list without pruning
  const double Sfree[9][2] = {{0.2, 0.2}, {0.3, 0.3}, {0.4, 0.4}, {0.2, 0.5}, {0.2, 0.7},
                              {0.3, 0.6}, {0.3, 0.8}, {0.3, 1.0}, {0.4, 0.9}};
  double Ss[9][2];
  int nS = 0;
  if (fixed_skin > 0) {
    const double extra[6] = {0.0, 0.3, 0.5, 0.7, 0.9, 1.1};
    for (int k = 0; k < 6; ++k) { Ss[nS][0] = fixed_skin; Ss[nS][1] = fixed_skin + extra[k]; ++nS; }
  } else {
    for (int k = 0; k < 9; ++k) { Ss[nS][0] = Sfree[k][0]; Ss[nS][1] = Sfree[k][1]; ++nS; }
  }
  // coordinate search: lanes x block size at the starting skins, then the
  // skins at the best of those, then lanes x block size again at the best skins
  for (int ti = 0; ti < 4; ++ti)
    for (int bi = 0; bi < 3; ++bi) probe(md_tuning{Ts[ti], Bs[bi], s0, so0});
  const md_tuning b1 = bt;
  for (int si = 0; si < nS; ++si)
    if (!(Ss[si][0] == s0 && Ss[si][1] == so0))
      probe(md_tuning{b1.threads_per_atom, b1.block_size, Ss[si][0], Ss[si][1]});
  const md_tuning b2 = bt;
  if (!(b2.skin == s0 && b2.skin_outer == so0))
    for (int ti = 0; ti < 4; ++ti)
      for (int bi = 0; bi < 3; ++bi)
        if (!(Ts[ti] == b2.threads_per_atom && Bs[bi] == b2.block_size))
          probe(md_tuning{Ts[ti], Bs[bi], b2.skin, b2.skin_outer});
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  md_status st2 = md_set_tuning(s, st == MD_OK ? &bt : &start);
  if (st2 == MD_OK) st2 = set_state_impl(s, saved, saved + n3, 1);
  if (st2 == MD_OK) {
    const int b = 256;
    k_set_images<<<blocks_for(s->n_total, b), b, 0, s->stream>>>(s->n_total, s->ntot, s->d_reps, s->d_rep_of_caller,
                                                                 saved_img, s->d_img);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) st2 = cuda_fail(s, ce, "k_set_images");
  }
  if (st2 == MD_OK) st2 = download_reps(s);
  if (st2 == MD_OK) {
    for (int r = 0; r < s->nrep; ++r) {
      RepDev& R = s->reps[r];
      const RepDev& O = saved_reps[r];
      R.T_target = O.T_target; R.Q = O.Q; R.xi = O.xi; R.g = O.g; R.lns = O.lns; R.lns_next = O.lns_next;
      R.xi_a = O.xi_a; R.rebuilds = O.rebuilds;
    }
    st2 = upload_reps(s);
  }
  if (st2 == MD_OK) {
    s->ctl.step = saved_step;
    st2 = upload_ctl(s);
  }
  if (st2 == MD_OK) st2 = reset_msd_ref(s);
  cudaStreamSynchronize(s->stream);
  dfree(s, saved);
  dfree(s, saved_img);
  if (st != MD_OK) return st;
  if (st2 != MD_OK) return st2;
  if (best) *best = bt;
  if (seconds_per_step) *seconds_per_step = (double)bms * 1e-3 / (double)probe_steps;
  return MD_OK;
}

md_status md_autotune(md_system* s, double dt, int64_t probe_steps, md_tuning* best, double* seconds_per_step) {
  return autotune_impl(s, dt, probe_steps, -1.0, best, seconds_per_step);
}

md_status md_autotune_skin(md_system* s, double dt, int64_t probe_steps, double skin, md_tuning* best,
                           double* seconds_per_step) {
  if (!(skin >= 0.05) || !(skin < 2.0)) return fail(s, MD_ERR_INVALID_ARG, "skin must be in [0.05, 2)");
  return autotune_impl(s, dt, probe_steps, skin, best, seconds_per_step);
}

md_status md_time_forces(md_system* s, int64_t repeats, double* seconds_per_eval) {
  if (!s || !seconds_per_eval) return fail(s, MD_ERR_INVALID_ARG, "NULL argument");
  if (!s->have_state) return fail(s, MD_ERR_INVALID_ARG, "no state: call md_set_state or md_init_lattice first");
  if (repeats < 1 || repeats > 100000) return fail(s, MD_ERR_INVALID_ARG, "repeats must be in [1, 100000]");
  // bring the lists up to date first (a rebuild would otherwise be timed too)
  CKS(download_ctl(s));
  if (s->ctl.drifted) return fail(s, MD_ERR_INVALID_ARG, "the state is between a position and a velocity update");
  if (s->ctl.pending & (MD_FLAG_REBUILD | MD_FLAG_PRUNE))
    CKS(run_op(s, MD_OP_REBUILD, MD_KIND_NVE, 0, 0, 0, 0, 0, 0, nullptr));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  md_status st = MD_OK;
  float ms = 0.0f, ms1 = 0.0f;
  // the launch's fixed cost (start, first barrier, end) is taken out by a
  // launch with one evaluation: seconds = (t(repeats) - t(1)) / (repeats - 1)
  for (int pass = 0; pass < 2 && st == MD_OK; ++pass) {
    const int64_t k = pass == 0 ? 1 : repeats;
    cudaEventRecord(e0, s->stream);
    st = run_op(s, MD_OP_FORCE_REPEAT, MD_KIND_NVE, 0.0, k, 0, 0, 0, 0, nullptr);
    cudaEventRecord(e1, s->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(pass == 0 ? &ms1 : &ms, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MD_OK) return st;
  *seconds_per_eval = repeats > 1 ? (double)(ms - ms1) * 1e-3 / (double)(repeats - 1) : (double)ms * 1e-3;
  return MD_OK;
}

md_status md_time_lists(md_system* s, int64_t repeats, double* seconds_per_build) {
  if (!s || !seconds_per_build) return fail(s, MD_ERR_INVALID_ARG, "NULL argument");
  if (!s->have_state) return fail(s, MD_ERR_INVALID_ARG, "no state: call md_set_state or md_init_lattice first");
  if (repeats < 2 || repeats > 10000) return fail(s, MD_ERR_INVALID_ARG, "repeats must be in [2, 10000]");
  CKS(download_ctl(s));
  if (s->ctl.drifted) return fail(s, MD_ERR_INVALID_ARG, "the state is between a position and a velocity update");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  md_status st = MD_OK;
  float ms = 0.0f, ms1 = 0.0f;
  // both launches start with the same full rebuild, which the difference
  // takes out with the launch's fixed cost
  for (int pass = 0; pass < 2 && st == MD_OK; ++pass) {
    const int64_t k = pass == 0 ? 1 : repeats;
    st = mark_rebuild_all(s);
    if (st != MD_OK) break;
    cudaEventRecord(e0, s->stream);
    st = run_op(s, MD_OP_LIST_REPEAT, MD_KIND_NVE, 0.0, k, 0, 0, 0, 0, nullptr);
    cudaEventRecord(e1, s->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(pass == 0 ? &ms1 : &ms, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MD_OK) return st;
  *seconds_per_build = (double)(ms - ms1) * 1e-3 / (double)(repeats - 1);
  return MD_OK;
}

md_status md_get_tuning(const md_system* s, md_tuning* t) {
  if (!s || !t) return MD_ERR_INVALID_ARG;
  *t = s->tun;
  return MD_OK;
}

md_status md_get_info(md_system* s, md_info* info) {
  if (!s || !info) return fail(s, MD_ERR_INVALID_ARG, "NULL argument");
  CKS(download_reps(s));
  CKS(download_ctl(s));
  std::memset(info, 0, sizeof(*info));
  info->n_total = s->n_total;
  info->n_replicas = s->nrep;
  info->grid_blocks = s->grid;
  info->steps_done = s->ctl.step;
  for (const auto& R : s->reps) {
    info->rebuilds += R.rebuilds;
    info->all_pairs_replicas += R.nc == 0;
  }
  CK(cudaMemsetAsync(s->d_count, 0, 8, s->stream));
  // entries of the list the force phase reads: the inner list when there are two
  const bool dual = s->tun.skin_outer > s->tun.skin;
  k_sum_i32<<<std::max(1, std::min(1024, blocks_for(s->ntot * s->tun.threads_per_atom, 256))), 256, 0, s->stream>>>(
      s->ntot * s->tun.threads_per_atom, dual ? s->d_nnb_in : s->d_nnb, s->d_count);
  CK(cudaGetLastError());
  unsigned long long entries = 0;
  CK(cudaMemcpyAsync(&entries, s->d_count, 8, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  info->list_entries = (int64_t)entries;
  info->list_capacity = (int64_t)s->maxrows * s->tun.threads_per_atom;
  info->device_bytes = (int64_t)s->bytes;
  info->precision = s->mixed ? MD_PREC_MIXED : MD_PREC_FP64;
  info->graph_launches = s->graph_launches;
  info->prunes = s->ctl.prunes;
  info->kernel_launches = s->kernel_launches;
  return MD_OK;
}

md_status md_count_pairs(md_system* s, int64_t* pairs) {
  if (!s || !pairs) return fail(s, MD_ERR_INVALID_ARG, "NULL argument");
  if (!s->have_state) return fail(s, MD_ERR_INVALID_ARG, "no state");
  CKS(download_ctl(s));
  if (s->ctl.pending & MD_FLAG_REBUILD) CKS(run_op(s, MD_OP_REBUILD, MD_KIND_NVE, 0, 0, 0, 0, 0, 0, nullptr));
  CKS(download_ctl(s));
  double rc2d[16];
  for (int t = 0; t < s->ntypes * s->ntypes; ++t) rc2d[t] = s->rc[t] * s->rc[t];
  CK(cudaMemcpyAsync(s->d_io, rc2d, sizeof(double) * s->ntypes * s->ntypes, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemsetAsync(s->d_count, 0, 8, s->stream));
  const int b = 128;
  k_count_pairs<<<blocks_for(s->ntot, b), b, 0, s->stream>>>(
      s->mixed, s->ntot, s->ntypes, rc_max(s) + s->tun.skin_outer, s->d_reps, s->d_tile_rep, s->d_pfx,
      s->d_p4[s->ctl.cur], s->d_typ, s->d_cstart, s->d_io, s->d_count);
  CK(cudaGetLastError());
  unsigned long long c = 0;
  CK(cudaMemcpyAsync(&c, s->d_count, 8, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  *pairs = (int64_t)c;
  return MD_OK;
}

md_status md_selftest_barrier(md_system* s, double timeout_s) {
  if (!s) return fail(nullptr, MD_ERR_INVALID_ARG, "NULL system");
  if (!(timeout_s > 0) || timeout_s > 60) return fail(s, MD_ERR_INVALID_ARG, "timeout_s must be in (0, 60]");
  CKS(download_ctl(s));
  const CtlDev saved = s->ctl;
  s->ctl.pending = 0;
  CKS(upload_ctl(s));
  KParams p = make_params(s);
  p.timeout_ns = (unsigned long long)(timeout_s * 1e9);
  CK(md_launch_barrier_selftest(p, 4, s->stream));
  CKS(download_ctl(s));
  const int pend = s->ctl.pending;
  // restore the control block so the system stays usable
  s->ctl = saved;
  CKS(upload_ctl(s));
  CK(cudaStreamSynchronize(s->stream));
  if (pend & MD_FLAG_TIMEOUT) return fail(s, MD_ERR_TIMEOUT, "barrier wait ran out as intended (self-test)");
  return fail(s, MD_ERR_CUDA, "barrier self-test: the wait did not run out");
}

#ifdef KAMD_PHASE_TIMERS
// profiling builds only: copy out (and clear) the per-barrier phase timers
md_status md_debug_phase_times(md_system* s, double* ns, double* cnt) {
  CKS(download_ctl(s));
  for (int k = 0; k < 128; ++k) {
    ns[k] = (double)s->ctl.phase_ns[k];
    cnt[k] = (double)s->ctl.phase_cnt[k];
    s->ctl.phase_ns[k] = 0;
    s->ctl.phase_cnt[k] = 0;
  }
  s->ctl.t_last = 0;
  return upload_ctl(s);
}
#endif

const char* md_last_error(const md_system* s) {
  if (!s) return g_create_err.c_str();
  return s->err.c_str();
}

void md_destroy(md_system* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  drop_graph(s);
  dfree(s, s->d_reps); dfree(s, s->d_tile_rep); dfree(s, s->d_ctl);
  dfree(s, s->d_pfx); dfree(s, s->d_pq[0]); dfree(s, s->d_pq[1]); dfree(s, s->d_velf); dfree(s, s->d_frcf); dfree(s, s->d_xbq);
  dfree(s, s->d_xbq_in); dfree(s, s->d_xbd_in); dfree(s, s->d_nbr_in); dfree(s, s->d_nnb_in);
  dfree(s, s->d_p4[0]); dfree(s, s->d_p4[1]); dfree(s, s->d_veld); dfree(s, s->d_frcd); dfree(s, s->d_xbd);
  dfree(s, s->d_gid); dfree(s, s->d_typ); dfree(s, s->d_img);
  dfree(s, s->d_tpfx); dfree(s, s->d_tp4); dfree(s, s->d_tvel); dfree(s, s->d_tfrc); dfree(s, s->d_tgid); dfree(s, s->d_ttyp);
  dfree(s, s->d_timg);
  dfree(s, s->d_cellof); dfree(s, s->d_cell_rep); dfree(s, s->d_ccount); dfree(s, s->d_cstart); dfree(s, s->d_ccursor); dfree(s, s->d_chunk); dfree(s, s->d_cta_sm); dfree(s, s->d_grp); dfree(s, s->d_redmap); dfree(s, s->d_redrep); dfree(s, s->d_redpart); dfree(s, s->d_scat);
  dfree(s, s->d_nbr); dfree(s, s->d_nnb); dfree(s, s->d_part[0]); dfree(s, s->d_part[1]); dfree(s, s->d_plog); dfree(s, s->d_plog_rec);
  dfree(s, s->d_typ_caller); dfree(s, s->d_rep_of_caller); dfree(s, s->d_thermo); dfree(s, s->d_io);
  dfree(s, s->d_io_i); dfree(s, s->d_rdf); dfree(s, s->d_msd_part); dfree(s, s->d_count);
  for (int k = 0; k < MD_MSD_SLOTS; ++k) dfree(s, s->d_msd_ref[k]);
  delete s;
}

}  // extern "C"
