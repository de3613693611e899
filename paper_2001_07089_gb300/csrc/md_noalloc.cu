// md_noalloc.cu -- md_forces_noalloc: forces of one configuration with no
// device allocation at all.
//
// Some callers cannot call cudaMalloc: code that enqueues work while a CUDA
// stream is being captured into a graph (a cudaMalloc there is illegal or
// silently leaves the graph), plugins and real-time loops that must not take
// the allocator's implicit device synchronisation, and hosts that hand the
// library a fixed memory budget they own. For them this entry point keeps all
// of its scratch (cell counts, cell starts, the cell-sorted index, per-block
// partial sums) in one file-scope device array of fixed size, allocated when
// the library is loaded and held until the process exits. The caller passes
// device pointers for every input and output.
//
// Arithmetic: all FP64, the same pair term and minimum-image rule as the FP64
// path of md_forces; one thread per particle gathers over the 27 neighbouring
// cells (every particle when fewer than 3 cells fit per box edge).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "kamd.h"
#include "md_internal.cuh"

namespace {

constexpr int64_t kMaxParticles = 131072;  // 2^17
constexpr int kMaxCells = 32768;
constexpr int kMaxCellsPerEdge = 32;  // kMaxCells = 32^3
constexpr int kBlock = 256;
constexpr int kMaxBlocks = (int)(kMaxParticles / kBlock);
constexpr int kMaxTypes = 4;

// Scratch layout (bytes): cellof[n] i32 | count[cells] i32 | start[cells+1] i32 |
// cursor[cells] i32 | sorted[n] i32 | partial[blocks][2] f64 | ticket u32
constexpr size_t kOffCellof = 0;
constexpr size_t kOffCount = kOffCellof + 4 * kMaxParticles;
constexpr size_t kOffStart = kOffCount + 4 * kMaxCells;
constexpr size_t kOffCursor = kOffStart + 4 * (kMaxCells + 1) + 4;  // keep 8-byte alignment below
constexpr size_t kOffSorted = kOffCursor + 4 * kMaxCells;
constexpr size_t kOffPart = (kOffSorted + 4 * kMaxParticles + 255) / 256 * 256;
constexpr size_t kOffTicket = kOffPart + 16 * (size_t)kMaxBlocks;
constexpr size_t kScratchBytes = (kOffTicket + 256 + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Table {
  double rc2[kMaxTypes * kMaxTypes], sig2[kMaxTypes * kMaxTypes], e48[kMaxTypes * kMaxTypes],
      e4[kMaxTypes * kMaxTypes], vsh[kMaxTypes * kMaxTypes];
};

struct Scratch {
  int32_t* cellof;
  int32_t* count;
  int32_t* start;
  int32_t* cursor;
  int32_t* sorted;
  double* part;
  unsigned int* ticket;
};

Scratch carve(unsigned char* base) {
  Scratch s;
  s.cellof = reinterpret_cast<int32_t*>(base + kOffCellof);
  s.count = reinterpret_cast<int32_t*>(base + kOffCount);
  s.start = reinterpret_cast<int32_t*>(base + kOffStart);
  s.cursor = reinterpret_cast<int32_t*>(base + kOffCursor);
  s.sorted = reinterpret_cast<int32_t*>(base + kOffSorted);
  s.part = reinterpret_cast<double*>(base + kOffPart);
  s.ticket = reinterpret_cast<unsigned int*>(base + kOffTicket);
  return s;
}

__device__ __forceinline__ double wrap01(double x, double L) {
  x -= L * floor(x / L);
  if (x >= L) x -= L;
  if (x < 0.0) x = 0.0;
  return x;
}

__device__ __forceinline__ int cell_index(const double* pos, int64_t i, int nc, double L) {
  int c[3];
  for (int k = 0; k < 3; ++k) {
    const double x = wrap01(pos[3 * i + k], L);
    c[k] = min(max((int)(x * nc / L), 0), nc - 1);
  }
  return (c[2] * nc + c[1]) * nc + c[0];
}

__global__ void k_clear(Scratch s, int ncells) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) s.count[c] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *s.ticket = 0u;
}

__global__ void k_bin(Scratch s, const double* pos, int64_t n, int nc, double L) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = cell_index(pos, i, nc, L);
  s.cellof[i] = c;
  atomicAdd(&s.count[c], 1);
}

// One block: exclusive scan of the cell counts into start and cursor.
__global__ void k_scan(Scratch s, int ncells) {
  __shared__ int warp_tot[32];
  const int per = (ncells + blockDim.x - 1) / blockDim.x;
  const int b0 = min((int)threadIdx.x * per, ncells), b1 = min(b0 + per, ncells);
  int sum = 0;
  for (int c = b0; c < b1; ++c) sum += s.count[c];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_tot[lane] = w;
  }
  __syncthreads();
  int run = (warp > 0 ? warp_tot[warp - 1] : 0) + x - sum;
  for (int c = b0; c < b1; ++c) {
    s.start[c] = run;
    s.cursor[c] = run;
    run += s.count[c];
  }
  if (threadIdx.x == blockDim.x - 1) s.start[ncells] = run;
}

__global__ void k_scatter(Scratch s, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int slot = atomicAdd(&s.cursor[s.cellof[i]], 1);
  s.sorted[slot] = (int32_t)i;
}

// One warp per cell: order the members by particle index (deterministic).
__global__ void k_order(Scratch s, int ncells) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < ncells; c += warps) {
    const int lo = s.start[c], m = s.start[c + 1] - lo;
    // members are at most a few dozen: sort in registers chunk by chunk
    for (int e0 = 0; e0 < m; e0 += 32) {
      const int mine = e0 + lane < m ? s.sorted[lo + e0 + lane] : 0x7fffffff;
      int rank = 0;
      for (int m0 = 0; m0 < m; m0 += 32) {
        const int other = m0 + lane < m ? s.sorted[lo + m0 + lane] : 0x7fffffff;
        const int lim = min(32, m - m0);
        for (int t = 0; t < lim; ++t) rank += (__shfl_sync(0xffffffffu, other, t) < mine);
      }
      // write into cellof (free after scatter) to avoid overwriting unread members
      if (e0 + lane < m) s.cellof[lo + rank] = mine;
    }
  }
}

__global__ void k_forces(Scratch s, const double* pos, const uint8_t* types, int64_t n, int ntypes, int nc, double L,
                         Table tab, double* f, double* pe_out, double* vir_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double fx = 0, fy = 0, fz = 0, pe = 0, vir = 0;
  if (i < n) {
    const double xi[3] = {wrap01(pos[3 * i], L), wrap01(pos[3 * i + 1], L), wrap01(pos[3 * i + 2], L)};
    const int ti = types[i];
    // a type outside [0, ntypes) never indexes the tables: the particle's
    // results (and those of particles that meet it) become NaN instead
    bool bad = ti >= ntypes;
    const double hL = 0.5 * L;
    auto pair = [&](int64_t j) {
      if (j == i || bad) return;
      double d[3];
      for (int k = 0; k < 3; ++k) {
        double e = xi[k] - wrap01(pos[3 * j + k], L);
        if (e > hL) e -= L;
        else if (e < -hL) e += L;
        d[k] = e;
      }
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      const int tj = types[j];
      if (tj >= ntypes) {
        bad = true;
        return;
      }
      const int t = ti * ntypes + tj;
      if (r2 < tab.rc2[t]) {
        const double ir2 = 1.0 / r2;
        const double s2 = tab.sig2[t] * ir2;
        const double s6 = s2 * s2 * s2;
        const double w = tab.e48[t] * s6 * (s6 - 0.5);
        const double fr = w * ir2;
        fx += fr * d[0];
        fy += fr * d[1];
        fz += fr * d[2];
        pe += tab.e4[t] * s6 * (s6 - 1.0) - tab.vsh[t];
        vir += w;
      }
    };
    if (nc >= 3) {
      int c[3];
      for (int k = 0; k < 3; ++k) c[k] = min(max((int)(xi[k] * nc / L), 0), nc - 1);
      for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            const int cc = (((c[2] + oz + nc) % nc) * nc + (c[1] + oy + nc) % nc) * nc + (c[0] + ox + nc) % nc;
            for (int q = s.start[cc]; q < s.start[cc + 1]; ++q) pair(s.cellof[q]);
          }
    } else {
      for (int64_t j = 0; j < n; ++j) pair(j);
    }
    if (bad) fx = fy = fz = pe = vir = __longlong_as_double(0x7ff8000000000000ll);
    f[3 * i] = fx;
    f[3 * i + 1] = fy;
    f[3 * i + 2] = fz;
  }
  // fixed-order block sums of the half pair energies and virials
  __shared__ double spe[kBlock], svir[kBlock];
  spe[threadIdx.x] = 0.5 * pe;
  svir[threadIdx.x] = 0.5 * vir;
  __syncthreads();
  for (int o = kBlock / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      spe[threadIdx.x] += spe[threadIdx.x + o];
      svir[threadIdx.x] += svir[threadIdx.x + o];
    }
    __syncthreads();
  }
  __shared__ bool last;
  if (threadIdx.x == 0) {
    s.part[2 * blockIdx.x] = spe[0];
    s.part[2 * blockIdx.x + 1] = svir[0];
    __threadfence();
    last = atomicAdd(s.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double a = 0, b = 0;
    for (unsigned k = 0; k < gridDim.x; ++k) {
      a += ((volatile double*)s.part)[2 * k];
      b += ((volatile double*)s.part)[2 * k + 1];
    }
    if (pe_out) *pe_out = a;
    if (vir_out) *vir_out = b;
  }
}

md_status noalloc_fail(md_status st, const std::string& m) {
  kamd_set_global_error(m);
  return st;
}

// Device address of the static scratch array, per CUDA context. The host-side
// name g_noalloc_scratch is a stand-in, not a device address, and the array
// moves whenever the module is loaded again (a new context after
// cudaDeviceReset, or another context on the same device). So the address is
// looked up afresh on every call made outside a stream capture, and the
// cached value of the current context is used only while a capture is open
// (where the look-up itself is not allowed).
typedef int (*CtxGetCurrentFn)(void**);

struct ScratchSlot {
  void* ctx;
  unsigned char* ptr;
};
constexpr int kSlots = 64;
ScratchSlot g_slots[kSlots];
int g_nslots = 0;
std::mutex g_slots_mu;

CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

md_status scratch_address(cudaStream_t st, unsigned char** out) {
  CtxGetCurrentFn get = ctx_get_current();
  if (!get) return noalloc_fail(MD_ERR_CUDA, "md_forces_noalloc: cuCtxGetCurrent is not available");
  // the capture query also sets up the runtime's context on this thread if
  // nothing else has yet
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return noalloc_fail(MD_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  void* ctx = nullptr;
  if (get(&ctx) != 0 || !ctx) return noalloc_fail(MD_ERR_CUDA, "md_forces_noalloc: no current CUDA context");
  std::lock_guard<std::mutex> lock(g_slots_mu);
  int k = 0;
  while (k < g_nslots && g_slots[k].ctx != ctx) ++k;
  if (cap != cudaStreamCaptureStatusNone) {
    if (k == g_nslots)
      return noalloc_fail(MD_ERR_INVALID_ARG,
                          "md_forces_noalloc: make one call in this CUDA context before capturing a stream");
    *out = g_slots[k].ptr;
    return MD_OK;
  }
  void* ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr)
    return noalloc_fail(MD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  if (k == g_nslots) {
    if (g_nslots == kSlots) k = 0;  // many contexts: reuse the oldest slot
    else ++g_nslots;
  }
  g_slots[k] = ScratchSlot{ctx, static_cast<unsigned char*>(ptr)};
  *out = g_slots[k].ptr;
  return MD_OK;
}

}  // namespace

extern "C" md_status md_forces_noalloc(int64_t n, const double* pos, const uint8_t* types, int ntypes, double L,
                                       const double* eps, const double* sigma, const double* rc, double* f, double* pe,
                                       double* virial, void* stream) {
  if (n < 2 || n > kMaxParticles)
    return noalloc_fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: n must be in [2, 131072] (fixed scratch size)");
  if (!pos || !types || !f || !eps || !sigma || !rc)
    return noalloc_fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: pos, types, f and the tables are required");
  if (ntypes < 1 || ntypes > kMaxTypes) return noalloc_fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: ntypes in [1, 4]");
  if (!(L > 0) || !std::isfinite(L)) return noalloc_fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: L must be > 0");
  Table tab;
  double rcmax = 0;
  for (int a = 0; a < ntypes; ++a)
    for (int b = 0; b < ntypes; ++b) {
      const int t = a * ntypes + b, u = b * ntypes + a;
      if (!(eps[t] > 0) || !(sigma[t] > 0) || !(rc[t] > 0) || eps[t] != eps[u] || sigma[t] != sigma[u] ||
          rc[t] != rc[u])
        return noalloc_fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: tables must be positive and symmetric");
      if (!(rc[t] < 0.5 * L)) return noalloc_fail(MD_ERR_INVALID_ARG, "md_forces_noalloc: every cutoff must be < L/2");
      const double sr6 = std::pow(sigma[t] / rc[t], 6.0);
      tab.rc2[t] = rc[t] * rc[t];
      tab.sig2[t] = sigma[t] * sigma[t];
      tab.e48[t] = 48.0 * eps[t];
      tab.e4[t] = 4.0 * eps[t];
      tab.vsh[t] = 4.0 * eps[t] * (sr6 * sr6 - sr6);
      rcmax = std::max(rcmax, rc[t]);
    }
  // cells of edge >= the largest cutoff, at most kMaxCellsPerEdge per edge
  // (clamped in double, so any finite L is safe); fewer than 3: all pairs
  int nc = (int)std::min(std::floor(L / rcmax), (double)kMaxCellsPerEdge);
  if (nc < 3) nc = 1;
  const int ncells = nc * nc * nc;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  const md_status as = scratch_address(st, &base);
  if (as != MD_OK) return as;
  const Scratch s = carve(base);
  cudaError_t e;
  const int nb = (int)((n + kBlock - 1) / kBlock);
  k_clear<<<std::max(1, std::min(64, (ncells + kBlock - 1) / kBlock)), kBlock, 0, st>>>(s, ncells);
  k_bin<<<nb, kBlock, 0, st>>>(s, pos, n, nc, L);
  k_scan<<<1, 1024, 0, st>>>(s, ncells);
  k_scatter<<<nb, kBlock, 0, st>>>(s, n);
  k_order<<<std::max(1, std::min(1024, (ncells * 32 + kBlock - 1) / kBlock)), kBlock, 0, st>>>(s, ncells);
  k_forces<<<nb, kBlock, 0, st>>>(s, pos, types, n, ntypes, nc >= 3 ? nc : 0, L, tab, f, pe, virial);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(MD_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return MD_OK;
}
