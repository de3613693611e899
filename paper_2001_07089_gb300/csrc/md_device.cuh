// md_device.cuh -- small device helpers shared by the library's kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kamd {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with the published multipliers, the key bumped by
// the published Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// 53-bit uniform in (0,1) from two words (top 32 bits of a, top 21 of b).
__device__ __forceinline__ double u01_53(uint32_t a, uint32_t b) {
  const uint64_t m = (((uint64_t)a << 21) ^ (uint64_t)(b >> 11)) & ((1ull << 53) - 1);
  return ((double)m + 0.5) * (1.0 / 9007199254740992.0);
}

enum { RNG_TAG_JITTER = 1, RNG_TAG_GAUSS = 2 };

// Three standard normals for particle p, draw d: two Philox blocks
// (counter = p, d_lo, tag<<16|block, d_hi; key = seed), Box-Muller on each
// pair of uniforms.
__device__ __forceinline__ void gauss3(uint64_t seed, uint64_t d, uint32_t p, double g[3]) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  double z[4];
#pragma unroll
  for (uint32_t blk = 0; blk < 2; ++blk) {
    const uint4 o = philox4x32_10(make_uint4(p, (uint32_t)d, (RNG_TAG_GAUSS << 16) | blk, (uint32_t)(d >> 32)), key);
    const double u1 = u01_53(o.x, o.y), u2 = u01_53(o.z, o.w);
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincos(2.0 * 3.14159265358979323846 * u2, &sn, &cs);
    z[2 * blk] = rad * cs;
    z[2 * blk + 1] = rad * sn;
  }
  g[0] = z[0];
  g[1] = z[1];
  g[2] = z[2];
}

// Three uniforms in (-1, 1) for the lattice jitter of particle p.
__device__ __forceinline__ void jitter3(uint64_t seed, uint32_t p, double u[3]) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const uint4 o = philox4x32_10(make_uint4(p, 0u, (RNG_TAG_JITTER << 16) | 0u, 0u), key);
  const uint4 o2 = philox4x32_10(make_uint4(p, 0u, (RNG_TAG_JITTER << 16) | 1u, 0u), key);
  u[0] = 2.0 * u01_53(o.x, o.y) - 1.0;
  u[1] = 2.0 * u01_53(o.z, o.w) - 1.0;
  u[2] = 2.0 * u01_53(o2.x, o2.y) - 1.0;
}

// Fixed point <-> length: u = x/L * 2^64 (mod 2^64).
__device__ __forceinline__ uint64_t to_fixed(double x, double invL) {
  double f = x * invL;
  f -= floor(f);                       // [0, 1]
  double s = f * 18446744073709551616.0;  // 2^64
  if (s >= 18446744073709551615.0) s = 0.0;  // f rounded to 1
  return (uint64_t)s;
}
__device__ __forceinline__ double from_fixed(uint64_t u, double L) {
  return (double)u * (L * (1.0 / 18446744073709551616.0));
}

__device__ __forceinline__ double wrap_box(double x, double L) {
  x -= L * floor(x / L);
  if (x >= L) x -= L;
  if (x < 0.0) x = 0.0;
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace kamd
