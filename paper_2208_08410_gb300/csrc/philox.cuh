// Counter-based start draws shared by the kernels that begin a power
// iteration (internal header).  Philox-4x32-10 (Salmon, Moraes, Dror & Shaw,
// SC'11) keyed by splitmix64(seed), one counter per pair of normals:
// (p mod 2^32, p div 2^32, l, 0x54535644); the two 64-bit halves of the
// output give u1 in (0, 1] and u2 in [0, 1), and Box-Muller in FP64 turns them
// into two standard normals (the start vector x ~ N(0, 1) of Alg. 2).
#pragma once

#include <stdint.h>

namespace tsvd {

__device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    philox_round(c, k0, k1);
  }
}

__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// normals 2p and 2p+1 of the start vector of triplet `lword` under key (k0, k1)
__device__ __forceinline__ void start_normal_pair(uint32_t k0, uint32_t k1, uint32_t lword, int64_t p, double *z0,
                                                  double *z1) {
  uint32_t c[4] = {(uint32_t)p, (uint32_t)((uint64_t)p >> 32), lword, 0x54535644u};
  philox10(c, k0, k1);
  const uint64_t a = ((uint64_t)c[0] << 32) | c[1];
  const uint64_t b = ((uint64_t)c[2] << 32) | c[3];
  const double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = (double)(b >> 11) * 0x1.0p-53;
  const double rad = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  *z0 = rad * cs;
  *z1 = rad * sn;
}

}  // namespace tsvd
