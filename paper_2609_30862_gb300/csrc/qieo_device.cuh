// qieo_device.cuh -- inline device helpers shared by the library's translation units:
// Philox4x32-10 and the CIP rotation of packed angle indices. No kernels live here.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qieo {

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC 2011). One round maps (c0, c1, c2, c3)
// to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key advances by
// the Weyl increments between rounds.
// ---------------------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

struct Draw4 {
    uint32_t a, b, c, d;
};

__device__ __forceinline__ Draw4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return {c0, c1, c2, c3};
}

// The same rounds with the ten round keys precomputed (kernel parameters, so each xor
// takes its key straight from the constant bank).
__device__ __forceinline__ Draw4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2,
                                                  uint32_t c3, const uint32_t (&rk0)[10],
                                                  const uint32_t (&rk1)[10])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk0[r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[r];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    return {c0, c1, c2, c3};
}

// ---------------------------------------------------------------------------------------
// CIP on a pair of scaled angle indices (4n) held in one uint32 (gene 2i low, 2i+1 high).
// d per half: 8 = step toward allele 1, 0 = step toward allele 0, 4 = no move.
// 4n' = min(max(4n + d, 4) - 4, 8K): saturates theta at 0 and pi/2 (the bounds of the
// angle index). No half can carry into the other: 4n + d <= 8K + 8 < 2^16.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t delta_pair(uint32_t e2, uint32_t m2)
{
    // e2: elite alleles of the two genes (bit 0, bit 1); m2: which of them move.
    const uint32_t lo = 4u - ((m2 & 1u) << 2) + ((m2 & e2 & 1u) << 3);
    const uint32_t hi = 4u - (((m2 >> 1) & 1u) << 2) + ((((m2 & e2) >> 1) & 1u) << 3);
    return lo | (hi << 16);
}

__device__ __forceinline__ uint32_t rotate_pair(uint32_t s, uint32_t d, uint32_t k8)
{
    return __vminu2(__vmaxu2(s + d, 0x00040004u) - 0x00040004u, k8);
}

// The same step with the delta given as a signed per-halfword step sd = d - 4 in {-4, 0, 4}
// (16-bit two's complement halves): 4n' = min(max(4n + sd, 0), 8K) with a per-halfword add
// (no carry between the halves) and a signed per-halfword maximum, three operations instead
// of four. 4n + sd lies in [-4, 8K + 4], inside the signed 16-bit range for 8K <= 8000.
__device__ __forceinline__ uint32_t signed_step(uint32_t d)
{
    return __vsub2(d, 0x00040004u);
}

__device__ __forceinline__ uint32_t rotate_pair_signed(uint32_t s, uint32_t sd, uint32_t k8)
{
    return __vminu2(__vmaxs2(__vadd2(s, sd), 0u), k8);
}

__device__ __forceinline__ uint4 rotate_vec(uint4 s, uint32_t e8, uint32_t m8, uint32_t k8)
{
    s.x = rotate_pair(s.x, delta_pair(e8 & 3u, m8 & 3u), k8);
    s.y = rotate_pair(s.y, delta_pair((e8 >> 2) & 3u, (m8 >> 2) & 3u), k8);
    s.z = rotate_pair(s.z, delta_pair((e8 >> 4) & 3u, (m8 >> 4) & 3u), k8);
    s.w = rotate_pair(s.w, delta_pair((e8 >> 6) & 3u, (m8 >> 6) & 3u), k8);
    return s;
}

}  // namespace qieo
