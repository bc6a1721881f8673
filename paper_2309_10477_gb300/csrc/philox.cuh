// philox.cuh -- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64
// multiplies, the high halves xored with the other two words and the round
// key; the key advances by the Weyl constants between rounds.  Also the same
// function split for the path kernels, where the counter is (j, p, h, 0) with
// j the step pair, p the low and h the high word of the path index: the
// products that depend on (j, h) alone are the same for every lane of a warp
// and are computed once per warp (philox_head), the one that depends on p
// alone once per path (philox_p1), and the rest per path and step pair
// (philox_tail).  Self-contained, so that a host program can include it.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

struct PhiloxKey {
    uint32_t k0, k1;
};

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// One round: (x, y, z, w) -> (hi(z M1) ^ y ^ k0, lo(z M1), hi(x M0) ^ w ^ k1, lo(x M0)).
__host__ __device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1)
{
    const unsigned long long p0 = (unsigned long long)c.x * kPhiloxM0;
    const unsigned long long p1 = (unsigned long long)c.z * kPhiloxM1;
    return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                      (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, PhiloxKey key)
{
    uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        c = philox_round(c, k0, k1);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// The split of philox4x32_10((j, p, h, 0), key), with the rounds numbered R0
// to R9.  With A = j M0 and B = h M1, R0 gives (hi(B) ^ p ^ k0, lo(B),
// hi(A) ^ k1, lo(A)); R1 multiplies x1 = p ^ hi(B) ^ k0 (P1 = x1 M0, per path,
// free of j) and z1 = hi(A) ^ k1 (Q = z1 M1, per (j, h)); R2 multiplies
// x2 = hi(Q) ^ lo(B) ^ k0' (P2, per (j, h)) and z2 = hi(P1) ^ lo(A) ^ k1'
// (per path).  philox_head returns the (j, h) words with their round keys
// folded in: (lo(A) ^ k1', lo(Q) ^ k0'', hi(P2) ^ k1'', lo(P2)), where ' and ''
// mark the keys of R1 and R2; lo_b = lo(B).
__host__ __device__ __forceinline__ uint4 philox_head(uint32_t j, uint32_t lo_b, PhiloxKey key)
{
    const unsigned long long A = (unsigned long long)j * kPhiloxM0;
    const uint32_t z1 = (uint32_t)(A >> 32) ^ key.k1;
    const unsigned long long Q = (unsigned long long)z1 * kPhiloxM1;
    const uint32_t x2 = (uint32_t)(Q >> 32) ^ lo_b ^ (key.k0 + kPhiloxW0);
    const unsigned long long P2 = (unsigned long long)x2 * kPhiloxM0;
    return make_uint4((uint32_t)A ^ (key.k1 + kPhiloxW1), (uint32_t)Q ^ (key.k0 + 2u * kPhiloxW0),
                      (uint32_t)(P2 >> 32) ^ (key.k1 + 2u * kPhiloxW1), (uint32_t)P2);
}

// P1 = (p ^ hi(B) ^ k0) M0; hi_b = hi(B).
__host__ __device__ __forceinline__ unsigned long long philox_p1(uint32_t p, uint32_t hi_b, PhiloxKey key)
{
    return (unsigned long long)(p ^ hi_b ^ key.k0) * kPhiloxM0;
}

// R1 (its per-path half) to R9 from the head t and the path's P1.
__host__ __device__ __forceinline__ uint4 philox_tail(uint4 t, unsigned long long P1, PhiloxKey key)
{
    const uint32_t z2 = (uint32_t)(P1 >> 32) ^ t.x;
    const unsigned long long Q2 = (unsigned long long)z2 * kPhiloxM1;
    uint4 c = make_uint4((uint32_t)(Q2 >> 32) ^ t.y, (uint32_t)Q2, t.z ^ (uint32_t)P1, t.w);
    uint32_t k0 = key.k0 + 3u * kPhiloxW0, k1 = key.k1 + 3u * kPhiloxW1;
#pragma unroll
    for (int i = 3; i < 10; ++i) {
        c = philox_round(c, k0, k1);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}
