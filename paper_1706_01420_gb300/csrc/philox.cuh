// Philox-4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11), written out here, and the 53-bit uniform built from
// two of its words.  Every draw is a pure function of (counter, key), so the
// generators address their random numbers by (index, toy, call) and the
// result of a draw does not depend on which thread makes it.  Also the block
// scan with which the accept-reject generators keep accepted candidates in
// candidate order.
#pragma once

#include <stdint.h>

#include "ipa_internal.cuh"

namespace ipa {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

struct U4 {
    uint32_t x, y, z, w;
};

// Ten rounds.  Round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
// c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); key bumped by (W0, W1) between rounds.
__device__ __forceinline__ U4 philox(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        const uint32_t lo0 = kPhiloxM0 * c.x, hi0 = __umulhi(kPhiloxM0, c.x);
        const uint32_t lo1 = kPhiloxM1 * c.z, hi1 = __umulhi(kPhiloxM1, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

// u = ((((a << 32) | b) >> 11) + 1) 2^-53, in (0, 1] (exact).
__device__ __forceinline__ double u01(uint32_t a, uint32_t b) {
    const unsigned long long v = ((((unsigned long long)a) << 32) | b) >> 11;
    return __dmul_rn(__ull2double_rn(v + 1ull), 0x1p-53);
}

// Counter (idx lo32, idx hi32, toy, call) with key (k0, k1).
__device__ __forceinline__ U4 draw(uint64_t idx, uint32_t toy, uint32_t call, uint32_t k0, uint32_t k1) {
    return philox(U4{(uint32_t)idx, (uint32_t)(idx >> 32), toy, call}, k0, k1);
}

// Exclusive scan of one int per thread over the block; returns the prefix and
// writes the block total to *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < kBlock / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        if (lane < kBlock / 32) warp_sums[lane] = s;   // inclusive warp prefix
    }
    __syncthreads();
    const int before = wid ? warp_sums[wid - 1] : 0;
    *total = warp_sums[kBlock / 32 - 1];
    __syncthreads();
    return before + x - v;
}

}  // namespace ipa
