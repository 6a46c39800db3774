// Shared pieces of the likelihood kernels (nll.cu, tagged.cu): the fixed-order
// FP64 reduction of per-tile accumulators, the tile-to-segment lookup, the
// per-lane log product and two bit-level helpers.
//
// Reduction order.  A tile of kTile events is owned by one warp; lane l adds
// events l, l+32, ... in order; the warp reduces its lanes with the butterfly
// below into one partial per tile.  The warp that completes the last tile of a
// group of kGroupTiles tiles reduces the group (lane l holding tile l), and the
// warp that completes a segment's last group adds the group partials in fixed
// order.  The order depends only on the segment's events, never on the launch
// geometry.
#pragma once

#include <stdint.h>

#include "fp64_math.cuh"
#include "ipa_internal.cuh"

namespace ipa {

// t > c for any doubles with c not NaN (integer compare of order-preserving keys).
__device__ __forceinline__ bool greater(double t, double c) {
    const long long a = __double_as_longlong(t), b = __double_as_longlong(c);
    const long long ka = a >= 0 ? a : (long long)(0x8000000000000000ull - (unsigned long long)a);
    const long long kb = b >= 0 ? b : (long long)(0x8000000000000000ull - (unsigned long long)b);
    return ka > kb;
}

// Position of the n-th (from 0) set bit of m; n < popc(m).
__device__ __forceinline__ int nth_set(unsigned m, int n) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const unsigned low = m & ((1u << w) - 1u);
        const int cnt = __popc(low);
        if (n >= cnt) {
            n -= cnt;
            m >>= w;
            pos += w;
        } else {
            m = low;
        }
    }
    return pos;
}

// P = m 2^e with m in [1, 2): *prod *= m and *esum += e, so that the log of the
// product of a lane's P values is log(*prod) + *esum ln 2 (bit operations on
// the integer pipe and one FP64 multiply per event instead of a log).  Zero,
// subnormal, negative, infinite and NaN P give what the sum of logs gives:
// -inf for +-0, the exact value for subnormals, +inf for +inf, NaN otherwise.
__device__ __forceinline__ void log_mul(double P, double* prod, int* esum) {
    const long long b = __double_as_longlong(P);
    long long mb = (b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll;
    int e = (int)(b >> 52) - 1023;
    if ((unsigned long long)(b - 0x0010000000000000ll) >= 0x7FE0000000000000ull) {
        if (b > 0 && b < 0x0010000000000000ll) {
            const int sh = __clzll(b) - 11;
            mb = ((b << sh) & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll;
            e = -1022 - sh;
        } else {
            mb = (b << 1) == 0 ? 0ll : (b == 0x7FF0000000000000ll ? b : 0x7FF8000000000000ll);
            e = 0;
        }
    }
    *prod *= __longlong_as_double(mb);
    *esum += e;
}

// log(prod) + esum ln 2
__device__ __forceinline__ double log_of(double prod, int esum, const MathTables* mt) {
    const double ed = (double)esum;
    return fma(ed, fp64tab::kLn2Hi, fma(ed, fp64tab::kLn2Lo, log_fast(prod, mt)));
}

// Butterfly reduction of NA accumulators over the 32 lanes of a warp (NA padded
// to the power of two NP).  The first log2(NP) levels halve the values each
// lane holds: at the level of lane bit j the lane keeps the half of its
// values selected by that bit and adds the partner's copy of that half, so
// every level costs NP / 2^(level+1) FP64 adds instead of NA.  The remaining
// levels add the partner's value of the same accumulator.  Afterwards lane l
// holds the full sum of accumulator acc_index<NA>(l) (two or more lanes hold
// each, with identical bits: addition is commutative), in an order fixed by
// the lane pairing.  NA = 15: 16 adds and 16 shuffles per warp instead of 75.
template <int NA>
struct Butterfly {
    static_assert(NA <= 16, "the butterfly takes at most 16 accumulators (see warp_allreduce_wide)");
    static constexpr int NP = NA <= 1 ? 1 : NA <= 2 ? 2 : NA <= 4 ? 4 : NA <= 8 ? 8 : 16;
    static constexpr int SPLITS = NP == 1 ? 0 : NP == 2 ? 1 : NP == 4 ? 2 : NP == 8 ? 3 : 4;
};

template <int NA>
__device__ __forceinline__ int acc_index(int lane) {
    constexpr int S = Butterfly<NA>::SPLITS;
    return (lane >> (5 - S)) & ((1 << S) - 1);
}

template <int NA>
__device__ __forceinline__ double warp_butterfly(const double* acc, int lane) {
    constexpr int NP = Butterfly<NA>::NP;
    constexpr int S = Butterfly<NA>::SPLITS;
    double v[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) v[a] = a < NA ? acc[a] : 0.0;
#pragma unroll
    for (int lev = 0; lev < S; ++lev) {
        const int mask = 16 >> lev;
        const int half = NP >> (lev + 1);
        const bool upper = (lane & mask) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const double keep = upper ? v[i + half] : v[i];
            const double give = upper ? v[i] : v[i + half];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, give, mask);
        }
    }
#pragma unroll
    for (int lev = S; lev < 5; ++lev) v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16 >> lev);
    return v[0];
}

// Every accumulator of a warp_butterfly result into acc[] of every lane.
template <int NA>
__device__ __forceinline__ void gather_butterfly(double v, double* acc) {
    constexpr int S = Butterfly<NA>::SPLITS;
#pragma unroll
    for (int a = 0; a < NA; ++a) acc[a] = __shfl_sync(0xffffffffu, v, a << (5 - S));
}

__device__ __forceinline__ int64_t clamp_off(int64_t v, int64_t n) {
    return v < 0 ? 0 : (v > n ? n : v);
}

// Segment s covers tiles [seg_tiles[s], seg_tiles[s+1]); find s for `tile`.
__device__ __forceinline__ int find_segment(const int64_t* seg_tiles, int n_seg, int64_t tile) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(seg_tiles + mid) <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Reduce the tile partials of one group (lane l holds tile g0 + l) or, with
// `stride` = kGroupTiles, the group partials of one segment (lane l adds groups
// l, l+32, ... in that order), then the butterfly; returns this lane's share
// (accumulator acc_index<NA>(lane)).
template <int NA>
__device__ __forceinline__ double reduce_partials(const double* partials, int64_t first, int64_t count,
                                                  int64_t stride, int lane) {
    double acc[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) acc[a] = 0.0;
#pragma unroll 4
    for (int64_t i = lane; i < count; i += 32) {
        const double* p = partials + (first + i * stride) * NA;
#pragma unroll
        for (int a = 0; a < NA; ++a) acc[a] += __ldcg(p + a);
    }
    return warp_butterfly<NA>(acc, lane);
}

// Lanes whose butterfly share is the first copy of an accumulator store it.
template <int NA>
__device__ __forceinline__ void store_share(double v, int lane, double* dst) {
    constexpr int S = Butterfly<NA>::SPLITS;
    const int a = acc_index<NA>(lane);
    if ((lane & ((1 << (5 - S)) - 1)) == 0 && a < NA) dst[a] = v;
}

// After a warp has reduced one tile into `share` (warp_butterfly): store the
// tile partial; if this warp completed the tile's group of kGroupTiles tiles,
// reduce the group into the partial slot of its first tile; if that completed
// the segment [t0, t1) of tiles, gather the segment's totals into acc[] of
// every lane and return true (the caller writes the segment's result and then
// resets counters[seg]).  gcount and counters return to zero for the next call.
template <int NA>
__device__ __forceinline__ bool tile_commit(double share, int lane, int64_t tile, int64_t t0, int64_t t1, int seg,
                                            double* partials, unsigned* gcount, unsigned* counters, double* acc) {
    const int64_t g0 = t0 + ((tile - t0) / kGroupTiles) * kGroupTiles;
    const int64_t g1 = g0 + kGroupTiles < t1 ? g0 + kGroupTiles : t1;
    int last = 0;
    store_share<NA>(share, lane, partials + tile * NA);
    __threadfence();
    __syncwarp();
    if (lane == 0) last = atomicAdd(gcount + g0, 1u) + 1u == (unsigned)(g1 - g0);
    if (!__shfl_sync(0xffffffffu, last, 0)) return false;
    __threadfence();
    const double gshare = reduce_partials<NA>(partials, g0, g1 - g0, 1, lane);
    // level 2: the warp that completes a segment's last group adds the
    // segment's group partials
    const int64_t n_groups = (t1 - t0 + kGroupTiles - 1) / kGroupTiles;
    __syncwarp();   // every lane has read the group's tile partials
    store_share<NA>(gshare, lane, partials + g0 * NA);
    __threadfence();
    __syncwarp();
    if (lane == 0) {
        gcount[g0] = 0u;
        last = atomicAdd(counters + seg, 1u) + 1u == (unsigned)n_groups;
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return false;
    __threadfence();
    gather_butterfly<NA>(reduce_partials<NA>(partials, t0, n_groups, kGroupTiles, lane), acc);
    return true;
}

// ---- the same protocol for more accumulators than the butterfly takes (16) ----
// Every lane ends with every sum: each accumulator goes through the full xor
// butterfly (at each level both partners add the same two values, so all lanes
// hold identical bits).  Costs 5 shuffles and adds per accumulator and tile.
template <int NA>
__device__ __forceinline__ void warp_allreduce_wide(double* acc) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    }
}

// Lane l stores accumulators l, l + 32, ... (register indices fixed at compile time).
template <int NA>
__device__ __forceinline__ void store_wide(const double* acc, int lane, double* dst) {
#pragma unroll
    for (int a = 0; a < NA; ++a)
        if ((a & 31) == lane) dst[a] = acc[a];
}

// acc = the warp's sums of the partials of `count` tiles (lane l adds tiles
// l, l+32, ... of first + i * stride in that order), on every lane.
template <int NA>
__device__ __forceinline__ void reduce_partials_wide(const double* partials, int64_t first, int64_t count,
                                                     int64_t stride, double* acc) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < NA; ++a) acc[a] = 0.0;
    for (int64_t i = lane; i < count; i += 32) {
        const double* p = partials + (first + i * stride) * NA;
#pragma unroll
        for (int a = 0; a < NA; ++a) acc[a] += __ldcg(p + a);
    }
    warp_allreduce_wide<NA>(acc);
}

// tile_commit for acc already reduced by warp_allreduce_wide: the group and
// segment levels in the same order; true with acc = the segment's totals.
template <int NA>
__device__ __forceinline__ bool tile_commit_wide(int lane, int64_t tile, int64_t t0, int64_t t1, int seg,
                                                 double* partials, unsigned* gcount, unsigned* counters, double* acc) {
    const int64_t g0 = t0 + ((tile - t0) / kGroupTiles) * kGroupTiles;
    const int64_t g1 = g0 + kGroupTiles < t1 ? g0 + kGroupTiles : t1;
    int last = 0;
    store_wide<NA>(acc, lane, partials + tile * NA);
    __threadfence();
    __syncwarp();
    if (lane == 0) last = atomicAdd(gcount + g0, 1u) + 1u == (unsigned)(g1 - g0);
    if (!__shfl_sync(0xffffffffu, last, 0)) return false;
    __threadfence();
    reduce_partials_wide<NA>(partials, g0, g1 - g0, 1, acc);
    const int64_t n_groups = (t1 - t0 + kGroupTiles - 1) / kGroupTiles;
    __syncwarp();   // every lane has read the group's tile partials
    store_wide<NA>(acc, lane, partials + g0 * NA);
    __threadfence();
    __syncwarp();
    if (lane == 0) {
        gcount[g0] = 0u;
        last = atomicAdd(counters + seg, 1u) + 1u == (unsigned)n_groups;
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return false;
    __threadfence();
    reduce_partials_wide<NA>(partials, t0, n_groups, kGroupTiles, acc);
    return true;
}

// The last warp of the grid to leave resets the two work counters (work[0]:
// tile takes handed out, work[1]: warps finished).
__device__ __forceinline__ void work_done(unsigned* work, int lane) {
    if (lane == 0) {
        const unsigned n_warps = gridDim.x * (blockDim.x >> 5);
        if (atomicAdd(work + 1, 1u) == n_warps - 1u) {
            work[0] = 0u;
            work[1] = 0u;
        }
    }
}

}  // namespace ipa
