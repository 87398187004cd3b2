// warp_keys.cuh -- (value, index) pairs as 64-bit keys and warp-wide bitonic sort / merge of
// one key per lane (selection support for the search kernels; no counterpart in the paper).
#pragma once

#include <cstdint>

namespace pts {

// (value, index) pairs as one 64-bit key ordered like the pair: the float's bits mapped to an
// unsigned order (negative values flipped) in the high word, the index in the low word.
__device__ __forceinline__ unsigned long long pack_key(float v, int i) {
    unsigned int u = __float_as_uint(v);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned int)i;
}
__device__ __forceinline__ float key_value(unsigned long long k) {
    unsigned int u = (unsigned int)(k >> 32);
    u = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    return __uint_as_float(u);
}
__device__ __forceinline__ int key_index(unsigned long long k) { return (int)(unsigned int)(k & 0xffffffffu); }

// Ascending bitonic sort of one key per lane, branch-free compare-exchange.
__device__ __forceinline__ void warp_sort_keys(unsigned long long &k, int lane) {
#pragma unroll
    for (int s = 2; s <= 32; s <<= 1) {
#pragma unroll
        for (int j = s >> 1; j > 0; j >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, k, j);
            const bool keep_min = ((lane & s) == 0) == ((lane & j) == 0);
            k = (keep_min == (o < k)) ? o : k;
        }
    }
}

// k := the 32 smallest of two ascending key lists k and w, ascending.
__device__ __forceinline__ void warp_merge_keys(unsigned long long &k, unsigned long long w, int lane) {
    const unsigned long long rw = __shfl_sync(0xffffffffu, w, 31 - lane);
    k = rw < k ? rw : k;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, k, s);
        k = (((lane & s) == 0) == (o < k)) ? o : k;
    }
}

}  // namespace pts
