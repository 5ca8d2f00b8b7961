// tc_tiles.cuh -- operand-tile helpers shared by the tensor-core kernels:
// 16-bit hi/lo splits and the byte offsets of the 128-row, 128-byte-swizzled
// K-major operand tiles that the phase builders write and the MMA
// descriptors address.
#pragma once
#include "internal.cuh"

namespace scm {

constexpr int kTileRows = 128;                 // M of one pixel tile
constexpr int kTileKBlock = 64;                // 64 x 16-bit = one 128-byte swizzle row
constexpr int kTileKBlockBytes = kTileRows * 128;

// Two values as a packed 16-bit pair (first value in the low half) and the
// packed pair of their remainders: v = hi + lo to about twice the format's
// precision.  One packed conversion per pair and part.
__device__ __forceinline__ void split_pair(float a, float b, int bf16, uint32_t *hi, uint32_t *lo) {
    if (bf16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 back = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - back.x, b - back.y);
        *hi = *reinterpret_cast<const uint32_t *>(&h);
        *lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 back = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - back.x, b - back.y);
        *hi = *reinterpret_cast<const uint32_t *>(&h);
        *lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

// Two values as one packed 16-bit pair (first value in the low half).
__device__ __forceinline__ uint32_t pack_pair(float a, float b, int bf16) {
    if (bf16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Byte offset of K element k (a multiple of 16) from the start of a 128-row
// operand made of 64-element K blocks: the descriptor start of that K step.
__device__ __forceinline__ uint32_t a_k_offset(int k) { return (uint32_t)((k >> 6) * kTileKBlockBytes + (k & 63) * 2); }

// Byte offset of 16-byte chunk `c` (8 elements) of row `m` in K-block `kb`
// of a 128-row operand laid out for the 128-byte swizzle.
__device__ __forceinline__ uint32_t a_chunk_offset(int m, int k) {
    const int kb = k >> 6, c = (k & 63) >> 3;
    return (uint32_t)(kb * kTileKBlockBytes + m * 128 + ((c ^ (m & 7)) << 4));
}

}  // namespace scm
