// common.cuh -- shared device helpers of the sm_103a SPH library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sphgb.h"

namespace sphgb {

constexpr int kCellMax = 2097151;          // 2^21 - 1 cells per axis
constexpr int kMaxLevels = 32;
constexpr unsigned long long kLevelSalt = 0x9E3779B97F4A7C15ull;

// Grid of the sorting stage as the kernels read it (device copy).
struct GridDev {
    float x0, y0, z0;
    int log2_L0;
    int n_levels;
    int log2_M;
};

// 2^e as FP32 for e in [-126, 127], built from its bits (exact).
__device__ __forceinline__ float pow2f(int e) {
    return __uint_as_float((unsigned)(e + 127) << 23);
}

// Level of a smoothing length: smallest l >= 0 with h <= L0 * 2^l, clamped.
// Integer arithmetic on the FP32 bits of the exact quotient h / L0.
__device__ __forceinline__ int level_of(float h, int log2_L0, int n_levels) {
    float q = __fmul_rn(h, pow2f(-log2_L0));
    int l;
    if (!(q > 1.0f)) {
        l = 0;
    } else {
        unsigned b = __float_as_uint(q);
        int e = (int)((b >> 23) & 0xffu) - 127;
        l = (b & 0x7fffffu) ? e + 1 : e;
    }
    return l < n_levels - 1 ? l : n_levels - 1;
}

// Cell coordinate floor((x - x0) * inv_c), clamped to [0, kCellMax]; NaN -> 0.
// Separate rounded subtract and multiply (no contraction) so the host-side
// definition of the grid reproduces it bit for bit.
__device__ __forceinline__ int cell_of(float x, float x0, float inv_c) {
    float u = __fmul_rn(__fsub_rn(x, x0), inv_c);
    if (!(u > 0.0f)) return 0;
    if (u >= (float)kCellMax) return kCellMax;
    return (int)u;
}

// Spread the low 10 bits of v to every third bit of a 32-bit word (bit b ->
// bit 3b).  The bucket keeps the low log2_M <= 30 bits of the full 63-bit
// interleave plus the level salt; carries only move upwards, so those bits
// depend only on the low 10 bits of each coordinate and 32-bit arithmetic
// gives the same bucket as the 64-bit definition.
constexpr unsigned kDilatedX = 0x09249249u;   // bits 0, 3, ..., 27
__device__ __forceinline__ unsigned spread3_lo(unsigned v) {
    unsigned x = v & 0x3ffu;
    x = (x | (x << 16)) & 0xff0000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & kDilatedX;
    return x;
}

// Bucket of cell (cx, cy, cz) on level tag l: (interleave + l * kLevelSalt)
// mod 2^log2_M, log2_M <= 30.
__device__ __forceinline__ int bucket_of(int cx, int cy, int cz, int l, int log2_M) {
    const unsigned m = spread3_lo((unsigned)cx) | (spread3_lo((unsigned)cy) << 1) |
                       (spread3_lo((unsigned)cz) << 2);
    return (int)((m + (unsigned)l * (unsigned)kLevelSalt) & ((1u << log2_M) - 1u));
}

// Occupancy bit of a super-cell (2 x 2 x 2 cells of one level): set by the
// sorting stage for every occupied super-cell, read by the neighbour search to
// skip levels with nobody near.  Hash collisions only cost a wasted probe.
// (Super-cells of 8^3 and 4^3 cells skipped fewer empty coarse levels: the
// list build took 4% longer at 2,097,152 gas particles; single cells gave
// the time of 2^3.)
constexpr int kSuperShift = 1;
constexpr unsigned long long kSuperSalt = 0xD1B54A32D192ED03ull;
__device__ __forceinline__ unsigned super_bit(int sx, int sy, int sz, int l, int log2_B) {
    const unsigned m = spread3_lo((unsigned)sx) | (spread3_lo((unsigned)sy) << 1) |
                       (spread3_lo((unsigned)sz) << 2);
    const unsigned mask = log2_B >= 32 ? 0xffffffffu : ((1u << log2_B) - 1u);
    return (m + (unsigned)(l + 1) * (unsigned)kSuperSalt) & mask;
}

// Tag of (level, cell): the level and the low 9 bits of each cell
// coordinate.  Two cells of one level share a tag only when they lie a
// multiple of 512 cells apart on every axis where they differ.
__device__ __forceinline__ unsigned cell_tag(int l, int cx, int cy, int cz) {
    return ((unsigned)l << 27) | (((unsigned)cx & 511u) << 18) | (((unsigned)cy & 511u) << 9) |
           ((unsigned)cz & 511u);
}

// FP32 neighbour predicate: ((dx*dx + dy*dy) + dz*dz) < (h_i + h_j)^2,
// every operation rounded separately.
__device__ __forceinline__ bool nb_pred(float4 a, float4 b) {
    float dx = __fsub_rn(a.x, b.x);
    float dy = __fsub_rn(a.y, b.y);
    float dz = __fsub_rn(a.z, b.z);
    float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    float s = __fadd_rn(a.w, b.w);
    return r2 < __fmul_rn(s, s);
}

// Ordered-integer image of a float for atomicMin/atomicMax.
__device__ __forceinline__ unsigned float_to_ordered(float f) {
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Kahan-compensated FP32 accumulation.
struct Kahan {
    float s, c;
    __device__ __forceinline__ void init() { s = 0.0f; c = 0.0f; }
    __device__ __forceinline__ void add(float x) {
        float y = __fsub_rn(x, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ float value() const { return s; }
};

__device__ __forceinline__ void set_flag(int *flags, int bit) {
    if (flags) atomicOr(flags, bit);
}

// Count kernel launches made by the library (read through sph_launch_count).
void note_launch(int k = 1);

// Streaming multiprocessors of the current device (152 on GB300).
int device_num_sms();
}  // namespace sphgb

// Host-side launch helpers shared by the translation units.
#define SPH_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return SPH_ERR_CUDA;          \
    } while (0)

#define SPH_LAUNCH_CHECK() SPH_CUDA_TRY(cudaGetLastError())
