// Device helpers shared by the per-signal kernels (internal header).
#pragma once

#include "cs_internal.cuh"

namespace cs {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// Packed pair of floats (element 0 in the low word) and the sm_100+ paired
// fp32 FMA, d = a * b + c on both halves with round-to-nearest.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi) {
    lo = __uint_as_float((unsigned)(v & 0xffffffffull));
    hi = __uint_as_float((unsigned)(v >> 32));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}


// E4M3 (FP8) round-to-nearest with saturation to +-448, and its value.
__device__ __forceinline__ uint32_t fp8_e4m3(float x) {
    return (uint32_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float fp8_e4m3_value(uint32_t q) {
    return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q, __NV_E4M3)));
}
// Scale that maps a vector's largest magnitude to the largest finite E4M3
// value (448); 1 for a zero vector.
__device__ __forceinline__ float fp8_scale(float amax) { return amax > 0.f ? amax / 448.f : 1.f; }

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One warp quantises x[0..m) (zero past m, up to mq, a multiple of 128) to
// E4M3 with the scale fp8_scale(max |x_i|): dst[i] = e4m3(x_i / scale).
// Returns the scale; *err receives ||x - scale * dst||_2.
__device__ __forceinline__ float quant_row_fp8(const float* __restrict__ x, int m, int mq, uint8_t* __restrict__ dst,
                                               float* err) {
    const int lane = threadIdx.x & 31;
    float amax = 0.f;
    for (int i = lane; i < m; i += 32) amax = fmaxf(amax, fabsf(x[i]));
    const float scale = fp8_scale(warp_max(amax));
    float e2 = 0.f;
    for (int i = 4 * lane; i < mq; i += 128) {
        uint32_t packed = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float v = i + u < m ? x[i + u] : 0.f;
            const uint32_t q = fp8_e4m3(v / scale);
            const float d = v - scale * fp8_e4m3_value(q);
            e2 = fmaf(d, d, e2);
            packed |= q << (8 * u);
        }
        *reinterpret_cast<uint32_t*>(dst + i) = packed;
    }
    *err = sqrtf(warp_sum(e2));
    return scale;
}

// Approximate reciprocal (rcp.approx.ftz, relative error ~2^-23).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------------- selection --

template <int MCH>
__device__ __forceinline__ void load_row(const float* __restrict__ base, int mp, float4 (&v)[MCH]) {
    const int lane = threadIdx.x & 31;
    const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int c = 0; c < MCH; ++c) {
        const int i4 = c * 32 + lane;
        v[c] = (i4 * 4 < mp) ? p[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Warp-cooperative dot products of up to 32 columns of A32 (atom index
// held by lane q, -1 = none) with the row-sliced vector x; lane q returns
// the full dot for its column.
template <int MCH>
__device__ __forceinline__ float warp_dots32(const float* __restrict__ A32, int mp, int my_atom,
                                             const float4 (&x)[MCH]) {
    const int lane = threadIdx.x & 31;
    float part[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int j = __shfl_sync(FULL, my_atom, q);
        float acc = 0.f;
        if (j >= 0) {
            const float4* col = reinterpret_cast<const float4*>(A32 + (size_t)j * mp);
#pragma unroll
            for (int c = 0; c < MCH; ++c) {
                const int i4 = c * 32 + lane;
                if (i4 * 4 < mp) acc += dot4(col[i4], x[c]);
            }
        }
        part[q] = acc;
    }
    warp_reduce_scatter32(part);
    return part[0];
}


inline int row_chunks(int mp) { return ceil_div(mp, 128); }

}  // namespace

// Number of CTAs that keep every SM of the current device busy with `kernel`
// (occupancy x SM count), capped at `needed`.  Kernels launched this way
// stride over their work items, so the grid never ends in a partial wave.
int resident_grid(const void* kernel, int block, int needed);

}  // namespace cs

#define CS_DISPATCH_MCH(MP, KERNEL, GRID, BLOCK, STREAM, ...)                     \
    do {                                                                          \
        switch (row_chunks(MP)) {                                                 \
            case 1: KERNEL<1><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;    \
            case 2: KERNEL<2><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;    \
            case 3:                                                               \
            case 4: KERNEL<4><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;    \
            default: KERNEL<8><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;   \
        }                                                                         \
    } while (0)

