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

