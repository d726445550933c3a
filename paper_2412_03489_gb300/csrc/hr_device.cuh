// Device helpers of the CUDA path: the counter-based RNG, the FP32 operation
// sequences that decide coverage and ray hits, and small reductions.
//
// Every FP32 operation whose result can change a discrete decision inside a
// renderer is written with an explicitly rounded intrinsic (__fmul_rn,
// __fadd_rn, __fsub_rn, __fmaf_rn, __fdiv_rn, __fsqrt_rn) so the compiler
// cannot fuse or reorder it: the renderers are defined by these sequences.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hr {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32 -> 64-bit multiplies with a Weyl key schedule.
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t a = 0xD2511F53u * c0, ha = __umulhi(0xD2511F53u, c0);
        const uint32_t b = 0xCD9E8D57u * c2, hb = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hb ^ c1 ^ k0, n2 = ha ^ c3 ^ k1;
        c0 = n0; c1 = b; c2 = n2; c3 = a;
    }
    return {c0, c1, c2, c3};
}

__device__ __forceinline__ u32x4 philox_seed(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
    return philox10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// uniform in (0,1): (x + 1/2) 2^-32, exact in FP64
__device__ __forceinline__ double u01d(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }
// 24-bit uniform in (0,1), exact in FP32: (2 (x >> 8) + 1) 2^-25
__device__ __forceinline__ float u24f(uint32_t x) {
    return __fadd_rn(__fmul_rn((float)(x >> 8), 0x1p-24f), 0x1p-25f);
}

constexpr uint32_t TAG_SAMPLE = 1u, TAG_PATH = 2u, TAG_TARGET = 3u;

// ---------------------------------------------------------------------------
// Screen-space edge functions (both rasterisers).  Edge P->Q:
//   A = Q.y - P.y, B = P.x - Q.x, C = RN(P.y Q.x) - RN(P.x Q.y)
//   E(x, y) = fma(A, x, fma(B, y, C))
// The reversed edge gives exactly -A, -B, -C (watertight shared edges);
// E == 0 counts as inside on a top-left edge: A > 0, or A == 0 and B > 0.
// ---------------------------------------------------------------------------
struct Edge { float A, B, C; };

__device__ __forceinline__ Edge edge_of(float px, float py, float qx, float qy) {
    Edge e;
    e.A = __fsub_rn(qy, py);
    e.B = __fsub_rn(px, qx);
    e.C = __fsub_rn(__fmul_rn(py, qx), __fmul_rn(px, qy));
    return e;
}
__device__ __forceinline__ float edge_eval(float A, float B, float C, float x, float y) {
    return __fmaf_rn(A, x, __fmaf_rn(B, y, C));
}
__device__ __forceinline__ bool edge_in(float A, float B, float v) {
    return (v > 0.0f) || (v == 0.0f && (A > 0.0f || (A == 0.0f && B > 0.0f)));
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP64 dot product of two shared/global n-vectors over the whole block;
// red holds one double per warp.  Every thread returns the same value.
__device__ __forceinline__ double block_dot(const double* a, const double* b, int n, double* red) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += a[i] * b[i];
    v = warp_sum_d(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
}

// Kahan-compensated FP32 accumulator
struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
};

}  // namespace hr
