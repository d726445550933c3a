// Device code of the hard-edged disc renderer fused with the L2 loss,
// shared by the disc kernels (render_disc.cu) and the persistent serving
// kernel (queue.cu).  One warp renders one perturbation: pixel centre
// ((x + 1/2)/W, (y + 1/2)/H) is inside when fma(dx, dx, dy*dy) < r*r in FP32,
// value 1 inside, 0 outside.
#pragma once
#include "hr.h"
#include "hr_device.cuh"

namespace hr {
namespace {

__device__ __forceinline__ float disc_value(int x, int y, int W, int H, float cx, float cy, float r2) {
    const float px = __fdiv_rn(__fadd_rn((float)x, 0.5f), (float)W);
    const float py = __fdiv_rn(__fadd_rn((float)y, 0.5f), (float)H);
    const float dx = __fsub_rn(px, cx);
    const float dy = __fsub_rn(py, cy);
    const float d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
    return d2 < r2 ? 1.0f : 0.0f;
}

// The pixel-centre coordinates (c + 1/2)/W of the columns and (r + 1/2)/H of
// the rows, rounded exactly as disc_value and boxes_value form them, filled
// once per CTA: a pixel then costs no division.  Lane l of a warp visits
// pixels i = l, l + 32, ... in row-major order (the order of its FP32 loss
// sum); (x, y) follow i by increments.
__device__ __forceinline__ void centre_tables(float* px, float* py, int W, int H) {
    for (int x = threadIdx.x; x < W; x += blockDim.x) px[x] = __fdiv_rn(__fadd_rn((float)x, 0.5f), (float)W);
    for (int y = threadIdx.x; y < H; y += blockDim.x) py[y] = __fdiv_rn(__fadd_rn((float)y, 0.5f), (float)H);
}

// kWide: W >= 32, so a step of 32 pixels wraps a row at most once
template <bool kWide>
__device__ __forceinline__ void next_pixel(int& x, int& y, int W) {
    x += 32;
    if (kWide) {
        if (x >= W) { x -= W; ++y; }
    } else {
        while (x >= W) { x -= W; ++y; }
    }
}

// Sum over this lane's pixels of (value(px, py) - target)^2, in pixel order;
// the target values of four pixels are loaded ahead of their arithmetic so
// that the loads overlap (one at a time, the loop waits on each load).
template <bool kWide, class Value>
__device__ __forceinline__ float lane_l2(const float* __restrict__ target, int W, int npx, int lane,
                                        const float* px, const float* py, Value value) {
    float acc = 0.0f;
    int y = lane / W, x = lane - y * W;
    int i = lane;
    for (; i + 96 < npx; i += 128) {
        float t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) t[u] = __ldg(target + i + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float d = __fsub_rn(value(px[x], py[y]), t[u]);
            acc = __fmaf_rn(d, d, acc);
            next_pixel<kWide>(x, y, W);
        }
    }
    for (; i < npx; i += 32) {
        const float d = __fsub_rn(value(px[x], py[y]), __ldg(target + i));
        acc = __fmaf_rn(d, d, acc);
        next_pixel<kWide>(x, y, W);
    }
    return acc;
}

// Disc loss of one lane for W = 32 kCpr (32 to 512): the lane's kCpr columns are fixed,
// so dx = px - cx is formed once per render and dy^2 once per row; a pixel is
// then the test fma(dx, dx, dy^2) < r^2 of disc_value.  Rows go in order and
// columns in order within a row: the pixel order of lane_l2, so the same sum.
template <int kCpr>
__device__ __forceinline__ float disc_rows(const float* __restrict__ target, int H, int lane, const float* px,
                                           const float* py, float cx, float cy, float r2) {
    constexpr int kRows = 16 / kCpr;   // target loads of kRows rows (16 loads) in flight
    constexpr int W = 32 * kCpr;
    float dx[kCpr];
#pragma unroll
    for (int c = 0; c < kCpr; ++c) dx[c] = __fsub_rn(px[lane + 32 * c], cx);
    float acc = 0.0f;
    int y = 0;
    for (; y + kRows <= H; y += kRows) {
        float t[kRows][kCpr];
#pragma unroll
        for (int r = 0; r < kRows; ++r)
#pragma unroll
            for (int c = 0; c < kCpr; ++c) t[r][c] = __ldg(target + (size_t)(y + r) * W + lane + 32 * c);
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const float dy = __fsub_rn(py[y + r], cy);
            const float dy2 = __fmul_rn(dy, dy);
#pragma unroll
            for (int c = 0; c < kCpr; ++c) {
                const float d = __fsub_rn(__fmaf_rn(dx[c], dx[c], dy2) < r2 ? 1.0f : 0.0f, t[r][c]);
                acc = __fmaf_rn(d, d, acc);
            }
        }
    }
    for (; y < H; ++y) {
        const float dy = __fsub_rn(py[y], cy);
        const float dy2 = __fmul_rn(dy, dy);
#pragma unroll
        for (int c = 0; c < kCpr; ++c) {
            const float d = __fsub_rn(__fmaf_rn(dx[c], dx[c], dy2) < r2 ? 1.0f : 0.0f,
                                      __ldg(target + (size_t)y * W + lane + 32 * c));
            acc = __fmaf_rn(d, d, acc);
        }
    }
    return acc;
}

// Loss of the disc at centre (cx, cy) against the target, by one warp (all
// 32 lanes call; every lane returns the loss): the FP32 sum of the squared
// differences over the image, per lane in pixel order, then a shuffle tree,
// divided by the pixel count.
__device__ __forceinline__ float disc_loss_warp(const float* __restrict__ target, int W, int H, float radius,
                                                const float* px, const float* py, float cx, float cy, int lane) {
    const float r2 = __fmul_rn(radius, radius);
    const int npx = W * H;
    auto value = [cx, cy, r2](float px_, float py_) {
        const float dx = __fsub_rn(px_, cx);
        const float dy = __fsub_rn(py_, cy);
        return __fmaf_rn(dx, dx, __fmul_rn(dy, dy)) < r2 ? 1.0f : 0.0f;
    };
    float acc;
    switch (W) {   // the widths with a fixed-column loop; any other takes lane_l2
        case 32: acc = disc_rows<1>(target, H, lane, px, py, cx, cy, r2); break;
        case 64: acc = disc_rows<2>(target, H, lane, px, py, cx, cy, r2); break;
        case 128: acc = disc_rows<4>(target, H, lane, px, py, cx, cy, r2); break;
        case 256: acc = disc_rows<8>(target, H, lane, px, py, cx, cy, r2); break;
        case 512: acc = disc_rows<16>(target, H, lane, px, py, cx, cy, r2); break;
        default:
            acc = W >= 32 ? lane_l2<true>(target, W, npx, lane, px, py, value)
                          : lane_l2<false>(target, W, npx, lane, px, py, value);
    }
    acc = warp_sum(acc);
    return __fdiv_rn(acc, (float)npx);
}

}  // namespace
}  // namespace hr
