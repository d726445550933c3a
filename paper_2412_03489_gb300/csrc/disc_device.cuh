// Device code of the hard-edged disc and squares renderers fused with the L2
// loss, shared by their kernels (render_disc.cu) and the persistent serving
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

// Binary targets (every pixel exactly 0 or 1).  Each pixel's squared
// difference is then 0 or 1, so the per-pixel FP32 sum is the count of pixels
// where the disc and the target differ: an integer below 2^24, exact in any
// order.  Both tests the pixel test is made of are monotone on either side of
// the disc's centre, because rounding is monotone:
//   - in a row, with dx = px - cx rounded to FP32, fma(dx, dx, dy^2) < r^2 is
//     non-increasing in x left of the centre column (the first column with
//     px >= cx) and non-decreasing from it, so the row's covered columns are
//     one interval [a, e);
//   - only rows with dy^2 = (py - cy)^2 < r^2 (rounded) can hold a covered
//     pixel, because fma(dx, dx, dy^2) >= dy^2.  The FP32 roundings of those
//     tests and of the band below move a row's position by less than
//     (|cy| + r) H 2^-22 + 1 rows, so every such row lies inside the
//     real-arithmetic band (cy -+ r) H - 1/2 widened by 2 + (|cy| + r) H 2^-20
//     rows; the rows [y0, y1) of that band are the only ones tested.
// A row's span ends are found with the exact test itself, in a window of four
// columns around the real-arithmetic ends cx -+ sqrt(r^2 - dy^2); an end
// outside the window falls back to a binary search on the same predicate.  Rows outside [y0, y1) differ from the target in its set pixels
// (a prefix sum of the rows' popcounts); a row inside differs in
// popc(target bits XOR span bits) over its words (an empty span when its
// dy^2 >= r^2).
// The bit-packed target of a binary image: bit x % 32 of word x / 32 of row y
// is pixel (x, y); rowpop [H + 1] the prefix sums of the rows' popcounts.
struct DiscBits {
    const uint32_t* bits;   // null: the target is not binary
    const int* rowpop;
};

// clamp of a float index estimate to [lo, hi] (NaN to lo)
__device__ __forceinline__ int clamp_col(float f, int lo, int hi) {
    return (int)fminf(fmaxf(f, (float)lo), (float)hi);
}

// first x in [lo, hi) with pred(x) true (hi if none), pred false..false true..true
template <class Pred>
__device__ __forceinline__ int first_true(int lo, int hi, Pred pred) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pred(mid)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// First index of [lo, hi) where in() holds (hi if none), for in() false..false
// true..true on [lo, hi), looked for around the guess g: the four tests of the
// window [w, w + 4) (w = g - 2, moved inside the range) are independent, so
// their latencies overlap; when the window does not hold the change from false
// to true, a binary search on the same predicate finds it.
template <class In>
__device__ __forceinline__ int first_in(int lo, int hi, int g, In in) {
    if (hi - lo <= 0) return hi;
    const int w = max(lo, min(g - 2, hi - 4));
    bool t[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) t[j] = w + j >= hi || in(w + j);
    if (t[0]) return w == lo ? lo : first_true(lo, w, in);
    if (!t[3]) return first_true(w + 4, hi, in);
    return w + 1 + (t[1] ? 0 : 1 + (t[2] ? 0 : 1));
}

// integer guess from a float estimate, clamped to [lo, hi] (NaN to lo)
__device__ __forceinline__ int guess_index(float f, int lo, int hi) { return clamp_col(ceilf(f), lo, hi); }

// [a, e): the indices i of the centre table ctr [N] (strictly increasing, the
// FP32 centres (i + 1/2)/N) where the test in(i) holds, given that in() is
// non-increasing in i below the first centre >= c and non-decreasing from it;
// half is the real-arithmetic half-width of the interval around c.
template <class In>
__device__ __forceinline__ void exact_span(const float* ctr, int N, float fN, float c, float half, In in, int& a,
                                           int& e) {
    // centre index: first i with ctr[i] >= c
    const int ic = first_in(0, N, guess_index(__fmaf_rn(c, fN, -0.5f), 0, N), [&](int i) { return ctr[i] >= c; });
    // lower end: first i of [0, ic) where the test holds; upper end: first i
    // of [ic, N) where it fails
    a = first_in(0, ic, guess_index(__fmaf_rn(__fsub_rn(c, half), fN, -0.5f), 0, N), in);
    e = first_in(ic, N, guess_index(__fmaf_rn(__fadd_rn(c, half), fN, -0.5f), 0, N), [&](int i) { return !in(i); });
}

// Mismatch count of the disc at (cx, cy) against a binary target, summed over
// the warp (every lane returns it): the rows [y0, y1) of the widened band go
// to lanes y0 + lane, y0 + lane + 32, ...; the others come from the prefix sums.
__device__ __forceinline__ int disc_mismatch_warp(const DiscBits& tb, int W, int H, const float* px,
                                                  const float* py, float cx, float cy, float radius, float r2,
                                                  int lane) {
    const int words = (W + 31) >> 5;
    const float fW = (float)W;
    const float fH = (float)H;
    const float mg = 2.0f + (fabsf(cy) + radius) * fH * 0x1p-20f;   // rows of margin (NaN: no rows)
    const int y0 = clamp_col(floorf(__fmaf_rn(__fsub_rn(cy, radius), fH, -0.5f) - mg), 0, H);
    const int y1 = max(y0, clamp_col(ceilf(__fmaf_rn(__fadd_rn(cy, radius), fH, -0.5f) + mg) + 1.0f, 0, H));
    int cnt = lane == 0 ? __ldg(tb.rowpop + H) - (__ldg(tb.rowpop + y1) - __ldg(tb.rowpop + y0)) : 0;
    for (int y = y0 + lane; y < y1; y += 32) {
        const float dy = __fsub_rn(py[y], cy);
        const float dy2 = __fmul_rn(dy, dy);
        int a = 0, e = 0;
        if (dy2 < r2)
            exact_span(px, W, fW, cx, sqrtf(__fsub_rn(r2, dy2)), [&](int x) {
                const float dx = __fsub_rn(px[x], cx);
                return __fmaf_rn(dx, dx, dy2) < r2;
            }, a, e);
        const uint32_t* row = tb.bits + (size_t)y * words;
        for (int j = 0; j < words; ++j) {
            const int lo = min(max(a - 32 * j, 0), 32), hi = min(max(e - 32 * j, 0), 32);
            const uint32_t m = (uint32_t)(((1ull << hi) - 1ull) & ~((1ull << lo) - 1ull));
            cnt += __popc(__ldg(row + j) ^ m);
        }
    }
    return __reduce_add_sync(0xffffffffu, cnt);
}

// Loss of the disc at centre (cx, cy) against the target, by one warp (all
// 32 lanes call; every lane returns the loss): the FP32 sum of the squared
// differences over the image, divided by the pixel count.  With a binary
// target (tb.bits non-null) the sum is the exact mismatch count of the spans;
// otherwise each lane sums its pixels in pixel order, then a shuffle tree adds
// the lanes.
__device__ __forceinline__ float disc_loss_warp(const float* __restrict__ target, const DiscBits& tb, int W, int H,
                                                float radius, const float* px, const float* py, float cx, float cy,
                                                int lane) {
    const float r2 = __fmul_rn(radius, radius);
    const int npx = W * H;
    if (tb.bits) return __fdiv_rn((float)disc_mismatch_warp(tb, W, H, px, py, cx, cy, radius, r2, lane), (float)npx);
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

// Squares (Box2 / Box10): K axis-aligned squares of half-size h centred at
// c[2k], c[2k + 1]; a pixel centre is 1 when |px - cx| < h and |py - cy| < h
// for some square (FP32).  Loss of one perturbation by one warp (every lane
// returns it).  With a binary target (tb.bits non-null) the sum is the exact
// mismatch count: |RN(px - cx)| is non-increasing in x left of the first
// column with px >= cx and non-decreasing from it, so square k covers the
// columns [a_k, e_k) in every row where |RN(py - cy_k)| < h; a row's covered
// pixels are the union of those intervals, its mismatches popc(target bits
// XOR union bits).  The intervals go to sp [2K] (this warp's shared memory).
// Otherwise each lane sums its pixels in pixel order, then a shuffle tree.
__device__ __forceinline__ float boxes_loss_warp(const float* __restrict__ target, const DiscBits& tb, int W, int H,
                                                 float h, const float* px, const float* py, const float* c, int* sp,
                                                 int K, int lane) {
    const int npx = W * H;
    if (tb.bits) {
        const float fW = (float)W;
        for (int k = lane; k < K; k += 32) {
            const float cx = c[2 * k];
            exact_span(px, W, fW, cx, h, [&](int x) { return fabsf(__fsub_rn(px[x], cx)) < h; }, sp[2 * k],
                       sp[2 * k + 1]);
        }
        __syncwarp();
        const int words = (W + 31) >> 5;
        int cnt = 0;
        for (int y = lane; y < H; y += 32) {
            const uint32_t* row = tb.bits + (size_t)y * words;
            for (int j = 0; j < words; ++j) {
                uint32_t m = 0u;
                for (int k = 0; k < K; ++k)
                    if (fabsf(__fsub_rn(py[y], c[2 * k + 1])) < h) {
                        const int lo = min(max(sp[2 * k] - 32 * j, 0), 32), hi = min(max(sp[2 * k + 1] - 32 * j, 0), 32);
                        m |= (uint32_t)(((1ull << hi) - 1ull) & ~((1ull << lo) - 1ull));
                    }
                cnt += __popc(__ldg(row + j) ^ m);
            }
        }
        return __fdiv_rn((float)__reduce_add_sync(0xffffffffu, cnt), (float)npx);
    }
    auto value = [c, K, h](float px_, float py_) {
        for (int k = 0; k < K; ++k)
            if (fabsf(__fsub_rn(px_, c[2 * k])) < h && fabsf(__fsub_rn(py_, c[2 * k + 1])) < h) return 1.0f;
        return 0.0f;
    };
    float acc = W >= 32 ? lane_l2<true>(target, W, npx, lane, px, py, value)
                        : lane_l2<false>(target, W, npx, lane, px, py, value);
    acc = warp_sum(acc);
    return __fdiv_rn(acc, (float)npx);
}

}  // namespace
}  // namespace hr
