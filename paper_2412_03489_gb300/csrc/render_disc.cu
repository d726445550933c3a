// K2: hard-edged disc renderer fused with the L2 loss (stand-in for the Box2
// plateau task, Sec. 4.1).  One warp renders one perturbation: pixel centre
// ((x + 1/2)/W, (y + 1/2)/H) is inside when fma(dx, dx, dy*dy) < r*r in FP32,
// value 1 inside, 0 outside.  With a 0/1 target every (v - t)^2 is 0 or 1 and
// the FP32 sum is an exact integer count.
#include <vector>

#include "disc_device.cuh"
#include "hr.h"
#include "hr_device.cuh"
#include "hr_internal.h"

namespace hr {
namespace {

template <int kW>
__global__ void __launch_bounds__(32 * kW) disc_loss_kernel(RenderBatch b, int W, int H, float radius,
                                                            const float* __restrict__ target,
                                                            DiscBits tb) {
    __shared__ float s_px[HR_MAX_IMAGE_SIDE], s_py[HR_MAX_IMAGE_SIDE];
    centre_tables(s_px, s_py, W, H);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.x * kW + warp;
    if (m >= b.M) return;
    const Pert pt = resolve(b, m);
    const float cx = __fadd_rn(pt.theta[0], pt.tau[0]);
    const float cy = __fadd_rn(pt.theta[1], pt.tau[1]);
    const float loss = disc_loss_warp(target, tb, W, H, radius, s_px, s_py, cx, cy, lane);
    if (lane == 0) *pt.loss = loss;
}

// Bit-packed target rows (bit x % 32 of word x / 32 of row y: pixel (x, y) is
// 1) and a flag raised by any pixel other than 0 or 1.
__global__ void disc_bits_kernel(const float* __restrict__ target, int W, int H, int words, uint32_t* bits,
                                 int* non_binary) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= words * H) return;
    const int y = i / words, j = i - y * words;
    uint32_t b = 0u;
    bool bad = false;
    for (int k = 0; k < 32 && 32 * j + k < W; ++k) {
        const float t = target[(size_t)y * W + 32 * j + k];
        if (t == 1.0f) b |= 1u << k;
        else if (t != 0.0f) bad = true;
    }
    bits[i] = b;
    if (bad) atomicOr(non_binary, 1);
}

__global__ void disc_image_kernel(const float* params, int W, int H, float radius, float* img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    const int y = i / W, x = i - y * W;
    img[i] = disc_value(x, y, W, H, params[0], params[1], __fmul_rn(radius, radius));
}

// Squares (Box2 / Box10): K axis-aligned squares of half-size h; a pixel
// centre is 1 when |px - cx| < h and |py - cy| < h for some square (FP32).
__device__ __forceinline__ float boxes_value(int x, int y, int W, int H, const float* c, int K, float h) {
    const float px = __fdiv_rn(__fadd_rn((float)x, 0.5f), (float)W);
    const float py = __fdiv_rn(__fadd_rn((float)y, 0.5f), (float)H);
    for (int k = 0; k < K; ++k)
        if (fabsf(__fsub_rn(px, c[2 * k])) < h && fabsf(__fsub_rn(py, c[2 * k + 1])) < h) return 1.0f;
    return 0.0f;
}

constexpr int kMaxBoxParams = 64;

template <int kW>
__global__ void __launch_bounds__(32 * kW) boxes_loss_kernel(RenderBatch b, int W, int H, float h,
                                                             const float* __restrict__ target, DiscBits tb) {
    __shared__ float s_c[kW][kMaxBoxParams];
    __shared__ int s_sp[kW][kMaxBoxParams];
    __shared__ float s_px[HR_MAX_IMAGE_SIDE], s_py[HR_MAX_IMAGE_SIDE];
    centre_tables(s_px, s_py, W, H);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.x * kW + warp;
    if (m >= b.M) return;
    const Pert pt = resolve(b, m);
    for (int d = lane; d < b.n; d += 32) s_c[warp][d] = __fadd_rn(pt.theta[d], pt.tau[d]);
    __syncwarp();
    const float loss = boxes_loss_warp(target, tb, W, H, h, s_px, s_py, s_c[warp], s_sp[warp], b.n / 2, lane);
    if (lane == 0) *pt.loss = loss;
}

__global__ void boxes_image_kernel(const float* params, int K, int W, int H, float h, float* img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    const int y = i / W, x = i - y * W;
    img[i] = boxes_value(x, y, W, H, params, K, h);
}

}  // namespace

// Launch-shape variants (autotuner): 8, 4 or 16 warps per CTA; one warp
// renders one perturbation in every shape, so the choice never changes a result.
void launch_boxes_loss(const DevScene& sc, const RenderBatch& b, cudaStream_t s) {
    const DiscBits tb{sc.tbinary ? sc.tbits : nullptr, sc.trowpop};
    switch (sc.render_variant) {
        case 1: boxes_loss_kernel<4><<<(b.M + 3) / 4, 128, 0, s>>>(b, sc.W, sc.H, sc.radius, sc.target, tb); break;
        case 2: boxes_loss_kernel<16><<<(b.M + 15) / 16, 512, 0, s>>>(b, sc.W, sc.H, sc.radius, sc.target, tb); break;
        default: boxes_loss_kernel<8><<<(b.M + 7) / 8, 256, 0, s>>>(b, sc.W, sc.H, sc.radius, sc.target, tb); break;
    }
}

void launch_boxes_image(const DevScene& sc, const float* params, float* img, cudaStream_t s) {
    const int npx = sc.W * sc.H;
    boxes_image_kernel<<<(npx + 255) / 256, 256, 0, s>>>(params, sc.n / 2, sc.W, sc.H, sc.radius, img);
}

void launch_disc_loss(const DevScene& sc, const RenderBatch& b, cudaStream_t s) {
    const DiscBits tb{sc.tbinary ? sc.tbits : nullptr, sc.trowpop};
    switch (sc.render_variant) {
        case 1: disc_loss_kernel<4><<<(b.M + 3) / 4, 128, 0, s>>>(b, sc.W, sc.H, sc.radius, sc.target, tb); break;
        case 2: disc_loss_kernel<16><<<(b.M + 15) / 16, 512, 0, s>>>(b, sc.W, sc.H, sc.radius, sc.target, tb); break;
        default: disc_loss_kernel<8><<<(b.M + 7) / 8, 256, 0, s>>>(b, sc.W, sc.H, sc.radius, sc.target, tb); break;
    }
}

cudaError_t disc_prepare_target(DevScene& sc, cudaStream_t s) {
    const int words = (sc.W + 31) / 32;
    int* d_flag = nullptr;
    cudaError_t e = cudaMalloc((void**)&sc.tbits, sizeof(uint32_t) * words * sc.H);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_flag, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        disc_bits_kernel<<<(words * sc.H + 255) / 256, 256, 0, s>>>(sc.target, sc.W, sc.H, words, sc.tbits, d_flag);
        e = cudaGetLastError();
    }
    int non_binary = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&non_binary, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_flag);
    // prefix sums of the rows' popcounts (rows the disc cannot reach differ
    // from the target in exactly its set pixels)
    std::vector<uint32_t> bits((size_t)words * sc.H);
    std::vector<int> pop((size_t)sc.H + 1, 0);
    if (e == cudaSuccess)
        e = cudaMemcpy(bits.data(), sc.tbits, sizeof(uint32_t) * bits.size(), cudaMemcpyDeviceToHost);
    for (int y = 0; y < sc.H; ++y) {
        int c = 0;
        for (int j = 0; j < words; ++j) c += __builtin_popcount(bits[(size_t)y * words + j]);
        pop[y + 1] = pop[y] + c;
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&sc.trowpop, sizeof(int) * pop.size());
    if (e == cudaSuccess) e = cudaMemcpy(sc.trowpop, pop.data(), sizeof(int) * pop.size(), cudaMemcpyHostToDevice);
    sc.tbinary = e == cudaSuccess && non_binary == 0;
    return e;
}

void launch_disc_image(const DevScene& sc, const float* params, float* img, cudaStream_t s) {
    const int npx = sc.W * sc.H;
    disc_image_kernel<<<(npx + 255) / 256, 256, 0, s>>>(params, sc.W, sc.H, sc.radius, img);
}

}  // namespace hr
