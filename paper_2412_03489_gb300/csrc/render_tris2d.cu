// Coloured-triangle rasteriser fused with the L2 loss (stand-in for the
// Box10 / mesh tasks of Sec. 4.1).  Vertex (x, y) in [0,1]^2 maps to pixel
// coordinates (x W, y H); both windings are drawn (edge coefficients negated
// when the signed area is negative, skipped when it is zero); painter's
// order: the highest covering triangle index wins.  One CTA renders one
// perturbation: the triangles are set up in shared memory, then each warp
// walks 8x4-pixel tiles with one pixel per lane, testing (warp-uniformly, from
// the highest index down) the triangles whose pixel box meets the tile.
#include "hr_device.cuh"
#include "hr_internal.h"

namespace hr {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxTris = 32;

struct __align__(16) T2Rec {
    float A0, B0, C0, A1;
    float B1, C1, A2, B2;
    float C2, r, g, bl;
    int xlo, xhi, ylo, yhi;
    float th0, th1, th2, pad;   // edge i passes when E_i > th_i (see tl_thr)
};

// E > 0, or E == 0 on a top-left edge (A > 0, or A == 0 and B > 0), is one
// compare E > th: th = 0, or th = -(smallest subnormal), no float lying
// strictly between the two
__device__ __forceinline__ float tl_thr(float A, float B) {
    return (A > 0.0f || (A == 0.0f && B > 0.0f)) ? -0x1p-149f : 0.0f;
}

__device__ __forceinline__ bool pixel_range2(float mn, float mx, int N, int& lo, int& hi) {
    if (!(mx >= 0.5f) || !(mn <= (float)N - 0.5f)) return false;
    lo = (mn <= 0.5f) ? 0 : (int)ceilf(__fsub_rn(mn, 0.5f));
    hi = (mx >= (float)N - 0.5f) ? N - 1 : (int)floorf(__fsub_rn(mx, 0.5f));
    return lo <= hi;
}

// Set up triangle t from its raw params q[9]; returns false when it covers no pixel.
__device__ bool setup_tri(const float* q, int W, int H, T2Rec& r) {
    const float fW = (float)W, fH = (float)H;
    const float ax = __fmul_rn(q[0], fW), ay = __fmul_rn(q[1], fH);
    const float bx = __fmul_rn(q[2], fW), by = __fmul_rn(q[3], fH);
    const float cx = __fmul_rn(q[4], fW), cy = __fmul_rn(q[5], fH);
    Edge e0 = edge_of(bx, by, cx, cy), e1 = edge_of(cx, cy, ax, ay), e2 = edge_of(ax, ay, bx, by);
    const float D2 = edge_eval(e2.A, e2.B, e2.C, cx, cy);
    if (D2 == 0.0f || D2 != D2) return false;
    if (D2 < 0.0f) {
        e0.A = -e0.A; e0.B = -e0.B; e0.C = -e0.C;
        e1.A = -e1.A; e1.B = -e1.B; e1.C = -e1.C;
        e2.A = -e2.A; e2.B = -e2.B; e2.C = -e2.C;
    }
    const float mnx = fminf(fminf(ax, bx), cx), mxx = fmaxf(fmaxf(ax, bx), cx);
    const float mny = fminf(fminf(ay, by), cy), mxy = fmaxf(fmaxf(ay, by), cy);
    if (!pixel_range2(mnx, mxx, W, r.xlo, r.xhi) || !pixel_range2(mny, mxy, H, r.ylo, r.yhi)) return false;
    r.A0 = e0.A; r.B0 = e0.B; r.C0 = e0.C;
    r.A1 = e1.A; r.B1 = e1.B; r.C1 = e1.C;
    r.A2 = e2.A; r.B2 = e2.B; r.C2 = e2.C;
    r.r = q[6]; r.g = q[7]; r.bl = q[8];
    r.th0 = tl_thr(e0.A, e0.B); r.th1 = tl_thr(e1.A, e1.B); r.th2 = tl_thr(e2.A, e2.B);
    r.pad = 0.0f;
    return true;
}

template <bool kImage>
__global__ void __launch_bounds__(kThreads)
tris2d_kernel(RenderBatch b, const float* __restrict__ raw, const int32_t* __restrict__ pidx, int n_tris, int W,
              int H, const float* __restrict__ target, const float* __restrict__ img_params, float* __restrict__ img) {
    __shared__ float s_raw[kMaxTris * 9];
    __shared__ T2Rec s_rec[kMaxTris];
    __shared__ int s_valid[kMaxTris];
    __shared__ float s_part[kThreads / 32];
    const int m = blockIdx.x;
    const int tid = threadIdx.x;
    for (int i = tid; i < n_tris * 9; i += kThreads) s_raw[i] = raw[i];
    __syncthreads();
    const int n = kImage ? 0 : b.n;
    if (kImage) {
        // img_params holds all raw params of the optimised subset
        for (int j = tid; j < (int)(b.n); j += kThreads) s_raw[pidx[j]] = img_params[j];
    } else {
        const Pert pt = resolve(b, m);
        for (int j = tid; j < n; j += kThreads) s_raw[pidx[j]] = __fadd_rn(pt.theta[j], pt.tau[j]);
    }
    __syncthreads();
    if (tid < n_tris) s_valid[tid] = setup_tri(&s_raw[9 * tid], W, H, s_rec[tid]) ? 1 : 0;
    __syncthreads();
    // warp-uniform raster: each warp walks 8x4 tiles (one pixel per lane); a
    // ballot gives the triangles whose pixel box meets the tile, tested from the
    // highest index down (painter's order) until every lane is covered
    float acc = 0.0f;
    const int npx = W * H;
    const int lane = tid & 31, warp = tid >> 5;
    const int TXn = (W + 7) / 8, TYn = (H + 3) / 4;
    constexpr int kWarps = kThreads / 32;
    // tile t = ty TXn + tx, stepped by kWarps without a division per tile
    int ty = warp / TXn, tx = warp - ty * TXn;
    for (int t = warp; t < TXn * TYn; t += kWarps) {
        const int x0 = tx * 8, y0 = ty * 4;
        tx += kWarps;
        while (tx >= TXn) { tx -= TXn; ++ty; }
        const int x = x0 + (lane & 7), y = y0 + (lane >> 3);
        bool over = false;
        if (lane < n_tris && s_valid[lane]) {
            const T2Rec& r = s_rec[lane];
            over = r.xlo <= x0 + 7 && r.xhi >= x0 && r.ylo <= y0 + 3 && r.yhi >= y0;
        }
        uint32_t mm = __ballot_sync(0xffffffffu, over);
        const bool inside_img = x < W && y < H;
        const float fx = __fadd_rn((float)x, 0.5f), fy = __fadd_rn((float)y, 0.5f);
        int win = -1;
        while (mm) {
            const int k = 31 - __clz(mm);
            mm &= ~(1u << k);
            if (win < 0 && inside_img) {
                const T2Rec& r = s_rec[k];
                if (x >= r.xlo && x <= r.xhi && y >= r.ylo && y <= r.yhi) {
                    const float E0 = edge_eval(r.A0, r.B0, r.C0, fx, fy);
                    const float E1 = edge_eval(r.A1, r.B1, r.C1, fx, fy);
                    const float E2 = edge_eval(r.A2, r.B2, r.C2, fx, fy);
                    if (E0 > r.th0 && E1 > r.th1 && E2 > r.th2) win = k;
                }
            }
            if (__all_sync(0xffffffffu, win >= 0 || !inside_img)) break;
        }
        if (inside_img) {
            const size_t p = (size_t)y * W + x;
            const float c0 = win >= 0 ? s_rec[win].r : 0.0f;
            const float c1 = win >= 0 ? s_rec[win].g : 0.0f;
            const float c2 = win >= 0 ? s_rec[win].bl : 0.0f;
            if (kImage) {
                img[3 * p] = c0; img[3 * p + 1] = c1; img[3 * p + 2] = c2;
            } else {
                const float d0 = c0 - target[3 * p], d1 = c1 - target[3 * p + 1], d2 = c2 - target[3 * p + 2];
                acc += d0 * d0 + d1 * d1 + d2 * d2;
            }
        }
    }
    (void)npx;
    if (!kImage) {
        acc = warp_sum(acc);
        if ((tid & 31) == 0) s_part[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            float v = 0.0f;
            for (int w = 0; w < kThreads / 32; ++w) v += s_part[w];
            *resolve(b, m).loss = v / (float)(W * H * 3);
        }
    }
}

}  // namespace

void launch_tris2d_loss(const DevScene& sc, const RenderBatch& b, cudaStream_t s) {
    tris2d_kernel<false><<<b.M, kThreads, 0, s>>>(b, sc.raw, sc.pidx, sc.n_tris, sc.W, sc.H, sc.target, nullptr,
                                                   nullptr);
}

void launch_tris2d_image(const DevScene& sc, const float* params, float* img, cudaStream_t s) {
    RenderBatch b{};
    b.n = sc.n;
    tris2d_kernel<true><<<1, kThreads, 0, s>>>(b, sc.raw, sc.pidx, sc.n_tris, sc.W, sc.H, sc.target, params, img);
}

}  // namespace hr
