// K3/K4: rasteriser of a triangle mesh (surface of revolution, stand-in for
// the Mug task of Sec. 4.1) fused with the per-pixel L2 loss and the block
// reduction, so that no image is written to HBM.
//
// One CTA (1024 threads, one per SM, persistent over perturbations) renders a
// whole perturbation:
//   1. rotation R = Rx(p0) Ry(p1) from RN32 of FP64 cos / sin (for every
//      perturbation after a CTA's first, computed during the previous raster);
//   2. vertex transform and projection (FP32, fixed operation order);
//   3. triangle setup: edge functions, back-face cull, depth plane of 1/Z,
//      pixel bounding box, flat Lambert shade; surviving triangles are
//      compacted into shared memory;
//   4. binning into 8x8 pixel tiles (count, scan, fill; all in shared memory),
//      skipping tiles that a conservative edge test shows the triangle misses;
//   5. warp-per-tile raster, tiles fetched dynamically: the two half-warps
//      take alternate bin entries, each lane testing 4 pixels of a row; nearest 1/Z
//      wins, ties to the lower triangle index (half-warp winners merged by a
//      shuffle); (colour - target)^2 per tile; tiles with an empty bin take
//      the precomputed sum of target^2;
//   6. per-tile losses summed in tile order, warp shuffle + block reduction to
//      one FP32 loss per perturbation.
// The FP32 sequences of steps 2-5 define the renderer (coverage and depth
// decisions), so they use explicitly rounded intrinsics.
#include <climits>
#include <cmath>

#include "hr_device.cuh"
#include "hr_internal.h"

namespace hr {
namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 8;
constexpr int kEntryCap = 16384;
constexpr int kHeavy = 6;   // tiles with at least this many entries are fetched first

struct __align__(16) TriRec {
    float A0, B0, C0, A1;
    float B1, C1, A2, B2;
    float C2, Aw, Bw, Cw;
    float shade;
    uint32_t key;  // triangle index | top-left flag of edge i at bit 29 + i
    uint32_t xr;   // x_lo | x_hi << 16 (pixel columns whose centre is inside the bbox)
    uint32_t yr;
};

// E > 0, or E == 0 on a top-left edge, is one compare: E > thr with thr = 0
// or thr = -(smallest subnormal) (no float lies strictly between the two)
__device__ __forceinline__ float tl_threshold(uint32_t key, int i) {
    return ((key >> (29 + i)) & 1u) ? -0x1p-149f : 0.0f;
}
__device__ __forceinline__ uint32_t tl_bit(float A, float B) {
    return (A > 0.0f || (A == 0.0f && B > 0.0f)) ? 1u : 0u;
}

struct RvArgs {
    const float* verts;
    const int32_t* tris;
    const float* tnrm;
    const float* target;
    const float* tile_t2;
    int nv, nt, W, H, TX, TY, T;
    uint64_t tx_recip;   // ceil(2^32 / TX): t / TX = (t tx_recip) >> 32 exactly for t, TX < 2^16
    unsigned long long* stats;   // [0]: renders whose bins overflowed (diagnostics)
    float alb0, alb1, alb2, l0, l1, l2, eye_dist, scale;
};

// pixel range [lo, hi] of centres c + 1/2 with mn <= c + 1/2 <= mx, c in [0, N)
__device__ __forceinline__ bool pixel_range(float mn, float mx, int N, int& lo, int& hi) {
    if (!(mx >= 0.5f) || !(mn <= (float)N - 0.5f)) return false;
    lo = (mn <= 0.5f) ? 0 : (int)ceilf(__fsub_rn(mn, 0.5f));
    hi = (mx >= (float)N - 0.5f) ? N - 1 : (int)floorf(__fsub_rn(mx, 0.5f));
    return lo <= hi;
}

// Does any pixel centre of tile (tx, ty) inside the triangle's bounding box
// pass all three edge tests?  Conservative: false only when, for some edge,
// the edge function at the corner of the (tile ∩ box) rectangle where it is
// largest lies below neg[i] = -1e-5 (|A| W + |B| H + |C|), minus 1e-5 times
// a bound on its term magnitudes anywhere in the image; the FP32 errors of
// the exact per-pixel test and of this test are below 3e-7 of that
// magnitude, so no rejected tile holds a covered pixel.
__device__ __forceinline__ bool tile_hits(const TriRec& r, const float neg[3], int tx, int ty) {
    const int x0 = max(tx * kTile, (int)(r.xr & 0xffffu)), x1 = min(tx * kTile + kTile - 1, (int)(r.xr >> 16));
    const int y0 = max(ty * kTile, (int)(r.yr & 0xffffu)), y1 = min(ty * kTile + kTile - 1, (int)(r.yr >> 16));
    const float fx0 = (float)x0 + 0.5f, fx1 = (float)x1 + 0.5f, fy0 = (float)y0 + 0.5f, fy1 = (float)y1 + 0.5f;
    const float A[3] = {r.A0, r.A1, r.A2}, B[3] = {r.B0, r.B1, r.B2}, C[3] = {r.C0, r.C1, r.C2};
    bool hit = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float x = A[i] > 0.0f ? fx1 : fx0, y = B[i] > 0.0f ? fy1 : fy0;
        hit = hit && !(fmaf(A[i], x, fmaf(B[i], y, C[i])) < neg[i]);
    }
    return hit;
}

// Exclusive scan of cnt[0..T) into off[0..T) and, in the same pass, the
// list of tiles with entries (olist[0..n_obj)): tiles with at least kHeavy
// entries first, then the others, each group in tile order, so that the
// dynamic fetch hands out the long tiles first and the raster ends on short
// ones.  Each tile contributes cnt + heavy 2^32 + light 2^48 to one 64-bit
// scan (cnt < 2^32, tile counts < 2^16).  Returns the total entry count (all
// threads) and sets n_obj.
__device__ int bin_scan(const int* cnt, int* off, uint16_t* olist, int T, unsigned long long* warp_tot,
                        int* n_obj) {
    const int per = (T + kThreads - 1) / kThreads;
    const int b = threadIdx.x * per;
    auto packed = [](int c) {
        return (unsigned long long)c + ((unsigned long long)(c >= kHeavy) << 32) +
               ((unsigned long long)(c > 0 && c < kHeavy) << 48);
    };
    unsigned long long local = 0ull;
    for (int i = 0; i < per; ++i)
        if (b + i < T) local += packed(cnt[b + i]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long wv = warp_tot[lane];
        unsigned long long wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        warp_tot[lane] = wi - wv;       // exclusive warp offsets
        if (lane == 31) warp_tot[32] = wi;
    }
    __syncthreads();
    unsigned long long run = warp_tot[warp] + incl - local;
    const unsigned long long total = warp_tot[32];
    const int n_heavy = (int)((total >> 32) & 0xffffull);
    for (int i = 0; i < per; ++i)
        if (b + i < T) {
            const int c = cnt[b + i];
            off[b + i] = (int)(run & 0xffffffffull);
            if (c >= kHeavy) olist[(run >> 32) & 0xffffull] = (uint16_t)(b + i);
            else if (c > 0) olist[n_heavy + (int)(run >> 48)] = (uint16_t)(b + i);
            run += packed(c);
        }
    __syncthreads();
    *n_obj = n_heavy + (int)(total >> 48);
    return (int)(total & 0xffffffffull);
}

// rotation angle d of perturbation m: RN32(theta32 + tau)
__device__ __forceinline__ float rotation_param(const RenderBatch& b, int m, int d) {
    const Pert pt = resolve(b, m);
    return __fadd_rn(pt.theta[d], pt.tau[d]);
}

template <bool kImage>
__global__ void __launch_bounds__(kThreads, 1)
revolve_kernel(RvArgs P, RenderBatch b, const float* __restrict__ img_params, float* __restrict__ img) {
    extern __shared__ __align__(16) unsigned char smem[];
    TriRec* rec = reinterpret_cast<TriRec*>(smem);
    float* vx = reinterpret_cast<float*>(rec + P.nt);
    float* vy = vx + P.nv;
    float* viz = vy + P.nv;
    int* tcnt = reinterpret_cast<int*>(vx + max(3 * P.nv, (P.T + 1) / 2));
    int* toff = tcnt + P.T;
    uint16_t* ent = reinterpret_cast<uint16_t*>(toff + P.T);

    __shared__ float s_cs[4], s_cs_next[4];
    __shared__ float sR[9];
    __shared__ float sL[3];
    __shared__ int s_count;
    __shared__ unsigned long long s_wtot[33];
    __shared__ float s_part[kWarps];
    __shared__ int s_tile;
    float* tshade = reinterpret_cast<float*>(ent + kEntryCap);   // [nt] shade by triangle index
    uint32_t* tmask = reinterpret_cast<uint32_t*>(tshade + P.nt);  // [nt] tiles hit, by record slot
    // [T] tiles with entries, in tile order: in the vertex arrays, free once
    // the triangles are set up (the region holds max(3 nv, T / 2) floats)
    uint16_t* olist = reinterpret_cast<uint16_t*>(vx);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int M = kImage ? 1 : b.M;
    for (int m = kImage ? 0 : (int)blockIdx.x; m < M; m += kImage ? 1 : (int)gridDim.x) {
        // ---- 1. parameters and rotation ----------------------------------
        if (tid < 4) {   // ca, sa, cb, sb
            if (kImage || m == (int)blockIdx.x) {
                const float p = kImage ? img_params[tid >> 1] : rotation_param(b, m, tid >> 1);
                const double a = (double)p;
                s_cs[tid] = (float)((tid & 1) ? sin(a) : cos(a));
            } else {
                s_cs[tid] = s_cs_next[tid];   // computed during the previous raster phase
            }
        }
        for (int i = tid; i < P.T; i += kThreads) tcnt[i] = 0;
        if (tid == 0) { s_count = 0; s_tile = 0; }
        __syncthreads();
        if (tid == 0) {
            const float ca = s_cs[0], sa = s_cs[1], cb = s_cs[2], sb = s_cs[3];
            sR[0] = cb;                 sR[1] = 0.0f; sR[2] = sb;
            sR[3] = __fmul_rn(sa, sb);  sR[4] = ca;   sR[5] = -__fmul_rn(sa, cb);
            sR[6] = -__fmul_rn(ca, sb); sR[7] = sa;   sR[8] = __fmul_rn(ca, cb);
            // light in model space: R^T l (shading value only)
            sL[0] = sR[0] * P.l0 + sR[3] * P.l1 + sR[6] * P.l2;
            sL[1] = sR[1] * P.l0 + sR[4] * P.l1 + sR[7] * P.l2;
            sL[2] = sR[2] * P.l0 + sR[5] * P.l1 + sR[8] * P.l2;
        }
        __syncthreads();
        // ---- 2. vertices ---------------------------------------------------
        const float halfW = __fmul_rn((float)P.W, 0.5f), halfH = __fmul_rn((float)P.H, 0.5f);
        for (int v = tid; v < P.nv; v += kThreads) {
            const float x = P.verts[3 * v], y = P.verts[3 * v + 1], z = P.verts[3 * v + 2];
            const float X = __fmaf_rn(sR[2], z, __fmaf_rn(sR[1], y, __fmul_rn(sR[0], x)));
            const float Y = __fmaf_rn(sR[5], z, __fmaf_rn(sR[4], y, __fmul_rn(sR[3], x)));
            const float w2 = __fmaf_rn(sR[8], z, __fmaf_rn(sR[7], y, __fmul_rn(sR[6], x)));
            const float Z = __fsub_rn(P.eye_dist, w2);
            const float qx = __fdiv_rn(X, Z), qy = __fdiv_rn(Y, Z);
            vx[v] = __fmaf_rn(P.scale, qx, halfW);
            vy[v] = __fmaf_rn(-P.scale, qy, halfH);
            viz[v] = (Z > 0.0f) ? __fdiv_rn(1.0f, Z) : -1.0f;
        }
        __syncthreads();
        // ---- 3. triangle setup ----------------------------------------------
        for (int t = tid; t < P.nt; t += kThreads) {
            const int ia = P.tris[3 * t], ib = P.tris[3 * t + 1], ic = P.tris[3 * t + 2];
            const float iza = viz[ia], izb = viz[ib], izc = viz[ic];
            if (!(iza > 0.0f && izb > 0.0f && izc > 0.0f)) continue;
            const float ax = vx[ia], ay = vy[ia], bx = vx[ib], by = vy[ib], cx = vx[ic], cy = vy[ic];
            const Edge e0 = edge_of(bx, by, cx, cy);
            const Edge e1 = edge_of(cx, cy, ax, ay);
            const Edge e2 = edge_of(ax, ay, bx, by);
            const float D2 = edge_eval(e2.A, e2.B, e2.C, cx, cy);
            if (!(D2 > 0.0f)) continue;
            int xlo, xhi, ylo, yhi;
            const float mnx = fminf(fminf(ax, bx), cx), mxx = fmaxf(fmaxf(ax, bx), cx);
            const float mny = fminf(fminf(ay, by), cy), mxy = fmaxf(fmaxf(ay, by), cy);
            if (!pixel_range(mnx, mxx, P.W, xlo, xhi) || !pixel_range(mny, mxy, P.H, ylo, yhi)) continue;
            const float invD = __fdiv_rn(1.0f, D2);
            TriRec r;
            r.A0 = e0.A; r.B0 = e0.B; r.C0 = e0.C;
            r.A1 = e1.A; r.B1 = e1.B; r.C1 = e1.C;
            r.A2 = e2.A; r.B2 = e2.B; r.C2 = e2.C;
            r.Aw = __fmul_rn(__fmaf_rn(e2.A, izc, __fmaf_rn(e1.A, izb, __fmul_rn(e0.A, iza))), invD);
            r.Bw = __fmul_rn(__fmaf_rn(e2.B, izc, __fmaf_rn(e1.B, izb, __fmul_rn(e0.B, iza))), invD);
            r.Cw = __fmul_rn(__fmaf_rn(e2.C, izc, __fmaf_rn(e1.C, izb, __fmul_rn(e0.C, iza))), invD);
            const float sh = P.tnrm[3 * t] * sL[0] + P.tnrm[3 * t + 1] * sL[1] + P.tnrm[3 * t + 2] * sL[2];
            r.shade = fmaxf(sh, 0.0f);
            tshade[t] = r.shade;
            r.key = (uint32_t)t | (tl_bit(e0.A, e0.B) << 29) | (tl_bit(e1.A, e1.B) << 30) | (tl_bit(e2.A, e2.B) << 31);
            r.xr = (uint32_t)xlo | ((uint32_t)xhi << 16);
            r.yr = (uint32_t)ylo | ((uint32_t)yhi << 16);
            const int slot = atomicAdd(&s_count, 1);
            rec[slot] = r;
        }
        __syncthreads();
        const int count = s_count;
        // ---- 4. binning -----------------------------------------------------
        // count pass: each record's tiles that pass the conservative edge test
        // go into a bit mask (row-major over its tile rectangle; rectangles of
        // more than 32 tiles skip the test), reused by the fill pass
        for (int s = tid; s < count; s += kThreads) {
            const TriRec r = rec[s];
            const int tx0 = (int)(r.xr & 0xffffu) / kTile, tx1 = (int)(r.xr >> 16) / kTile;
            const int ty0 = (int)(r.yr & 0xffffu) / kTile, ty1 = (int)(r.yr >> 16) / kTile;
            const bool test = (tx1 - tx0 + 1) * (ty1 - ty0 + 1) <= 32;
            const float fW = (float)P.W, fH = (float)P.H;
            const float neg[3] = {-1e-5f * fmaf(fabsf(r.A0), fW, fmaf(fabsf(r.B0), fH, fabsf(r.C0))),
                                  -1e-5f * fmaf(fabsf(r.A1), fW, fmaf(fabsf(r.B1), fH, fabsf(r.C1))),
                                  -1e-5f * fmaf(fabsf(r.A2), fW, fmaf(fabsf(r.B2), fH, fabsf(r.C2)))};
            uint32_t mask = 0;
            int bit = 0;
            for (int ty = ty0; ty <= ty1; ++ty)
                for (int tx = tx0; tx <= tx1; ++tx, ++bit)
                    if (!test || tile_hits(r, neg, tx, ty)) {
                        atomicAdd(&tcnt[ty * P.TX + tx], 1);
                        if (test) mask |= 1u << bit;
                    }
            tmask[s] = test ? mask : 0xFFFFFFFFu;
        }
        __syncthreads();
        int n_obj = 0;
        const int total = bin_scan(tcnt, toff, olist, P.T, s_wtot, &n_obj);
        const bool overflow = total > kEntryCap;
        if (overflow && tid == 0 && P.stats) atomicAdd(P.stats, 1ull);
        for (int i = tid; i < P.T; i += kThreads) tcnt[i] = 0;   // becomes the fill cursor
        __syncthreads();
        if (!overflow) {
            for (int s = tid; s < count; s += kThreads) {
                const uint32_t xr = rec[s].xr, yr = rec[s].yr, mask = tmask[s];
                const int tx0 = (int)(xr & 0xffffu) / kTile, tx1 = (int)(xr >> 16) / kTile;
                const int ty0 = (int)(yr & 0xffffu) / kTile, ty1 = (int)(yr >> 16) / kTile;
                int bit = 0;
                for (int ty = ty0; ty <= ty1; ++ty)
                    for (int tx = tx0; tx <= tx1; ++tx, ++bit) {
                        if (mask != 0xFFFFFFFFu && !((mask >> bit) & 1u)) continue;
                        const int tile = ty * P.TX + tx;
                        const int pos = atomicAdd(&tcnt[tile], 1);
                        ent[toff[tile] + pos] = (uint16_t)s;
                    }
            }
        }
        __syncthreads();
        // ---- 5. raster + loss ------------------------------------------------
        // warps fetch tiles dynamically (object tiles cost far more than
        // background tiles); each tile's loss goes to its own slot (the fill cursor array is free
        // again) and the slots are summed in tile order below, so the loss does
        // not depend on which warp took which tile
        float* tile_loss = reinterpret_cast<float*>(tcnt);
        // Half-warp pairing: lanes 0-15 and 16-31 walk alternate entries of the
        // bin.  Lane (row ry, half-row hx) of a half covers the 4 pixels
        // (x0 .. x0 + 3, y): the row term fma(B, y + 1/2, C) of each edge and of
        // the depth plane is formed once per entry and shared by the 4 pixels.
        // The per-entry work (record loads, unpacking, thresholds) is paid once
        // per pair of entries; the halves' per-pixel winners merge with a
        // shuffle (largest 1/Z, lower index on ties: order-independent).
        const int half = lane >> 4, hl = lane & 15;
        const int ry = hl >> 1, hx = hl & 1;
        // the FP64 cos / sin of this CTA's next perturbation, off the critical
        // path: one warp computes them before it joins the tile loop
        if (!kImage && warp == kWarps - 1 && lane < 4) {
            const int mn = m + (int)gridDim.x;
            if (mn < M) {
                const double a = (double)rotation_param(b, mn, lane >> 1);
                s_cs_next[lane] = (float)((lane & 1) ? sin(a) : cos(a));
            }
        }
        // each warp reserves its next tile when it starts the current one, so
        // the shared atomic's latency overlaps the tile's work
        // tiles without entries are not visited: their loss, the sum of
        // target^2, is taken in the reduction (an image visits every tile)
        const bool all_tiles = kImage || overflow;
        const int n_iter = all_tiles ? P.T : n_obj;
        int t_next = 0;
        if (lane == 0) t_next = atomicAdd(&s_tile, 1);
        for (int it = __shfl_sync(0xffffffffu, t_next, 0); it < n_iter; it = __shfl_sync(0xffffffffu, t_next, 0)) {
            if (lane == 0) t_next = atomicAdd(&s_tile, 1);
            const int t = all_tiles ? it : (int)olist[it];
            int beg, end;
            if (overflow) { beg = 0; end = count; }
            else { beg = toff[t]; end = (t + 1 < P.T) ? toff[t + 1] : total; }
            // division by multiplication with the rounded-up reciprocal
            // (Granlund and Montgomery, PLDI 1994): exact for t, TX < 2^16
            const int ty = (int)(((uint64_t)(uint32_t)t * P.tx_recip) >> 32), tx = t - ty * P.TX;
            const int x0 = tx * kTile + 4 * hx, y = ty * kTile + ry;
            // loss pixels of this lane after the merge: columns x0 + 2 half, x0 + 2 half + 1
            const int xa = x0 + 2 * half, xb = xa + 1;
            const bool va = xa < P.W && y < P.H, vb = xb < P.W && y < P.H;
            float tga[3] = {0.f, 0.f, 0.f}, tgb[3] = {0.f, 0.f, 0.f};
            if (!kImage) {
                if (va) for (int c = 0; c < 3; ++c) tga[c] = P.target[3 * ((size_t)y * P.W + xa) + c];
                if (vb) for (int c = 0; c < 3; ++c) tgb[c] = P.target[3 * ((size_t)y * P.W + xb) + c];
            }
            const float fy = __fadd_rn((float)y, 0.5f);
            float fx[4], bw[4];
            int bi[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                fx[c] = __fadd_rn((float)(x0 + c), 0.5f);
                bw[c] = -INFINITY;
                bi[c] = INT_MAX;
            }
            for (int jj = beg; jj < end; jj += 2) {
                const int j = jj + half;
                if (j < end) {
                    const int s = overflow ? j : (int)ent[j];
                    const float4* rp = reinterpret_cast<const float4*>(&rec[s]);
                    const float4 q0 = rp[0], q1 = rp[1], q2 = rp[2], q3 = rp[3];
                    const uint32_t key = __float_as_uint(q3.y);
                    const uint32_t xr = __float_as_uint(q3.z), yr = __float_as_uint(q3.w);
                    const int ti = (int)(key & 0x1FFFFFFFu);
                    const float th0 = tl_threshold(key, 0), th1 = tl_threshold(key, 1), th2 = tl_threshold(key, 2);
                    const int lo = (int)(xr & 0xffffu) - x0, hi = (int)(xr >> 16) - x0;
                    const int ylo = (int)(yr & 0xffffu);
                    const bool yok = (unsigned)(y - ylo) <= (yr >> 16) - (unsigned)ylo;
                    const float r0 = __fmaf_rn(q0.y, fy, q0.z);
                    const float r1 = __fmaf_rn(q1.x, fy, q1.y);
                    const float r2 = __fmaf_rn(q1.w, fy, q2.x);
                    const float rw = __fmaf_rn(q2.z, fy, q2.w);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float E0 = __fmaf_rn(q0.x, fx[c], r0);
                        const float E1 = __fmaf_rn(q0.w, fx[c], r1);
                        const float E2 = __fmaf_rn(q1.z, fx[c], r2);
                        const float wz = __fmaf_rn(q2.y, fx[c], rw);
                        const bool in = yok && c >= lo && c <= hi && (E0 > th0) && (E1 > th1) && (E2 > th2);
                        const bool better = in && (wz > bw[c] || (wz == bw[c] && ti < bi[c]));
                        bw[c] = better ? wz : bw[c];
                        bi[c] = better ? ti : bi[c];
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float ow = __shfl_xor_sync(0xffffffffu, bw[c], 16);
                const int oi = __shfl_xor_sync(0xffffffffu, bi[c], 16);
                const bool take = ow > bw[c] || (ow == bw[c] && oi < bi[c]);
                bw[c] = take ? ow : bw[c];
                bi[c] = take ? oi : bi[c];
            }
            // this lane's two pixels: columns 2 half and 2 half + 1 of its four
            const int ia = half ? bi[2] : bi[0], ib = half ? bi[3] : bi[1];
            const float sha = ia != INT_MAX ? tshade[ia] : 0.0f;
            const float shb = ib != INT_MAX ? tshade[ib] : 0.0f;
            const float ca0 = sha * P.alb0, ca1 = sha * P.alb1, ca2 = sha * P.alb2;
            const float cb0 = shb * P.alb0, cb1 = shb * P.alb1, cb2 = shb * P.alb2;
            if (kImage) {
                if (va) {
                    const size_t p = 3 * ((size_t)y * P.W + xa);
                    img[p] = ca0; img[p + 1] = ca1; img[p + 2] = ca2;
                }
                if (vb) {
                    const size_t p = 3 * ((size_t)y * P.W + xb);
                    img[p] = cb0; img[p + 1] = cb1; img[p + 2] = cb2;
                }
            } else {
                float acc = 0.0f;
                if (va) {
                    const float d0 = ca0 - tga[0], d1 = ca1 - tga[1], d2 = ca2 - tga[2];
                    acc += d0 * d0 + d1 * d1 + d2 * d2;
                }
                if (vb) {
                    const float d0 = cb0 - tgb[0], d1 = cb1 - tgb[1], d2 = cb2 - tgb[2];
                    acc += d0 * d0 + d1 * d1 + d2 * d2;
                }
                acc = warp_sum(acc);
                if (lane == 0) tile_loss[t] = acc;
            }
        }
        // ---- 6. reduction -----------------------------------------------------
        if (!kImage) {
            __syncthreads();
            // thread i sums tiles i, i + 1024, ...; then a fixed shuffle tree
            float acc = 0.0f;
            for (int t = tid; t < P.T; t += kThreads) {
                const bool has = overflow || ((t + 1 < P.T) ? toff[t + 1] : total) > toff[t];
                acc += has ? tile_loss[t] : P.tile_t2[t];
            }
            acc = warp_sum(acc);
            if (lane == 0) s_part[warp] = acc;
            __syncthreads();
            if (warp == 0) {
                float v = s_part[lane];
                v = warp_sum(v);
                if (lane == 0) *resolve(b, m).loss = v / (float)(P.W * P.H * 3);
            }
        }
        __syncthreads();
    }
}

__global__ void normals_kernel(const float* verts, const int32_t* tris, int nt, float* tnrm) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const float* A = verts + 3 * tris[3 * t];
    const float* B = verts + 3 * tris[3 * t + 1];
    const float* C = verts + 3 * tris[3 * t + 2];
    const double u0 = (double)B[0] - A[0], u1 = (double)B[1] - A[1], u2 = (double)B[2] - A[2];
    const double v0 = (double)C[0] - A[0], v1 = (double)C[1] - A[1], v2 = (double)C[2] - A[2];
    const double n0 = u1 * v2 - u2 * v1, n1 = u2 * v0 - u0 * v2, n2 = u0 * v1 - u1 * v0;
    const double len = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    const double inv = len > 0.0 ? 1.0 / len : 0.0;
    tnrm[3 * t] = (float)(n0 * inv);
    tnrm[3 * t + 1] = (float)(n1 * inv);
    tnrm[3 * t + 2] = (float)(n2 * inv);
}

__global__ void tile_t2_kernel(const float* target, int W, int H, int TX, int T, float* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int ty = t / TX, tx = t - ty * TX;
    float s = 0.0f;
    for (int yy = 0; yy < kTile; ++yy)
        for (int xx = 0; xx < kTile; ++xx) {
            const int x = tx * kTile + xx, y = ty * kTile + yy;
            if (x >= W || y >= H) continue;
            const size_t p = (size_t)y * W + x;
            for (int c = 0; c < 3; ++c) s += target[3 * p + c] * target[3 * p + c];
        }
    out[t] = s;
}

RvArgs make_args(const DevScene& sc) {
    RvArgs a;
    a.verts = sc.verts; a.tris = sc.tris; a.tnrm = sc.tnrm; a.target = sc.target; a.tile_t2 = sc.tile_t2;
    a.nv = sc.nv; a.nt = sc.nt; a.W = sc.W; a.H = sc.H;
    a.TX = (sc.W + kTile - 1) / kTile; a.TY = (sc.H + kTile - 1) / kTile; a.T = a.TX * a.TY;
    a.tx_recip = ((uint64_t(1) << 32) + (uint64_t)a.TX - 1) / (uint64_t)a.TX;
    a.alb0 = sc.albedo[0]; a.alb1 = sc.albedo[1]; a.alb2 = sc.albedo[2];
    a.l0 = sc.light[0]; a.l1 = sc.light[1]; a.l2 = sc.light[2];
    a.eye_dist = sc.eye_dist; a.scale = sc.scale;
    a.stats = sc.rv_stats;
    return a;
}

}  // namespace

size_t revolve_smem_bytes(int nv, int nt, int W, int H) {
    const int T = ((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile);
    const size_t vreg = 3 * (size_t)nv > (size_t)(T + 1) / 2 ? 3 * (size_t)nv : (size_t)(T + 1) / 2;
    return sizeof(TriRec) * (size_t)nt + sizeof(float) * vreg + 2 * sizeof(int) * (size_t)T +
           sizeof(uint16_t) * kEntryCap + sizeof(float) * (size_t)nt + sizeof(uint32_t) * (size_t)nt;
}

void revolve_prepare(DevScene& sc, cudaStream_t s) {
    normals_kernel<<<(sc.nt + 255) / 256, 256, 0, s>>>(sc.verts, sc.tris, sc.nt, sc.tnrm);
    sc.rv_smem = revolve_smem_bytes(sc.nv, sc.nt, sc.W, sc.H);
    cudaFuncSetAttribute(revolve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc.rv_smem);
    cudaFuncSetAttribute(revolve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc.rv_smem);
}

void revolve_tile_t2(DevScene& sc, cudaStream_t s) {
    const int TX = (sc.W + kTile - 1) / kTile, TY = (sc.H + kTile - 1) / kTile;
    tile_t2_kernel<<<(TX * TY + 127) / 128, 128, 0, s>>>(sc.target, sc.W, sc.H, TX, TX * TY, sc.tile_t2);
}

int revolve_tiles(int W, int H) { return ((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile); }

void launch_revolve_loss(const DevScene& sc, const RenderBatch& b, cudaStream_t s) {
    const int grid = b.M < num_sms() ? b.M : num_sms();
    revolve_kernel<false><<<grid, kThreads, sc.rv_smem, s>>>(make_args(sc), b, nullptr, nullptr);
}

void launch_revolve_image(const DevScene& sc, const float* params, float* img, cudaStream_t s) {
    RenderBatch b{};
    revolve_kernel<true><<<1, kThreads, sc.rv_smem, s>>>(make_args(sc), b, params, img);
}

}  // namespace hr
