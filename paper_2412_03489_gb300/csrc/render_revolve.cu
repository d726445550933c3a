// K3/K4: rasteriser of a triangle mesh (surface of revolution, stand-in for
// the Mug task of Sec. 4.1) fused with the per-pixel L2 loss and the block
// reduction, so that no image is written to HBM.
//
// One CTA (persistent over perturbations) renders a whole perturbation.  Two
// shared-memory layouts:
//   compact  records of surviving triangles only, by slot, in half an SM's
//            shared memory: two CTAs of 512 threads per SM, so that one's
//            barrier-bound set-up phases overlap the other's raster; a render
//            with more survivors than slots or more bin entries than fit is
//            handed over (its loss set to a marker NaN);
//   full     records by triangle, one CTA of 1024 threads per SM, bins that do
//            not fit rastered in bands; it renders the handed-over
//            perturbations (a second launch that reads the loss words), every
//            scene too large for the compact layout, and images.
// Both take the same coverage and depth decisions:
//   1. rotation R = Rx(p0) Ry(p1) from RN32 of FP64 cos / sin (for every
//      perturbation after a CTA's first, computed during the previous raster);
//   2. vertex transform and projection (FP32, fixed operation order);
//   3. triangle setup: edge functions with their top-left thresholds, back-face
//      cull, depth plane of 1/Z, pixel bounding box, flat Lambert shade; each
//      record stays at its triangle's index (full) or takes the next slot
//      (compact, where the record carries the triangle's index);
//   4. binning into 8x4 pixel tiles (8x8 where shared memory is short; count,
//      scan, fill; all in shared memory), skipping tiles that a conservative
//      edge test shows the triangle misses; each bin entry carries the
//      triangle index and the rows / columns of its tile that lie inside the
//      triangle's bounding box; bins that do not fit at once are filled and
//      rastered in bands of tile rows;
//   5. group-per-tile raster (8 lanes per 8x4 tile, 16 per 8x8 tile), tiles
//      fetched dynamically in groups ordered by entry count; each lane tests 4
//      pixels of a row against every entry of its tile's bin; nearest 1/Z
//      wins, ties to the lower triangle index (a strict compare, and a
//      second walk of the rare tile where equal depths met); (colour -
//      target)^2 per tile; tiles with an empty bin take the precomputed sum
//      of target^2;
//   6. per-tile losses summed in tile order, warp shuffle + block reduction to
//      one FP32 loss per perturbation.
// The FP32 sequences of steps 2-5 define the renderer (coverage and depth
// decisions), so they use explicitly rounded intrinsics.
#include <algorithm>
#include <climits>
#include <cmath>
#include <type_traits>

#include "hr_device.cuh"
#include "hr_internal.h"

namespace hr {
namespace {

constexpr int kThreads = 1024;      // full layout: one CTA per SM
constexpr int kCompactThreads = 512; // compact layout: two CTAs per SM
constexpr int kTW = 8;              // tile width; tiles are 8 x 4 or 8 x 8 pixels
constexpr int kEntryCapMax = 16384;  // bin entries per render (less where shared memory is short)
constexpr int kEntryCapMin = 2048;
constexpr int kStaticSmem = 1024;    // the kernel's static shared memory, rounded up
// compact layout: at least this many bin entries, and slots for at least
// half the triangles (a closed mesh shows about half of them)
constexpr int kCompactCapMin = 4096;
// loss written by a compact-layout render that did not fit (more survivors
// than slots, or more entries than the entry array holds): a NaN no
// arithmetic produces, which the full-layout launch that follows renders again
constexpr uint32_t kRedoLoss = 0x7FC0DEADu;
// compact layout: a launch's loss words start as kFreeLoss (marked by a kernel
// that runs first); a CTA claims a perturbation by turning its word into
// kTakenLoss with one compare-and-swap, then writes the loss over it
constexpr uint32_t kFreeLoss = 0x7FC0F4EEu;
constexpr uint32_t kTakenLoss = 0x7FC07A4Eu;

// One surviving triangle.  E > 0, or E == 0 on a top-left edge, is one
// compare: E > th with th = 0 or th = -(smallest subnormal) (no float lies
// strictly between the two).  The last word is the flat shade (full layout:
// records by triangle) or the triangle's index (compact layout: records by
// survivor slot, the index decides depth ties); the raster reads the shades
// from their own array.
struct __align__(16) TriRec {
    float A0, B0, C0, th0;
    float A1, B1, C1, th1;
    float A2, B2, C2, th2;
    float Aw, Bw, Cw, shade;
};

// bin entry: triangle << 16 | (tile rows OUTSIDE the bounding box) << 8 |
// (tile columns outside it): a pixel of the tile lies in the box iff neither
// its row bit nor its column bit is set, one AND per pixel
__device__ __forceinline__ uint32_t entry_word(int tri, uint32_t rows, uint32_t cols) {
    return ((uint32_t)tri << 16) | ((~rows & 0xFFu) << 8) | (~cols & 0xFFu);
}
// an entry no pixel is in (record 0, every row and column outside)
constexpr uint32_t kSentinel = 0x0000FFFFu;
// bits lo..hi (clamped to 0..7) of a byte
__device__ __forceinline__ uint32_t span_bits(int lo, int hi) {
    lo = max(lo, 0);
    hi = min(hi, 7);
    return lo > hi ? 0u : ((0xFFu >> (7 - hi)) & (0xFFu << lo));
}
__device__ __forceinline__ float tl_threshold(float A, float B) {
    return (A > 0.0f || (A == 0.0f && B > 0.0f)) ? -0x1p-149f : 0.0f;
}

struct RvArgs {
    const float* verts;
    const int32_t* tris;
    const float* tnrm;
    const float* target;
    const float* tile_t2;
    int nv, nt, W, H, TX, TY, T;
    int cap;             // bin entry capacity
    int vreg;            // floats in the vertex region
    int th;              // tile height (the kernel's template argument)
    int slots;           // compact layout: survivor slots (records by slot)
    int redo;            // full layout: render only the perturbations whose loss is kRedoLoss
    uint64_t tx_recip;   // ceil(2^32 / TX): t / TX = (t tx_recip) >> 32 exactly for t, TX < 2^16
    unsigned long long* stats;   // diagnostics [8], see hr_scene_stats
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
template <int kTH>
__device__ __forceinline__ bool tile_hits(const float A[3], const float B[3], const float C[3], uint2 bb,
                                          const float neg[3], int tx, int ty) {
    const int x0 = max(tx * kTW, (int)(bb.x & 0xffffu)), x1 = min(tx * kTW + kTW - 1, (int)(bb.x >> 16));
    const int y0 = max(ty * kTH, (int)(bb.y & 0xffffu)), y1 = min(ty * kTH + kTH - 1, (int)(bb.y >> 16));
    const float fx0 = (float)x0 + 0.5f, fx1 = (float)x1 + 0.5f, fy0 = (float)y0 + 0.5f, fy1 = (float)y1 + 0.5f;
    bool hit = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float x = A[i] > 0.0f ? fx1 : fx0, y = B[i] > 0.0f ? fy1 : fy0;
        hit = hit && !(fmaf(A[i], x, fmaf(B[i], y, C[i])) < neg[i]);
    }
    return hit;
}

constexpr int kCountClasses = 32;   // tiles ordered by entry count, counts >= 31 share a class

// Exclusive scan of cnt[0..T) into off[0..T) and, in the same barriers, the
// list of tiles with entries (olist[0..n_obj)) ordered by entry count,
// largest first (a counting sort over count classes; the order within a
// class is arbitrary, which only affects which warp takes which tile).  The
// raster fetches the tiles of a warp together, one per lane group, so groups
// of nearly equal counts waste few iterations, and the long tiles go first.  hist
// [kCountClasses] must be zero on entry.  Returns the total entry count (all
// threads) and sets n_obj.
template <int kT, class OffT>
__device__ int bin_scan(const int* cnt, OffT* off, uint16_t* olist, int T, int* warp_tot, int* hist, int* n_obj) {
    const int per = (T + kT - 1) / kT;
    const int b = threadIdx.x * per;
    int local = 0;
    for (int i = 0; i < per; ++i)
        if (b + i < T) {
            const int c = cnt[b + i];
            local += c;
            if (c > 0) atomicAdd(&hist[kCountClasses - 1 - min(c, kCountClasses - 1)], 1);
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp < 2) {   // warp 0: offsets of the warps' tile ranges; warp 1: the count classes
        int* arr = warp == 0 ? warp_tot : hist;
        const int wv = (warp == 0 && lane >= kT / 32) ? 0 : arr[lane];
        int wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        arr[lane] = wi - wv;
        if (lane == 31) arr[32] = wi;
    }
    __syncthreads();
    int run = warp_tot[warp] + incl - local;
    for (int i = 0; i < per; ++i)
        if (b + i < T) {
            const int c = cnt[b + i];
            off[b + i] = (OffT)run;
            if (c > 0) olist[atomicAdd(&hist[kCountClasses - 1 - min(c, kCountClasses - 1)], 1)] = (uint16_t)(b + i);
            run += c;
        }
    __syncthreads();
    *n_obj = hist[32];
    return warp_tot[32];
}

// The four pixels of a lane against one bin entry, as PTX predicate chains.
// Pixel c (x coordinate fx_c) is in when its row and column bits of the
// entry's outside mask are clear (row bit row_out, column bit c) and
// E_i = fma(A_i, fx_c, r_i) > th_i for the three edges; it takes the entry
// when also wz = fma(Aw, fx_c, rw) > bw_c (strict).  t4 becomes non-zero when
// some wz == bw_c (an exact depth tie, resolved by a second, exact walk of
// the tile).
__device__ __forceinline__ void pixels4(const float4& q0, const float4& q1, const float4& q2, float Aw, float r0,
                                        float r1, float r2, float rw, const float fx[4], uint32_t outside,
                                        uint32_t row_out, int s, float bw[4], int bs[4], uint32_t& t4) {
    asm("{\n\t"
        ".reg .pred p, q;\n\t"
        ".reg .b32 m;\n\t"
        ".reg .f32 e0, e1, e2, w;\n\t"
        "setp.ne.u32 q, 0, 0;\n\t"
#define HR_PIXEL(C, FX, BW, BS)                                 \
        "lop3.b32 m, %18, %19, " #C ", 0xE0;\n\t"              \
        "setp.eq.u32 p, m, 0;\n\t"                             \
        "fma.rn.f32 e0, %9, " FX ", %13;\n\t"                  \
        "fma.rn.f32 e1, %10, " FX ", %14;\n\t"                 \
        "fma.rn.f32 e2, %11, " FX ", %15;\n\t"                 \
        "fma.rn.f32 w, %12, " FX ", %16;\n\t"                  \
        "setp.gt.and.f32 p, e0, %21, p;\n\t"                   \
        "setp.gt.and.f32 p, e1, %22, p;\n\t"                   \
        "setp.gt.and.f32 p, e2, %23, p;\n\t"                   \
        "setp.eq.or.f32 q, w, " BW ", q;\n\t"                  \
        "setp.gt.and.f32 p, w, " BW ", p;\n\t"                 \
        "selp.f32 " BW ", w, " BW ", p;\n\t"                   \
        "selp.b32 " BS ", %20, " BS ", p;\n\t"
        HR_PIXEL(1, "%17", "%0", "%4")
        HR_PIXEL(2, "%24", "%1", "%5")
        HR_PIXEL(4, "%25", "%2", "%6")
        HR_PIXEL(8, "%26", "%3", "%7")
#undef HR_PIXEL
        "@q or.b32 %8, %8, 1;\n\t"
        "}"
        : "+f"(bw[0]), "+f"(bw[1]), "+f"(bw[2]), "+f"(bw[3]), "+r"(bs[0]), "+r"(bs[1]), "+r"(bs[2]), "+r"(bs[3]),
          "+r"(t4)
        : "f"(q0.x), "f"(q1.x), "f"(q2.x), "f"(Aw), "f"(r0), "f"(r1), "f"(r2), "f"(rw), "f"(fx[0]), "r"(outside),
          "r"(row_out), "r"(s), "f"(q0.w), "f"(q1.w), "f"(q2.w), "f"(fx[1]), "f"(fx[2]), "f"(fx[3]));
}

// rotation angle d of perturbation m: RN32(theta32 + tau)
__device__ __forceinline__ float rotation_param(const RenderBatch& b, int m, int d) {
    const Pert pt = resolve(b, m);
    return __fadd_rn(pt.theta[d], pt.tau[d]);
}

// one triangle's setup (vertex indices ia, ib, ic; model-space unit normal
// n); false if it is clipped, culled or outside the image
__device__ __forceinline__ bool setup_triangle(const RvArgs& P, int ia, int ib, int ic, const float n[3],
                                               const float* vx, const float* vy, const float* viz, const float sL[3],
                                               TriRec& r, uint2& bb) {
    const float iza = viz[ia], izb = viz[ib], izc = viz[ic];
    if (!(iza > 0.0f && izb > 0.0f && izc > 0.0f)) return false;
    const float ax = vx[ia], ay = vy[ia], bx = vx[ib], by = vy[ib], cx = vx[ic], cy = vy[ic];
    const Edge e0 = edge_of(bx, by, cx, cy);
    const Edge e1 = edge_of(cx, cy, ax, ay);
    const Edge e2 = edge_of(ax, ay, bx, by);
    const float D2 = edge_eval(e2.A, e2.B, e2.C, cx, cy);
    if (!(D2 > 0.0f)) return false;
    int xlo, xhi, ylo, yhi;
    const float mnx = fminf(fminf(ax, bx), cx), mxx = fmaxf(fmaxf(ax, bx), cx);
    const float mny = fminf(fminf(ay, by), cy), mxy = fmaxf(fmaxf(ay, by), cy);
    if (!pixel_range(mnx, mxx, P.W, xlo, xhi) || !pixel_range(mny, mxy, P.H, ylo, yhi)) return false;
    const float invD = __fdiv_rn(1.0f, D2);
    r.A0 = e0.A; r.B0 = e0.B; r.C0 = e0.C; r.th0 = tl_threshold(e0.A, e0.B);
    r.A1 = e1.A; r.B1 = e1.B; r.C1 = e1.C; r.th1 = tl_threshold(e1.A, e1.B);
    r.A2 = e2.A; r.B2 = e2.B; r.C2 = e2.C; r.th2 = tl_threshold(e2.A, e2.B);
    r.Aw = __fmul_rn(__fmaf_rn(e2.A, izc, __fmaf_rn(e1.A, izb, __fmul_rn(e0.A, iza))), invD);
    r.Bw = __fmul_rn(__fmaf_rn(e2.B, izc, __fmaf_rn(e1.B, izb, __fmul_rn(e0.B, iza))), invD);
    r.Cw = __fmul_rn(__fmaf_rn(e2.C, izc, __fmaf_rn(e1.C, izb, __fmul_rn(e0.C, iza))), invD);
    const float sh = n[0] * sL[0] + n[1] * sL[1] + n[2] * sL[2];
    r.shade = fmaxf(sh, 0.0f);
    bb.x = (uint32_t)xlo | ((uint32_t)xhi << 16);
    bb.y = (uint32_t)ylo | ((uint32_t)yhi << 16);
    return true;
}

// kCompact: records by survivor slot in about half the shared memory, so
// that two CTAs of 512 threads share an SM and one's barrier-bound set-up
// phases overlap the other's raster; a render that does not fit (more
// survivors than slots, more bin entries than the entry array) writes
// kRedoLoss instead of its loss.  Otherwise (full layout) records by
// triangle, one 1024-thread CTA per SM, bins too large for the shared memory
// rastered in bands; with P.redo only the kRedoLoss perturbations are rendered.
template <int kTH, bool kImage, bool kCompact>
__global__ void __launch_bounds__(kCompact ? kCompactThreads : kThreads, kCompact ? 2 : 1)
revolve_kernel(RvArgs P, RenderBatch b, const float* __restrict__ img_params, float* __restrict__ img,
               int32_t* __restrict__ ids) {
    constexpr int kT = kCompact ? kCompactThreads : kThreads;   // threads per CTA
    constexpr int kW = kT / 32;
    constexpr int kG = 2 * kTH;          // lanes per tile: kTH rows x 2 four-pixel strips
    constexpr int kPer = 32 / kG;        // tiles per warp
    using OffT = typename std::conditional<kCompact, uint16_t, int>::type;   // bin offsets (< kEntryCapMax)
    extern __shared__ __align__(16) unsigned char smem[];
    const int nrec = kCompact ? P.slots : P.nt;
    TriRec* rec = reinterpret_cast<TriRec*>(smem);      // [nrec] by triangle (full) or by slot (compact)
    uint2* bbx = reinterpret_cast<uint2*>(rec + nrec);  // [nrec] pixel bounding boxes
    float* vx;            // projected vertices x, y, 1/Z [nv] each
    float* tshade;        // [nrec] flat shades
    int* tcnt;            // [T] bin counts, then fill cursors, then tile losses
    OffT* toff;           // [T] bin offsets
    uint16_t* surv = nullptr;              // full: [nt] surviving triangles (any order)
    uint32_t* ent;                         // [cap] bin entries
    unsigned long long* tmask = nullptr;   // full: [nt] tile masks of the count pass, by survivor
    uint16_t* tm16 = nullptr;              // compact: [slots] tile masks of rectangles of <= 16 tiles
    uint16_t* olist;                       // [T] tiles with entries, ordered by entry count
    if constexpr (kCompact) {
        tshade = reinterpret_cast<float*>(bbx + nrec);
        tcnt = reinterpret_cast<int*>(tshade + nrec);
        toff = reinterpret_cast<OffT*>(tcnt + P.T);
        olist = reinterpret_cast<uint16_t*>(toff + P.T);
        tm16 = olist + P.T;
        ent = reinterpret_cast<uint32_t*>(tm16 + ((nrec + 1) & ~1));
        vx = reinterpret_cast<float*>(ent);   // the vertices are dead before the first entry is written
    } else {
        vx = reinterpret_cast<float*>(bbx + nrec);   // vertex region, P.vreg floats (8 B aligned)
        tshade = vx + P.vreg;
        tcnt = reinterpret_cast<int*>(tshade + nrec);
        toff = reinterpret_cast<OffT*>(tcnt + P.T);
        surv = reinterpret_cast<uint16_t*>(toff + P.T);
        ent = reinterpret_cast<uint32_t*>(surv + ((P.nt + 1) & ~1));
        // after the triangle setup the vertex region holds the count pass's
        // tile masks and the list of tiles with entries
        tmask = reinterpret_cast<unsigned long long*>(vx);
        olist = reinterpret_cast<uint16_t*>(tmask + P.nt);
    }
    float* vy = vx + P.nv;
    float* viz = vy + P.nv;

    __shared__ float s_cs[4], s_cs_next[4];
    __shared__ float sR[9];
    __shared__ float sL[3];
    __shared__ int s_count;
    __shared__ int s_wtot[33];
    __shared__ int s_hist[33];
    __shared__ float s_part[kW];
    __shared__ int s_tile;
    __shared__ int s_band[2];   // the current band's end row and whether it walks every triangle

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int M = kImage ? 1 : b.M;
    unsigned long long steps = 0ull;   // lane 0: this warp's raster steps (diagnostics)
    // Redo mode: the first of this CTA's perturbations m0, m0 + G, ... (G the
    // grid) whose loss is kRedoLoss, M if none; warp 0 reads 32 loss words at
    // a time.  Every thread calls it (one barrier); s_next is rewritten only
    // by the next call, after the render's barriers.
    __shared__ int s_next;
    auto next_redo = [&](int m0) -> int {
        if (warp == 0) {
            const int G = (int)gridDim.x;
            int found = M;
            for (int base = m0; base < M && found == M; base += 32 * G) {
                const int mm = base + lane * G;
                const bool want = mm < M && __float_as_uint(*resolve(b, mm).loss) == kRedoLoss;
                const unsigned bal = __ballot_sync(0xffffffffu, want);
                if (bal) found = base + (__ffs(bal) - 1) * G;
            }
            if (lane == 0) s_next = found;
        }
        __syncthreads();
        return s_next;
    };
    const bool redo = !kImage && !kCompact && P.redo;
    // Compact layout: CTA c walks its perturbations c, c + G, ... and renders
    // those it claims (one compare-and-swap on the loss word; the next one is
    // claimed during the raster, with its rotation); after its own it steals
    // free ones among the last 2G, so that CTAs that drew cheaper renders
    // take over the last renders of the others.  Each perturbation is
    // claimed, and rendered, exactly once.
    __shared__ int s_pref;   // the perturbation claimed ahead (its rotation in s_cs_next), M if none
    auto claim = [&](int i) -> bool {
        unsigned int* w = reinterpret_cast<unsigned int*>(resolve(b, i).loss);
        return atomicCAS(w, kFreeLoss, kTakenLoss) == kFreeLoss;
    };
    auto claim_from = [&](int i) -> int {   // one thread: the first of i, i + G, ... it claims, M if none
        for (; i < M; i += (int)gridDim.x)
            if (claim(i)) return i;
        return M;
    };
    auto steal = [&]() -> int {   // every thread (one barrier); warp 0 scans 32 loss words at a time
        if (warp == 0) {
            const int lo = max(0, M - 2 * (int)gridDim.x);
            int got = M;
            for (int top = M - 1; top >= lo && got == M; top -= 32) {
                const int i = top - lane;
                const bool is_free =
                    i >= lo && __ldcv(reinterpret_cast<const unsigned int*>(resolve(b, i).loss)) == kFreeLoss;
                unsigned bal = __ballot_sync(0xffffffffu, is_free);
                while (bal && got == M) {
                    const int src = __ffs(bal) - 1;
                    int ok = 0;
                    if (lane == src) ok = claim(i) ? 1 : 0;
                    if (__shfl_sync(0xffffffffu, ok, src)) got = top - src;
                    bal &= bal - 1;
                }
            }
            if (lane == 0) s_next = got;
        }
        __syncthreads();
        return s_next;
    };
    bool have_cs = false;   // compact: s_cs_next holds this perturbation's rotation
    auto first_m = [&]() -> int {
        if constexpr (kImage) {
            return 0;
        } else if constexpr (kCompact) {
            if (tid == 0) s_next = claim_from((int)blockIdx.x);
            __syncthreads();
            const int f = s_next;
            __syncthreads();
            return f < M ? f : steal();
        } else {
            return redo ? next_redo((int)blockIdx.x) : (int)blockIdx.x;
        }
    };
    auto next_m = [&](int m) -> int {
        if constexpr (kImage) {
            return m + 1;
        } else if constexpr (kCompact) {
            const int p = s_pref;
            have_cs = p < M;
            return p < M ? p : steal();
        } else {
            return redo ? next_redo(m + (int)gridDim.x) : m + (int)gridDim.x;
        }
    };
    for (int m = first_m(); m < M; m = next_m(m)) {
        // ---- 1. parameters and rotation ----------------------------------
        if (tid < 4) {   // ca, sa, cb, sb
            if (kCompact ? !have_cs : (kImage || m == (int)blockIdx.x || P.redo)) {
                const float p = kImage ? img_params[tid >> 1] : rotation_param(b, m, tid >> 1);
                const double a = (double)p;
                s_cs[tid] = (float)((tid & 1) ? sin(a) : cos(a));
            } else {
                s_cs[tid] = s_cs_next[tid];   // computed during the previous raster phase
            }
        }
        // scene constants this thread uses in the render (two vertices, two
        // triangles, the target's sum of squares on two tiles), loaded now so
        // that their latency overlaps the rotation
        float pv[2][3], pn[2][3], pt2[2];
        int pt[2][3];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int v = tid + k * kT, t = tid + k * kT;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                pv[k][c] = v < P.nv ? P.verts[3 * v + c] : 0.0f;
                pt[k][c] = t < P.nt ? P.tris[3 * t + c] : 0;
                pn[k][c] = t < P.nt ? P.tnrm[3 * t + c] : 0.0f;
            }
            pt2[k] = (!kImage && tid + k * kT < P.T) ? P.tile_t2[tid + k * kT] : 0.0f;
        }
        for (int i = tid; i < P.T; i += kT) tcnt[i] = 0;
        if (tid < 33) s_hist[tid] = 0;
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
        auto project = [&](int v, float x, float y, float z) {
            const float X = __fmaf_rn(sR[2], z, __fmaf_rn(sR[1], y, __fmul_rn(sR[0], x)));
            const float Y = __fmaf_rn(sR[5], z, __fmaf_rn(sR[4], y, __fmul_rn(sR[3], x)));
            const float w2 = __fmaf_rn(sR[8], z, __fmaf_rn(sR[7], y, __fmul_rn(sR[6], x)));
            const float Z = __fsub_rn(P.eye_dist, w2);
            const float qx = __fdiv_rn(X, Z), qy = __fdiv_rn(Y, Z);
            vx[v] = __fmaf_rn(P.scale, qx, halfW);
            vy[v] = __fmaf_rn(-P.scale, qy, halfH);
            viz[v] = (Z > 0.0f) ? __fdiv_rn(1.0f, Z) : -1.0f;
        };
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (tid + k * kT < P.nv) project(tid + k * kT, pv[k][0], pv[k][1], pv[k][2]);
        for (int v = tid + 2 * kT; v < P.nv; v += kT)
            project(v, P.verts[3 * v], P.verts[3 * v + 1], P.verts[3 * v + 2]);
        __syncthreads();
        // ---- 3. triangle setup ------------------------------------------------
        // records stay at their triangle's index (bin entries carry it for the
        // tie rule); the survivors are listed for the binning, and a clipped,
        // culled or off-image triangle gets an empty bounding box (lo > hi),
        // which the all-triangles fallback of the raster skips
        // (compact layout: a survivor takes the next slot; past the last slot
        // it is only counted, and the render is handed to the full layout)
        auto setup = [&](int t, const int id[3], const float n[3]) {
            TriRec r;
            uint2 bb;
            if constexpr (kCompact) {
                if (setup_triangle(P, id[0], id[1], id[2], n, vx, vy, viz, sL, r, bb)) {
                    const int k = atomicAdd(&s_count, 1);
                    if (k < nrec) {
                        tshade[k] = r.shade;
                        r.shade = __int_as_float(t);
                        rec[k] = r;
                        bbx[k] = bb;
                    }
                }
            } else {
                if (setup_triangle(P, id[0], id[1], id[2], n, vx, vy, viz, sL, r, bb)) {
                    rec[t] = r;
                    tshade[t] = r.shade;
                    surv[atomicAdd(&s_count, 1)] = (uint16_t)t;
                } else {
                    bb = make_uint2(1u, 1u);
                }
                bbx[t] = bb;
            }
        };
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (tid + k * kT < P.nt) setup(tid + k * kT, pt[k], pn[k]);
        for (int t = tid + 2 * kT; t < P.nt; t += kT) {
            const int id[3] = {P.tris[3 * t], P.tris[3 * t + 1], P.tris[3 * t + 2]};
            const float n[3] = {P.tnrm[3 * t], P.tnrm[3 * t + 1], P.tnrm[3 * t + 2]};
            setup(t, id, n);
        }
        __syncthreads();
        const int count = s_count;
        // (one warp, before the raster) the CTA's next perturbation and the
        // FP64 cos / sin of its rotation, off the critical path: full layout
        // m + G; compact, the next of its own that it claims (s_pref)
        auto prefetch_next = [&]() {
            int mn;
            if constexpr (kCompact) {
                mn = M;
                if (lane == 0) mn = claim_from(m + (int)gridDim.x);
                mn = __shfl_sync(0xffffffffu, mn, 0);
                if (lane == 0) s_pref = mn;
            } else {
                mn = m + (int)gridDim.x;
            }
            if (lane < 4 && mn < M) {
                const double a = (double)rotation_param(b, mn, lane >> 1);
                s_cs_next[lane] = (float)((lane & 1) ? sin(a) : cos(a));
            }
        };
        // A compact-layout render that does not fit writes kRedoLoss (the full
        // layout renders it again) and claims the CTA's next perturbation,
        // which its skipped raster phase would have done.
        auto hand_over = [&]() {
            if (tid == 0) {
                *resolve(b, m).loss = __uint_as_float(kRedoLoss);
                if (P.stats) atomicAdd(&P.stats[7], 1ull);
            }
            if (warp == kW - 1) prefetch_next();
            __syncthreads();
        };
        if constexpr (kCompact) {
            if (count > nrec) {
                hand_over();
                continue;
            }
        }
        // ---- 4. binning -----------------------------------------------------
        // count pass: each survivor's tiles that pass the conservative edge
        // test go into a bit mask (row-major over its tile rectangle;
        // rectangles of more than 64 tiles, 16 in the compact layout, skip the
        // test), reused by the fill
        for (int k = tid; k < count; k += kT) {
            const int s = kCompact ? k : (int)surv[k];
            const uint2 bb = bbx[s];
            const float4* rp = reinterpret_cast<const float4*>(&rec[s]);
            const float4 q0 = rp[0], q1 = rp[1], q2 = rp[2];
            const float A[3] = {q0.x, q1.x, q2.x}, B[3] = {q0.y, q1.y, q2.y}, C[3] = {q0.z, q1.z, q2.z};
            const int tx0 = (int)(bb.x & 0xffffu) / kTW, tx1 = (int)(bb.x >> 16) / kTW;
            const int ty0 = (int)(bb.y & 0xffffu) / kTH, ty1 = (int)(bb.y >> 16) / kTH;
            const bool test = (tx1 - tx0 + 1) * (ty1 - ty0 + 1) <= (kCompact ? 16 : 64);
            const float fW = (float)P.W, fH = (float)P.H;
            float neg[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) neg[i] = -1e-5f * fmaf(fabsf(A[i]), fW, fmaf(fabsf(B[i]), fH, fabsf(C[i])));
            unsigned long long mask = 0ull;
            int bit = 0;
            const int xlo = (int)(bb.x & 0xffffu), xhi = (int)(bb.x >> 16);
            const int ylo = (int)(bb.y & 0xffffu), yhi = (int)(bb.y >> 16);
            for (int ty = ty0; ty <= ty1; ++ty) {
                // per edge, the row term at the (tile row ∩ box) edge where
                // B y is largest: the tile test is fma(A, x*, rowterm)
                const float fy0 = (float)max(ty * kTH, ylo) + 0.5f, fy1 = (float)min(ty * kTH + kTH - 1, yhi) + 0.5f;
                float rt[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) rt[i] = fmaf(B[i], B[i] > 0.0f ? fy1 : fy0, C[i]);
                for (int tx = tx0; tx <= tx1; ++tx, ++bit) {
                    bool hit = true;
                    if (test) {
                        const float fx0 = (float)max(tx * kTW, xlo) + 0.5f, fx1 = (float)min(tx * kTW + kTW - 1, xhi) + 0.5f;
#pragma unroll
                        for (int i = 0; i < 3; ++i) hit = hit && !(fmaf(A[i], A[i] > 0.0f ? fx1 : fx0, rt[i]) < neg[i]);
                    }
                    if (hit) {
                        atomicAdd(&tcnt[ty * P.TX + tx], 1);
                        if (test) mask |= 1ull << bit;
                    }
                }
            }
            if constexpr (kCompact) tm16[k] = (uint16_t)mask;
            else tmask[k] = test ? mask : ~0ull;
        }
        __syncthreads();
        int n_obj = 0;
        const int total = bin_scan<kT>(tcnt, toff, olist, P.T, s_wtot, s_hist, &n_obj);
        if constexpr (kCompact) {
            if (total > P.cap) {
                hand_over();
                continue;
            }
        }
        // Bins that do not fit the shared memory at once are filled and
        // rastered in bands of whole tile rows, each with at most capb entries;
        // meanwhile the count pass's per-row totals sit at the end of the
        // entry array.  A tile row whose entries alone exceed capb is a band of
        // its own whose tiles walk every triangle.  A band only decides which
        // tiles are rastered together: every pixel's decisions are the same.
        const bool banded = !kCompact && total > P.cap;
        const int capb = banded ? P.cap - P.TY : P.cap;
        int* rowtot = reinterpret_cast<int*>(ent) + capb;
        if (banded) {
            for (int r = warp; r < P.TY; r += kW) {
                int sum = 0;
                for (int tx = lane; tx < P.TX; tx += 32) sum += tcnt[r * P.TX + tx];
                sum = __reduce_add_sync(0xffffffffu, sum);
                if (lane == 0) rowtot[r] = sum;
            }
        }
        if (!kImage && tid == 0 && P.stats) {   // diagnostics: see hr_scene_stats
            if (banded) atomicAdd(&P.stats[0], 1ull);
            atomicAdd(&P.stats[1], 1ull);
            atomicAdd(&P.stats[2], (unsigned long long)count);
            atomicAdd(&P.stats[3], (unsigned long long)total);
            atomicAdd(&P.stats[4], (unsigned long long)n_obj);
        }
        // one band: fill and raster of tile rows [r0, r1), the whole image when
        // the bins fit (then every argument but the row count is a constant)
        auto band = [&](const int r0, const int r1, const int total_b, const bool walk_all) {
            const int tb = r0 * P.TX, Tb = (r1 - r0) * P.TX;   // the band's tiles [tb, tb + Tb)
            for (int i = tid; i < Tb; i += kT) tcnt[tb + i] = 0;   // becomes the fill cursor
            if (tid == 0) s_tile = 0;
            __syncthreads();
            if (!walk_all) {
                // tiles without entries keep the sum of target^2 as their loss
                // (the raster writes the others)
                float* tl = reinterpret_cast<float*>(tcnt);
                auto empty = [&](int i) { return ((i + 1 < Tb) ? toff[tb + i + 1] : total_b) == toff[tb + i]; };
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int i = tid + k * kT;
                    if (i < Tb && empty(i)) tl[tb + i] = tb == 0 ? pt2[k] : P.tile_t2[tb + i];
                }
                for (int i = tid + 2 * kT; i < Tb; i += kT)
                    if (empty(i)) tl[tb + i] = P.tile_t2[tb + i];
                for (int k = tid; k < count; k += kT) {
                    const int s = kCompact ? k : (int)surv[k];
                    const uint2 bb = bbx[s];
                    const int xlo = (int)(bb.x & 0xffffu), xhi = (int)(bb.x >> 16);
                    const int ylo = (int)(bb.y & 0xffffu), yhi = (int)(bb.y >> 16);
                    const int tx0 = xlo / kTW, tx1 = xhi / kTW, ty0 = ylo / kTH, ty1 = yhi / kTH;
                    const int ya = max(ty0, r0), yb = min(ty1, r1 - 1);
                    if (ya > yb) continue;
                    unsigned long long mask;   // ~0: every tile of the rectangle (not tested)
                    if constexpr (kCompact) mask = (tx1 - tx0 + 1) * (ty1 - ty0 + 1) <= 16 ? tm16[k] : ~0ull;
                    else mask = tmask[k];
                    int bit = (ya - ty0) * (tx1 - tx0 + 1);   // row-major over the whole tile rectangle
                    for (int ty = ya; ty <= yb; ++ty) {
                        // rows of this tile inside the box (bits >= kTH are never tested)
                        const uint32_t rows = span_bits(ylo - ty * kTH, yhi - ty * kTH);
                        for (int tx = tx0; tx <= tx1; ++tx, ++bit) {
                            if (mask != ~0ull && !((mask >> bit) & 1ull)) continue;
                            const int tile = ty * P.TX + tx;
                            const int pos = atomicAdd(&tcnt[tile], 1);
                            ent[toff[tile] + pos] = entry_word(s, rows, span_bits(xlo - tx * kTW, xhi - tx * kTW));
                        }
                    }
                }
            }
            __syncthreads();
            // ---- 5. raster + loss ------------------------------------------------
            // Warps fetch tiles dynamically, kPer at a time, from the
            // count-ordered list, one tile per group of kG lanes; each tile's loss
            // goes to its own slot (the fill cursor array is free again) and the
            // slots are summed in tile order below, so the loss does not depend on
            // which warp took which tile.  Lane (row ry, half-row hx) of a group
            // owns the 4 pixels (x0 .. x0 + 3, y) of its tile and walks the tile's
            // whole bin: the row term fma(B, y + 1/2, C) of each edge and of the
            // depth plane is formed once per entry and shared by the 4 pixels.
            const int grp = lane / kG, gl = lane % kG;
            const int ry = gl >> 1, hx = gl & 1;
            // the next perturbation and its rotation: one warp, before it joins
            // the tile loop
            if (!kImage && !P.redo && r0 == 0 && warp == kW - 1) prefetch_next();
            // tiles without entries are not visited: their loss, the sum of
            // target^2, is taken in the reduction (an image visits every tile)
            float* tile_loss = reinterpret_cast<float*>(tcnt);
            const bool all_tiles = kImage || walk_all;
            const int n_iter = all_tiles ? Tb : n_obj;
            const int col_shift = 4 * hx;
            const uint32_t row_out = 1u << (8 + ry - col_shift);   // this lane's row bit after the shift
            const bool vec_target = (P.W & 3) == 0;
            // each warp reserves its next tiles when it starts the current ones,
            // so the shared atomic's latency overlaps the tiles' work
            int t_next = 0;
            if (lane == 0) t_next = atomicAdd(&s_tile, kPer);
            for (int it = __shfl_sync(0xffffffffu, t_next, 0); it < n_iter; it = __shfl_sync(0xffffffffu, t_next, 0)) {
                if (lane == 0) t_next = atomicAdd(&s_tile, kPer);
                const int my = it + grp;
                const bool has_tile = my < n_iter;
                const int t = !has_tile ? 0 : tb + (all_tiles ? my : (int)olist[my]);
                const int beg = has_tile && !walk_all ? toff[t] : 0;
                const int n_mine = has_tile && !walk_all ? ((t + 1 < tb + Tb) ? toff[t + 1] : total_b) - beg : 0;
                // division by multiplication with the rounded-up reciprocal
                // (Granlund and Montgomery, PLDI 1994): exact for t, TX < 2^16
                const int ty = (int)(((uint64_t)(uint32_t)t * P.tx_recip) >> 32), tx = t - ty * P.TX;
                const int x0 = tx * kTW + 4 * hx, y = ty * kTH + ry;
                const float fy = __fadd_rn((float)y, 0.5f);
                const float fx0 = __fadd_rn((float)x0, 0.5f);
                float fx[4], bw[4];
                int bs[4];
    #pragma unroll
                for (int c = 0; c < 4; ++c) {
                    fx[c] = __fadd_rn(fx0, (float)c);   // exact: small integers + 1/2
                    bw[c] = -INFINITY;
                    bs[c] = INT_MAX;
                }
                // One bin entry against this lane's 4 pixels.  Bins are in fill
                // (arbitrary) order, so the strict depth compare alone would give
                // an exact depth tie to whichever triangle came first; every time
                // a depth equals the pixel's current best (covered or not: one
                // compare instead of two, at the price of re-walking about 4 % of
                // the tile groups, where adjacent triangles' depth planes agree to
                // the last bit) the lane notes it, and a tile group where any lane
                // did is walked again with the full rule (larger 1/Z, lower index
                // on equal 1/Z).
                uint32_t tie_u = 0u;
                // (outside: the entry's complement masks shifted so that bit c is
                // this lane's column c and bit 8 + ry - 4 hx its row)
                auto raster_entry = [&](int s, uint32_t outside, bool exact) {
                    const float4* rp = reinterpret_cast<const float4*>(&rec[s]);
                    const float4 q0 = rp[0], q1 = rp[1], q2 = rp[2], q3 = rp[3];
                    const float r0 = __fmaf_rn(q0.y, fy, q0.z);
                    const float r1 = __fmaf_rn(q1.y, fy, q1.z);
                    const float r2 = __fmaf_rn(q2.y, fy, q2.z);
                    const float rw = __fmaf_rn(q3.y, fy, q3.z);
                    if (exact) {
    #pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float E0 = __fmaf_rn(q0.x, fx[c], r0);
                            const float E1 = __fmaf_rn(q1.x, fx[c], r1);
                            const float E2 = __fmaf_rn(q2.x, fx[c], r2);
                            const float wz = __fmaf_rn(q3.x, fx[c], rw);
                            const bool in = ((outside & (row_out | (1u << c))) == 0u) && (E0 > q0.w) &&
                                            (E1 > q1.w) && (E2 > q2.w);
                            // equal depths: the lower triangle index (records by
                            // slot carry it in their last word)
                            bool lower;
                            if constexpr (kCompact)
                                lower = bs[c] == INT_MAX || __float_as_int(rec[s].shade) < __float_as_int(rec[bs[c]].shade);
                            else
                                lower = s < bs[c];
                            const bool better = in && (wz > bw[c] || (wz == bw[c] && lower));
                            bw[c] = better ? wz : bw[c];
                            bs[c] = better ? s : bs[c];
                        }
                    } else {
                        uint32_t t4 = 0u;
                        pixels4(q0, q1, q2, q3.x, r0, r1, r2, rw, fx, outside, row_out, s, bw, bs, t4);
                        tie_u |= t4;
                    }
                };
                if (!walk_all) {
                    const int n_max = (int)__reduce_max_sync(0xffffffffu, (unsigned)n_mine);
                    if (!kImage && lane == 0) steps += (unsigned long long)n_max;
                    // a group whose bin is shorter walks a sentinel entry (every
                    // row and column outside: no pixel is in) instead of
                    // branching around the step
                    // (the next entry is loaded one step ahead)
                    uint32_t e = 0 < n_mine ? ent[beg] : kSentinel;
                    for (int k = 0; k < n_max; ++k) {
                        const uint32_t en = k + 1 < n_mine ? ent[beg + k + 1] : kSentinel;
                        raster_entry((int)(e >> 16), e >> col_shift, false);
                        e = en;
                    }
                    if (__any_sync(0xffffffffu, tie_u != 0u)) {
    #pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            bw[c] = -INFINITY;
                            bs[c] = INT_MAX;
                        }
                        for (int k = 0; k < n_max; ++k) {
                            const uint32_t e = k < n_mine ? ent[beg + k] : kSentinel;
                            raster_entry((int)(e >> 16), e >> col_shift, true);
                        }
                    }
                } else if constexpr (!kCompact) {
                    // every triangle in index order (culled ones have an empty
                    // box), so the strict compare already keeps the lower index
                    for (int s = 0; s < P.nt; ++s) {
                        const uint2 bb = bbx[s];
                        const int xlo = (int)(bb.x & 0xffffu), xhi = (int)(bb.x >> 16);
                        const int ylo = (int)(bb.y & 0xffffu), yhi = (int)(bb.y >> 16);
                        if (has_tile && xlo <= xhi && y >= ylo && y <= yhi)
                            raster_entry(s, ((~span_bits(xlo - tx * kTW, xhi - tx * kTW) & 0xFFu) >> col_shift) & 0xFu,
                                         false);
                    }
                }
                // (every group runs the shuffles below, a group without a tile too)
                float sh[4];
    #pragma unroll
                for (int c = 0; c < 4; ++c) sh[c] = bs[c] != INT_MAX ? tshade[bs[c]] : 0.0f;
                const bool rowv = has_tile && y < P.H;
                if (kImage) {
    #pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (rowv && x0 + c < P.W) {
                            const size_t q = (size_t)y * P.W + x0 + c;
                            if (ids) {
                                ids[q] = bs[c] != INT_MAX ? bs[c] : -1;
                            } else {
                                img[3 * q] = sh[c] * P.alb0; img[3 * q + 1] = sh[c] * P.alb1; img[3 * q + 2] = sh[c] * P.alb2;
                            }
                        }
                } else {
                    float tg[12];
                    if (rowv && vec_target && x0 + 3 < P.W) {
                        const float4* tp = reinterpret_cast<const float4*>(P.target + 3 * ((size_t)y * P.W + x0));
                        const float4 a0 = tp[0], a1 = tp[1], a2 = tp[2];
                        tg[0] = a0.x; tg[1] = a0.y; tg[2] = a0.z; tg[3] = a0.w;
                        tg[4] = a1.x; tg[5] = a1.y; tg[6] = a1.z; tg[7] = a1.w;
                        tg[8] = a2.x; tg[9] = a2.y; tg[10] = a2.z; tg[11] = a2.w;
                    } else {
    #pragma unroll
                        for (int c = 0; c < 4; ++c)
    #pragma unroll
                            for (int ch = 0; ch < 3; ++ch)
                                tg[3 * c + ch] = (rowv && x0 + c < P.W) ? P.target[3 * ((size_t)y * P.W + x0 + c) + ch] : 0.0f;
                    }
                    float acc = 0.0f;
    #pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (rowv && x0 + c < P.W) {
                            const float d0 = sh[c] * P.alb0 - tg[3 * c], d1 = sh[c] * P.alb1 - tg[3 * c + 1];
                            const float d2 = sh[c] * P.alb2 - tg[3 * c + 2];
                            acc += d0 * d0 + d1 * d1 + d2 * d2;
                        }
                    // sum over the group's kG lanes
    #pragma unroll
                    for (int o = kG / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (gl == 0 && has_tile) tile_loss[t] = acc;
                }
            }
        };
        bool walked = false;   // some band walked every triangle
        if (!banded) {
            band(0, P.TY, total, false);
        } else {
            for (int r0 = 0, r1 = 0; r0 < P.TY; r0 = r1) {
                __syncthreads();   // row totals written; the previous band's raster done
                if (tid == 0) {
                    int r = r0, sum = 0;
                    while (r < P.TY && sum + rowtot[r] <= capb) sum += rowtot[r++];
                    s_band[0] = r > r0 ? r : r0 + 1;
                    s_band[1] = r > r0 ? 0 : 1;
                }
                if (tid < 33) s_hist[tid] = 0;
                __syncthreads();
                r1 = s_band[0];
                const bool walk_all = s_band[1] != 0;
                walked = walked || walk_all;
                const int total_b = walk_all ? 0
                                             : bin_scan<kT>(tcnt + r0 * P.TX, toff + r0 * P.TX, olist, (r1 - r0) * P.TX,
                                                        s_wtot, s_hist, &n_obj);
                band(r0, r1, total_b, walk_all);
            }
        }
        if (!kImage && tid == 0 && P.stats && walked) atomicAdd(&P.stats[6], 1ull);
        // ---- 6. reduction -----------------------------------------------------
        if (!kImage) {
            __syncthreads();
            // thread i sums tiles i, i + kT, ...; then a fixed shuffle tree
            float acc = 0.0f;
            const float* tile_loss = reinterpret_cast<const float*>(tcnt);
            for (int t = tid; t < P.T; t += kT) acc += tile_loss[t];
            acc = warp_sum(acc);
            if (lane == 0) s_part[warp] = acc;
            __syncthreads();
            if (warp == 0) {
                float v = lane < kW ? s_part[lane] : 0.0f;
                v = warp_sum(v);
                if (lane == 0) *resolve(b, m).loss = v / (float)(P.W * P.H * 3);
            }
        }
        __syncthreads();
    }
    // each warp's raster steps go to the diagnostics once per launch
    if (!kImage && lane == 0 && P.stats && steps) atomicAdd(&P.stats[5], steps);
}

// every loss word of the launch to kFreeLoss (before a compact-layout launch)
__global__ void mark_free_kernel(RenderBatch b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < b.M) *reinterpret_cast<unsigned int*>(resolve(b, i).loss) = kFreeLoss;
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

__global__ void tile_t2_kernel(const float* target, int W, int H, int TX, int TH, int T, float* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int ty = t / TX, tx = t - ty * TX;
    float s = 0.0f;
    for (int yy = 0; yy < TH; ++yy)
        for (int xx = 0; xx < kTW; ++xx) {
            const int x = tx * kTW + xx, y = ty * TH + yy;
            if (x >= W || y >= H) continue;
            const size_t p = (size_t)y * W + x;
            for (int c = 0; c < 3; ++c) s += target[3 * p + c] * target[3 * p + c];
        }
    out[t] = s;
}

RvArgs make_args(const DevScene& sc, bool compact = false, bool redo = false) {
    RvArgs a;
    a.verts = sc.verts; a.tris = sc.tris; a.tnrm = sc.tnrm; a.target = sc.target; a.tile_t2 = sc.tile_t2;
    a.nv = sc.nv; a.nt = sc.nt; a.W = sc.W; a.H = sc.H;
    a.th = sc.rv_th;
    a.TX = (sc.W + kTW - 1) / kTW; a.TY = (sc.H + sc.rv_th - 1) / sc.rv_th; a.T = a.TX * a.TY;
    a.tx_recip = ((uint64_t(1) << 32) + (uint64_t)a.TX - 1) / (uint64_t)a.TX;
    a.alb0 = sc.albedo[0]; a.alb1 = sc.albedo[1]; a.alb2 = sc.albedo[2];
    a.l0 = sc.light[0]; a.l1 = sc.light[1]; a.l2 = sc.light[2];
    a.eye_dist = sc.eye_dist; a.scale = sc.scale;
    a.cap = compact ? sc.rv_ccap : sc.rv_cap;
    a.vreg = sc.rv_vreg;
    a.slots = sc.rv_cslots;
    a.redo = redo ? 1 : 0;
    a.stats = sc.rv_stats;
    return a;
}

// Compact layout of one render with tile height th in `budget` bytes:
// records (64 B), bounding boxes (8 B), shades (4 B) and 16-bit tile masks
// by survivor slot, tile counts (4 B), offsets and the list of tiles with
// entries (2 B each) by tile, and the bin entries, which first hold the
// projected vertices.  Slots for every triangle when they fit (the rest
// of the budget to entries, at most kEntryCapMax), else kCompactCapMin
// entries and the rest to slots; false under half the triangles' slots.
bool compact_layout_for(int nv, int nt, int W, int H, int th, long long budget, size_t* bytes, int* cap,
                        int* slots) {
    const long long T = (long long)((W + kTW - 1) / kTW) * ((H + th - 1) / th);
    const long long per_slot = (long long)(sizeof(TriRec) + sizeof(uint2) + sizeof(float) + sizeof(uint16_t));
    const long long fixed = (long long)(sizeof(int) + 2 * sizeof(uint16_t)) * T + 4;   // + the mask array's padding
    const long long cap_min = std::max<long long>(kCompactCapMin, 3LL * nv);   // the vertices live in the entries
    if (cap_min > kEntryCapMax) return false;
    long long s = (budget - kStaticSmem - fixed - 4 * cap_min) / per_slot;
    long long c = cap_min;
    if (s >= nt) {
        s = nt;
        c = std::min<long long>(kEntryCapMax, (budget - kStaticSmem - fixed - per_slot * nt) / 4);
    }
    if (s < 1 || 2 * s < nt) return false;
    *slots = (int)s;
    *cap = (int)c;
    *bytes = (size_t)(per_slot * s + fixed + 4 * c);
    return true;
}

// bytes and entry capacity of one render's layout with tile height th
bool layout_for(int nv, int nt, int W, int H, int th, int max_smem, size_t* bytes, int* cap, int* vreg) {
    const int T = ((W + kTW - 1) / kTW) * ((H + th - 1) / th);
    const int vr = 3 * nv > 2 * nt + (T + 1) / 2 ? 3 * nv : 2 * nt + (T + 1) / 2;
    const size_t fixed = (sizeof(TriRec) + sizeof(uint2) + sizeof(float)) * (size_t)nt +
                         sizeof(float) * (size_t)vr + 2 * sizeof(int) * (size_t)T +
                         sizeof(uint16_t) * (size_t)((nt + 1) & ~1);
    const long long avail = (long long)max_smem - kStaticSmem - (long long)fixed;
    const long long c = avail / (long long)sizeof(uint32_t);
    if (c < kEntryCapMin) return false;
    *cap = c < kEntryCapMax ? (int)c : kEntryCapMax;
    *vreg = vr;
    *bytes = fixed + sizeof(uint32_t) * (size_t)*cap;
    return true;
}

}  // namespace

// Shared-memory layout of one render: records (64 B) and bounding boxes (8 B)
// by triangle, the vertex region (the projected vertices, later the 64-bit
// tile masks and the list of tiles with entries), shades (4 B) by triangle,
// tile counts and offsets, the survivor list (2 B per triangle), and the bin
// entries in what remains of max_smem (at most kEntryCapMax).  8x4 tiles
// when that leaves room for 8,192 entries, else 8x8 tiles; false when fewer
// than kEntryCapMin entries fit either way.  The tile height is a function of
// the scene's sizes only (both layouts use it), so each layout sums a render's
// loss in one fixed order, and which layout renders a perturbation depends on
// that render's own survivors and entries only: results are deterministic.
//
// The compact layout (two CTAs per SM, each with half of smem_per_sm less
// the 1 KB the hardware reserves per CTA) serves the renders it fits, with
// the same tile height; the full layout renders the rest and every image.
bool revolve_layout(DevScene& sc, int max_smem, int smem_per_sm) {
    size_t bytes = 0;
    int cap = 0, vreg = 0;
    if (layout_for(sc.nv, sc.nt, sc.W, sc.H, 4, max_smem, &bytes, &cap, &vreg) && cap >= 8192) {
        sc.rv_th = 4;
    } else if (layout_for(sc.nv, sc.nt, sc.W, sc.H, 8, max_smem, &bytes, &cap, &vreg)) {
        sc.rv_th = 8;
    } else {
        return false;
    }
    sc.rv_smem = bytes;
    sc.rv_cap = cap;
    sc.rv_vreg = vreg;
    size_t cbytes = 0;
    int ccap = 0, cslots = 0;
    const long long budget = std::min<long long>(max_smem, smem_per_sm / 2 - 1024);
    if (compact_layout_for(sc.nv, sc.nt, sc.W, sc.H, sc.rv_th, budget, &cbytes, &ccap, &cslots)) {
        sc.rv_csmem = cbytes;
        sc.rv_ccap = ccap;
        sc.rv_cslots = cslots;
    } else {
        sc.rv_csmem = 0;
        sc.rv_ccap = 0;
        sc.rv_cslots = 0;
    }
    return true;
}

void revolve_prepare(DevScene& sc, cudaStream_t s) {
    normals_kernel<<<(sc.nt + 255) / 256, 256, 0, s>>>(sc.verts, sc.tris, sc.nt, sc.tnrm);
    const int bytes = (int)sc.rv_smem;
    cudaFuncSetAttribute(revolve_kernel<4, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(revolve_kernel<4, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(revolve_kernel<8, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(revolve_kernel<8, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (sc.rv_csmem) {
        const int cb = (int)sc.rv_csmem;
        cudaFuncSetAttribute(revolve_kernel<4, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cb);
        cudaFuncSetAttribute(revolve_kernel<8, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cb);
        // all of the SM's unified memory as shared memory, so that two CTAs fit
        cudaFuncSetAttribute(revolve_kernel<4, false, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(revolve_kernel<8, false, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
}

void revolve_tile_t2(DevScene& sc, cudaStream_t s) {
    const int TX = (sc.W + kTW - 1) / kTW, TY = (sc.H + sc.rv_th - 1) / sc.rv_th;
    tile_t2_kernel<<<(TX * TY + 127) / 128, 128, 0, s>>>(sc.target, sc.W, sc.H, TX, sc.rv_th, TX * TY, sc.tile_t2);
}

int revolve_tiles(const DevScene& sc) {
    return ((sc.W + kTW - 1) / kTW) * ((sc.H + sc.rv_th - 1) / sc.rv_th);
}

// With a compact layout: the loss words marked free, the compact launch (two
// CTAs per SM), then the full-layout launch in redo mode, which renders only
// the perturbations the compact one handed over (its CTAs read M loss words
// when there are none).
void launch_revolve_loss(const DevScene& sc, const RenderBatch& b, cudaStream_t s) {
    if (b.M <= 0) return;   // nothing to render (and no empty grid to launch)
    const int grid = b.M < num_sms() ? b.M : num_sms();
    const bool compact = sc.rv_csmem != 0;
    if (compact) {
        mark_free_kernel<<<(b.M + 255) / 256, 256, 0, s>>>(b);
        const int cgrid = b.M < 2 * num_sms() ? b.M : 2 * num_sms();
        if (sc.rv_th == 4)
            revolve_kernel<4, false, true><<<cgrid, kCompactThreads, sc.rv_csmem, s>>>(make_args(sc, true), b, nullptr,
                                                                                        nullptr, nullptr);
        else
            revolve_kernel<8, false, true><<<cgrid, kCompactThreads, sc.rv_csmem, s>>>(make_args(sc, true), b, nullptr,
                                                                                        nullptr, nullptr);
    }
    if (sc.rv_th == 4)
        revolve_kernel<4, false, false><<<grid, kThreads, sc.rv_smem, s>>>(make_args(sc, false, compact), b, nullptr,
                                                                           nullptr, nullptr);
    else
        revolve_kernel<8, false, false><<<grid, kThreads, sc.rv_smem, s>>>(make_args(sc, false, compact), b, nullptr,
                                                                           nullptr, nullptr);
}

// one image at params: colours into img [H][W][3], or, with ids non-null,
// the index of the triangle each pixel shows (-1: background) into ids [H][W]
void launch_revolve_image(const DevScene& sc, const float* params, float* img, int32_t* ids, cudaStream_t s) {
    RenderBatch b{};
    if (sc.rv_th == 4)
        revolve_kernel<4, true, false><<<1, kThreads, sc.rv_smem, s>>>(make_args(sc), b, params, img, ids);
    else
        revolve_kernel<8, true, false><<<1, kThreads, sc.rv_smem, s>>>(make_args(sc), b, params, img, ids);
}

}  // namespace hr
