// K1: perturbation sampler and kernel weights (Sec. 3.2-3.5).
//
// Two threads draw one antithetic pair k of one sample group: a + leg from
// the positive lobe and a - leg from the negative lobe of the chosen kernel,
// every other dimension N(0, sigma^2) shared by both legs (Sec. 3.2,
// separability; Suppl. "Smooth Gradient Marginalization").  Lobe samples are
// computed in FP64 and rounded once to FP32: that FP32 value is the
// perturbation every renderer sees.  Weights are evaluated in FP64 at the
// FP32 perturbation and stored in FP32.
//
// Philox counter of pair k: (k, block, (1 << 24) | sub, request), key = seed.
// Block 0 = (component word, lobe uniform a, lobe uniform b, sign word);
// block 1 + b holds the Box-Muller uniforms of dims 4b .. 4b + 3.
#include <cmath>

#include "hr_device.cuh"
#include "hr_internal.h"
#include "sample_device.cuh"

namespace hr {
namespace {

constexpr int kSampleThreadsMax = 128;   // launch shapes 32 / 64 / 128 threads per block

__global__ void __launch_bounds__(kSampleThreadsMax) sample_kernel(SampleArgs a, Lobes host_lobes) {
    const SampleGroup G = a.n_inline > 0 ? a.inline_groups[blockIdx.y] : a.groups[blockIdx.y];
    // two threads per pair: leg 0 writes the + perturbation, leg 1 the -
    // one; both derive the pair's component and shared dims from the same
    // Philox words, so the FP64-heavy lobe inverse and weights of the two
    // legs run side by side (FP64 latency dominates this kernel)
    if (a.theta_out && blockIdx.x == 0 && blockIdx.y == 0) {
        for (int d = threadIdx.x; d < a.theta_n; d += blockDim.x)
            a.theta_out[d] = a.theta_in ? __double2float_rn(a.theta_in[d]) : a.theta_vals[d];
    }
    const int n = a.n;
    const uint32_t sub = G.sub + (a.step ? 64u * (uint32_t)(*a.step) : 0u);
    const uint32_t c2 = (TAG_SAMPLE << 24) | (sub & 0xFFFFFFu);
    const int leg = threadIdx.x & 1;
    const int kb = blockIdx.x * (blockDim.x >> 1);   // first pair of this block
    int k = kb + (threadIdx.x >> 1);
    if (G.comp_i == -1 && G.lobe == 1 && blockDim.x >= 64 && n > 1) {
        // Aggregate Hessian lobes: a pair's component is diagonal (the long
        // Lambert-W root) or off-diagonal (two half-Rayleigh radii).  With two
        // or more warps per block, the block's pairs are taken diagonal ones
        // first, so that most warps run one of the two paths instead of both;
        // every pair is computed by the same code either way.
        __shared__ int s_order[kSampleThreadsMax / 2];
        __shared__ int s_cnt[2][2];
        const int np = blockDim.x >> 1, p = threadIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        bool valid = false, diag = false;
        if (p < np && kb + p < G.P) {
            valid = true;
            const u32x4 wq = philox_seed(a.seed, (uint32_t)(kb + p), 0u, c2, G.request);
            const int e = (int)(((uint64_t)wq.x * (uint64_t)(n * n)) >> 32);
            diag = e / n == e - (e / n) * n;
        }
        unsigned bd = 0u, bo = 0u;
        if (w < 2) {
            bd = __ballot_sync(0xffffffffu, valid && diag);
            bo = __ballot_sync(0xffffffffu, valid && !diag);
            if (lane == 0) { s_cnt[0][w] = __popc(bd); s_cnt[1][w] = __popc(bo); }
        }
        __syncthreads();
        if (w < 2 && p < np) {
            const unsigned lt = (1u << lane) - 1u;
            const int nd = s_cnt[0][0] + s_cnt[0][1];
            int pos = p;   // pairs past the end of the group keep their place (after all valid ones)
            if (valid && diag) pos = __popc(bd & lt) + (w ? s_cnt[0][0] : 0);
            else if (valid) pos = nd + __popc(bo & lt) + (w ? s_cnt[1][0] : 0);
            s_order[pos] = p;
        }
        __syncthreads();
        k = kb + s_order[threadIdx.x >> 1];
    }
    if (k >= G.P) return;
    sample_leg(a, G, lobes_for(a, G, host_lobes), k, leg);
}

// K6: estimator sums.  Element e sums w[m][e] * loss[m] over its row range in
// a fixed order: 256 contiguous chunks, each a Kahan-compensated FP32 sum,
// then an FP64 tree over the chunks, times 1/(2P).
constexpr int kFinThreads = 256;

__global__ void __launch_bounds__(kFinThreads) finalize_kernel(FinalizeArgs a) {
    __shared__ double sh[kFinThreads], sa[kFinThreads];
    const int e = blockIdx.x;
    const int m0 = a.elementwise ? e * a.pairs2 : 0;
    const int cnt = a.pairs2;
    const int chunk = (cnt + kFinThreads - 1) / kFinThreads;
    const int b = m0 + threadIdx.x * chunk;
    const int end = min(m0 + cnt, b + chunk);
    Kahan ks, ka;
    int m = b;
    // four items' loads go out before their sums, which stay in item order
    for (; m + 3 < end; m += 4) {
        float x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = __fmul_rn(__ldg(a.w + (size_t)(m + u) * a.E + e), __ldg(a.loss + m + u));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            ks.add(x[u]);
            ka.add(fabsf(x[u]));
        }
    }
    for (; m < end; ++m) {
        const float x = __fmul_rn(a.w[(size_t)m * a.E + e], a.loss[m]);
        ks.add(x);
        ka.add(fabsf(x));
    }
    const int t = threadIdx.x;
    sh[t] = (double)ks.s - (double)ks.c;
    sa[t] = (double)ka.s - (double)ka.c;
    __syncthreads();
    // pairwise tree (t, t + o); its last five levels by warp shuffles
    for (int o = kFinThreads / 2; o >= 32; o >>= 1) {
        if (t < o) {
            sh[t] += sh[t + o];
            sa[t] += sa[t + o];
        }
        __syncthreads();
    }
    if (t >= 32) return;
    double vs = sh[t], va = sa[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vs += __shfl_down_sync(0xffffffffu, vs, o);
        va += __shfl_down_sync(0xffffffffu, va, o);
    }
    if (t == 0) {
        const double val = vs * a.inv2P;
        a.out_flat[e] = val;
        if (a.out_scale) a.out_scale[e] = va * a.inv2P;
        if (a.hessian && a.out_full) {
            // e -> (row, col) of the upper triangle
            int r = 0, rem = e;
            while (rem >= a.n - r) { rem -= a.n - r; ++r; }
            const int c = r + rem;
            a.out_full[r * a.n + c] = val;
            a.out_full[c * a.n + r] = val;
        }
    }
}

}  // namespace

void launch_sample(const SampleArgs& a, int n_groups, int max_P, cudaStream_t s) {
    // FP64-latency bound: few threads per block spread the pairs over many SMs
    const int t = (a.threads == 16 || a.threads == 64 || a.threads == 128) ? a.threads : 32;
    dim3 grid((2 * max_P + t - 1) / t, n_groups);   // one thread per perturbation (pair leg)
    sample_kernel<<<grid, t, 0, s>>>(a, make_lobes(a.sigma, a.Zg, a.Zd, a.Zo, a.n));
}

void launch_finalize(const FinalizeArgs& a, cudaStream_t s) {
    finalize_kernel<<<a.E, kFinThreads, 0, s>>>(a);
}

}  // namespace hr
