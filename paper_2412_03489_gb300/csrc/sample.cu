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

namespace hr {
namespace {

constexpr int kMaxN = 64;
constexpr double kPi = 3.141592653589793238462643383279502884;

// Root s > 0 of  log(s) - s + 1 + L = 0  for L >= 0, i.e. s e^{-s} = e^{-1-L}.
// upper: the root s >= 1 (tails of the diagonal lobe, |t| > 1), else s <= 1.
// Halley's method on the log form, started from the branch-point expansion
// s = 1 +- u + u^2/3 (u = sqrt(2L)) or from the asymptotics of each branch.
__device__ double lobe_root(double L, bool upper) {
    const double u = sqrt(2.0 * L);
    if (u < 1e-9) return upper ? 1.0 + u : 1.0 - u;
    double s;
    if (upper) {
        s = (u < 2.0) ? 1.0 + u + u * u / 3.0 : (1.0 + L) + log(1.0 + L);
    } else {
        const double y = exp(-1.0 - L);
        s = (u < 1.0) ? 1.0 - u + u * u / 3.0 : y * (1.0 + y);
    }
    // Away from the branch point the same Halley iteration first runs in
    // FP32 (an FP64 log costs thousands of cycles on this GPU, an FP32 one
    // tens), so the FP64 iteration below starts within a few FP32 ulps of the
    // root and stops after about two steps.  Near s = 1 (small u) FP32 cannot
    // resolve g, and the FP64 iteration starts from the series as before.
    if (u > 0.05) {
        float sf = (float)s;
        const float Lf = (float)L;
        for (int it = 0; it < 8; ++it) {
            const float g = __logf(sf) - sf + 1.0f + Lf;
            const float r = 1.0f / sf;
            const float g1 = r - 1.0f;
            float sn = sf - 2.0f * g * g1 / (2.0f * g1 * g1 + g * r * r);
            if (!(sn > 0.0f)) sn = 0.5f * sf;
            if (upper && sn < 1.0f) sn = 0.5f * (sf + 1.0f);
            if (!upper && sn > 1.0f) sn = 0.5f * (sf + 1.0f);
            const bool done = fabsf(sn - sf) <= 2e-6f * sn;
            sf = sn;
            if (done) break;
        }
        if (sf > 0.0f && (upper ? sf >= 1.0f : sf <= 1.0f)) s = (double)sf;
    }
    // Stops at a relative step of 4e-16, or once a step fails to halve the
    // previous one: the residual log(s) - s + 1 + L carries rounding noise of
    // about 1e-16 max(|log s|, s, L), which for small s (the middle of the
    // lobe near c = 1/2) sits far above 4e-16 s, so the step can stall at
    // that noise level without meeting the relative test.
    double prev = INFINITY;
    for (int it = 0; it < 16; ++it) {
        const double g = log(s) - s + 1.0 + L;
        const double r = 1.0 / s;
        const double g1 = r - 1.0;
        double sn = s - 2.0 * g * g1 / (2.0 * g1 * g1 + g * (r * r));
        if (!(sn > 0.0)) sn = 0.5 * s;
        if (upper && sn < 1.0) sn = 0.5 * (s + 1.0);
        if (!upper && sn > 1.0) sn = 0.5 * (s + 1.0);
        const double step = fabs(sn - s);
        s = sn;
        if (step <= 4e-16 * s) break;
        if (it >= 2 && step >= 0.5 * prev) break;
        prev = step;
    }
    return s;
}

// Inverse of the diagonal-lobe CDF (standardised t = tau / sigma): with tail
// mass m (or middle offset a = |c - 1/2|), t^2 e^{-t^2} = 16 m^2 / e, i.e.
// s = t^2 solves s e^{-s} = e^{-1-L}, L = -log(16 m^2).
__device__ double diag_inverse(double c) {
    if (c < 0.25 || c > 0.75) {
        const double m = c < 0.25 ? c : 1.0 - c;
        const double m16 = 16.0 * m * m;
        const double L = m16 < 0.5 ? -log(m16) : -log1p(-((1.0 - 4.0 * m) * (1.0 + 4.0 * m)));
        const double t = sqrt(lobe_root(L, true));
        return c < 0.25 ? -t : t;
    }
    const double d = c - 0.5;
    if (d == 0.0) return 0.0;
    const double a = fabs(d);
    const double a16 = 16.0 * a * a;
    const double L = a16 < 0.5 ? -log(a16) : -log1p(-((1.0 - 4.0 * a) * (1.0 + 4.0 * a)));
    const double t = sqrt(lobe_root(L, false));
    return d < 0.0 ? -t : t;
}

__device__ __forceinline__ int upper_index(int a, int b, int n) {
    return a * n - a * (a - 1) / 2 + (b - a);
}

// e^{-1/2}, rounded to double
constexpr double kExpMinusHalf = 0.60653065971263342360;

// Bandwidth of a group and the masses of its lobes (Sec. 3.2-3.3):
// Zg = sqrt(2/pi)/sigma, Zd = 4 e^{-1/2} / (sqrt(2 pi) sigma^2), Zo = Zg^2,
// with the reciprocals the weights use.  A dependent FP64 operation costs
// tens of cycles on this GPU and a division hundreds, so the weights below
// multiply by these reciprocals (within an FP64 ulp or two of dividing).
struct Lobes {
    double sigma, Zg, Zd, Zo;
    double s2, is2, is4, iZg, iZd, iZo;
};

__device__ __forceinline__ Lobes make_lobes(double s, double zg, double zd, double zo) {
    Lobes L;
    L.sigma = s; L.Zg = zg; L.Zd = zd; L.Zo = zo;
    L.s2 = s * s;
    L.is2 = 1.0 / L.s2;
    L.is4 = L.is2 * L.is2;
    L.iZg = 1.0 / zg; L.iZd = 1.0 / zd; L.iZo = 1.0 / zo;
    return L;
}

__device__ __forceinline__ Lobes lobes_for(const SampleArgs& a, const SampleGroup& G) {
    if (!a.sigma_row) return make_lobes(a.sigma, a.Zg, a.Zd, a.Zo);
    const double s = a.sigma_row[G.theta_row];
    const double zg = sqrt(2.0 / kPi) / s;
    return make_lobes(s, zg, 4.0 * kExpMinusHalf / (sqrt(2.0 * kPi) * (s * s)), zg * zg);
}

// S(tau): n^2 q(tau) / N(tau) for the Hessian mixture, O(n) via
// sum_{i != j} |t_i t_j| = (sum |t_i|)^2 - sum t_i^2.
__device__ double hess_mixture(const float* t, int n, const Lobes& L) {
    double sd = 0.0, sa = 0.0, sq = 0.0;
    for (int d = 0; d < n; ++d) {
        const double x = (double)t[d];
        sd += fabs(x * x - L.s2);
        sa += fabs(x);
        sq += x * x;
    }
    const double off = sa * sa - sq;
    return (sd * L.is4 * L.iZd + (off > 0.0 ? off : 0.0) * L.is4 * L.iZo) / ((double)n * (double)n);
}

__device__ void write_weights(const SampleArgs& a, const Lobes& L, const SampleGroup& G, int m, const float* t,
                              double sign) {
    const int n = a.n;
    const double s2 = L.s2, is2 = L.is2, is4 = L.is4;
    if (G.quantity == 3) {
        const double S = hess_mixture(t, n, L);
        a.invS[m] = (float)(S > 0.0 ? 1.0 / S : 0.0);
        return;
    }
    float* wm = a.w + (size_t)m * a.E;
    for (int e = 0; e < a.E; ++e) wm[e] = 0.0f;
    if (G.comp_i == -3) {
        // plain Gaussian sampling: the weight is the kernel factor c(tau)
        if (G.quantity == 0) {
            for (int d = 0; d < n; ++d) wm[d] = (float)((double)t[d] * is2);
        } else if (G.quantity == 1) {
            int e = 0;
            for (int i = 0; i < n; ++i) {
                const double ti = (double)t[i];
                for (int jj = i; jj < n; ++jj, ++e)
                    wm[e] = (float)((i == jj) ? (ti * ti - s2) * is4 : ti * (double)t[jj] * is4);
            }
        } else {
            double tv = 0.0;
            for (int d = 0; d < n; ++d) tv += (double)t[d] * a.v[d];
            for (int kk = 0; kk < n; ++kk) wm[kk] = (float)((double)t[kk] * tv * is4 - a.v[kk] * is2);
        }
        return;
    }
    if (G.quantity == 4) {
        // element-wise HVP, row i: h_i^v / q_i of the row mixture
        const int i = G.comp_i;
        const double ti = (double)t[i];
        double hv = 0.0, den = 0.0, tot = 0.0;
        for (int b = 0; b < n; ++b) {
            const double c = (b == i) ? (ti * ti - s2) * is4 : ti * (double)t[b] * is4;
            hv += c * a.v[b];
            den += fabs(a.v[b]) * fabs(c);
            tot += fabs(a.v[b]) * (b == i ? L.Zd : L.Zo);
        }
        wm[i] = (float)(den > 0.0 ? hv * tot / den : 0.0);
        return;
    }
    if (G.comp_i >= 0) {
        if (G.quantity == 0) {
            wm[G.comp_i] = (float)(sign * L.Zg);
        } else {
            const int lo = min(G.comp_i, G.comp_j), hi = max(G.comp_i, G.comp_j);
            wm[upper_index(lo, hi, n)] = (float)(sign * (lo == hi ? L.Zd : L.Zo));
        }
        return;
    }
    if (G.quantity == 0) {
        double S = 0.0;
        for (int d = 0; d < n; ++d) S += fabs((double)t[d] * is2);
        S = S * L.iZg / (double)n;
        const double iS = S > 0.0 ? 1.0 / S : 0.0;
        for (int d = 0; d < n; ++d) wm[d] = (float)(((double)t[d] * is2) * iS);
        return;
    }
    const double S = hess_mixture(t, n, L);
    if (!(S > 0.0)) return;
    const double iS = 1.0 / S;
    if (G.quantity == 1) {
        int e = 0;
        for (int i = 0; i < n; ++i) {
            const double ti = (double)t[i];
            for (int j = i; j < n; ++j, ++e) {
                const double c = (i == j) ? (ti * ti - s2) * is4 : ti * (double)t[j] * is4;
                wm[e] = (float)(c * iS);
            }
        }
    } else {
        double tv = 0.0;
        for (int d = 0; d < n; ++d) tv += (double)t[d] * a.v[d];
        for (int k = 0; k < n; ++k) {
            const double hv = (double)t[k] * tv * is4 - a.v[k] * is2;
            wm[k] = (float)(hv * iS);
        }
    }
}

constexpr int kSampleThreadsMax = 128;   // launch shapes 32 / 64 / 128 threads per block

__global__ void __launch_bounds__(kSampleThreadsMax) sample_kernel(SampleArgs a) {
    const SampleGroup G = a.n_inline > 0 ? a.inline_groups[blockIdx.y] : a.groups[blockIdx.y];
    // two threads per pair: leg 0 writes the + perturbation, leg 1 the -
    // one; both derive the pair's component and shared dims from the same
    // Philox words, so the FP64-heavy lobe inverse and weights of the two
    // legs run side by side (FP64 latency dominates this kernel)
    const int tk = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = tk >> 1, leg = tk & 1;
    if (k >= G.P) return;
    const int n = a.n;
    const Lobes L = lobes_for(a, G);
    const double sigma = L.sigma;
    const uint32_t sub = G.sub + (a.step ? 64u * (uint32_t)(*a.step) : 0u);
    const uint32_t c2 = (TAG_SAMPLE << 24) | (sub & 0xFFFFFFu);
    const u32x4 w0 = philox_seed(a.seed, (uint32_t)k, 0u, c2, G.request);
    int i, j;
    if (G.comp_i == -3) {
        i = -1; j = -1;            // no importance sampling: every dim Gaussian
    } else if (G.comp_i >= 0 && G.comp_j == -2) {
        // element-wise HVP: component j of row i with probability
        // |v_j| Z_ij / sum_l |v_l| Z_il (cumulative sums in index order)
        i = G.comp_i;
        double tot = 0.0;
        for (int l = 0; l < n; ++l) tot += fabs(a.v[l]) * (l == i ? L.Zd : L.Zo);
        const double u = u01d(w0.x) * tot;
        double acc = 0.0;
        j = i;
        int last = i;
        bool found = false;
        for (int l = 0; l < n; ++l) {
            const double p = fabs(a.v[l]) * (l == i ? L.Zd : L.Zo);
            if (p > 0.0) last = l;
            acc += p;
            if (!found && p > 0.0 && u < acc) { j = l; found = true; }
        }
        if (!found) j = last;
    } else if (G.comp_i >= 0) {
        i = G.comp_i;
        j = G.lobe == 0 ? G.comp_i : G.comp_j;
    } else if (G.lobe == 0) {
        i = (int)(((uint64_t)w0.x * (uint64_t)n) >> 32);
        j = i;
    } else {
        const int e = (int)(((uint64_t)w0.x * (uint64_t)(n * n)) >> 32);
        i = e / n;
        j = e - i * n;
    }
    // Box-Muller dims (skipped where the lobe sample overwrites them; the
    // words are the same either way)
    double g[kMaxN];
    for (int d = 0; d < n; d += 4) {
        const bool need[4] = {d != i && d != j, d + 1 < n && d + 1 != i && d + 1 != j,
                              d + 2 < n && d + 2 != i && d + 2 != j, d + 3 < n && d + 3 != i && d + 3 != j};
        if (!(need[0] || need[1] || need[2] || need[3])) continue;
        const u32x4 r = philox_seed(a.seed, (uint32_t)k, (uint32_t)(1 + d / 4), c2, G.request);
        const uint32_t words[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (!(need[2 * q] || need[2 * q + 1])) continue;
            const double R = sqrt(-2.0 * log(u01d(words[2 * q])));
            const double ph = 2.0 * kPi * u01d(words[2 * q + 1]);
            if (need[2 * q]) g[d + 2 * q] = sigma * (R * cos(ph));
            if (need[2 * q + 1]) g[d + 2 * q + 1] = sigma * (R * sin(ph));
        }
    }
    const double ua = u01d(w0.y), ub = u01d(w0.z);
    const double sign = leg ? -1.0 : 1.0;
    const int m = G.m0 + 2 * k + leg;
    float* tm = a.tau + (size_t)m * n;
    if (G.comp_i == -3) {
        // legs +tau and -tau of tau ~ N(0, sigma^2 I)
        for (int d = 0; d < n; ++d) tm[d] = leg ? (float)(-g[d]) : (float)g[d];
        if (a.meta) a.meta[m] = make_uint2(sub, (uint32_t)k);
        if (a.w) write_weights(a, L, G, m, tm, sign);
        return;
    }
    double vi, vj;   // this leg's values in dims i and j
    if (G.lobe == 0) {
        const double r = sigma * sqrt(-2.0 * log(ua));
        vi = leg ? -r : r;
        vj = vi;
    } else if (i == j) {
        // + leg: the tails (c in (0, 1/4) or (3/4, 1)); - leg: the middle
        const double c = leg ? 0.25 + 0.5 * ua : (ua < 0.5 ? 0.5 * ua : 0.5 + 0.5 * ua);
        vi = sigma * diag_inverse(c);
        vj = vi;
    } else {
        const double ri = sigma * sqrt(-2.0 * log(ua));
        const double rj = sigma * sqrt(-2.0 * log(ub));
        const double sg = (w0.w & 1u) ? -1.0 : 1.0;
        vi = sg * ri;
        vj = leg ? -sg * rj : sg * rj;
    }
    for (int d = 0; d < n; ++d) {
        double vv;
        if (d == i) vv = vi;
        else if (d == j) vv = vj;
        else vv = g[d];
        tm[d] = (float)vv;
    }
    if (a.meta) a.meta[m] = make_uint2(sub, (uint32_t)k);
    if (a.w || a.invS) write_weights(a, L, G, m, tm, sign);
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
    for (int m = b; m < end; ++m) {
        const float x = __fmul_rn(a.w[(size_t)m * a.E + e], a.loss[m]);
        ks.add(x);
        ka.add(fabsf(x));
    }
    sh[threadIdx.x] = (double)ks.s - (double)ks.c;
    sa[threadIdx.x] = (double)ka.s - (double)ka.c;
    __syncthreads();
    for (int o = kFinThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[threadIdx.x] += sh[threadIdx.x + o];
            sa[threadIdx.x] += sa[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double val = sh[0] * a.inv2P;
        a.out_flat[e] = val;
        if (a.out_scale) a.out_scale[e] = sa[0] * a.inv2P;
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
    sample_kernel<<<grid, t, 0, s>>>(a);
}

void launch_finalize(const FinalizeArgs& a, cudaStream_t s) {
    finalize_kernel<<<a.E, kFinThreads, 0, s>>>(a);
}

}  // namespace hr
