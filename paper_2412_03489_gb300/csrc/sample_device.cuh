// Device code of the perturbation sampler (Sec. 3.2-3.5), shared by the
// sampler kernel (sample.cu) and the persistent serving kernel (queue.cu):
// FP64 lobe inverses, the mixture densities and the weights, and one pair
// leg's draw.
#pragma once
#include <cmath>

#include "hr_device.cuh"
#include "hr_internal.h"

namespace hr {
namespace {

constexpr int kMaxN = 64;
constexpr double kPi = 3.141592653589793238462643383279502884;

// 1/x for x in the normal FP32 range by the Newton-Raphson iteration for the
// reciprocal, r' = r + r (1 - x r), started from the FP32 reciprocal (relative
// error ~1e-7): one step leaves ~1e-14, two leave FP64 rounding.  An FP64
// division costs hundreds of cycles on this GPU, a step two dependent FMAs.
__device__ __forceinline__ double recip_nr(double x) {
    const double r = (double)__frcp_rn((float)x);
    return fma(r, fma(-x, r, 1.0), r);
}
__device__ __forceinline__ double recip_nr2(double x) {
    const double r = recip_nr(x);
    return fma(r, fma(-x, r, 1.0), r);
}

// Root s > 0 of  log(s) - s + 1 + L = 0  for L >= 0, i.e. s e^{-s} = e^{-1-L}.
// upper: the root s >= 1 (tails of the diagonal lobe, |t| > 1), else s <= 1.
// Halley's method on the log form.  A dependent FP64 operation costs tens of
// cycles on this GPU, an FP64 log thousands, so:
//   1. away from the branch point (u = sqrt(2L) > 0.05) the start comes from
//      the same iteration in FP32, begun at the branch-point expansion
//      s = 1 +- u + u^2/3 or at the asymptotics of each branch; near it
//      (u <= 0.05) FP32 cannot resolve g and the start is the expansion in FP64;
//   2. the FP64 iteration takes one log, of the start s0, and evaluates
//      log s = log s0 + log1p(d), d = (s - s0)/s0, by the series of log1p
//      (|d| <= 1e-4 on this path: the start is within ~1e-5 of the root;
//      otherwise it falls back to log(s)); its divisions are Newton-refined
//      reciprocals (a step needs ~1e-14 relative, not a rounded quotient);
//   3. it stops by the cubic convergence of Halley's method: after a step of
//      relative size D the error is about D^3 / (4 (1 - s)^2), below 1e-17
//      once D <= 1e-7 min(1, |1 - s|).
__device__ double lobe_root(double L, bool upper) {
    const float Lf = (float)L;
    const float uf = sqrtf(2.0f * Lf);
    double s0 = -1.0;
    if (uf > 0.05f) {
        float sf;
        if (upper) {
            sf = (uf < 2.0f) ? 1.0f + uf + uf * uf * (1.0f / 3.0f) : (1.0f + Lf) + __logf(1.0f + Lf);
        } else {
            const float y = __expf(-1.0f - Lf);
            sf = (uf < 1.0f) ? 1.0f - uf + uf * uf * (1.0f / 3.0f) : y * (1.0f + y);
        }
        for (int it = 0; it < 8; ++it) {
            const float g = __logf(sf) - sf + 1.0f + Lf;
            const float r = __frcp_rn(sf);
            const float g1 = r - 1.0f;
            float sn = sf - __fdividef(2.0f * g * g1, 2.0f * g1 * g1 + g * r * r);
            if (!(sn > 0.0f)) sn = 0.5f * sf;
            if (upper && sn < 1.0f) sn = 0.5f * (sf + 1.0f);
            if (!upper && sn > 1.0f) sn = 0.5f * (sf + 1.0f);
            const bool done = fabsf(sn - sf) <= 2e-6f * sn;
            sf = sn;
            if (done) break;
        }
        if (sf > 0.0f && (upper ? sf >= 1.0f : sf <= 1.0f)) s0 = (double)sf;
    }
    if (s0 < 0.0) {
        const double u = sqrt(2.0 * L);
        if (u < 1e-9) return upper ? 1.0 + u : 1.0 - u;
        if (u < (upper ? 2.0 : 1.0)) {
            s0 = 1.0 + (upper ? u : -u) + u * u * (1.0 / 3.0);
        } else if (upper) {
            s0 = (1.0 + L) + log(1.0 + L);
        } else {
            const double y = exp(-1.0 - L);
            s0 = y * (1.0 + y);
        }
    }
    const double lg0 = log(s0);
    const double r0 = recip_nr(s0);
    double s = s0;
    for (int it = 0; it < 16; ++it) {
        const double d = (s - s0) * r0;
        const double ls = fabs(d) <= 1e-4 ? lg0 + d * (1.0 - d * (0.5 - d * (1.0 / 3.0 - 0.25 * d))) : log(s);
        const double g = ls - s + 1.0 + L;
        const double om = 1.0 - s;
        // Halley: s - 2 g g' / (2 g'^2 - g g''), g' = (1 - s)/s, g'' = -1/s^2
        double sn = s - 2.0 * g * om * s * recip_nr(2.0 * om * om + g);
        if (!(sn > 0.0)) sn = 0.5 * s;
        if (upper && sn < 1.0) sn = 0.5 * (s + 1.0);
        if (!upper && sn > 1.0) sn = 0.5 * (s + 1.0);
        const double step = fabs(sn - s);
        s = sn;
        if (step <= 1e-7 * s * fmin(1.0, fabs(om))) break;
    }
    return s;
}

// L = -log(16 m^2) for m in (0, 1/4], with one log either way: below
// 16 m^2 = 1/2 the log of 16 m^2 itself; above it -log1p(y), y = -(1 - 4m)(1 + 4m)
// (16 m^2 - 1 without cancellation), by Goldberg's identity
// log1p(y) = y log(w) / (w - 1), w = 1 + y, where w - 1 is exact for w in
// [1/2, 1] (D. Goldberg, "What every computer scientist should know about
// floating-point arithmetic", ACM Computing Surveys 1991, Theorem 4).  The
// lanes of a warp then share one log call instead of running a log and a log1p.
__device__ __forceinline__ double neg_log16(double m) {
    const double x = 16.0 * m * m;
    const double y = -((1.0 - 4.0 * m) * (1.0 + 4.0 * m));
    const bool direct = x < 0.5;
    const double w = 1.0 + y;
    const double lg = log(direct ? x : w);
    if (direct) return -lg;
    return w == 1.0 ? -y : -(y * (lg * recip_nr2(w - 1.0)));
}

// Inverse of the diagonal-lobe CDF (standardised t = tau / sigma): with tail
// mass m (or middle offset a = |c - 1/2|), t^2 e^{-t^2} = 16 m^2 / e, i.e.
// s = t^2 solves s e^{-s} = e^{-1-L}, L = -log(16 m^2).  Tails and middle go
// through one call of the root solve (the two legs of a pair sit in adjacent
// lanes, so separate calls would run the solve twice per warp).
__device__ double diag_inverse(double c) {
    const bool tail = c < 0.25 || c > 0.75;
    const double d = c - 0.5;
    if (!tail && d == 0.0) return 0.0;
    const double m = tail ? (c < 0.25 ? c : 1.0 - c) : fabs(d);
    const double t = sqrt(lobe_root(neg_log16(m), tail));
    return (tail ? c < 0.25 : d < 0.0) ? -t : t;
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
// With a single bandwidth per launch the host computes them once and passes
// them in; per-instance bandwidths (sigma_row) are expanded in the kernel.
struct Lobes {
    double sigma, Zg, Zd, Zo;
    double s2, is2, is4, iZg, iZd, iZo;
    double inv_n, inv_n2;   // 1/n, 1/n^2 of the mixture densities
};

__host__ __device__ inline Lobes make_lobes(double s, double zg, double zd, double zo, int n) {
    Lobes L;
    L.sigma = s; L.Zg = zg; L.Zd = zd; L.Zo = zo;
    L.s2 = s * s;
    L.is2 = 1.0 / L.s2;
    L.is4 = L.is2 * L.is2;
    L.iZg = 1.0 / zg; L.iZd = 1.0 / zd; L.iZo = 1.0 / zo;
    L.inv_n = 1.0 / (double)n;
    L.inv_n2 = 1.0 / ((double)n * (double)n);
    return L;
}

__device__ __forceinline__ Lobes lobes_for(const SampleArgs& a, const SampleGroup& G, const Lobes& host) {
    if (!a.sigma_row) return host;
    const double s = a.sigma_row[G.theta_row];
    const double zg = sqrt(2.0 / kPi) / s;
    return make_lobes(s, zg, 4.0 * kExpMinusHalf / (sqrt(2.0 * kPi) * (s * s)), zg * zg, a.n);
}

// 1/S for the mixture densities: S > 0 is far inside the FP32 range except in
// degenerate draws, which take the division
__device__ __forceinline__ double recip_mixture(double S) {
    return (S > 1e-30 && S < 1e30) ? recip_nr2(S) : 1.0 / S;
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
    return (sd * L.is4 * L.iZd + (off > 0.0 ? off : 0.0) * L.is4 * L.iZo) * L.inv_n2;
}

// Args: SampleArgs, or any type with the fields read here and in sample_leg
// (n, E, seed, v, tau, w, invS, meta, step).
template <class Args>
__device__ void write_weights(const Args& a, const Lobes& L, const SampleGroup& G, int m, const float* t,
                              double sign) {
    const int n = a.n;
    const double s2 = L.s2, is2 = L.is2, is4 = L.is4;
    if (G.quantity == 3) {
        const double S = hess_mixture(t, n, L);
        a.invS[m] = (float)(S > 0.0 ? recip_mixture(S) : 0.0);
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
        S = S * L.iZg * L.inv_n;
        const double iS = S > 0.0 ? recip_mixture(S) : 0.0;
        for (int d = 0; d < n; ++d) wm[d] = (float)(((double)t[d] * is2) * iS);
        return;
    }
    const double S = hess_mixture(t, n, L);
    if (!(S > 0.0)) return;
    const double iS = recip_mixture(S);
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

// One leg (0: + lobe, 1: - lobe) of antithetic pair k of group G: its
// perturbation, path key and weights (Sec. 3.2-3.5).  Called by the sampler
// kernel (two threads per pair) and by the persistent serving kernel.
template <class Args>
__device__ __forceinline__ void sample_leg(const Args& a, const SampleGroup& G, const Lobes& L, int k, int leg) {
    const int n = a.n;
    const uint32_t sub = G.sub + (a.step ? 64u * (uint32_t)(*a.step) : 0u);
    const uint32_t c2 = (TAG_SAMPLE << 24) | (sub & 0xFFFFFFu);
    const double sigma = L.sigma;
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

}  // namespace
}  // namespace hr
