/*
 * Oracle for the stochastic Hessian / HVP / gradient estimator of a
 * Gaussian-smoothed rendering loss (Wang, Fischer, Ritschel: "Stochastic
 * Gradient Estimation for Higher-order Differentiable Rendering").
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Plain, slow,
 * single-threaded C; values in FP64.  Renderer decisions (coverage, depth
 * order, ray hits) are taken in FP32 with the operation sequence that defines
 * each renderer, because the renderer under test renders in FP32; every such
 * operation is written out below with an explicit fmaf or a plain FP32
 * operator (compile with -ffp-contract=off).
 *
 * Convention: smoothed loss  fbar(theta) = E_{tau ~ N(0, s^2 I)} f(theta + tau).
 * (The paper writes the convolution with f(theta - tau), Sec. 3.1; the
 * gradient kernel then flips sign, the Hessian kernel is even and does not.)
 *
 * parity pinned by: tests/test_oracle_*.py (Philox known-answer vectors,
 * Lambert W vs an independent library, CDF landmarks, lobe masses by
 * quadrature, closed-form smoothed derivatives of a quadratic, a step edge,
 * the disc scene and a negated Gaussian; brute-force coverage; a furnace
 * and an analytic direct-lighting case for the path tracer).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_E 2.71828182845904523536

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11.  Ten rounds of the S-box (two 32x32->64 bit      */
/* multiplies) with a Weyl key schedule.                                     */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double or_u01(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

static void philox_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Lambert W by Halley's iteration (Corless, Gonnet, Hare, Jeffrey, Knuth,   */
/* "On the Lambert W function", 1996): branch-point series start near -1/e,  */
/* asymptotic start for W_{-1} near 0-.                                      */
/* ------------------------------------------------------------------------ */
static double lambertw_p(double z, double p, int branch)
{
    /* p = sqrt(2 (1 + e z)), supplied accurately by the caller. */
    double w;
    if (branch == 0) {
        w = -1.0 + p - p * p / 3.0 + 11.0 / 72.0 * p * p * p;
    } else if (z < -0.25) {
        w = -1.0 - p - p * p / 3.0 - 11.0 / 72.0 * p * p * p;
    } else {
        double L1 = log(-z), L2 = log(-L1);
        w = L1 - L2 + L2 / L1;
    }
    if (p < 1e-9) return w; /* series error O(p^4) is below FP64 resolution */
    for (int it = 0; it < 60; ++it) {
        double ew = exp(w);
        double f = w * ew - z;
        double wp1 = w + 1.0;
        double step = f / (ew * wp1 - (w + 2.0) * f / (2.0 * wp1));
        double wn = w - step;
        if (fabs(wn - w) <= 4e-16 * fabs(wn)) { w = wn; break; }
        w = wn;
    }
    return w;
}

double or_lambertw(double z, int branch)
{
    double one_plus_ez = 1.0 + OR_E * z;
    if (one_plus_ez < 0.0) one_plus_ez = 0.0;
    return lambertw_p(z, sqrt(2.0 * one_plus_ez), branch);
}

/* ------------------------------------------------------------------------ */
/* Diagonal Hessian lobe, standardised t = tau / sigma (Sec. 3.3, CDF        */
/* P^H_ii): left tail -t/4 e^{1/2 - t^2/2}, middle 1/2 + t/4 e^{...}, right  */
/* tail 1 - t/4 e^{...}.  Values 1/4, 1/2, 3/4 at t = -1, 0, 1.              */
/* ------------------------------------------------------------------------ */
double or_diag_cdf(double t)
{
    double g = t / 4.0 * exp(0.5 - t * t / 2.0);
    if (t < -1.0) return -g;
    if (t <= 1.0) return 0.5 + g;
    return 1.0 - g;
}

/* Inverse: with m the tail mass (c or 1 - c) or d = c - 1/2 in the middle,
 * t^2 e^{-t^2} = 16 m^2 / e, so -t^2 = W(-16 m^2 / e): branch -1 in the tails
 * (|t| > 1), branch 0 in the middle (|t| < 1).  1 + e z = (1 - 4m)(1 + 4m) is
 * formed without cancellation. */
double or_diag_inv_cdf(double c)
{
    if (c < 0.25) {
        double m = c;
        double z = -16.0 * m * m / OR_E;
        double p = sqrt(2.0 * (1.0 - 4.0 * m) * (1.0 + 4.0 * m));
        return -sqrt(-lambertw_p(z, p, -1));
    }
    if (c > 0.75) {
        double m = 1.0 - c;
        double z = -16.0 * m * m / OR_E;
        double p = sqrt(2.0 * (1.0 - 4.0 * m) * (1.0 + 4.0 * m));
        return sqrt(-lambertw_p(z, p, -1));
    }
    double d = c - 0.5;
    if (d == 0.0) return 0.0;
    double ad = fabs(d);
    double z = -16.0 * ad * ad / OR_E;
    double p = sqrt(2.0 * (1.0 - 4.0 * ad) * (1.0 + 4.0 * ad));
    double t = sqrt(-lambertw_p(z, p, 0));
    return d < 0 ? -t : t;
}

/* ------------------------------------------------------------------------ */
/* Lobe masses: Z = integral of |kernel| (positive lobe = negative lobe =    */
/* Z/2).  Gradient: 2 N1(0); diagonal: 4 N1(sigma)/sigma; off-diagonal: Zg^2 */
/* ------------------------------------------------------------------------ */
static double n1(double x, double s) { return exp(-0.5 * x * x / (s * s)) / (s * sqrt(2.0 * OR_PI)); }
double or_Zg(double s) { return 2.0 * n1(0.0, s); }
double or_Zd(double s) { return 4.0 * n1(s, s) / s; }
double or_Zo(double s) { return or_Zg(s) * or_Zg(s); }

/* ------------------------------------------------------------------------ */
/* Sampling.  Philox counter (pair k, block b, (1 << 24) | sub, request),     */
/* key = seed.  Block 0 = (component word, lobe uniform a, lobe uniform b,   */
/* sign word); blocks 1.. = Box-Muller uniforms, dims 4(b-1)..4(b-1)+3.      */
/* ------------------------------------------------------------------------ */
#define TAG_SAMPLE 1u

/* Row mixture of the HVP kernel sum_j c_ij v_j (element-wise HVP): component
 * j of row i is drawn with probability |v_j| Z_ij / sum_l |v_l| Z_il, the mass
 * of |c_ij v_j N|; the cumulative table is summed in index order. */
static int row_component(uint32_t word, int i, int n, double sigma, const double* v)
{
    double tot = 0.0;
    for (int l = 0; l < n; ++l) tot += fabs(v[l]) * (l == i ? or_Zd(sigma) : or_Zo(sigma));
    double u = or_u01(word) * tot, acc = 0.0;
    int last = i;
    for (int l = 0; l < n; ++l) {
        double p = fabs(v[l]) * (l == i ? or_Zd(sigma) : or_Zo(sigma));
        if (p > 0.0) last = l;
        acc += p;
        if (p > 0.0 && u < acc) return l;
    }
    return last;
}

static const double* g_row_v = 0;   /* v for row-mixture draws (set by or_draw_hvp_rows) */

int or_draw(int lobe, int n, double sigma, int64_t P, uint64_t seed,
            uint32_t request, uint32_t sub, int comp_i, int comp_j,
            float* tau, int32_t* comp_out)
{
    if (n < 1 || P < 1 || !(sigma > 0)) return -1;
    if (comp_j == -2 && !g_row_v) return -1;
    double* g = (double*)malloc(sizeof(double) * n);
    double* tp = (double*)malloc(sizeof(double) * n);
    double* tm = (double*)malloc(sizeof(double) * n);
    uint32_t c2 = (TAG_SAMPLE << 24) | (sub & 0xFFFFFFu);
    for (int64_t k = 0; k < P; ++k) {
        uint32_t w[4], gw[4];
        philox_words(seed, (uint32_t)k, 0u, c2, request, w);
        /* dims not being differentiated: N(0, sigma^2) by Box-Muller, shared
         * by both legs of the pair (Sec. 3.2 "separability"; Suppl. B) */
        for (int d = 0; d < n; ++d) {
            if (d % 4 == 0) philox_words(seed, (uint32_t)k, (uint32_t)(1 + d / 4), c2, request, gw);
            int q = (d % 4) / 2;
            double u1 = or_u01(gw[2 * q]), u2 = or_u01(gw[2 * q + 1]);
            double R = sqrt(-2.0 * log(u1));
            double z = (d % 2 == 0) ? R * cos(2.0 * OR_PI * u2) : R * sin(2.0 * OR_PI * u2);
            g[d] = sigma * z;
        }
        if (comp_i == -3) {
            /* no importance sampling (Tab. 1 "no IS" column): tau ~ N(0, s^2 I),
             * antithetic legs +tau and -tau */
            for (int d = 0; d < n; ++d) {
                tau[(2 * k) * n + d] = (float)g[d];
                tau[(2 * k + 1) * n + d] = (float)(-g[d]);
            }
            if (comp_out) comp_out[k] = -1;
            continue;
        }
        int i, j;
        if (comp_i >= 0 && comp_j == -2) {
            i = comp_i;
            j = row_component(w[0], comp_i, n, sigma, g_row_v);
        } else if (comp_i >= 0) {
            i = comp_i;
            j = lobe == 0 ? comp_i : comp_j;
        } else if (lobe == 0) {
            i = (int)(((uint64_t)w[0] * (uint64_t)n) >> 32);
            j = i;
        } else {
            int e = (int)(((uint64_t)w[0] * (uint64_t)(n * n)) >> 32);
            i = e / n;
            j = e % n;
        }
        if (comp_out) comp_out[k] = lobe == 0 ? i : i * n + j;
        memcpy(tp, g, sizeof(double) * n);
        memcpy(tm, g, sizeof(double) * n);
        double ua = or_u01(w[1]), ub = or_u01(w[2]);
        if (lobe == 0) {
            /* gradient lobe: positive part tau_i > 0, half-Rayleigh radius */
            double r = sigma * sqrt(-2.0 * log(ua));
            tp[i] = r;
            tm[i] = -r;
        } else if (i == j) {
            /* diagonal: + lobe = tails (CDF in (0,1/4) u (3/4,1)), - lobe =
             * middle (CDF in (1/4,3/4)); one uniform drives both legs */
            double cp = ua < 0.5 ? 0.5 * ua : 0.5 + 0.5 * ua;
            double cm = 0.25 + 0.5 * ua;
            tp[i] = sigma * or_diag_inv_cdf(cp);
            tm[i] = sigma * or_diag_inv_cdf(cm);
        } else {
            /* off-diagonal: product of two gradient lobes (Sec. 3.3); + lobe
             * has sign(tau_i) = sign(tau_j) */
            double ri = sigma * sqrt(-2.0 * log(ua));
            double rj = sigma * sqrt(-2.0 * log(ub));
            double s = (w[3] & 1u) ? -1.0 : 1.0;
            tp[i] = s * ri; tp[j] = s * rj;
            tm[i] = s * ri; tm[j] = -s * rj;
        }
        for (int d = 0; d < n; ++d) {
            tau[(2 * k) * n + d] = (float)tp[d];
            tau[(2 * k + 1) * n + d] = (float)tm[d];
        }
    }
    free(g); free(tp); free(tm);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Weights.  Kernel factors c with h = c N: gradient c_i = tau_i / s^2;      */
/* Hessian c_ii = (tau_i^2 - s^2)/s^4, c_ij = tau_i tau_j / s^4 (Sec. 3.3).  */
/* Aggregate (Sec. 3.5): the mixture of all normalised element kernels,      */
/* q = (1/E) sum |h_e| / Z_e, weight h / q (the N factor cancels).           */
/* ------------------------------------------------------------------------ */
int or_weights(int quantity, int n, double sigma, const double* v, int64_t M,
               const float* tau, int comp_i, int comp_j, double* w)
{
    int E = quantity == 1 ? n * (n + 1) / 2 : n;
    double s2 = sigma * sigma, s4 = s2 * s2;
    if (quantity == 3 && (!v || comp_i < 0)) return -1;
    double Zg = or_Zg(sigma), Zd = or_Zd(sigma), Zo = or_Zo(sigma);
    double* t = (double*)malloc(sizeof(double) * n);
    double* C = (double*)malloc(sizeof(double) * n * n);
    for (int64_t m = 0; m < M; ++m) {
        double* wm = w + m * E;
        for (int e = 0; e < E; ++e) wm[e] = 0.0;
        double sign = (m % 2 == 0) ? 1.0 : -1.0;
        if (comp_i == -3) {
            /* plain Gaussian sampling: the weight is the kernel factor c(tau) */
            for (int d = 0; d < n; ++d) t[d] = (double)tau[m * n + d];
            if (quantity == 0) {
                for (int d = 0; d < n; ++d) wm[d] = t[d] / s2;
            } else {
                int e = 0;
                for (int a = 0; a < n; ++a) {
                    double hv = 0.0;
                    for (int b = 0; b < n; ++b) {
                        double c = (a == b) ? (t[a] * t[a] - s2) / s4 : t[a] * t[b] / s4;
                        if (quantity == 1 && b >= a) wm[e++] = c;
                        if (quantity != 1) hv += c * v[b];
                    }
                    if (quantity != 1) wm[a] = hv;
                }
            }
            continue;
        }
        if (quantity == 3) {
            /* h_i^v / q_i with q_i the row mixture: (sum_j c_ij v_j) (sum_l |v_l| Z_il) / sum_j |v_j| |c_ij| */
            for (int d = 0; d < n; ++d) t[d] = (double)tau[m * n + d];
            int i = comp_i;
            double hv = 0.0, den = 0.0, tot = 0.0;
            for (int b = 0; b < n; ++b) {
                double c = (b == i) ? (t[i] * t[i] - s2) / s4 : t[i] * t[b] / s4;
                hv += c * v[b];
                den += fabs(v[b]) * fabs(c);
                tot += fabs(v[b]) * (b == i ? Zd : Zo);
            }
            wm[i] = den > 0.0 ? hv * tot / den : 0.0;
            continue;
        }
        if (comp_i >= 0) {
            if (quantity == 0) {
                wm[comp_i] = sign * Zg;
            } else if (quantity == 1) {
                int a = comp_i < comp_j ? comp_i : comp_j;
                int b = comp_i < comp_j ? comp_j : comp_i;
                int e = a * n - a * (a - 1) / 2 + (b - a);
                wm[e] = sign * (a == b ? Zd : Zo);
            } else {
                free(t); free(C);
                return -1;
            }
            continue;
        }
        for (int d = 0; d < n; ++d) t[d] = (double)tau[m * n + d];
        if (quantity == 0) {
            double S = 0.0;
            for (int d = 0; d < n; ++d) S += fabs(t[d] / s2) / Zg;
            S /= (double)n;            /* q / N = S / n */
            for (int d = 0; d < n; ++d) wm[d] = S > 0 ? (t[d] / s2) / S : 0.0;
            continue;
        }
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b)
                C[a * n + b] = (a == b) ? (t[a] * t[a] - s2) / s4 : t[a] * t[b] / s4;
        double S = 0.0;
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b)
                S += fabs(C[a * n + b]) / (a == b ? Zd : Zo);
        S /= (double)(n * n);          /* q / N = S / n^2 */
        if (quantity == 1) {
            int e = 0;
            for (int a = 0; a < n; ++a)
                for (int b = a; b < n; ++b, ++e) wm[e] = S > 0 ? C[a * n + b] / S : 0.0;
        } else {
            for (int a = 0; a < n; ++a) {
                double hv = 0.0;
                for (int b = 0; b < n; ++b) hv += C[a * n + b] * v[b];
                wm[a] = S > 0 ? hv / S : 0.0;
            }
        }
    }
    free(t); free(C);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Disc renderer: pixel centre ((x + 1/2)/W, (y + 1/2)/H) is inside when    */
/* dx^2 + dy^2 < r^2, decided in FP32 as fma(dx, dx, dy*dy) < r*r.           */
/* ------------------------------------------------------------------------ */
double or_disc_loss(int W, int H, float r, const float p[2], const float* target, float* img)
{
    float r2 = r * r;
    double acc = 0.0;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            float px = ((float)x + 0.5f) / (float)W;
            float py = ((float)y + 0.5f) / (float)H;
            float dx = px - p[0];
            float dy = py - p[1];
            float d2 = fmaf(dx, dx, dy * dy);
            double v = d2 < r2 ? 1.0 : 0.0;
            if (img) img[y * W + x] = (float)v;
            if (target) {
                double diff = v - (double)target[y * W + x];
                acc += diff * diff;
            }
        }
    }
    return acc / ((double)W * (double)H);
}

/* ------------------------------------------------------------------------ */
/* Squares renderer (the Box2 / Box10 plateau tasks of Sec. 4.1): K          */
/* axis-aligned squares of half-size h centred at (p[2s], p[2s+1]); a pixel  */
/* centre is 1 when it lies strictly inside any square, decided in FP32 as   */
/* |px - cx| < h and |py - cy| < h.                                          */
/* ------------------------------------------------------------------------ */
double or_boxes_loss(int W, int H, int K, float h, const float* p, const float* target, float* img)
{
    double acc = 0.0;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            float px = ((float)x + 0.5f) / (float)W;
            float py = ((float)y + 0.5f) / (float)H;
            double v = 0.0;
            for (int k = 0; k < K; ++k) {
                float dx = px - p[2 * k], dy = py - p[2 * k + 1];
                if (fabsf(dx) < h && fabsf(dy) < h) { v = 1.0; break; }
            }
            if (img) img[y * W + x] = (float)v;
            if (target) {
                double d = v - (double)target[y * W + x];
                acc += d * d;
            }
        }
    }
    return acc / ((double)W * (double)H);
}

/* ------------------------------------------------------------------------ */
/* Screen-space triangle edges shared by the two rasterisers.                */
/* Edge P->Q: A = Q.y - P.y, B = P.x - Q.x, C = P.y Q.x - P.x Q.y (products   */
/* rounded, then the difference), E(x, y) = fma(A, x, fma(B, y, C)).  The    */
/* edge reversed gives exactly -A, -B, -C, so a shared edge is watertight;   */
/* E == 0 counts as inside only on a "top-left" edge: A > 0, or A == 0 and  */
/* B > 0.                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct { float A, B, C; } edge32;

static edge32 edge_of(float px, float py, float qx, float qy)
{
    edge32 e;
    e.A = qy - py;
    e.B = px - qx;
    float m1 = py * qx;
    float m2 = px * qy;
    e.C = m1 - m2;
    return e;
}
static float edge_eval(edge32 e, float x, float y) { return fmaf(e.A, x, fmaf(e.B, y, e.C)); }
static int edge_inside(edge32 e, float v)
{
    if (v > 0.0f) return 1;
    if (v < 0.0f) return 0;
    return (e.A > 0.0f) || (e.A == 0.0f && e.B > 0.0f);
}
static float fmin3(float a, float b, float c) { float m = a < b ? a : b; return m < c ? m : c; }
static float fmax3(float a, float b, float c) { float m = a > b ? a : b; return m > c ? m : c; }

/* ------------------------------------------------------------------------ */
/* Surface-of-revolution rasteriser (stand-in for the Mug task, Sec. 4.1).   */
/* FP32 geometry: R = Rx(p0) Ry(p1) from RN32 of FP64 cos/sin; camera at z = */
/* D looking down -z; screen x = fma(k, X/Z, W/2), y = fma(-k, Y/Z, H/2);    */
/* back faces (signed area <= 0) culled; nearest 1/Z wins, ties to the lower */
/* triangle index.  Flat Lambert shading max(0, n.l) * albedo in FP64.       */
/* ------------------------------------------------------------------------ */
double or_revolve_loss(const or_revolve_scene* s, const float p[2], const float* target, float* img)
{
    return or_revolve_render(s, p, target, img, 0);
}

/* The mesh renderer; also writes, if ids is not NULL, the index of the
 * triangle that each pixel shows (-1: background). */
double or_revolve_render(const or_revolve_scene* s, const float p[2], const float* target, float* img, int* ids)
{
    const int W = s->W, H = s->H, nv = s->nv, nt = s->nt;
    float ca = (float)cos((double)p[0]), sa = (float)sin((double)p[0]);
    float cb = (float)cos((double)p[1]), sb = (float)sin((double)p[1]);
    float R[3][3];
    R[0][0] = cb;      R[0][1] = 0.0f; R[0][2] = sb;
    R[1][0] = sa * sb; R[1][1] = ca;   R[1][2] = -(sa * cb);
    R[2][0] = -(ca * sb); R[2][1] = sa; R[2][2] = ca * cb;

    float* sx = (float*)malloc(sizeof(float) * nv);
    float* sy = (float*)malloc(sizeof(float) * nv);
    float* iz = (float*)malloc(sizeof(float) * nv);
    float* zc = (float*)malloc(sizeof(float) * nv);
    for (int v = 0; v < nv; ++v) {
        const float* P = s->verts + 3 * v;
        float w[3];
        for (int r = 0; r < 3; ++r) w[r] = fmaf(R[r][2], P[2], fmaf(R[r][1], P[1], R[r][0] * P[0]));
        float X = w[0], Y = w[1], Z = s->eye_dist - w[2];
        float qx = X / Z, qy = Y / Z;
        sx[v] = fmaf(s->scale, qx, (float)W * 0.5f);
        sy[v] = fmaf(-s->scale, qy, (float)H * 0.5f);
        iz[v] = 1.0f / Z;
        zc[v] = Z;
    }
    /* FP64 rotation for shading values */
    double Rd[3][3];
    {
        double a = p[0], b = p[1];
        double cad = cos(a), sad = sin(a), cbd = cos(b), sbd = sin(b);
        Rd[0][0] = cbd;        Rd[0][1] = 0.0; Rd[0][2] = sbd;
        Rd[1][0] = sad * sbd;  Rd[1][1] = cad; Rd[1][2] = -sad * cbd;
        Rd[2][0] = -cad * sbd; Rd[2][1] = sad; Rd[2][2] = cad * cbd;
    }
    int npx = W * H;
    float* best_w = (float*)malloc(sizeof(float) * npx);
    int* best_t = (int*)malloc(sizeof(int) * npx);
    for (int i = 0; i < npx; ++i) { best_w[i] = 0.0f; best_t[i] = -1; }

    for (int t = 0; t < nt; ++t) {
        int ia = s->tris[3 * t], ib = s->tris[3 * t + 1], ic = s->tris[3 * t + 2];
        if (!(zc[ia] > 0.0f && zc[ib] > 0.0f && zc[ic] > 0.0f)) continue;
        edge32 e0 = edge_of(sx[ib], sy[ib], sx[ic], sy[ic]);
        edge32 e1 = edge_of(sx[ic], sy[ic], sx[ia], sy[ia]);
        edge32 e2 = edge_of(sx[ia], sy[ia], sx[ib], sy[ib]);
        float D2 = edge_eval(e2, sx[ic], sy[ic]);
        if (!(D2 > 0.0f)) continue;                 /* back face or degenerate */
        float invD = 1.0f / D2;
        float Aw = fmaf(e2.A, iz[ic], fmaf(e1.A, iz[ib], e0.A * iz[ia])) * invD;
        float Bw = fmaf(e2.B, iz[ic], fmaf(e1.B, iz[ib], e0.B * iz[ia])) * invD;
        float Cw = fmaf(e2.C, iz[ic], fmaf(e1.C, iz[ib], e0.C * iz[ia])) * invD;
        float minx = fmin3(sx[ia], sx[ib], sx[ic]), maxx = fmax3(sx[ia], sx[ib], sx[ic]);
        float miny = fmin3(sy[ia], sy[ib], sy[ic]), maxy = fmax3(sy[ia], sy[ib], sy[ic]);
        for (int y = 0; y < H; ++y) {
            float cy = (float)y + 0.5f;
            if (cy < miny || cy > maxy) continue;
            for (int x = 0; x < W; ++x) {
                float cx = (float)x + 0.5f;
                if (cx < minx || cx > maxx) continue;
                if (!edge_inside(e0, edge_eval(e0, cx, cy))) continue;
                if (!edge_inside(e1, edge_eval(e1, cx, cy))) continue;
                if (!edge_inside(e2, edge_eval(e2, cx, cy))) continue;
                float wz = fmaf(Aw, cx, fmaf(Bw, cy, Cw));
                int i = y * W + x;
                if (best_t[i] < 0 || wz > best_w[i]) { best_w[i] = wz; best_t[i] = t; }
            }
        }
    }
    double acc = 0.0;
    for (int i = 0; i < npx; ++i) {
        double col[3] = {0.0, 0.0, 0.0};
        int t = best_t[i];
        if (t >= 0) {
            const float* A = s->verts + 3 * s->tris[3 * t];
            const float* B = s->verts + 3 * s->tris[3 * t + 1];
            const float* C = s->verts + 3 * s->tris[3 * t + 2];
            double u[3], v[3], nm[3], nw[3];
            for (int c = 0; c < 3; ++c) { u[c] = (double)B[c] - A[c]; v[c] = (double)C[c] - A[c]; }
            nm[0] = u[1] * v[2] - u[2] * v[1];
            nm[1] = u[2] * v[0] - u[0] * v[2];
            nm[2] = u[0] * v[1] - u[1] * v[0];
            double len = sqrt(nm[0] * nm[0] + nm[1] * nm[1] + nm[2] * nm[2]);
            for (int r = 0; r < 3; ++r) nw[r] = (Rd[r][0] * nm[0] + Rd[r][1] * nm[1] + Rd[r][2] * nm[2]) / len;
            double sh = nw[0] * s->light[0] + nw[1] * s->light[1] + nw[2] * s->light[2];
            if (sh < 0.0) sh = 0.0;
            for (int c = 0; c < 3; ++c) col[c] = sh * (double)s->albedo[c];
        }
        for (int c = 0; c < 3; ++c) {
            if (img) img[3 * i + c] = (float)col[c];
            if (target) {
                double d = col[c] - (double)target[3 * i + c];
                acc += d * d;
            }
        }
    }
    if (ids)
        for (int i = 0; i < npx; ++i) ids[i] = best_t[i];
    free(sx); free(sy); free(iz); free(zc); free(best_w); free(best_t);
    return acc / ((double)npx * 3.0);
}

/* ------------------------------------------------------------------------ */
/* Coloured-triangle rasteriser (stand-in for Box10 / mesh tasks).  Vertex   */
/* (x, y) in [0,1]^2 maps to pixels (x W, y H); both windings drawn (edge    */
/* coefficients negated when the signed area is negative); painter's order: */
/* the highest covering index wins.  p holds the optimised raw params.       */
/* ------------------------------------------------------------------------ */
double or_tris2d_loss(const or_tris2d_scene* s, const float* p, const float* target, float* img)
{
    const int W = s->W, H = s->H, nt = s->n_tris;
    float* raw = (float*)malloc(sizeof(float) * 9 * nt);
    memcpy(raw, s->raw, sizeof(float) * 9 * nt);
    for (int j = 0; j < s->n_params; ++j) raw[s->index[j]] = p[j];
    int npx = W * H;
    int* win = (int*)malloc(sizeof(int) * npx);
    for (int i = 0; i < npx; ++i) win[i] = -1;
    for (int t = 0; t < nt; ++t) {
        const float* q = raw + 9 * t;
        float ax = q[0] * (float)W, ay = q[1] * (float)H;
        float bx = q[2] * (float)W, by = q[3] * (float)H;
        float cx_ = q[4] * (float)W, cy_ = q[5] * (float)H;
        edge32 e0 = edge_of(bx, by, cx_, cy_);
        edge32 e1 = edge_of(cx_, cy_, ax, ay);
        edge32 e2 = edge_of(ax, ay, bx, by);
        float D2 = edge_eval(e2, cx_, cy_);
        if (D2 == 0.0f || D2 != D2) continue;
        if (D2 < 0.0f) {
            e0.A = -e0.A; e0.B = -e0.B; e0.C = -e0.C;
            e1.A = -e1.A; e1.B = -e1.B; e1.C = -e1.C;
            e2.A = -e2.A; e2.B = -e2.B; e2.C = -e2.C;
        }
        float minx = fmin3(ax, bx, cx_), maxx = fmax3(ax, bx, cx_);
        float miny = fmin3(ay, by, cy_), maxy = fmax3(ay, by, cy_);
        for (int y = 0; y < H; ++y) {
            float py = (float)y + 0.5f;
            if (py < miny || py > maxy) continue;
            for (int x = 0; x < W; ++x) {
                float px = (float)x + 0.5f;
                if (px < minx || px > maxx) continue;
                if (!edge_inside(e0, edge_eval(e0, px, py))) continue;
                if (!edge_inside(e1, edge_eval(e1, px, py))) continue;
                if (!edge_inside(e2, edge_eval(e2, px, py))) continue;
                win[y * W + x] = t;
            }
        }
    }
    double acc = 0.0;
    for (int i = 0; i < npx; ++i) {
        for (int c = 0; c < 3; ++c) {
            double v = win[i] >= 0 ? (double)raw[9 * win[i] + 6 + c] : 0.0;
            if (img) img[3 * i + c] = (float)v;
            if (target) {
                double d = v - (double)target[3 * i + c];
                acc += d * d;
            }
        }
    }
    free(raw); free(win);
    return acc / ((double)npx * 3.0);
}

/* ------------------------------------------------------------------------ */
/* Path tracer for the procedural box (stand-in for the Shadow task).        */
/* Primitives: 12 axis-aligned quads (index 0..11), the light quad (12,      */
/* horizontal, emitting downward), 3 spheres (13..15).  Rays and hits in     */
/* FP32 with the operation order below; radiance and throughput in FP64.     */
/* Path random numbers: Philox (pixel sample, (k << 8) | (vertex << 4) |     */
/* block, (tag << 24) | sub, request), key = seed; both legs of a pair share */
/* them.  Vertex 0 = camera (jitter); vertices 1..depth: block 0 words 0,1   */
/* pick the light point, words 2,3 the first disc try; blocks 1..3 hold      */
/* tries 1..6 (rejection from the square; all 7 rejected -> normal).         */
/* ------------------------------------------------------------------------ */
#define PT_NQUAD 12
#define PT_LIGHT 12
#define PT_NPRIM 16

typedef struct {
    int axis[13];
    float plane[13], lo_u[13], lo_v[13], hi_u[13], hi_v[13];
    float sc[3][3], sr[3];
} pt_geom;

static float u24(uint32_t x) { return (float)(x >> 8) * 0x1p-24f + 0x1p-25f; }
static float dot3f(const float* a, const float* b) { return fmaf(a[2], b[2], fmaf(a[1], b[1], a[0] * b[0])); }

static void pt_setup(const or_ptbox_scene* s, const float p[6], pt_geom* g)
{
    for (int q = 0; q < PT_NQUAD; ++q) {
        g->axis[q] = s->quad_axis[q];
        g->plane[q] = s->quad_geom[5 * q + 0];
        g->lo_u[q] = s->quad_geom[5 * q + 1];
        g->lo_v[q] = s->quad_geom[5 * q + 2];
        g->hi_u[q] = s->quad_geom[5 * q + 3];
        g->hi_v[q] = s->quad_geom[5 * q + 4];
    }
    g->axis[PT_LIGHT] = 1;
    g->plane[PT_LIGHT] = p[1];
    g->lo_u[PT_LIGHT] = p[0] - s->light_half;
    g->hi_u[PT_LIGHT] = p[0] + s->light_half;
    g->lo_v[PT_LIGHT] = p[2] - s->light_half;
    g->hi_v[PT_LIGHT] = p[2] + s->light_half;
    for (int i = 0; i < 3; ++i) {
        for (int c = 0; c < 3; ++c) g->sc[i][c] = i == 0 ? p[3 + c] : s->sph_center[3 * i + c];
        g->sr[i] = s->sph_radius[i];
    }
}

/* closest hit with t > 0; ties go to the lower primitive index.  Plane
 * distances use the ray's per-axis reciprocal: t = RN(RN(plane - o_a) * RN(1/d_a)). */
static int pt_intersect(const pt_geom* g, const float o[3], const float d[3], float* t_out)
{
    float best = INFINITY;
    int prim = -1;
    float inv[3];
    for (int c = 0; c < 3; ++c) inv[c] = 1.0f / d[c];
    for (int q = 0; q <= PT_LIGHT; ++q) {
        int a = g->axis[q];
        int u = a == 0 ? 1 : 0;
        int v = a == 2 ? 1 : 2;
        if (d[a] == 0.0f) continue;
        float t = (g->plane[q] - o[a]) * inv[a];
        if (!(t > 0.0f)) continue;
        float hu = fmaf(t, d[u], o[u]);
        float hv = fmaf(t, d[v], o[v]);
        if (hu < g->lo_u[q] || hu > g->hi_u[q] || hv < g->lo_v[q] || hv > g->hi_v[q]) continue;
        if (t < best) { best = t; prim = q; }
    }
    for (int i = 0; i < 3; ++i) {
        float oc[3] = {o[0] - g->sc[i][0], o[1] - g->sc[i][1], o[2] - g->sc[i][2]};
        float b = dot3f(oc, d);
        float cc = dot3f(oc, oc) - g->sr[i] * g->sr[i];
        float disc = fmaf(b, b, -cc);
        if (disc < 0.0f) continue;
        float sq = sqrtf(disc);
        float t = -b - sq;
        if (!(t > 0.0f)) {
            t = sq - b;
            if (!(t > 0.0f)) continue;
        }
        if (t < best) { best = t; prim = 13 + i; }
    }
    *t_out = best;
    return prim;
}

static void pt_normal(const pt_geom* g, int prim, const float x[3], const float d[3], float n[3])
{
    if (prim <= PT_LIGHT) {
        int a = g->axis[prim];
        n[0] = n[1] = n[2] = 0.0f;
        n[a] = d[a] > 0.0f ? -1.0f : 1.0f;
        return;
    }
    int i = prim - 13;
    float ir = 1.0f / g->sr[i];
    for (int c = 0; c < 3; ++c) n[c] = (x[c] - g->sc[i][c]) * ir;
    if (dot3f(n, d) > 0.0f) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
}

static const float* pt_albedo(const or_ptbox_scene* s, int prim)
{
    if (prim < PT_NQUAD) return s->quad_albedo + 3 * prim;
    if (prim >= 13) return s->sph_albedo + 3 * (prim - 13);
    return NULL;
}

static void pt_normalize(float v[3])
{
    float il = 1.0f / sqrtf(dot3f(v, v));
    v[0] = v[0] * il; v[1] = v[1] * il; v[2] = v[2] * il;
}

/* one path sample; adds its radiance to L */
/* cnt (may be NULL) counts closest-hit rays [0], shadow rays [1] and shaded
 * vertices [2] */
static void pt_path(const or_ptbox_scene* s, const pt_geom* g, int depth, uint64_t seed,
                    uint32_t request, uint32_t c2, uint32_t k, uint32_t idx,
                    const float o0[3], const float d0[3], double L[3], long long* cnt)
{
    double beta[3] = {1.0, 1.0, 1.0};
    float o[3] = {o0[0], o0[1], o0[2]}, d[3] = {d0[0], d0[1], d0[2]};
    float t;
    if (cnt) ++cnt[0];
    int prim = pt_intersect(g, o, d, &t);
    if (prim < 0) return;
    if (s->emit_all) {
        for (int c = 0; c < 3; ++c) L[c] += s->emission[c];
    } else if (prim == PT_LIGHT) {
        if (d[1] > 0.0f) for (int c = 0; c < 3; ++c) L[c] += s->emission[c];
        return;
    }
    for (int v = 1; v <= depth; ++v) {
        if (prim == PT_LIGHT && !s->emit_all) return;
        float x[3], n[3], o2[3];
        for (int c = 0; c < 3; ++c) x[c] = fmaf(t, d[c], o[c]);
        pt_normal(g, prim, x, d, n);
        for (int c = 0; c < 3; ++c) o2[c] = fmaf(n[c], 1e-4f, x[c]);
        const float* rho = s->emit_all && prim == PT_LIGHT ? s->quad_albedo : pt_albedo(s, prim);
        if (cnt) ++cnt[2];
        uint32_t w0[4];
        philox_words(seed, idx, (k << 8) | ((uint32_t)v << 4) | 0u, c2, request, w0);
        if (s->nee) {
            float ly[3];
            float ul1 = u24(w0[0]), ul2 = u24(w0[1]);
            ly[0] = fmaf(ul1, g->hi_u[PT_LIGHT] - g->lo_u[PT_LIGHT], g->lo_u[PT_LIGHT]);
            ly[1] = g->plane[PT_LIGHT];
            ly[2] = fmaf(ul2, g->hi_v[PT_LIGHT] - g->lo_v[PT_LIGHT], g->lo_v[PT_LIGHT]);
            float wv[3] = {ly[0] - o2[0], ly[1] - o2[1], ly[2] - o2[2]};
            float dist2 = dot3f(wv, wv);
            float idist = 1.0f / sqrtf(dist2);
            float om[3] = {wv[0] * idist, wv[1] * idist, wv[2] * idist};
            float cosx = dot3f(n, om);
            float cosl = om[1];
            if (cosx > 0.0f && cosl > 0.0f) {
                float ts;
                if (cnt) ++cnt[1];
                int ps = pt_intersect(g, o2, om, &ts);
                if (ps == PT_LIGHT) {
                    double area = ((double)g->hi_u[PT_LIGHT] - g->lo_u[PT_LIGHT]) *
                                  ((double)g->hi_v[PT_LIGHT] - g->lo_v[PT_LIGHT]);
                    double geo = (double)cosx * (double)cosl / (double)dist2 * area;
                    for (int c = 0; c < 3; ++c)
                        L[c] += beta[c] * (double)rho[c] / OR_PI * (double)s->emission[c] * geo;
                }
            }
        }
        if (v == depth) return;
        /* cosine-weighted direction (Malley): uniform disc point lifted to
         * the hemisphere; disc point by rejection from the square */
        float a = 0.0f, b = 0.0f;
        int found = 0;
        for (int tr = 0; tr < 7 && !found; ++tr) {
            uint32_t wb[4];
            const uint32_t* src;
            int off;
            if (tr == 0) { src = w0; off = 2; }
            else {
                philox_words(seed, idx, (k << 8) | ((uint32_t)v << 4) | (uint32_t)((tr + 1) / 2), c2, request, wb);
                src = wb;
                off = (tr % 2 == 1) ? 0 : 2;
            }
            float ta = fmaf(u24(src[off]), 2.0f, -1.0f);
            float tb = fmaf(u24(src[off + 1]), 2.0f, -1.0f);
            if (fmaf(ta, ta, tb * tb) < 1.0f) { a = ta; b = tb; found = 1; }
        }
        float r2 = fmaf(a, a, b * b);
        float cz = sqrtf(1.0f - r2);
        /* orthonormal basis around n (Duff et al., "Building an Orthonormal
         * Basis, Revisited", JCGT 2017) */
        float sg = copysignf(1.0f, n[2]);
        float aa = -1.0f / (sg + n[2]);
        float bb = (n[0] * n[1]) * aa;
        float t1[3] = {fmaf(sg * (n[0] * n[0]), aa, 1.0f), sg * bb, -(sg * n[0])};
        float t2[3] = {bb, fmaf(n[1] * n[1], aa, sg), -n[1]};
        float nd[3];
        for (int c = 0; c < 3; ++c) nd[c] = fmaf(cz, n[c], fmaf(b, t2[c], a * t1[c]));
        for (int c = 0; c < 3; ++c) beta[c] *= (double)rho[c];
        if (cnt) ++cnt[0];
        prim = pt_intersect(g, o2, nd, &t);
        if (prim < 0) return;
        if (s->emit_all)
            for (int c = 0; c < 3; ++c) L[c] += beta[c] * s->emission[c];
        for (int c = 0; c < 3; ++c) { o[c] = o2[c]; d[c] = nd[c]; }
    }
}

double or_ptbox_render(const or_ptbox_scene* s, const float p[6], int spp, int depth,
                       uint64_t seed, uint32_t request, uint32_t sub, uint32_t k,
                       uint32_t tag, const float* target, double* img)
{
    return or_ptbox_render_counted(s, p, spp, depth, seed, request, sub, k, tag, target, img, 0);
}

/* The path tracer; also adds, if cnt is not NULL, its closest-hit rays,
 * shadow rays and shaded vertices to cnt[0..2]. */
double or_ptbox_render_counted(const or_ptbox_scene* s, const float p[6], int spp, int depth,
                               uint64_t seed, uint32_t request, uint32_t sub, uint32_t k,
                               uint32_t tag, const float* target, double* img, long long* cnt)
{
    pt_geom g;
    pt_setup(s, p, &g);
    const int W = s->W, H = s->H;
    uint32_t c2 = (tag << 24) | (sub & 0xFFFFFFu);
    double acc = 0.0;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            double L[3] = {0.0, 0.0, 0.0};
            for (int sidx = 0; sidx < spp; ++sidx) {
                uint32_t idx = (uint32_t)((y * W + x) * spp + sidx);
                uint32_t wj[4];
                philox_words(seed, idx, k << 8, c2, request, wj);
                float fx = (float)x + u24(wj[0]);
                float fy = (float)y + u24(wj[1]);
                float d[3] = {fmaf(fx, s->pix_scale, -s->tan_half), fmaf(-fy, s->pix_scale, s->tan_half), -1.0f};
                pt_normalize(d);
                float o[3] = {0.0f, 0.0f, s->cam_z};
                pt_path(s, &g, depth, seed, request, c2, k, idx, o, d, L, cnt);
            }
            int i = y * W + x;
            for (int c = 0; c < 3; ++c) {
                double v = L[c] / (double)spp;
                if (img) img[3 * i + c] = v;
                if (target) {
                    double df = v - (double)target[3 * i + c];
                    acc += df * df;
                }
            }
        }
    }
    return acc / ((double)W * (double)H * 3.0);
}

/* Exposed for pins: one ray's closest hit, and one path from a given ray. */
int or_ptbox_intersect(const or_ptbox_scene* s, const float p[6], const float o[3],
                       const float d[3], float* t)
{
    pt_geom g;
    pt_setup(s, p, &g);
    return pt_intersect(&g, o, d, t);
}

void or_ptbox_trace(const or_ptbox_scene* s, const float p[6], const float o[3], const float d[3],
                    int depth, uint64_t seed, uint32_t request, uint32_t sub, uint32_t k,
                    uint32_t tag, uint32_t idx, double out[3])
{
    pt_geom g;
    pt_setup(s, p, &g);
    out[0] = out[1] = out[2] = 0.0;
    pt_path(s, &g, depth, seed, request, (tag << 24) | (sub & 0xFFFFFFu), k, idx, o, d, out, 0);
}

/* p = RN32(RN32(theta) + tau): the perturbed parameters every renderer sees */
void or_perturb(int n, const double* theta, const float* tau, float* p)
{
    for (int j = 0; j < n; ++j) p[j] = (float)theta[j] + tau[j];
}

/* Element-wise HVP draws: P pairs for output row i from its |v|-weighted
 * row mixture (v is read during the call only). */
int or_draw_hvp_rows(int n, double sigma, const double* v, int64_t P, uint64_t seed,
                     uint32_t request, uint32_t sub, int row, float* tau, int32_t* comp_out)
{
    g_row_v = v;
    int rc = or_draw(1, n, sigma, P, seed, request, sub, row, -2, tau, comp_out);
    g_row_v = 0;
    return rc;
}
