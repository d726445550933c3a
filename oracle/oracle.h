/*
 * Oracle for the stochastic Hessian / HVP / gradient estimator of a
 * Gaussian-smoothed rendering loss (Wang, Fischer, Ritschel, "Stochastic
 * Gradient Estimation for Higher-order Differentiable Rendering").
 *
 * TEST INFRASTRUCTURE ONLY.  A plain, slow, single-threaded CPU restatement
 * of the method in FP64.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * Precision rule: every value (kernel weights, lobe samples before their
 * final rounding, shading, radiance, losses, sums) is FP64.  Where floating
 * point decides a discrete outcome inside the renderer (pixel coverage,
 * depth order, ray hit/miss, which primitive is closest, NEE validity,
 * rejection of a disc sample) the decision is taken in FP32 with the
 * operation sequence that defines the renderer, because the renderer under
 * test renders in FP32.
 */
#ifndef HR_ORACLE_H
#define HR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- counter-based RNG (Salmon et al., SC'11) ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_u01(uint32_t x);                 /* (x + 1/2) 2^-32 */

/* ---- Lambert W and the diagonal-lobe CDF (Sec. 3.3, Suppl. D) ---- */
double or_lambertw(double z, int branch);  /* branch 0 or -1, z in [-1/e, 0) */
double or_diag_cdf(double t);              /* t = tau / sigma */
double or_diag_inv_cdf(double c);          /* exact inverse, FP64 */

/* ---- lobe masses ---- */
double or_Zg(double sigma);
double or_Zd(double sigma);
double or_Zo(double sigma);

/* ---- sampling (Sec. 3.2-3.5) ----
 * lobe: 0 = gradient lobes, 1 = Hessian lobes.
 * comp_i = -1: aggregate (component drawn from Philox word 0).
 * comp_i = -3: no importance sampling: tau ~ N(0, s^2 I), legs +tau / -tau.
 * comp_i >= 0: element-wise importance sampling of element (comp_i, comp_j)
 *              (comp_j ignored for gradient lobes).
 * Writes tau[2P][n] as FP32 (the canonical perturbation) and, when comp_out is
 * not NULL, the drawn component (i*n+j, or i for gradient lobes) per pair.
 */
int or_draw(int lobe, int n, double sigma, int64_t P, uint64_t seed,
            uint32_t request, uint32_t sub, int comp_i, int comp_j,
            float* tau, int32_t* comp_out);

/* Element-wise HVP (Tab. 1 IS column): pairs for output row `row`, component
 * (row, j) drawn with probability |v_j| Z_rowj / sum_l |v_l| Z_rowl. */
int or_draw_hvp_rows(int n, double sigma, const double* v, int64_t P, uint64_t seed,
                     uint32_t request, uint32_t sub, int row, float* tau, int32_t* comp_out);

/* ---- estimator weights ----
 * quantity: 0 = gradient (E = n), 1 = Hessian upper triangle (E = n(n+1)/2),
 *           2 = HVP (E = n, needs v), 3 = element-wise HVP of row comp_i
 *           (E = n, needs v; weight h_i^v / q_i of the row mixture).
 * For element-wise sampling (comp_i >= 0) the weight is +-Z of that element
 * and zero elsewhere.  Weights are evaluated at the FP32 perturbation.
 */
int or_weights(int quantity, int n, double sigma, const double* v, int64_t M,
               const float* tau, int comp_i, int comp_j, double* w);

/* ---- renderers: loss of one image against a target ---- */
/* disc: value 1 inside radius r of the centre p, else 0; grayscale. */
/* squares: K axis-aligned squares of half-size h centred at p[2s], p[2s+1]. */
double or_boxes_loss(int W, int H, int K, float h, const float* p, const float* target, float* img);
double or_disc_loss(int W, int H, float r, const float p[2], const float* target, float* img);

typedef struct {
    int W, H, nv, nt;
    const float* verts;      /* nv x 3 */
    const int32_t* tris;     /* nt x 3 */
    float albedo[3], light[3];
    float eye_dist, scale;
} or_revolve_scene;
double or_revolve_loss(const or_revolve_scene* s, const float p[2], const float* target, float* img);
double or_revolve_render(const or_revolve_scene* s, const float p[2], const float* target, float* img, int* ids);

typedef struct {
    int W, H, n_tris, n_params;
    const float* raw;        /* n_tris x 9 : x0 y0 x1 y1 x2 y2 r g b */
    const int32_t* index;    /* n_params indices into raw */
} or_tris2d_scene;
double or_tris2d_loss(const or_tris2d_scene* s, const float* p, const float* target, float* img);

typedef struct {
    int W, H;
    const int32_t* quad_axis;   /* 12 */
    const float* quad_geom;     /* 12 x 5: plane, lo_u, lo_v, hi_u, hi_v */
    const float* quad_albedo;   /* 12 x 3 */
    const float* sph_center;    /* 3 x 3 (sphere 0 centre replaced by params) */
    const float* sph_radius;    /* 3 */
    const float* sph_albedo;    /* 3 x 3 */
    float light_half, cam_z, tan_half, pix_scale;
    float emission[3];
    int emit_all;               /* furnace mode: every surface emits `emission` to camera rays */
    int nee;                    /* 1 = next-event estimation on */
} or_ptbox_scene;
/* Renders at params p (light centre xyz, sphere-0 centre xyz) with `spp`
 * samples per pixel and the path random numbers of (seed, request, sub,
 * pair k, tag); returns the loss against target (if not NULL) and writes the
 * FP64 image into img (W*H*3, may be NULL). */
double or_ptbox_render(const or_ptbox_scene* s, const float p[6], int spp, int depth,
                       uint64_t seed, uint32_t request, uint32_t sub, uint32_t k,
                       uint32_t tag, const float* target, double* img);
double or_ptbox_render_counted(const or_ptbox_scene* s, const float p[6], int spp, int depth,
                               uint64_t seed, uint32_t request, uint32_t sub, uint32_t k,
                               uint32_t tag, const float* target, double* img, long long* cnt);

/* one ray's closest primitive (-1 = none) and its distance */
int or_ptbox_intersect(const or_ptbox_scene* s, const float p[6], const float o[3],
                       const float d[3], float* t);
/* radiance of one path from ray (o, d) with path sample index idx */
void or_ptbox_trace(const or_ptbox_scene* s, const float p[6], const float o[3], const float d[3],
                    int depth, uint64_t seed, uint32_t request, uint32_t sub, uint32_t k,
                    uint32_t tag, uint32_t idx, double out[3]);

/* p_j = RN32(RN32(theta_j) + tau_j) */
void or_perturb(int n, const double* theta, const float* tau, float* p);

#ifdef __cplusplus
}
#endif
#endif
