/*
 * hr — stochastic gradient, Hessian and Hessian-vector-product estimation of
 * a Gaussian-smoothed rendering loss on one GB300 GPU (sm_103a).
 *
 * Method: Wang, Fischer, Ritschel, "Stochastic Gradient Estimation for
 * Higher-order Differentiable Rendering".  The loss f(theta) (a renderer
 * followed by an image-space L2 loss against a target) is smoothed by a
 * Gaussian in parameter space,
 *     fbar(theta) = E_{tau ~ N(0, sigma^2 I)} f(theta + tau)         (Sec. 3.1)
 * and its derivatives are estimated by Monte Carlo over perturbations tau
 * drawn by importance sampling the positive and negative lobes of the
 * Gaussian derivative kernels: gradient (Sec. 3.2, Eq. "gradient"),
 * Hessian (Sec. 3.3), HVP (Sec. 3.4) and the aggregate strategy that samples
 * the mixture of all element kernels and renders once per sample (Sec. 3.5,
 * Tab. 1).  Each estimate is
 *     est_e = 1/(2P) * sum_m w_e(tau_m) * f(theta + tau_m)
 * over the 2P perturbations (P antithetic +/- pairs) of a request.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: HR_OK (0) or a negative hr_status.  No exception crosses
 *   the ABI.  hr_last_error() gives a message for the calling thread's most
 *   recent failure.
 * - Memory: pointers named h_* / plain are HOST memory; pointers named d_*
 *   are DEVICE memory of the current CUDA device.  The library copies what it
 *   needs and never frees or retains caller memory after a call returns.
 * - Streams: opts->stream (a cudaStream_t, NULL = the library's own stream;
 *   to run on the legacy default stream pass cudaStreamLegacy).
 *   Host-pointer calls are synchronous; the *_dev call is asynchronous on
 *   that stream.
 * - Validation happens before any launch: n must match the scene, M even and
 *   >= 2, sigma > 0, sizes within the stated maxima; otherwise
 *   HR_ERR_INVALID_ARG and nothing is launched.
 * - Thread safety: calls on different scenes may run concurrently from
 *   different threads; calls on one scene are serialised by the library.
 */
#ifndef HR_H
#define HR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hr_status;
#define HR_OK 0
#define HR_ERR_INVALID_ARG (-1)
#define HR_ERR_OOM (-2)
#define HR_ERR_CUDA (-3)
#define HR_ERR_TIMEOUT (-4)
#define HR_ERR_BUSY (-5)
#define HR_ERR_UNSUPPORTED (-6)

/* Scene kinds (synthetic stand-ins for the paper's tasks, Sec. 4.1):
 * DISC2D     one hard-edged disc, 2 params (centre x, y in [0,1]^2), grayscale;
 * REVOLVE3D  closed triangle mesh of a surface of revolution, 2 params
 *            (rotation about x, then y), flat Lambert shading, RGB;
 * PTBOX      path-traced box: 12 axis-aligned quads, 3 spheres, 1 emitting
 *            quad; 6 params (light centre xyz, sphere-0 centre xyz), RGB;
 * TRIS2D     coloured 2D triangles drawn in painter's order; params are a
 *            subset (param_index) of the 9 raw values per triangle
 *            (x0 y0 x1 y1 x2 y2 r g b);
 * BOXES2D    K = n_params / 2 axis-aligned squares (the Box2 / Box10 plateau
 *            tasks), params = square centres, grayscale; a pixel centre is 1
 *            inside any square (|dx| < h and |dy| < h in FP32);
 * analytic test functions in place of a renderer (the "loss" is f(p) itself,
 * evaluated in FP64 at the FP32 perturbed parameters and stored in FP32; the
 * image is 1 x 1 x 1 holding f; no target):
 * QUADRATIC  f = 1/2 p^T A p + b^T p (quad_A [n][n] row-major, quad_b [n]);
 *            its smoothed gradient is A theta + b and Hessian (A + A^T)/2
 *            exactly;
 * STEP1D     f = 1 if p_0 > 0 else 0 (n = 1), the 1D hard edge;
 * NEGGAUSS   f = -exp(-|p|^2 / (2 s^2)) / (2 pi s^2)^(n/2), s = gauss_sigma;
 *            smoothing gives -N(0, (s^2 + sigma^2) I). */
#define HR_SCENE_DISC2D 0
#define HR_SCENE_REVOLVE3D 1
#define HR_SCENE_PTBOX 2
#define HR_SCENE_TRIS2D 3
#define HR_SCENE_BOXES2D 4
#define HR_SCENE_QUADRATIC 5
#define HR_SCENE_STEP1D 6
#define HR_SCENE_NEGGAUSS 7

/* Sampling strategy: element-wise importance sampling (one sample set of M
 * perturbations per unique element: n for the gradient, n(n+1)/2 for the
 * Hessian, n rows for the HVP; Tab. 1 IS column), aggregate sampling (one set
 * of M for all elements, Tab. 1 AIS column), or no importance sampling
 * (tau ~ N(0, sigma^2 I) with antithetic legs +tau / -tau, weight = the kernel
 * factor; Tab. 1 no-IS column). */
#define HR_ELEMENTWISE 0
#define HR_AGGREGATE 1
#define HR_PLAIN 2

/* Estimated quantity */
#define HR_GRAD 0
#define HR_HESSIAN 1
#define HR_HVP 2

/* Maxima (validated) */
#define HR_MAX_PARAMS 64
#define HR_MAX_IMAGE_SIDE 1024
#define HR_MAX_TRIANGLES 4096
#define HR_MAX_VERTICES 4096
#define HR_MAX_TRIS2D 32

typedef struct hr_scene_s* hr_scene;

/* Scene description.  All arrays are host memory, read during
 * hr_create_scene only.  Fields that a kind does not use are ignored. */
typedef struct {
    int32_t kind;                 /* HR_SCENE_* */
    int32_t width, height;        /* image size in pixels */
    int32_t n_params;             /* DISC2D 2, REVOLVE3D 2, PTBOX 6, TRIS2D = len(param_index),
                                     BOXES2D 2K (K <= 32) */
    const double* theta_target;   /* [n_params] target parameters */
    const float* target_image;    /* optional [H][W][C] FP32 (C = 1 for DISC2D, else 3);
                                     NULL: the library renders it at theta_target */
    /* DISC2D: disc radius; BOXES2D: square half-size */
    float radius;
    /* REVOLVE3D: model-space vertices [n_vertices][3], triangles [n_triangles][3]
       (outward winding), albedo RGB, unit light direction, camera distance on +z
       and projection scale (pixels per unit of X/Z).  One render's triangle
       records, projected vertices and tile bins live in shared memory: 78 B
       per triangle, 12 B per vertex, 8 B per raster tile (8x4 pixels, or 8x8
       where fewer than 8,192 bin entries would fit) and at least 2,048 bin
       entries of 4 B, within the 227 KB one CTA may use: about 2,400 triangles
       at 256x256 on a GB300; larger meshes are rejected with
       HR_ERR_UNSUPPORTED.  Where records of half the triangles (the ones that
       survive culling, by slot) and 4,096 bin entries also fit half an SM,
       two renders share each SM (the compact layout; mesh_compact_slots in
       hr_scene_stats), and a render that does not fit it is rendered again
       in the full layout.  Both layouts take the same coverage and depth
       decisions; they sum the per-tile losses in different orders.  At most
       HR_MAX_VERTICES vertices and HR_MAX_TRIANGLES triangles (else
       HR_ERR_INVALID_ARG). */
    const float* vertices;
    int32_t n_vertices;
    const int32_t* triangles;
    int32_t n_triangles;
    float albedo[3];
    float light[3];
    float eye_dist;
    float scale;
    /* TRIS2D: raw params [n_tris][9] (n_tris <= 32), optimised subset
       param_index[n_params] (n_params <= 64) */
    const float* raw_params;
    int32_t n_tris;
    const int32_t* param_index;
    /* PTBOX: quads [12] (axis, {plane, lo_u, lo_v, hi_u, hi_v}, albedo RGB),
       spheres [3] (centre xyz, radius, albedo RGB; sphere 0 centre = params 3..5),
       light half-size, camera z, tan(fov/2), pixel scale 2 tan(fov/2)/H,
       emitted radiance RGB, samples per pixel, target samples per pixel,
       path depth, and the seed of the target's path random numbers */
    const int32_t* quad_axis;
    const float* quad_geom;
    const float* quad_albedo;
    const float* sph_center;
    const float* sph_radius;
    const float* sph_albedo;
    float light_half, cam_z, tan_half, pix_scale;
    float emission[3];
    int32_t spp, target_spp, depth;
    uint64_t seed;
    /* QUADRATIC: A [n][n] row-major and b [n] (FP64); NEGGAUSS: s.  The
       analytic kinds need neither theta_target nor target_image. */
    const double* quad_A;
    const double* quad_b;
    double gauss_sigma;
} hr_scene_desc;

/* Options of one estimate. */
typedef struct {
    double sigma;          /* smoothing bandwidth, > 0 */
    int64_t n_perturb;     /* M: renders per request (aggregate) or per unique
                              element (element-wise); even, >= 2 */
    int32_t strategy;      /* HR_ELEMENTWISE, HR_AGGREGATE or HR_PLAIN */
    uint64_t seed;         /* Philox key */
    uint32_t request_id;   /* Philox counter word 3 */
    uint32_t sub;          /* first sub-stream (counter word 2, low 24 bits);
                              element e of element-wise sampling uses sub + e */
    void* stream;          /* cudaStream_t or NULL */
    /* Optional HOST outputs for inspection (may be NULL), in launch order
       m = group * M + 2k + leg (leg 0 = + lobe):
       out_tau [M_total][n] FP32 perturbations, out_weights [M_total][E] FP32,
       out_losses [M_total] FP32 per-render losses, out_scale [E] FP64
       A_e = 1/(2P) sum_m |w_e f_m|. */
    float* out_tau;
    float* out_weights;
    float* out_losses;
    double* out_scale;
} hr_opts;

/* Create a scene: uploads geometry, renders the target when target_image is
 * NULL, and allocates its device workspace.  *out receives the handle. */
hr_status hr_create_scene(const hr_scene_desc* desc, hr_scene* out);
hr_status hr_destroy_scene(hr_scene scene);

/* Smoothed gradient (Sec. 3.2): h_theta [n] host, h_out_g [n] host. */
hr_status hr_estimate_grad(hr_scene scene, const double* h_theta, const hr_opts* opts, double* h_out_g);

/* Smoothed Hessian (Sec. 3.3, 3.5): h_out_H [n][n] row-major, symmetric. */
hr_status hr_estimate_hessian(hr_scene scene, const double* h_theta, const hr_opts* opts, double* h_out_H);

/* Smoothed Hessian-vector product (Sec. 3.4, 3.5): the HVP kernel
 * sum_j h_ij v_j.  Aggregate: sampled from the Hessian mixture (M renders),
 * so that on the same samples it equals the aggregate Hessian times v.
 * Element-wise (Tab. 1 IS column, n sample sets of M): output row i draws
 * lobe (i, j) with probability |v_j| Z_ij / sum_l |v_l| Z_il and is weighted by
 * the row kernel over that mixture. */
hr_status hr_estimate_hvp(hr_scene scene, const double* h_theta, const double* h_v,
                          const hr_opts* opts, double* h_out_Hv);

/* HVP as the central difference of two smoothed-gradient estimates,
 * (g(theta + eps v) - g(theta - eps v)) / (2 eps) (Sec. 2 central differences
 * of gradients; Sec. 3.4), both estimates on the same perturbations (common
 * random numbers): one sampling pass, 2 M renders per sample set (element-wise
 * gradient: n sets).  theta +- eps v is formed in FP64 and rounded to FP32.
 * Inspection outputs in opts are ignored.  eps > 0. */
hr_status hr_estimate_hvp_fd(hr_scene scene, const double* h_theta, const double* h_v, double eps,
                             const hr_opts* opts, double* h_out_Hv);

/* Grey-box composition (Suppl. "Grey-box differentials"): the loss is
 * f(g(x)) with a white-box inner map g, whose Jacobian J = dg/dx at x the
 * caller supplies (h_J [n][n_x] row-major, n = the scene's parameter count),
 * and the black-box renderer loss f, estimated at y = g(x) (h_y [n]).
 *   HR_GRAD:    h_out [n_x]       = J^T grad_y fbar(y)
 *   HR_HESSIAN: h_out [n_x][n_x]  = J^T H_y J  (n_x <= 4096; drops the curvature
 *                                   of g, exact when g is affine)
 *   HR_HVP:     h_out [n_x]       = J^T H_y (J h_vx), h_vx [n_x]
 * The products with J run on the device in FP64; opts as for the estimates
 * (inspection outputs ignored).  1 <= n_x <= 2^24. */
hr_status hr_estimate_greybox(hr_scene scene, int32_t quantity, const double* h_y, const double* h_J, int32_t n_x,
                              const double* h_vx, const hr_opts* opts, double* h_out);

/* Device-pointer form of the three estimates, asynchronous on opts->stream:
 * d_theta [n], d_v [n] (HVP only, else NULL), d_out [n], [n][n] or [n]
 * FP64 device memory.  Debug outputs in opts are ignored.  Every estimate on
 * a scene works in that scene's one workspace: calls are serialised on the
 * host, but on the device two calls on the same scene must not overlap, so
 * issue them on one stream (or order the streams).  Independent estimates run
 * concurrently on separate scenes or through the server. */
hr_status hr_estimate_dev(hr_scene scene, int32_t quantity, const double* d_theta, const double* d_v,
                          const hr_opts* opts, double* d_out);

/* Device-pointer estimate that allocates nothing.  Same arguments, results
 * and stream behaviour as hr_estimate_dev (bit-identical outputs: the same
 * kernels run in the same order on the same values); the paper has no
 * counterpart.  Inspection outputs in opts are ignored.
 *
 * For callers that cannot allocate device memory while they run: real-time
 * or latency-bound loops that must not take the allocator's locks or pay the
 * device-wide synchronisation that cudaFree implies, and host applications
 * that hand the library a fixed device-memory budget up front and forbid
 * allocations outside it.  Its working memory is one fixed 4 MiB array of
 * device memory inside the library, present on every GPU that loads the
 * library until the process exits; a request needing more than that (about
 * 130,000 perturbations for a 2 x 2 aggregate Hessian, fewer for larger n)
 * fails with HR_ERR_INVALID_ARG before anything is launched, and
 * hr_estimate_dev remains the entry point for such requests.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents (every call overwrites all of it that it reads, so
 * nothing needs clearing): two calls that can run at the same time on the GPU
 * (different streams, or work not ordered one after the other) race and
 * corrupt each other's results, so issue them in order on one stream.  On
 * the host the call takes the scene's lock like every other call on the
 * scene. */
hr_status hr_estimate_dev_noalloc(hr_scene scene, int32_t quantity, const double* d_theta, const double* d_v,
                                  const hr_opts* opts, double* d_out);

/* ---------------------------------------------------------------------------
 * Newton-CG (Sec. 2 "Newton Conjugate Gradient"): per step and instance, an
 * aggregate gradient estimate g, then K linear-CG iterations on
 * (H + lambda I) d = -g from d = 0, each Hessian product an aggregate HVP with
 * fresh samples; alpha = r.r / p.(H + lambda I)p capped at Delta/|p| (the
 * paper's trust-region step truncation), Fletcher-Reeves beta, exit on
 * non-positive curvature (first iteration: step Delta along -g);
 * lambda = lambda_rel |g|; theta += d.  B instances share the scene and run in
 * the same launches; with use_graph the step is one CUDA graph replay.
 * Sub-streams: gradient 64 s, product i: 64 s + 1 + i (s = step index);
 * request id of instance b = request_base + b.
 * ------------------------------------------------------------------------- */
typedef struct hr_optstate_s* hr_optstate;

typedef struct {
    double sigma;
    int32_t n_grad;        /* perturbations for the gradient (even) */
    int32_t n_hvp;         /* perturbations per Hessian product (even) */
    int32_t cg_iters;      /* K <= 63 */
    double lambda_rel;     /* lambda = lambda_rel * |g| */
    double trust_radius;   /* Delta */
    uint64_t seed;
    uint32_t request_base;
    int32_t use_graph;     /* 1: capture the step once, replay it */
    void* stream;
} hr_cg_opts;

typedef struct {
    double grad_norm;
    double lambda;
    int32_t iters;         /* CG iterations taken */
    int32_t exit_reason;   /* 0 max iterations, 1 non-positive curvature, 2 zero residual */
    double step_norm;
} hr_step_info;

hr_status hr_optstate_create(hr_scene scene, int32_t n_instances, const double* h_theta0,
                             const hr_cg_opts* opts, hr_optstate* out);
hr_status hr_optstate_destroy(hr_optstate st);
/* One step for all instances; h_info [n_instances] may be NULL. */
hr_status hr_newton_cg_step(hr_scene scene, hr_optstate st, hr_step_info* h_info);
/* Current parameters, h_theta [n_instances][n]. */
hr_status hr_optstate_theta(hr_optstate st, double* h_theta);
/* What the last step computed, for inspection (waits for the state's
 * stream): h_g [n_instances][n] the gradient estimates, h_p
 * [n_instances][cg_iters][n] the CG directions p_i and h_Hp (same shape) the
 * aggregate HVP estimates of H p_i (without the lambda p_i term), all at the
 * step's starting parameters; rows i >= hr_step_info.iters are unspecified.
 * Any pointer may be NULL. */
hr_status hr_optstate_trace(hr_optstate st, double* h_g, double* h_p, double* h_Hp);

/* ---------------------------------------------------------------------------
 * The optimiser as the paper runs it (Sec. 2 "Newton Conjugate Gradient" with
 * the point moved at every iteration; Suppl. "Hyperparameters": linear sigma
 * annealing, line-search iterations and tolerance, recompute period, trust
 * region).  Per instance it keeps x, a direction d, a residual r and an outer
 * iteration counter i.  One evaluation is one line-search step at the
 * current x:
 *   g = aggregate gradient estimate at x (n_grad perturbations, sub 64 e),
 *   Hd = aggregate Hessian-vector product at x (n_hvp perturbations, sub
 *        64 e + 1; the perturbations do not depend on d) plus lambda d,
 *        lambda = lambda_rel |g|;
 *   at the first step of outer iteration i the direction is updated:
 *     i % recompute == 0: r = d = -g (recompute / restart),
 *     else r' = r (residual_mode 0, the printed recurrence) or -g (mode 1),
 *          d = r' + (r'.r' / r.r) d (Fletcher-Reeves), d = r' if r'.d <= 0;
 *   alpha = -g.d / d.Hd (Eq. pertubation), or +-Delta/|d| downhill when
 *   d.Hd <= 0; |alpha| <= Delta/|d| (trust region); x += alpha d; mode 0
 *   also r -= alpha Hd;
 *   the line search ends after ls_iters steps or once |alpha| |d| <= ls_tol;
 *   then i += 1 and sigma_i = sigma_start + (sigma_end - sigma_start) i/(T-1)
 *   (sigma_end from i >= T-1; T = anneal_iters, T = 1: sigma_start always).
 * Each instance follows its own line search, so instances in one launch can
 * be at different outer iterations and bandwidths.  Request id of instance b
 * = request_base + b; evaluation e counts from 0 per state (at most 262,144).
 * Limits: n <= 64, n_hvp <= 512, 1 <= n_instances <= 4096.
 * ------------------------------------------------------------------------- */
typedef struct hr_ncg_s* hr_ncg;

typedef struct {
    double sigma_start;
    double sigma_end;
    int32_t anneal_iters;  /* T >= 1 */
    int32_t n_grad;        /* perturbations per gradient estimate (even, >= 2) */
    int32_t n_hvp;         /* perturbations per Hessian product (even, 2..512) */
    int32_t ls_iters;      /* J >= 1 */
    double ls_tol;         /* line search ends once |alpha| |d| <= ls_tol */
    int32_t recompute;     /* R >= 1 */
    int32_t residual_mode; /* 0 recurrence r -= alpha Hd, 1 r = -g each outer iteration */
    double trust_radius;   /* Delta > 0 */
    double lambda_rel;     /* >= 0 */
    uint64_t seed;
    uint32_t request_base;
    int32_t use_graph;     /* 1: capture one evaluation into a CUDA graph, replay it */
    void* stream;          /* cudaStream_t or NULL (own stream) */
} hr_ncg_opts;

typedef struct {
    int32_t iter;          /* outer iteration i of this evaluation */
    int32_t ls_step;       /* line-search step within it (0: direction updated here) */
    int32_t restarted;     /* 1: r and d were reset to -g here */
    int32_t pad;
    double sigma;          /* bandwidth the estimates used */
    double grad_norm;      /* |g| */
    double gd;             /* g.d */
    double dHd;            /* d.(H + lambda I) d */
    double alpha;          /* step along d after truncation */
    double step_norm;      /* |alpha| |d| */
} hr_ncg_info;

/* Allocates the state (device memory for B instances) and copies h_theta0
 * [n_instances][n]; returns HR_ERR_INVALID_ARG on bad options, HR_ERR_OOM if
 * device memory runs out.  The state belongs to `scene`. */
hr_status hr_ncg_create(hr_scene scene, int32_t n_instances, const double* h_theta0, const hr_ncg_opts* opts,
                        hr_ncg* out);
hr_status hr_ncg_destroy(hr_ncg st);
/* Runs n_evals evaluations for all instances and waits for them.  h_info, if
 * not NULL, receives [n_evals][n_instances] records. */
hr_status hr_ncg_run(hr_scene scene, hr_ncg st, int32_t n_evals, hr_ncg_info* h_info);
/* Current parameters, h_theta [n_instances][n] (waits for the state's stream). */
hr_status hr_ncg_theta(hr_ncg st, double* h_theta);
/* What the last evaluation computed, for inspection (waits for the state's
 * stream): h_g [n_instances][n] the gradient estimates, h_d the direction d
 * the evaluation stepped along and h_Hd the aggregate HVP estimates of H d
 * (without the lambda d term), all at the evaluation's starting point.  Any
 * pointer may be NULL. */
hr_status hr_ncg_trace(hr_ncg st, double* h_g, double* h_d, double* h_Hd);

/* Render one image at h_params [n] (rounded to FP32) into h_img [H][W][C]
 * (host).  For PTBOX the path random numbers are those of (seed, request,
 * sub, pair k, tag) with spp samples per pixel (tag 2: perturbation renders,
 * tag 3: the target); other kinds ignore these arguments.  Used to compare
 * renderers pixel by pixel. */
hr_status hr_render(hr_scene scene, const double* h_params, uint64_t seed, uint32_t request, uint32_t sub,
                    uint32_t k, uint32_t tag, int32_t spp, float* h_img);

/* Mesh scenes (REVOLVE3D) only: the index of the triangle each pixel shows
 * at h_params [2] (rounded to FP32) into h_ids [H][W] (host), -1 for the
 * background: the rasteriser's coverage and depth decisions (largest 1/Z,
 * lower index on equal 1/Z) without shading, for exact comparison with
 * another renderer.  HR_ERR_UNSUPPORTED for other kinds. */
hr_status hr_render_ids(hr_scene scene, const double* h_params, int32_t* h_ids);

/* ---------------------------------------------------------------------------
 * Serving with continuous batching.  A server owns one device arena of
 * hbm_budget bytes (allocated at creation) and a worker thread.  Submitted
 * requests wait in a queue until a slot (max_active) and arena space for
 * their state are free; once admitted, their perturbations are sampled and
 * rendered in chunks, and every batched render launch carries chunks of all
 * active requests on the same scene, so requests that arrive while others
 * run join the next launch and their work overlaps on the device.  Scenes
 * (geometry, targets) and Newton-CG states stay resident; a Newton-CG step
 * request advances its state by one step.  A request's result does not
 * depend on what else is in flight: each render and each request's sums run
 * the same code in the same order as hr_estimate_*.
 * ------------------------------------------------------------------------- */
#define HR_NEWTON_STEP 3

typedef struct hr_server_s* hr_server;

typedef struct {
    int64_t hbm_budget;     /* bytes of device memory for request state */
    int32_t max_active;     /* requests admitted at once, 1..48 */
    int32_t chunk;          /* perturbations per request per batched launch (0: 2048) */
} hr_server_opts;

typedef struct {
    hr_scene scene;
    int32_t quantity;       /* HR_GRAD, HR_HESSIAN, HR_HVP or HR_NEWTON_STEP */
    const double* h_theta;  /* [n] host, copied at submission (estimates) */
    const double* h_v;      /* [n] host, copied at submission (HVP) */
    hr_opts opts;           /* sigma, n_perturb, strategy, seed, request_id, sub;
                               stream and inspection outputs are ignored */
    hr_optstate optstate;   /* HR_NEWTON_STEP: the state to advance (same scene) */
} hr_request;

typedef struct {
    double submit_ms, admit_ms, done_ms;   /* host clock, ms since server creation */
    int32_t status;                         /* HR_OK or the request's failure code */
    int32_t batches;                        /* batched launches that carried its renders */
} hr_request_info;

hr_status hr_server_create(const hr_server_opts* opts, hr_server* out);
/* Stops admitting, finishes admitted work, fails queued requests with
 * HR_ERR_BUSY, frees the arena. */
hr_status hr_server_destroy(hr_server srv);
/* Queue a request (inputs copied); *ticket identifies it.  HR_ERR_OOM if its
 * state can never fit the arena. */
hr_status hr_server_submit(hr_server srv, const hr_request* req, uint64_t* ticket);
/* Wait for a request.  h_out (host) receives n (gradient, HVP) or n*n
 * (Hessian) doubles, or B hr_step_info records for HR_NEWTON_STEP; info may be
 * NULL.  timeout_ms < 0 waits without limit; on timeout HR_ERR_TIMEOUT is
 * returned and the ticket stays valid.  A ticket can be waited for once. */
hr_status hr_server_wait(hr_server srv, uint64_t ticket, void* h_out, hr_request_info* info, int32_t timeout_ms);

/* ---------------------------------------------------------------------------
 * Persistent queue (disc and squares scenes): estimate requests of one DISC2D
 * or BOXES2D scene (at most 8 parameters) served by one long-running kernel
 * (Sec. 3.2-3.5 estimators, Sec. 4.1 Box2 task).
 * A request's perturbations are sampled, rendered and summed inside that
 * kernel, in units of 16 antithetic pairs taken by whichever warp is free;
 * the warp that finishes a request's last unit forms its sums in the same
 * order as hr_estimate_*, so the result is bit-identical to hr_estimate_* with
 * the same options.  Submission makes no driver call: the descriptor goes into
 * host-mapped memory that the kernel polls.
 *
 * The kernel leaves after idle_budget_us without a new request (its polling
 * is bounded by clock64(), never an unbounded spin) and records HR_ERR_TIMEOUT
 * as its exit status; the next hr_queue_submit or hr_queue_wait launches it
 * again.  It occupies every SM while it runs, so other work on the GPU shares
 * the SMs with it during that time.
 *
 * One queue per scene at a time; destroy the queue before its scene.  The
 * functions may be called from several host threads (one lock per queue).
 * ------------------------------------------------------------------------- */
typedef struct hr_queue_s* hr_queue;

typedef struct {
    int32_t max_requests;    /* ring slots: requests submitted and not yet waited for, 1..16384
                                (4 KiB of device memory and 0.5 KiB host-mapped each) */
    int32_t idle_budget_us;  /* the kernel leaves after this long without a new request, 1..10^7 */
    int64_t arena_bytes;     /* device bytes for the perturbations, weights and losses of
                                unfinished requests (>= 1 MiB); a request takes
                                about G M (n + E + 1) 4 bytes */
} hr_queue_opts;

/* HR_ERR_UNSUPPORTED unless the scene is DISC2D, or BOXES2D with at most 4
 * squares; HR_ERR_OOM if the device or host-mapped memory cannot be had. */
hr_status hr_queue_create(hr_scene scene, const hr_queue_opts* opts, hr_queue* out);
/* Queue one estimate (HR_GRAD, HR_HESSIAN or HR_HVP; h_theta [n] and h_v [n]
 * host, copied).  opts: sigma, n_perturb, strategy, seed, request_id and sub
 * as in hr_estimate_*; stream and inspection outputs are ignored.  At most 4
 * sample groups (element-wise Hessians of n = 2 have 3).  HR_ERR_BUSY, with
 * nothing queued, when the ring slot of the next ticket still holds a result
 * not waited for, or when the arena has no room until earlier requests
 * finish: wait for an earlier ticket and submit again. */
hr_status hr_queue_submit(hr_queue q, int32_t quantity, const double* h_theta, const double* h_v,
                          const hr_opts* opts, uint64_t* ticket);
/* Queue count estimates of one quantity in one call: h_theta [count][n],
 * h_v [count][n] (HVP, else NULL), opts [count] (host).  All are checked
 * first (HR_ERR_INVALID_ARG queues none); then they are queued in order until
 * the ring or the arena is full.  *submitted receives how many were queued and
 * tickets [0, *submitted) their tickets; HR_ERR_BUSY when fewer than count. */
hr_status hr_queue_submit_many(hr_queue q, int32_t count, int32_t quantity, const double* h_theta,
                               const double* h_v, const hr_opts* opts, uint64_t* tickets, int32_t* submitted);
/* Wait for a ticket; h_out (host) receives n doubles (gradient, HVP) or n*n
 * (Hessian).  timeout_ms < 0 waits without limit; on timeout HR_ERR_TIMEOUT is
 * returned and the ticket stays valid.  A ticket can be waited for once. */
hr_status hr_queue_wait(hr_queue q, uint64_t ticket, double* h_out, int32_t timeout_ms);
/* Wait for count tickets in order; result i goes to h_out + i * out_stride
 * (host; out_stride >= every result's size, else HR_ERR_INVALID_ARG before any
 * wait).  timeout_ms bounds the whole call; on an error, the results of the
 * tickets before the failing one have been delivered. */
hr_status hr_queue_wait_many(hr_queue q, int32_t count, const uint64_t* tickets, double* h_out,
                             int32_t out_stride, int32_t timeout_ms);
/* *kernel_status: 1 while the kernel runs; after it left, HR_ERR_TIMEOUT (idle
 * budget spent) or HR_OK.  *launches (may be NULL): launches so far. */
hr_status hr_queue_status(hr_queue q, int32_t* kernel_status, uint64_t* launches);
/* Lets the kernel finish the requests already submitted, then frees the queue. */
hr_status hr_queue_destroy(hr_queue q);

/* Diagnostics of a scene's mesh renders since its creation, summed over
 * renders (waits for the device); all 0 for kinds other than REVOLVE3D.
 *   mesh_overflow_renders   renders whose tile bins held more (triangle,
 *                           tile) entries than the render's shared memory
 *                           holds at once (at most 16,384), so that they were
 *                           binned and rastered in bands of tile rows that fit
 *                           (same pixels, same decisions);
 *   mesh_renders            renders of estimates (images not counted);
 *   mesh_survivors          triangles that passed clipping, culling and the
 *                           image bounds;
 *   mesh_bin_entries        (triangle, tile) bin entries;
 *   mesh_tiles_with_entries tiles with at least one entry;
 *   mesh_raster_steps       raster loop trips of the warps (a warp's tiles
 *                           take as many trips as the longest bin among
 *                           them);
 *   mesh_tile_height        rows of the 8-pixel-wide raster tiles (4 or 8);
 *   mesh_walk_all_renders   renders with a tile row whose entries alone did
 *                           not fit, so that its tiles walked every triangle
 *                           (same pixels, same decisions, slower);
 *   mesh_redo_renders       renders that did not fit the compact layout
 *                           (more survivors than its slots, or more entries
 *                           than it holds) and were rendered again in the
 *                           full layout (counted once in mesh_renders);
 *   mesh_compact_slots      survivor slots of the scene's compact layout,
 *                           which puts two renders on an SM with the records
 *                           of surviving triangles only (0: the scene's mesh
 *                           or image is too large for it, every render uses
 *                           the full layout).  Both layouts take the same
 *                           coverage and depth decisions.
 * The sums divided by mesh_renders give per-render averages.  Path-traced
 * scenes (PTBOX) count their work only while hr_scene_count_work is on
 * (those launches use a counting build of the default launch shape; the
 * images and losses are the same):
 *   pt_counted_renders      renders launched while counting;
 *   pt_hit_rays             closest-hit rays (camera rays and continuations);
 *   pt_shadow_rays          shadow rays of next-event estimation;
 *   pt_vertices             shaded path vertices. */
typedef struct {
    int64_t mesh_overflow_renders;
    int64_t mesh_renders;
    int64_t mesh_survivors;
    int64_t mesh_bin_entries;
    int64_t mesh_tiles_with_entries;
    int64_t mesh_raster_steps;
    int64_t mesh_tile_height;
    int64_t pt_counted_renders;
    int64_t pt_hit_rays;
    int64_t pt_shadow_rays;
    int64_t pt_vertices;
    int64_t mesh_walk_all_renders;
    int64_t mesh_redo_renders;
    int64_t mesh_compact_slots;
} hr_scene_stats;
hr_status hr_scene_get_stats(hr_scene scene, hr_scene_stats* out);
/* PTBOX only: on != 0 makes the scene's following render launches count
 * their rays (see hr_scene_stats); HR_ERR_UNSUPPORTED for other kinds. */
hr_status hr_scene_count_work(hr_scene scene, int32_t on);

/* Stage timing: when enabled (on != 0), every estimate records CUDA events
 * on its stream around its three launches (sampler, render + loss, sums) and
 * hr_profile_last writes their durations in milliseconds, ms[3], for the
 * calling thread's last estimate on that scene (after it completed).
 * Returns HR_ERR_INVALID_ARG when nothing was recorded. */
hr_status hr_profile_enable(hr_scene scene, int32_t on);
hr_status hr_profile_last(hr_scene scene, float* ms3);

/* ---------------------------------------------------------------------------
 * Autotuning of launch shapes.  Each scene kind has render+loss launch-shape
 * variants (path tracer: minimum resident CTAs per SM 3 / 2 / 4, i.e. register
 * caps; disc and squares: 8 / 4 / 16 warps per CTA, one warp per
 * perturbation; mesh and 2D triangles: one shape) and the sampler runs with
 * 16, 32, 64 or 128 threads per block (16 spreads small requests over more
 * SMs; with 64 or 128, a block takes its aggregate Hessian pairs diagonal-lobe
 * ones first so that most warps run one lobe path).  Every variant computes
 * each value with the same operations in the same order, so results are
 * bit-identical whatever is chosen.
 * hr_autotune times each variant on profiled aggregate HVP estimates of
 * max(n_probe, 8 x the SM count) perturbations at h_theta [n] (v = ones,
 * sigma 0.05; median of 3 after a warm-up; the floor keeps the GPU full so
 * that occupancy shows), keeps the fastest for the scene and, if info is not NULL,
 * reports the choice and the timings (ms).  hr_set_tuning sets a choice
 * directly (HR_ERR_INVALID_ARG when out of range).  Scenes start at variant 0
 * and 32 sampler threads.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t render_variant;     /* chosen render variant */
    int32_t sample_threads;     /* chosen sampler threads per block */
    int32_t n_render_variants;
    int32_t n_sample_variants;  /* 4: 32, 64, 128, 16 threads */
    float render_ms[4];         /* median render+loss time per variant */
    float sample_ms[4];         /* median sampler time per shape */
} hr_tune_info;

hr_status hr_autotune(hr_scene scene, const double* h_theta, int32_t n_probe, hr_tune_info* info);
hr_status hr_set_tuning(hr_scene scene, int32_t render_variant, int32_t sample_threads);

/* Thread-local message of the last failure (empty if none); returns the
 * message length.  buf may be NULL to query the length. */
size_t hr_last_error(char* buf, size_t len);

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t hr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HR_H */
