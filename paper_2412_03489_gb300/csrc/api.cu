// C-ABI entry points of libhr: scene lifetime, the three estimators, the
// device-pointer form, single-image rendering, error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hr.h"
#include "hr_api_internal.h"
#include "hr_device.cuh"
#include "hr_internal.h"

namespace hr {

void launch_disc_loss(const DevScene&, const RenderBatch&, cudaStream_t);
void launch_disc_image(const DevScene&, const float*, float*, cudaStream_t);
void launch_boxes_loss(const DevScene&, const RenderBatch&, cudaStream_t);
void launch_boxes_image(const DevScene&, const float*, float*, cudaStream_t);
void launch_revolve_loss(const DevScene&, const RenderBatch&, cudaStream_t);
void launch_revolve_image(const DevScene&, const float*, float*, int32_t*, cudaStream_t);
void launch_tris2d_loss(const DevScene&, const RenderBatch&, cudaStream_t);
void launch_tris2d_image(const DevScene&, const float*, float*, cudaStream_t);
void launch_ptbox_loss(const DevScene&, const RenderBatch&, cudaStream_t);
void launch_analytic_loss(const DevScene&, const RenderBatch&, cudaStream_t);
void launch_analytic_image(const DevScene&, const float*, float*, cudaStream_t);
void launch_ptbox_image(const DevScene&, const float*, uint64_t, uint32_t, uint32_t, uint32_t, uint32_t, int, float*,
                        cudaStream_t);

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

void launch_render_loss(const DevScene& sc, const RenderBatch& b, cudaStream_t s) {
    switch (sc.kind) {
        case HR_SCENE_DISC2D: launch_disc_loss(sc, b, s); break;
        case HR_SCENE_REVOLVE3D: launch_revolve_loss(sc, b, s); break;
        case HR_SCENE_TRIS2D: launch_tris2d_loss(sc, b, s); break;
        case HR_SCENE_PTBOX: launch_ptbox_loss(sc, b, s); break;
        case HR_SCENE_BOXES2D: launch_boxes_loss(sc, b, s); break;
        case HR_SCENE_QUADRATIC:
        case HR_SCENE_STEP1D:
        case HR_SCENE_NEGGAUSS: launch_analytic_loss(sc, b, s); break;
    }
}

void launch_render_image(const DevScene& sc, const float* d_params, uint64_t seed, uint32_t request, uint32_t sub,
                         uint32_t k, uint32_t tag, int spp, float* d_img, cudaStream_t s) {
    switch (sc.kind) {
        case HR_SCENE_DISC2D: launch_disc_image(sc, d_params, d_img, s); break;
        case HR_SCENE_REVOLVE3D: launch_revolve_image(sc, d_params, d_img, nullptr, s); break;
        case HR_SCENE_TRIS2D: launch_tris2d_image(sc, d_params, d_img, s); break;
        case HR_SCENE_PTBOX: launch_ptbox_image(sc, d_params, seed, request, sub, k, tag, spp, d_img, s); break;
        case HR_SCENE_BOXES2D: launch_boxes_image(sc, d_params, d_img, s); break;
        case HR_SCENE_QUADRATIC:
        case HR_SCENE_STEP1D:
        case HR_SCENE_NEGGAUSS: launch_analytic_image(sc, d_params, d_img, s); break;
    }
}

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

hr_status fail(hr_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

void clear_error() { g_err.clear(); }

const std::string& last_error() { return g_err; }

// ---------------------------------------------------------------------------
// device buffer that grows on demand
// ---------------------------------------------------------------------------
cudaError_t DevBuf::reserve(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    const cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
}
void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
}

}  // namespace hr

using namespace hr;

namespace {

template <class T>
cudaError_t upload(T** dst, const T* src, size_t count) {
    cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * (count ? count : 1));
    if (e != cudaSuccess) return e;
    if (count) e = cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice);
    return e;
}

__global__ void fd_combine_kernel(const double* gp, const double* gm, double inv2eps, int n, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (gp[i] - gm[i]) * inv2eps;
}

}  // namespace

// ---------------------------------------------------------------------------
// estimator pipeline shared by the host- and device-pointer entry points
// ---------------------------------------------------------------------------
namespace hr {

int n_elements(int quantity, int n) { return quantity == HR_HESSIAN ? n * (n + 1) / 2 : n; }

hr_status validate_opts(const hr_scene_s* s, int quantity, const hr_opts* o) {
    if (!s) return fail(HR_ERR_INVALID_ARG, "scene is NULL");
    if (!o) return fail(HR_ERR_INVALID_ARG, "opts is NULL");
    if (!(o->sigma > 0.0) || !std::isfinite(o->sigma)) return fail(HR_ERR_INVALID_ARG, "sigma must be > 0");
    if (o->n_perturb < 2 || (o->n_perturb & 1)) return fail(HR_ERR_INVALID_ARG, "n_perturb must be even and >= 2");
    if (o->strategy != HR_ELEMENTWISE && o->strategy != HR_AGGREGATE && o->strategy != HR_PLAIN)
        return fail(HR_ERR_INVALID_ARG, "unknown strategy %d", o->strategy);
    const int n = s->sc.n;
    const int G = o->strategy == HR_ELEMENTWISE ? n_elements(quantity, n) : 1;
    const int64_t total = (int64_t)G * o->n_perturb;
    if (o->n_perturb / 2 >= (1 << 24)) return fail(HR_ERR_INVALID_ARG, "at most 2^24 - 1 pairs per request");
    if (total > (int64_t)1 << 28) return fail(HR_ERR_INVALID_ARG, "too many perturbations (%lld)", (long long)total);
    if ((uint64_t)o->sub + (uint64_t)G > (1u << 24)) return fail(HR_ERR_INVALID_ARG, "sub-stream out of range");
    return HR_OK;
}

hr_status run_estimate(hr_scene_s* s, int quantity, const double* h_theta, const double* d_theta,
                       const double* h_v, const double* d_v, const hr_opts* o, double* h_out, double* d_out) {
    hr_status st = validate_opts(s, quantity, o);
    if (st != HR_OK) return st;
    DevScene& sc = s->sc;
    Workspace& ws = s->ws;
    const int n = sc.n;
    const int E = n_elements(quantity, n);
    const int G = o->strategy == HR_ELEMENTWISE ? E : 1;
    const int64_t M = o->n_perturb;
    const int P = (int)(M / 2);
    const int64_t Mt = (int64_t)G * M;
    cudaStream_t stream = o->stream ? (cudaStream_t)o->stream : s->stream;

#define WS_TRY(x)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (x);                                                                  \
        if (e_ != cudaSuccess) return fail(HR_ERR_OOM, "workspace: %s", cudaGetErrorString(e_)); \
    } while (0)
    WS_TRY(ws.theta32.reserve(sizeof(float) * n));
    WS_TRY(ws.v.reserve(sizeof(double) * n));
    WS_TRY(ws.tau.reserve(sizeof(float) * Mt * n));
    WS_TRY(ws.w.reserve(sizeof(float) * Mt * E));
    WS_TRY(ws.meta.reserve(sizeof(uint2) * Mt));
    WS_TRY(ws.loss.reserve(sizeof(float) * Mt));
    WS_TRY(ws.flat.reserve(sizeof(double) * E));
    WS_TRY(ws.scale.reserve(sizeof(double) * E));
    WS_TRY(ws.full.reserve(sizeof(double) * n * n));
    WS_TRY(ws.groups.reserve(sizeof(SampleGroup) * G));
#undef WS_TRY

#define CU_TRY(x)                                                                               \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) return fail(HR_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_));  \
    } while (0)
    // theta in FP32 is written by the sampler launch (its first block): from
    // the device array, or from values passed by value (n <= 64: no host
    // staging, no wait)
    float* theta32 = (float*)ws.theta32.ptr;
    const double* vdev = d_v;
    if (quantity == HR_HVP && h_v) {
        CU_TRY(cudaMemcpyAsync(ws.v.ptr, h_v, sizeof(double) * n, cudaMemcpyHostToDevice, stream));
        vdev = (const double*)ws.v.ptr;
    }
    s->host_groups.resize(G);
    for (int g = 0; g < G; ++g) {
        SampleGroup& gr = s->host_groups[g];
        gr.m0 = (int32_t)(g * M);
        gr.P = P;
        gr.lobe = quantity == HR_GRAD ? 0 : 1;
        gr.quantity = quantity;
        gr.sub = o->sub + (uint32_t)g;
        gr.request = o->request_id;
        gr.theta_row = 0;
        gr.pad = 0;
        if (o->strategy == HR_AGGREGATE) {
            gr.comp_i = -1; gr.comp_j = -1;
        } else if (o->strategy == HR_PLAIN) {
            gr.comp_i = -3; gr.comp_j = -3;
        } else if (quantity == HR_GRAD) {
            gr.comp_i = g; gr.comp_j = g;
        } else if (quantity == HR_HVP) {
            gr.comp_i = g; gr.comp_j = -2; gr.quantity = 4;   // row g of the HVP, row-mixture draws
        } else {
            int r = 0, rem = g;
            while (rem >= n - r) { rem -= n - r; ++r; }
            gr.comp_i = r; gr.comp_j = r + rem;
        }
    }
    if (G > kInlineGroups) {
        CU_TRY(cudaMemcpyAsync(ws.groups.ptr, s->host_groups.data(), sizeof(SampleGroup) * G, cudaMemcpyHostToDevice,
                               stream));
        CU_TRY(cudaStreamSynchronize(stream));   // host group table may be reused by the next call
    }

    SampleArgs sa{};
    sa.theta_out = theta32;
    sa.theta_n = n;
    sa.theta_in = h_theta ? nullptr : d_theta;
    if (h_theta)
        for (int i = 0; i < n; ++i) sa.theta_vals[i] = (float)h_theta[i];
    sa.groups = (const SampleGroup*)ws.groups.ptr;
    sa.n = n;
    sa.E = E;
    sa.sigma = o->sigma;
    const double s2 = o->sigma * o->sigma;
    sa.Zg = std::sqrt(2.0 / M_PI) / o->sigma;
    sa.Zd = 4.0 * std::exp(-0.5) / (std::sqrt(2.0 * M_PI) * s2);
    sa.Zo = sa.Zg * sa.Zg;
    sa.seed = o->seed;
    sa.v = vdev;
    sa.tau = (float*)ws.tau.ptr;
    sa.w = (float*)ws.w.ptr;
    sa.invS = nullptr;
    sa.meta = (uint2*)ws.meta.ptr;
    sa.threads = s->sc.sample_threads;
    if (G <= kInlineGroups) {
        sa.n_inline = G;
        for (int g = 0; g < G; ++g) sa.inline_groups[g] = s->host_groups[g];
    }
    if (s->profile) cudaEventRecord(s->ev[0], stream);
    launch_sample(sa, G, P, stream);
    if (s->profile) cudaEventRecord(s->ev[1], stream);

    RenderBatch rb{};
    rb.theta32 = theta32;
    rb.tau = (const float*)ws.tau.ptr;
    rb.meta = (const uint2*)ws.meta.ptr;
    rb.loss = (float*)ws.loss.ptr;
    rb.M = (int32_t)Mt;
    rb.n = n;
    rb.per_row = (int32_t)Mt;
    rb.request0 = o->request_id;
    rb.seed = o->seed;
    launch_render_loss(sc, rb, stream);
    if (s->profile) cudaEventRecord(s->ev[2], stream);

    FinalizeArgs fa{};
    fa.w = (const float*)ws.w.ptr;
    fa.loss = (const float*)ws.loss.ptr;
    fa.E = E;
    fa.n = n;
    fa.pairs2 = (int32_t)M;
    fa.elementwise = o->strategy == HR_ELEMENTWISE;
    fa.hessian = quantity == HR_HESSIAN;
    fa.inv2P = 1.0 / (double)M;
    fa.out_flat = (double*)ws.flat.ptr;
    fa.out_scale = (double*)ws.scale.ptr;
    fa.out_full = quantity == HR_HESSIAN ? (d_out ? d_out : (double*)ws.full.ptr) : nullptr;
    if (quantity != HR_HESSIAN && d_out) fa.out_flat = d_out;
    launch_finalize(fa, stream);
    if (s->profile) {
        cudaEventRecord(s->ev[3], stream);
        s->profile_valid = true;
    }
    CU_TRY(cudaGetLastError());

    if (h_out) {
        if (quantity == HR_HESSIAN)
            CU_TRY(cudaMemcpyAsync(h_out, ws.full.ptr, sizeof(double) * n * n, cudaMemcpyDeviceToHost, stream));
        else
            CU_TRY(cudaMemcpyAsync(h_out, ws.flat.ptr, sizeof(double) * n, cudaMemcpyDeviceToHost, stream));
        if (o->out_tau)
            CU_TRY(cudaMemcpyAsync(o->out_tau, ws.tau.ptr, sizeof(float) * Mt * n, cudaMemcpyDeviceToHost, stream));
        if (o->out_weights)
            CU_TRY(cudaMemcpyAsync(o->out_weights, ws.w.ptr, sizeof(float) * Mt * E, cudaMemcpyDeviceToHost, stream));
        if (o->out_losses)
            CU_TRY(cudaMemcpyAsync(o->out_losses, ws.loss.ptr, sizeof(float) * Mt, cudaMemcpyDeviceToHost, stream));
        if (o->out_scale)
            CU_TRY(cudaMemcpyAsync(o->out_scale, ws.scale.ptr, sizeof(double) * E, cudaMemcpyDeviceToHost, stream));
        CU_TRY(cudaStreamSynchronize(stream));
    }
#undef CU_TRY
    return HR_OK;
}

// Central difference of two gradient estimates on shared perturbations: the
// sampler runs once, one launch renders both parameter rows (theta +- eps v)
// through a two-row batch table, each row gets its own sums.
hr_status run_hvp_fd(hr_scene_s* s, const double* h_theta, const double* h_v, double eps, const hr_opts* o,
                     double* h_out) {
    DevScene& sc = s->sc;
    Workspace& ws = s->ws;
    const int n = sc.n;
    const int E = n;
    const int G = o->strategy == HR_ELEMENTWISE ? n : 1;
    const int64_t M = o->n_perturb;
    const int P = (int)(M / 2);
    const int64_t Mt = (int64_t)G * M;
    cudaStream_t stream = o->stream ? (cudaStream_t)o->stream : s->stream;
    if (ws.theta32.reserve(sizeof(float) * 2 * n) != cudaSuccess || ws.tau.reserve(sizeof(float) * Mt * n) != cudaSuccess ||
        ws.w.reserve(sizeof(float) * Mt * E) != cudaSuccess || ws.meta.reserve(sizeof(uint2) * Mt) != cudaSuccess ||
        ws.loss.reserve(sizeof(float) * 2 * Mt) != cudaSuccess || ws.flat.reserve(sizeof(double) * 3 * E) != cudaSuccess ||
        ws.groups.reserve(sizeof(SampleGroup) * G) != cudaSuccess)
        return fail(HR_ERR_OOM, "workspace");
    std::vector<float> t32(2 * n);
    for (int i = 0; i < n; ++i) {
        t32[i] = (float)(h_theta[i] + eps * h_v[i]);
        t32[n + i] = (float)(h_theta[i] - eps * h_v[i]);
    }
    s->host_groups.resize(G);
    for (int g = 0; g < G; ++g) {
        SampleGroup& gr = s->host_groups[g];
        gr.m0 = (int32_t)(g * M);
        gr.P = P;
        gr.lobe = 0;
        gr.quantity = HR_GRAD;
        gr.sub = o->sub + (uint32_t)g;
        gr.request = o->request_id;
        gr.theta_row = 0;
        gr.pad = 0;
        gr.comp_i = o->strategy == HR_ELEMENTWISE ? g : (o->strategy == HR_PLAIN ? -3 : -1);
        gr.comp_j = gr.comp_i;
    }
    cudaError_t e = cudaMemcpyAsync(ws.theta32.ptr, t32.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws.groups.ptr, s->host_groups.data(), sizeof(SampleGroup) * G, cudaMemcpyHostToDevice,
                            stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    SampleArgs sa{};
    sa.groups = (const SampleGroup*)ws.groups.ptr;
    sa.n = n;
    sa.E = E;
    sa.sigma = o->sigma;
    sa.Zg = std::sqrt(2.0 / M_PI) / o->sigma;
    sa.Zd = 4.0 * std::exp(-0.5) / (std::sqrt(2.0 * M_PI) * o->sigma * o->sigma);
    sa.Zo = sa.Zg * sa.Zg;
    sa.seed = o->seed;
    sa.tau = (float*)ws.tau.ptr;
    sa.w = (float*)ws.w.ptr;
    sa.meta = (uint2*)ws.meta.ptr;
    sa.threads = s->sc.sample_threads;
    launch_sample(sa, G, P, stream);
    RenderBatch rb{};
    rb.M = (int32_t)(2 * Mt);
    rb.n = n;
    rb.per_row = 1;
    rb.table_rows = 2;
    for (int r = 0; r < 2; ++r) {
        BatchRow& br = rb.rows[r];
        br.theta32 = (const float*)ws.theta32.ptr + r * n;
        br.tau = (const float*)ws.tau.ptr;
        br.meta = (const uint2*)ws.meta.ptr;
        br.loss = (float*)ws.loss.ptr + r * Mt;
        br.seed = o->seed;
        br.request = o->request_id;
        br.m_begin = 0;
        br.start = (int32_t)(r * Mt);
        br.pad = 0;
    }
    launch_render_loss(sc, rb, stream);
    double* flat = (double*)ws.flat.ptr;
    for (int r = 0; r < 2; ++r) {
        FinalizeArgs fa{};
        fa.w = (const float*)ws.w.ptr;
        fa.loss = (const float*)ws.loss.ptr + r * Mt;
        fa.E = E;
        fa.n = n;
        fa.pairs2 = (int32_t)M;
        fa.elementwise = o->strategy == HR_ELEMENTWISE;
        fa.hessian = 0;
        fa.inv2P = 1.0 / (double)M;
        fa.out_flat = flat + r * E;
        launch_finalize(fa, stream);
    }
    fd_combine_kernel<<<1, 64, 0, stream>>>(flat, flat + E, 0.5 / eps, n, flat + 2 * E);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(HR_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpyAsync(h_out, flat + 2 * E, sizeof(double) * n, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(stream)) != cudaSuccess)
        return fail(HR_ERR_CUDA, "result: %s", cudaGetErrorString(e));
    return HR_OK;
}

}  // namespace hr

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int32_t hr_version(void) { return 100; }

size_t hr_last_error(char* buf, size_t len) {
    const std::string& e = last_error();
    if (buf && len) {
        const size_t c = e.size() < len - 1 ? e.size() : len - 1;
        memcpy(buf, e.data(), c);
        buf[c] = 0;
    }
    return e.size();
}

hr_status hr_create_scene(const hr_scene_desc* d, hr_scene* out) {
    clear_error();
    if (!d || !out) return fail(HR_ERR_INVALID_ARG, "desc/out is NULL");
    *out = nullptr;
    if (d->width < 1 || d->height < 1 || d->width > HR_MAX_IMAGE_SIDE || d->height > HR_MAX_IMAGE_SIDE)
        return fail(HR_ERR_INVALID_ARG, "image size %dx%d out of range", d->width, d->height);
    int expect_n = -1, C = 3;
    switch (d->kind) {
        case HR_SCENE_DISC2D: expect_n = 2; C = 1;
            if (!(d->radius > 0.0f)) return fail(HR_ERR_INVALID_ARG, "disc radius must be > 0");
            break;
        case HR_SCENE_BOXES2D: C = 1;
            if (!(d->radius > 0.0f)) return fail(HR_ERR_INVALID_ARG, "square half-size must be > 0");
            if (d->n_params < 2 || (d->n_params & 1)) return fail(HR_ERR_INVALID_ARG, "n_params must be 2K");
            expect_n = d->n_params;
            break;
        case HR_SCENE_REVOLVE3D: expect_n = 2;
            if (!d->vertices || !d->triangles || d->n_vertices < 3 || d->n_triangles < 1 ||
                d->n_vertices > HR_MAX_VERTICES || d->n_triangles > HR_MAX_TRIANGLES)
                return fail(HR_ERR_INVALID_ARG, "mesh needs 3..%d vertices and 1..%d triangles", HR_MAX_VERTICES,
                            HR_MAX_TRIANGLES);
            if (d->width > 512 || d->height > 512) return fail(HR_ERR_UNSUPPORTED, "mesh images are at most 512x512");
            for (int i = 0; i < 3 * d->n_triangles; ++i)
                if (d->triangles[i] < 0 || d->triangles[i] >= d->n_vertices)
                    return fail(HR_ERR_INVALID_ARG, "triangle index out of range");
            if (!(d->eye_dist > 0.0f) || !(d->scale > 0.0f)) return fail(HR_ERR_INVALID_ARG, "bad camera");
            break;
        case HR_SCENE_PTBOX: expect_n = 6;
            if (!d->quad_axis || !d->quad_geom || !d->quad_albedo || !d->sph_center || !d->sph_radius || !d->sph_albedo)
                return fail(HR_ERR_INVALID_ARG, "path-traced box needs quads and spheres");
            if (d->spp < 1 || d->target_spp < 1 || d->depth < 1 || d->depth > 15 || d->spp > 4096)
                return fail(HR_ERR_INVALID_ARG, "spp/depth out of range");
            if ((int64_t)d->width * d->height * (d->target_spp > d->spp ? d->target_spp : d->spp) >= ((int64_t)1 << 32))
                return fail(HR_ERR_INVALID_ARG, "pixel samples exceed 2^32");
            for (int q = 0; q < 12; ++q)
                if (d->quad_axis[q] < 0 || d->quad_axis[q] > 2) return fail(HR_ERR_INVALID_ARG, "quad axis");
            break;
        case HR_SCENE_TRIS2D:
            if (!d->raw_params || !d->param_index || d->n_tris < 1 || d->n_tris > HR_MAX_TRIS2D)
                return fail(HR_ERR_INVALID_ARG, "need 1..%d triangles", HR_MAX_TRIS2D);
            expect_n = d->n_params;
            for (int j = 0; j < d->n_params; ++j)
                if (d->param_index[j] < 0 || d->param_index[j] >= 9 * d->n_tris)
                    return fail(HR_ERR_INVALID_ARG, "param_index out of range");
            break;
        case HR_SCENE_QUADRATIC: C = 1; expect_n = d->n_params;
            if (!d->quad_A || !d->quad_b) return fail(HR_ERR_INVALID_ARG, "quadratic needs A and b");
            break;
        case HR_SCENE_STEP1D: C = 1; expect_n = 1; break;
        case HR_SCENE_NEGGAUSS: C = 1; expect_n = d->n_params;
            if (!(d->gauss_sigma > 0.0) || !std::isfinite(d->gauss_sigma))
                return fail(HR_ERR_INVALID_ARG, "gauss_sigma must be finite and > 0");
            break;
        default: return fail(HR_ERR_INVALID_ARG, "unknown scene kind %d", d->kind);
    }
    const bool analytic = d->kind == HR_SCENE_QUADRATIC || d->kind == HR_SCENE_STEP1D || d->kind == HR_SCENE_NEGGAUSS;
    if (d->n_params != expect_n || d->n_params < 1 || d->n_params > HR_MAX_PARAMS)
        return fail(HR_ERR_INVALID_ARG, "n_params %d invalid for this scene", d->n_params);
    if (analytic && (d->width != 1 || d->height != 1))
        return fail(HR_ERR_INVALID_ARG, "analytic scenes have a 1 x 1 image");
    if (!analytic && !d->theta_target && !d->target_image)
        return fail(HR_ERR_INVALID_ARG, "need theta_target or target_image");

    hr_scene_s* s = new hr_scene_s();
    DevScene& sc = s->sc;
    sc.kind = d->kind; sc.W = d->width; sc.H = d->height; sc.C = C; sc.n = d->n_params;
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    auto bail = [&](cudaError_t err, const char* what) {
        hr_destroy_scene(s);
        return fail(err == cudaErrorMemoryAllocation ? HR_ERR_OOM : HR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(err));
    };
    if (e != cudaSuccess) { delete s; return fail(HR_ERR_CUDA, "stream: %s", cudaGetErrorString(e)); }
    const size_t npx = (size_t)sc.W * sc.H * C;
    if ((e = cudaMalloc(&sc.target, sizeof(float) * npx)) != cudaSuccess) return bail(e, "target");
    switch (d->kind) {
        case HR_SCENE_DISC2D: sc.radius = d->radius; break;
        case HR_SCENE_BOXES2D: sc.radius = d->radius; break;
        case HR_SCENE_REVOLVE3D: {
            sc.nv = d->n_vertices; sc.nt = d->n_triangles;
            for (int c = 0; c < 3; ++c) { sc.albedo[c] = d->albedo[c]; sc.light[c] = d->light[c]; }
            sc.eye_dist = d->eye_dist; sc.scale = d->scale;
            int dev = 0, maxsm = 0, smpm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaDeviceGetAttribute(&smpm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            if (!revolve_layout(sc, maxsm, smpm)) {
                hr_destroy_scene(s);
                return fail(HR_ERR_UNSUPPORTED, "mesh of %d triangles at %dx%d does not fit in %d B of shared memory",
                            sc.nt, sc.W, sc.H, maxsm);
            }
            if ((e = upload(&sc.verts, d->vertices, 3 * (size_t)sc.nv)) != cudaSuccess) return bail(e, "vertices");
            if ((e = upload(&sc.tris, d->triangles, 3 * (size_t)sc.nt)) != cudaSuccess) return bail(e, "triangles");
            if ((e = cudaMalloc(&sc.tnrm, sizeof(float) * 3 * sc.nt)) != cudaSuccess) return bail(e, "normals");
            if ((e = cudaMalloc(&sc.tile_t2, sizeof(float) * revolve_tiles(sc))) != cudaSuccess)
                return bail(e, "tiles");
            if ((e = cudaMalloc(&sc.rv_stats, 8 * sizeof(unsigned long long))) != cudaSuccess) return bail(e, "stats");
            if ((e = cudaMemset(sc.rv_stats, 0, 8 * sizeof(unsigned long long))) != cudaSuccess) return bail(e, "stats");
            revolve_prepare(sc, s->stream);
            break;
        }
        case HR_SCENE_TRIS2D:
            sc.n_tris = d->n_tris;
            if ((e = upload(&sc.raw, d->raw_params, 9 * (size_t)sc.n_tris)) != cudaSuccess) return bail(e, "raw");
            if ((e = upload(&sc.pidx, d->param_index, (size_t)sc.n)) != cudaSuccess) return bail(e, "param_index");
            break;
        case HR_SCENE_PTBOX:
            for (int q = 0; q < 12; ++q) {
                sc.qaxis[q] = d->quad_axis[q];
                for (int c = 0; c < 5; ++c) sc.qgeom[q][c] = d->quad_geom[5 * q + c];
                for (int c = 0; c < 3; ++c) sc.qalb[q][c] = d->quad_albedo[3 * q + c];
            }
            for (int i = 0; i < 3; ++i) {
                for (int c = 0; c < 3; ++c) { sc.sc_[i][c] = d->sph_center[3 * i + c]; sc.salb[i][c] = d->sph_albedo[3 * i + c]; }
                sc.sr[i] = d->sph_radius[i];
            }
            sc.light_half = d->light_half; sc.cam_z = d->cam_z; sc.tan_half = d->tan_half; sc.pix_scale = d->pix_scale;
            for (int c = 0; c < 3; ++c) sc.emission[c] = d->emission[c];
            sc.spp = d->spp; sc.target_spp = d->target_spp; sc.depth = d->depth; sc.scene_seed = d->seed;
            if ((e = cudaMalloc(&sc.pt_stats, 4 * sizeof(unsigned long long))) != cudaSuccess) return bail(e, "stats");
            if ((e = cudaMemset(sc.pt_stats, 0, 4 * sizeof(unsigned long long))) != cudaSuccess) return bail(e, "stats");
            break;
        case HR_SCENE_QUADRATIC:
            if ((e = upload(&sc.qA, d->quad_A, (size_t)sc.n * sc.n)) != cudaSuccess) return bail(e, "A");
            if ((e = upload(&sc.qb, d->quad_b, (size_t)sc.n)) != cudaSuccess) return bail(e, "b");
            break;
        case HR_SCENE_NEGGAUSS:
            sc.gauss_sigma = d->gauss_sigma;
            break;
    }
    if (analytic) {
        // no target: the loss is f itself
        if ((e = cudaMemset(sc.target, 0, sizeof(float) * npx)) != cudaSuccess) return bail(e, "target");
    } else if (d->target_image) {
        if ((e = cudaMemcpy(sc.target, d->target_image, sizeof(float) * npx, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail(e, "target upload");
    } else {
        std::vector<float> p32(sc.n);
        for (int i = 0; i < sc.n; ++i) p32[i] = (float)d->theta_target[i];
        float* dp = nullptr;
        if ((e = upload(&dp, p32.data(), (size_t)sc.n)) != cudaSuccess) return bail(e, "target params");
        launch_render_image(sc, dp, sc.scene_seed, 0, 0, 0, hr::TAG_TARGET, sc.target_spp, sc.target, s->stream);
        e = cudaStreamSynchronize(s->stream);
        cudaFree(dp);
        if (e != cudaSuccess) return bail(e, "target render");
    }
    if (sc.kind == HR_SCENE_REVOLVE3D) revolve_tile_t2(sc, s->stream);
    if ((sc.kind == HR_SCENE_DISC2D || sc.kind == HR_SCENE_BOXES2D) &&
        (e = disc_prepare_target(sc, s->stream)) != cudaSuccess)
        return bail(e, "target bits");
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return bail(e, "scene setup");
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(e, "scene setup launch");
    *out = s;
    return HR_OK;
}

hr_status hr_destroy_scene(hr_scene s) {
    if (!s) return HR_OK;
    DevScene& sc = s->sc;
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFree(sc.target); cudaFree(sc.verts); cudaFree(sc.tris); cudaFree(sc.tnrm); cudaFree(sc.tile_t2);
    cudaFree(sc.raw); cudaFree(sc.pidx); cudaFree(sc.qA); cudaFree(sc.qb); cudaFree(sc.rv_stats);
    cudaFree(sc.pt_stats); cudaFree(sc.tbits); cudaFree(sc.trowpop);
    s->ws.release_all();
    for (cudaEvent_t& e : s->ev)
        if (e) cudaEventDestroy(e);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return HR_OK;
}

hr_status hr_estimate_grad(hr_scene s, const double* theta, const hr_opts* o, double* out) {
    clear_error();
    if (!theta || !out) return fail(HR_ERR_INVALID_ARG, "theta/out is NULL");
    if (!s) return fail(HR_ERR_INVALID_ARG, "scene is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    return run_estimate(s, HR_GRAD, theta, nullptr, nullptr, nullptr, o, out, nullptr);
}

hr_status hr_estimate_hessian(hr_scene s, const double* theta, const hr_opts* o, double* out) {
    clear_error();
    if (!theta || !out) return fail(HR_ERR_INVALID_ARG, "theta/out is NULL");
    if (!s) return fail(HR_ERR_INVALID_ARG, "scene is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    return run_estimate(s, HR_HESSIAN, theta, nullptr, nullptr, nullptr, o, out, nullptr);
}

hr_status hr_estimate_hvp(hr_scene s, const double* theta, const double* v, const hr_opts* o, double* out) {
    clear_error();
    if (!theta || !out || !v) return fail(HR_ERR_INVALID_ARG, "theta/v/out is NULL");
    if (!s) return fail(HR_ERR_INVALID_ARG, "scene is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    return run_estimate(s, HR_HVP, theta, nullptr, v, nullptr, o, out, nullptr);
}

hr_status hr_estimate_dev(hr_scene s, int32_t quantity, const double* d_theta, const double* d_v, const hr_opts* o,
                          double* d_out) {
    clear_error();
    if (!s) return fail(HR_ERR_INVALID_ARG, "scene is NULL");
    if (quantity < HR_GRAD || quantity > HR_HVP) return fail(HR_ERR_INVALID_ARG, "unknown quantity %d", quantity);
    if (!d_theta || !d_out || (quantity == HR_HVP && !d_v)) return fail(HR_ERR_INVALID_ARG, "NULL device pointer");
    std::lock_guard<std::mutex> lk(s->mu);
    return run_estimate(s, quantity, nullptr, d_theta, nullptr, d_v, o, nullptr, d_out);
}

hr_status hr_scene_get_stats(hr_scene s, hr_scene_stats* out) {
    clear_error();
    if (!s || !out) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    if (s->sc.rv_stats) {
        unsigned long long v[8] = {};
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(v, s->sc.rv_stats, sizeof v, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(HR_ERR_CUDA, "stats: %s", cudaGetErrorString(e));
        out->mesh_overflow_renders = (int64_t)v[0];
        out->mesh_renders = (int64_t)v[1];
        out->mesh_survivors = (int64_t)v[2];
        out->mesh_bin_entries = (int64_t)v[3];
        out->mesh_tiles_with_entries = (int64_t)v[4];
        out->mesh_raster_steps = (int64_t)v[5];
        out->mesh_tile_height = s->sc.rv_th;
        out->mesh_walk_all_renders = (int64_t)v[6];
        out->mesh_redo_renders = (int64_t)v[7];
        out->mesh_compact_slots = s->sc.rv_cslots;
    }
    if (s->sc.pt_stats) {
        unsigned long long v[4] = {};
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(v, s->sc.pt_stats, sizeof v, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(HR_ERR_CUDA, "stats: %s", cudaGetErrorString(e));
        out->pt_counted_renders = (int64_t)v[0];
        out->pt_hit_rays = (int64_t)v[1];
        out->pt_shadow_rays = (int64_t)v[2];
        out->pt_vertices = (int64_t)v[3];
    }
    return HR_OK;
}

hr_status hr_scene_count_work(hr_scene s, int32_t on) {
    clear_error();
    if (!s) return fail(HR_ERR_INVALID_ARG, "NULL scene");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->sc.kind != HR_SCENE_PTBOX) return fail(HR_ERR_UNSUPPORTED, "work counting exists for path-traced scenes only");
    s->sc.count_work = on ? 1 : 0;
    return HR_OK;
}

hr_status hr_profile_enable(hr_scene s, int32_t on) {
    clear_error();
    if (!s) return fail(HR_ERR_INVALID_ARG, "scene is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    if (on && !s->ev[0]) {
        for (cudaEvent_t& e : s->ev) {
            const cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return fail(HR_ERR_CUDA, "event: %s", cudaGetErrorString(err));
        }
    }
    s->profile = on != 0;
    s->profile_valid = false;
    return HR_OK;
}

hr_status hr_profile_last(hr_scene s, float* ms3) {
    clear_error();
    if (!s || !ms3) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->profile_valid) return fail(HR_ERR_INVALID_ARG, "no profiled estimate");
    const cudaError_t es = cudaEventSynchronize(s->ev[3]);
    if (es != cudaSuccess) return fail(HR_ERR_CUDA, "event: %s", cudaGetErrorString(es));
    for (int i = 0; i < 3; ++i) {
        const cudaError_t e = cudaEventElapsedTime(&ms3[i], s->ev[i], s->ev[i + 1]);
        if (e != cudaSuccess) return fail(HR_ERR_CUDA, "event timing: %s", cudaGetErrorString(e));
    }
    return HR_OK;
}

hr_status hr_estimate_hvp_fd(hr_scene s, const double* h_theta, const double* h_v, double eps, const hr_opts* o,
                             double* h_out) {
    clear_error();
    if (!s || !h_theta || !h_v || !h_out) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(HR_ERR_INVALID_ARG, "eps must be > 0");
    std::lock_guard<std::mutex> lk(s->mu);
    hr_status st = validate_opts(s, HR_GRAD, o);
    if (st != HR_OK) return st;
    return run_hvp_fd(s, h_theta, h_v, eps, o, h_out);
}

hr_status hr_render_ids(hr_scene s, const double* h_params, int32_t* h_ids) {
    clear_error();
    if (!s || !h_params || !h_ids) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    DevScene& sc = s->sc;
    if (sc.kind != HR_SCENE_REVOLVE3D) return fail(HR_ERR_UNSUPPORTED, "triangle indices exist for mesh scenes only");
    const size_t npx = (size_t)sc.W * sc.H;
    float p32[2] = {(float)h_params[0], (float)h_params[1]};
    if (s->ws.render_img.reserve(sizeof(int32_t) * npx) != cudaSuccess ||
        s->ws.render_params.reserve(sizeof(p32)) != cudaSuccess)
        return fail(HR_ERR_OOM, "render buffers");
    cudaError_t e = cudaMemcpy(s->ws.render_params.ptr, p32, sizeof(p32), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "params: %s", cudaGetErrorString(e));
    launch_revolve_image(sc, (const float*)s->ws.render_params.ptr, nullptr, (int32_t*)s->ws.render_img.ptr, s->stream);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(HR_ERR_CUDA, "render: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpyAsync(h_ids, s->ws.render_img.ptr, sizeof(int32_t) * npx, cudaMemcpyDeviceToHost, s->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
        return fail(HR_ERR_CUDA, "render: %s", cudaGetErrorString(e));
    return HR_OK;
}

hr_status hr_render(hr_scene s, const double* h_params, uint64_t seed, uint32_t request, uint32_t sub, uint32_t k,
                    uint32_t tag, int32_t spp, float* h_img) {
    clear_error();
    if (!s || !h_params || !h_img) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    DevScene& sc = s->sc;
    if (sc.kind == HR_SCENE_PTBOX && (spp < 1 || (int64_t)sc.W * sc.H * spp >= ((int64_t)1 << 32)))
        return fail(HR_ERR_INVALID_ARG, "spp out of range");
    const size_t npx = (size_t)sc.W * sc.H * sc.C;
    std::vector<float> p32(sc.n);
    for (int i = 0; i < sc.n; ++i) p32[i] = (float)h_params[i];
    if (s->ws.render_img.reserve(sizeof(float) * npx) != cudaSuccess ||
        s->ws.render_params.reserve(sizeof(float) * sc.n) != cudaSuccess)
        return fail(HR_ERR_OOM, "render buffers");
    cudaError_t e = cudaMemcpy(s->ws.render_params.ptr, p32.data(), sizeof(float) * sc.n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "params: %s", cudaGetErrorString(e));
    launch_render_image(sc, (const float*)s->ws.render_params.ptr, seed, request, sub, k, tag, spp,
                        (float*)s->ws.render_img.ptr, s->stream);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(HR_ERR_CUDA, "render: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpyAsync(h_img, s->ws.render_img.ptr, sizeof(float) * npx, cudaMemcpyDeviceToHost, s->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
        return fail(HR_ERR_CUDA, "render: %s", cudaGetErrorString(e));
    return HR_OK;
}

}  // extern "C"
