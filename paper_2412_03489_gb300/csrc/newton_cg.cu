// K7: batched Newton-CG (Sec. 2 "Newton Conjugate Gradient"; trust-region
// step truncation alpha = min(alpha, Delta / |p|); non-positive curvature
// exit, Suppl. "Positive-Definite Hessians").
//
// One step for B instances is four launches, captured once into a CUDA graph
// and replayed:
//   1. sampler: per instance one aggregate-gradient group (sub 64 s) and K
//      aggregate-Hessian groups (sub 64 s + 1 + i) whose HVP weights depend
//      on the CG direction and are formed later from the stored 1/S(tau);
//   2. renders of all B (M_g + K M_h) perturbations in one launch (the
//      renders do not depend on the CG direction, only on theta);
//   3. gradient sums (Kahan FP32 chunks, FP64 tree) per instance;
//   4. one CTA per instance runs the K CG iterations in FP64; each Hessian
//      product is the HVP estimate of its own fresh sample group, its sums in
//      Kahan FP32; theta += d; the device step counter advances.
#include <cmath>
#include <cstring>
#include <vector>

#include "hr.h"
#include "hr_api_internal.h"
#include "hr_device.cuh"
#include "hr_internal.h"

namespace hr {
namespace {

constexpr int kCgThreads = 128;
constexpr int kMaxN = 64;

__global__ void theta32_kernel(const double* th, float* th32, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) th32[i] = __double2float_rn(th[i]);
}

// g[b][e] = 1/Mg sum over the instance's gradient rows of w[m][e] loss[m]
__global__ void __launch_bounds__(256) grad_reduce_kernel(const float* w, const float* loss, int n, int per_inst,
                                                          int Mg, double* g) {
    __shared__ double sh[256];
    const int e = blockIdx.x, b = blockIdx.y;
    const int m0 = b * per_inst;
    const int chunk = (Mg + 255) / 256;
    const int beg = m0 + threadIdx.x * chunk, end = min(m0 + Mg, beg + chunk);
    Kahan k;
    for (int m = beg; m < end; ++m) k.add(__fmul_rn(w[(size_t)m * n + e], loss[m]));
    sh[threadIdx.x] = (double)k.s - (double)k.c;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) g[b * n + e] = sh[0] / (double)Mg;
}

struct CgArgs {
    int n, per_inst, Mg, Mh, K;
    double sigma, lambda_rel, delta;
    const float* tau;
    const float* invS;
    const float* loss;
    const double* g;
    double* theta;
    hr_step_info* info;
    int32_t* step;
    double* tr_p;     // [B][K][n] CG directions of the step
    double* tr_Hp;    // [B][K][n] their HVP estimates (without lambda p)
};

__global__ void __launch_bounds__(kCgThreads) cg_kernel(CgArgs a) {
    __shared__ double d[kMaxN], r[kMaxN], p[kMaxN], Hp[kMaxN], red[kCgThreads / 32];
    __shared__ double tp[512];
    const int b = blockIdx.x, n = a.n;
    const double s2 = a.sigma * a.sigma, is2 = 1.0 / s2, is4 = is2 * is2;   // reciprocals: FP64 division is slow here
    const double* g = a.g + (size_t)b * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) { d[i] = 0.0; r[i] = -g[i]; p[i] = r[i]; }
    __syncthreads();
    const double gn = sqrt(block_dot(g, g, n, red));
    const double lam = a.lambda_rel * gn;
    double rr = block_dot(r, r, n, red);
    int iters = 0, reason = 0;
    for (int it = 0; it < a.K; ++it) {
        iters = it + 1;
        const int m0 = b * a.per_inst + a.Mg + it * a.Mh;
        // tau_m . p for the product's perturbations (n_hvp <= 512)
        for (int q = threadIdx.x; q < a.Mh; q += blockDim.x) {
            const float* t = a.tau + (size_t)(m0 + q) * n;
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += (double)t[j] * p[j];
            tp[q] = s;
        }
        __syncthreads();
        // HVP_k = 1/Mh sum_m loss_m w_mk, w_mk = (tau_mk (tau_m.p)/s^4 - p_k/s^2) n^2/S(tau_m)
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            Kahan acc;
            for (int q = 0; q < a.Mh; ++q) {
                const int m = m0 + q;
                const double tq = tp[q];
                const double w = ((double)a.tau[(size_t)m * n + k] * tq * is4 - p[k] * is2) * (double)a.invS[m];
                acc.add(__fmul_rn((float)w, a.loss[m]));
            }
            const double hv = ((double)acc.s - (double)acc.c) / (double)a.Mh;
            Hp[k] = hv + lam * p[k];
            const size_t tr = ((size_t)b * a.K + it) * n + k;
            a.tr_p[tr] = p[k];
            a.tr_Hp[tr] = hv;
        }
        __syncthreads();
        const double pHp = block_dot(p, Hp, n, red);
        const double pn = sqrt(block_dot(p, p, n, red));
        if (!(pHp > 0.0) || pn == 0.0) {
            if (it == 0 && pn > 0.0)
                for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = p[i] * (a.delta / pn);
            reason = 1;
            __syncthreads();
            break;
        }
        const double alpha = fmin(rr / pHp, a.delta / pn);
        for (int i = threadIdx.x; i < n; i += blockDim.x) { d[i] += alpha * p[i]; r[i] -= alpha * Hp[i]; }
        __syncthreads();
        const double rr_new = block_dot(r, r, n, red);
        if (rr_new == 0.0) { reason = 2; break; }
        const double beta = rr_new / rr;
        for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = r[i] + beta * p[i];
        __syncthreads();
        rr = rr_new;
    }
    __syncthreads();
    const double dn = sqrt(block_dot(d, d, n, red));
    for (int i = threadIdx.x; i < n; i += blockDim.x) a.theta[(size_t)b * n + i] += d[i];
    if (threadIdx.x == 0) {
        hr_step_info& inf = a.info[b];
        inf.grad_norm = gn;
        inf.lambda = lam;
        inf.iters = iters;
        inf.exit_reason = reason;
        inf.step_norm = dn;
    }
}

__global__ void advance_step_kernel(int32_t* step) { *step += 1; }

}  // namespace

void launch_grad_reduce(const float* w, const float* loss, int n, int per_inst, int Mg, int B, double* g,
                        cudaStream_t s) {
    grad_reduce_kernel<<<dim3(n, B), 256, 0, s>>>(w, loss, n, per_inst, Mg, g);
}

}  // namespace hr

using namespace hr;

struct hr_optstate_s {
    hr_scene scene = nullptr;
    int B = 0, n = 0, Mg = 0, Mh = 0, K = 0, per_inst = 0;
    hr_cg_opts opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevBuf theta, theta32, tau, w, invS, meta, loss, groups, g, info, step, tr_p, tr_Hp;
    hr_step_info* h_info = nullptr;   // pinned
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

hr_status enqueue_step(hr_optstate_s* st) {
    DevScene& sc = st->scene->sc;
    const int B = st->B, n = st->n;
    const int Mt = B * st->per_inst;
    SampleArgs sa{};
    sa.groups = (const SampleGroup*)st->groups.ptr;
    sa.n = n;
    sa.E = n;
    sa.sigma = st->opts.sigma;
    sa.Zg = std::sqrt(2.0 / M_PI) / st->opts.sigma;
    sa.Zd = 4.0 * std::exp(-0.5) / (std::sqrt(2.0 * M_PI) * st->opts.sigma * st->opts.sigma);
    sa.Zo = sa.Zg * sa.Zg;
    sa.seed = st->opts.seed;
    sa.tau = (float*)st->tau.ptr;
    sa.w = (float*)st->w.ptr;
    sa.invS = (float*)st->invS.ptr;
    sa.meta = (uint2*)st->meta.ptr;
    sa.step = (const int32_t*)st->step.ptr;
    const int maxP = (st->Mg > st->Mh ? st->Mg : st->Mh) / 2;
    sa.threads = sc.sample_threads;
    launch_sample(sa, B * (1 + st->K), maxP, st->stream);
    theta32_kernel<<<(B * n + 127) / 128, 128, 0, st->stream>>>((const double*)st->theta.ptr, (float*)st->theta32.ptr,
                                                                 B * n);
    RenderBatch rb{};
    rb.theta32 = (const float*)st->theta32.ptr;
    rb.tau = (const float*)st->tau.ptr;
    rb.meta = (const uint2*)st->meta.ptr;
    rb.loss = (float*)st->loss.ptr;
    rb.M = Mt;
    rb.n = n;
    rb.per_row = st->per_inst;
    rb.request0 = st->opts.request_base;
    rb.seed = st->opts.seed;
    launch_render_loss(sc, rb, st->stream);
    launch_grad_reduce((const float*)st->w.ptr, (const float*)st->loss.ptr, n, st->per_inst, st->Mg, B,
                       (double*)st->g.ptr, st->stream);
    CgArgs ca{};
    ca.n = n; ca.per_inst = st->per_inst; ca.Mg = st->Mg; ca.Mh = st->Mh; ca.K = st->K;
    ca.sigma = st->opts.sigma; ca.lambda_rel = st->opts.lambda_rel; ca.delta = st->opts.trust_radius;
    ca.tau = (const float*)st->tau.ptr;
    ca.invS = (const float*)st->invS.ptr;
    ca.loss = (const float*)st->loss.ptr;
    ca.g = (const double*)st->g.ptr;
    ca.theta = (double*)st->theta.ptr;
    ca.info = (hr_step_info*)st->info.ptr;
    ca.step = (int32_t*)st->step.ptr;
    ca.tr_p = (double*)st->tr_p.ptr;
    ca.tr_Hp = (double*)st->tr_Hp.ptr;
    cg_kernel<<<B, kCgThreads, 0, st->stream>>>(ca);
    advance_step_kernel<<<1, 1, 0, st->stream>>>((int32_t*)st->step.ptr);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "newton-cg launch: %s", cudaGetErrorString(e));
    return HR_OK;
}

}  // namespace

extern "C" {

hr_status hr_optstate_create(hr_scene scene, int32_t B, const double* theta0, const hr_cg_opts* o, hr_optstate* out) {
    clear_error();
    if (!scene || !theta0 || !o || !out) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    const int n = scene->sc.n;
    if (B < 1 || B > 4096) return fail(HR_ERR_INVALID_ARG, "n_instances must be 1..4096");
    if (!(o->sigma > 0.0)) return fail(HR_ERR_INVALID_ARG, "sigma must be > 0");
    if (o->n_grad < 2 || (o->n_grad & 1) || o->n_hvp < 2 || (o->n_hvp & 1) || o->n_hvp > 512)
        return fail(HR_ERR_INVALID_ARG, "n_grad, n_hvp must be even and >= 2 (n_hvp <= 512)");
    if (o->cg_iters < 1 || o->cg_iters > 63) return fail(HR_ERR_INVALID_ARG, "cg_iters must be 1..63");
    if (!(o->trust_radius > 0.0) || !(o->lambda_rel >= 0.0)) return fail(HR_ERR_INVALID_ARG, "bad trust radius/lambda");
    if (n > kMaxN) return fail(HR_ERR_INVALID_ARG, "n > %d", kMaxN);
    hr_optstate_s* st = new hr_optstate_s();
    st->scene = scene; st->B = B; st->n = n; st->opts = *o;
    st->Mg = o->n_grad; st->Mh = o->n_hvp; st->K = o->cg_iters;
    st->per_inst = st->Mg + st->K * st->Mh;
    const size_t Mt = (size_t)B * st->per_inst;
    if (o->stream) st->stream = (cudaStream_t)o->stream;
    else {
        cudaStreamCreateWithFlags(&st->stream, cudaStreamNonBlocking);
        st->own_stream = true;
    }
    cudaError_t e = cudaSuccess;
    for (auto pr : {std::make_pair(&st->theta, sizeof(double) * B * n), std::make_pair(&st->theta32, sizeof(float) * B * n),
                    std::make_pair(&st->tau, sizeof(float) * Mt * n), std::make_pair(&st->w, sizeof(float) * Mt * n),
                    std::make_pair(&st->invS, sizeof(float) * Mt), std::make_pair(&st->meta, sizeof(uint2) * Mt),
                    std::make_pair(&st->loss, sizeof(float) * Mt),
                    std::make_pair(&st->groups, sizeof(SampleGroup) * B * (1 + st->K)),
                    std::make_pair(&st->g, sizeof(double) * B * n), std::make_pair(&st->info, sizeof(hr_step_info) * B),
                    std::make_pair(&st->step, sizeof(int32_t)),
                    std::make_pair(&st->tr_p, sizeof(double) * B * st->K * n),
                    std::make_pair(&st->tr_Hp, sizeof(double) * B * st->K * n)}) {
        if (e == cudaSuccess) e = pr.first->reserve(pr.second);
    }
    if (e == cudaSuccess) e = cudaMallocHost((void**)&st->h_info, sizeof(hr_step_info) * B);
    if (e != cudaSuccess) {
        hr_optstate_destroy(st);
        return fail(HR_ERR_OOM, "optimizer state: %s", cudaGetErrorString(e));
    }
    std::vector<SampleGroup> groups(B * (1 + st->K));
    for (int b = 0; b < B; ++b) {
        for (int j = 0; j <= st->K; ++j) {
            SampleGroup& G = groups[b * (1 + st->K) + j];
            G.m0 = b * st->per_inst + (j == 0 ? 0 : st->Mg + (j - 1) * st->Mh);
            G.P = (j == 0 ? st->Mg : st->Mh) / 2;
            G.lobe = j == 0 ? 0 : 1;
            G.comp_i = -1; G.comp_j = -1;
            G.quantity = j == 0 ? 0 : 3;
            G.sub = (uint32_t)j;
            G.request = o->request_base + (uint32_t)b;
            G.theta_row = b;
            G.pad = 0;
        }
    }
    const int32_t zero = 0;
    if ((e = cudaMemcpy(st->groups.ptr, groups.data(), sizeof(SampleGroup) * groups.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(st->theta.ptr, theta0, sizeof(double) * B * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(st->step.ptr, &zero, sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess) {
        hr_optstate_destroy(st);
        return fail(HR_ERR_CUDA, "optimizer state upload: %s", cudaGetErrorString(e));
    }
    *out = st;
    return HR_OK;
}

hr_status hr_optstate_destroy(hr_optstate st) {
    if (!st) return HR_OK;
    if (st->stream) cudaStreamSynchronize(st->stream);
    if (st->exec) cudaGraphExecDestroy(st->exec);
    if (st->graph) cudaGraphDestroy(st->graph);
    for (DevBuf* b : {&st->theta, &st->theta32, &st->tau, &st->w, &st->invS, &st->meta, &st->loss, &st->groups, &st->g,
                      &st->info, &st->step, &st->tr_p, &st->tr_Hp})
        b->release();
    if (st->h_info) cudaFreeHost(st->h_info);
    if (st->own_stream && st->stream) cudaStreamDestroy(st->stream);
    delete st;
    return HR_OK;
}

hr_status hr_newton_cg_step(hr_scene scene, hr_optstate st, hr_step_info* h_info) {
    clear_error();
    if (!scene || !st || st->scene != scene) return fail(HR_ERR_INVALID_ARG, "state does not belong to this scene");
    std::lock_guard<std::mutex> lk(scene->mu);
    const hr_status s = hr::optstate_launch_step(st, h_info != nullptr);
    if (s != HR_OK) return s;
    const cudaError_t e = cudaStreamSynchronize(st->stream);
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "step: %s", cudaGetErrorString(e));
    if (h_info) memcpy(h_info, st->h_info, sizeof(hr_step_info) * st->B);
    return HR_OK;
}

}  // extern "C"

namespace hr {

// One step on the state's stream (graph replay or direct launches) and, if
// asked, the step records copied to the state's pinned buffer; returns
// without waiting.
hr_status optstate_launch_step(hr_optstate st, bool copy_info) {
    cudaError_t e;
    if (st->opts.use_graph) {
        if (!st->exec) {
            if ((e = cudaStreamBeginCapture(st->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return fail(HR_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
            const hr_status s = enqueue_step(st);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(st->stream, &g);
            if (s != HR_OK) { if (g) cudaGraphDestroy(g); return s; }
            if (e != cudaSuccess) return fail(HR_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
            st->graph = g;
            if ((e = cudaGraphInstantiate(&st->exec, g, 0)) != cudaSuccess)
                return fail(HR_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
        }
        if ((e = cudaGraphLaunch(st->exec, st->stream)) != cudaSuccess)
            return fail(HR_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    } else {
        const hr_status s = enqueue_step(st);
        if (s != HR_OK) return s;
    }
    if (copy_info) {
        if ((e = cudaMemcpyAsync(st->h_info, st->info.ptr, sizeof(hr_step_info) * st->B, cudaMemcpyDeviceToHost,
                                 st->stream)) != cudaSuccess)
            return fail(HR_ERR_CUDA, "info: %s", cudaGetErrorString(e));
    }
    return HR_OK;
}

cudaStream_t optstate_stream(hr_optstate st) { return st->stream; }
int optstate_instances(hr_optstate st) { return st->B; }
hr_scene optstate_scene(hr_optstate st) { return st->scene; }
void optstate_copy_info(hr_optstate st, hr_step_info* out) { memcpy(out, st->h_info, sizeof(hr_step_info) * st->B); }

}  // namespace hr

extern "C" {

hr_status hr_optstate_trace(hr_optstate st, double* h_g, double* h_p, double* h_Hp) {
    clear_error();
    if (!st) return fail(HR_ERR_INVALID_ARG, "NULL state");
    cudaError_t e = cudaStreamSynchronize(st->stream);
    const size_t nk = (size_t)st->B * st->K * st->n;
    if (e == cudaSuccess && h_g) e = cudaMemcpy(h_g, st->g.ptr, sizeof(double) * st->B * st->n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_p) e = cudaMemcpy(h_p, st->tr_p.ptr, sizeof(double) * nk, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_Hp) e = cudaMemcpy(h_Hp, st->tr_Hp.ptr, sizeof(double) * nk, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "trace: %s", cudaGetErrorString(e));
    return HR_OK;
}

hr_status hr_optstate_theta(hr_optstate st, double* h_theta) {
    clear_error();
    if (!st || !h_theta) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    const cudaError_t e = cudaMemcpy(h_theta, st->theta.ptr, sizeof(double) * st->B * st->n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "theta: %s", cudaGetErrorString(e));
    return HR_OK;
}

}  // extern "C"
