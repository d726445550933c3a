// The optimiser as the paper runs it: conjugate directions with the point
// moved at every iteration (Sec. 2 "Newton Conjugate Gradient", Eq.
// pertubation for the step, Fletcher-Reeves directions, trust-region
// truncation), a Newton-Raphson line search of at most J steps with a
// tolerance, a recompute period for the residual, and linear annealing of the
// smoothing bandwidth per outer iteration (Suppl. "Hyperparameters").
//
// One evaluation for B instances is five launches, captured once into a CUDA
// graph and replayed:
//   1. sampler: per instance an aggregate-gradient group (sub 64 e) and an
//      aggregate-Hessian group (sub 64 e + 1) that stores 1/S(tau) only, both
//      at the instance's own bandwidth sigma_b read from device memory;
//   2. theta -> FP32; 3. renders of all B (M_g + M_h) perturbations;
//   4. gradient sums per instance (Kahan FP32 chunks, FP64 tree);
//   5. one CTA per instance: direction update (first line-search step of an
//      outer iteration), the Hessian-vector product Hd from the stored
//      perturbations (the renders do not depend on d), the step alpha, x, r,
//      the line-search and annealing state; then the evaluation counter
//      advances.
#include <cmath>
#include <cstring>
#include <vector>

#include "hr.h"
#include "hr_api_internal.h"
#include "hr_device.cuh"
#include "hr_internal.h"

namespace hr {
namespace {

constexpr int kNcgThreads = 128;
constexpr int kMaxN = 64;
constexpr int kMaxHvp = 512;
constexpr int kMaxEvals = 1 << 18;   // sub 64 e + 1 must fit 24 bits

// sigma_i of the linear schedule: start + (end - start) i / (T - 1), end from
// i >= T - 1, start throughout for T <= 1
__host__ __device__ inline double anneal(double start, double end, int T, int i) {
    if (T <= 1) return start;
    if (i >= T - 1) return end;
    return start + (end - start) * (double)i / (double)(T - 1);
}

struct NcgArgs {
    int n, per_inst, Mg, Mh, J, R, T, mode;
    double sigma_start, sigma_end, tol, delta, lambda_rel;
    const float* tau;
    const float* invS;
    const float* loss;
    const double* g;      // [B][n]
    double* theta;        // [B][n]
    double* d;            // [B][n]
    double* r;            // [B][n]
    double* rr;           // [B]
    int32_t* it;          // [B]
    int32_t* ls;          // [B]
    double* sigma;        // [B]
    hr_ncg_info* info;    // [B]
    double* tr_q;         // [B][n] HVP estimate H d of the evaluation (without lambda d)
};

__global__ void __launch_bounds__(kNcgThreads) ncg_kernel(NcgArgs a) {
    __shared__ double d[kMaxN], r[kMaxN], q[kMaxN], red[kNcgThreads / 32];
    __shared__ double tp[kMaxHvp];
    const int b = blockIdx.x, n = a.n;
    const double* g = a.g + (size_t)b * n;
    double* gd_ = a.d + (size_t)b * n;
    double* gr_ = a.r + (size_t)b * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) { d[i] = gd_[i]; r[i] = gr_[i]; }
    const int it = a.it[b], j = a.ls[b];
    const double sigma = a.sigma[b];
    double rr = a.rr[b];
    int restarted = 0;
    __syncthreads();
    if (j == 0) {
        if (it % a.R == 0) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) { r[i] = -g[i]; d[i] = -g[i]; }
            __syncthreads();
            rr = block_dot(r, r, n, red);
            restarted = 1;
        } else {
            if (a.mode == 1) {
                for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] = -g[i];
                __syncthreads();
            }
            const double rr_new = block_dot(r, r, n, red);
            const double beta = rr > 0.0 ? rr_new / rr : 0.0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = r[i] + beta * d[i];
            __syncthreads();
            if (!(block_dot(r, d, n, red) > 0.0)) {
                for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = r[i];
                __syncthreads();
                restarted = 1;
            }
            rr = rr_new;
        }
    }
    const double gn = sqrt(block_dot(g, g, n, red));
    const double lam = a.lambda_rel * gn;
    // Hd = 1/Mh sum_m loss_m (tau_m (tau_m.d)/s^4 - d/s^2) n^2/S(tau_m) + lambda d
    const double s2 = sigma * sigma, is2 = 1.0 / s2, is4 = is2 * is2;   // reciprocals: FP64 division is slow here
    const int m0 = b * a.per_inst + a.Mg;
    for (int k = threadIdx.x; k < a.Mh; k += blockDim.x) {
        const float* t = a.tau + (size_t)(m0 + k) * n;
        double s = 0.0;
        for (int c = 0; c < n; ++c) s += (double)t[c] * d[c];
        tp[k] = s;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        Kahan acc;
        for (int k = 0; k < a.Mh; ++k) {
            const int m = m0 + k;
            const double w = ((double)a.tau[(size_t)m * n + c] * tp[k] * is4 - d[c] * is2) * (double)a.invS[m];
            acc.add(__fmul_rn((float)w, a.loss[m]));
        }
        const double hv = ((double)acc.s - (double)acc.c) / (double)a.Mh;
        q[c] = hv + lam * d[c];
        a.tr_q[(size_t)b * n + c] = hv;
    }
    __syncthreads();
    const double gdv = block_dot(g, d, n, red);
    const double dHd = block_dot(d, q, n, red);
    const double dn = sqrt(block_dot(d, d, n, red));
    double alpha = 0.0;
    if (dn > 0.0) {
        const double cap = a.delta / dn;
        if (dHd > 0.0) alpha = -gdv / dHd;
        else if (gdv < 0.0) alpha = cap;
        else if (gdv > 0.0) alpha = -cap;
        alpha = fmin(fmax(alpha, -cap), cap);
    }
    double* th = a.theta + (size_t)b * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        th[i] += alpha * d[i];
        gd_[i] = d[i];
        gr_[i] = a.mode == 0 ? r[i] - alpha * q[i] : r[i];
    }
    if (threadIdx.x == 0) {
        hr_ncg_info& inf = a.info[b];
        inf.iter = it;
        inf.ls_step = j;
        inf.restarted = restarted;
        inf.pad = 0;
        inf.sigma = sigma;
        inf.grad_norm = gn;
        inf.gd = gdv;
        inf.dHd = dHd;
        inf.alpha = alpha;
        inf.step_norm = fabs(alpha) * dn;
        a.rr[b] = rr;
        if (j + 1 >= a.J || fabs(alpha) * dn <= a.tol) {
            a.ls[b] = 0;
            a.it[b] = it + 1;
            a.sigma[b] = anneal(a.sigma_start, a.sigma_end, a.T, it + 1);
        } else {
            a.ls[b] = j + 1;
        }
    }
}

__global__ void ncg_theta32_kernel(const double* th, float* th32, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) th32[i] = __double2float_rn(th[i]);
}

__global__ void ncg_advance_kernel(int32_t* e) { *e += 1; }

}  // namespace
}  // namespace hr

using namespace hr;

struct hr_ncg_s {
    hr_scene scene = nullptr;
    int B = 0, n = 0, per_inst = 0;
    int64_t evals = 0;                 // evaluations issued (host count)
    hr_ncg_opts opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevBuf theta, theta32, tau, w, invS, meta, loss, groups, g, d, r, rr, it, ls, sigma, info, evc, tr_q;
    hr_ncg_info* h_info = nullptr;     // pinned [cap][B]
    int h_cap = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

hr_status enqueue_eval(hr_ncg_s* st) {
    DevScene& sc = st->scene->sc;
    const int B = st->B, n = st->n;
    const hr_ncg_opts& o = st->opts;
    SampleArgs sa{};
    sa.groups = (const SampleGroup*)st->groups.ptr;
    sa.n = n;
    sa.E = n;
    sa.sigma = o.sigma_start;        // unused: every group reads sigma_row
    sa.seed = o.seed;
    sa.tau = (float*)st->tau.ptr;
    sa.w = (float*)st->w.ptr;
    sa.invS = (float*)st->invS.ptr;
    sa.meta = (uint2*)st->meta.ptr;
    sa.step = (const int32_t*)st->evc.ptr;
    sa.sigma_row = (const double*)st->sigma.ptr;
    sa.threads = sc.sample_threads;
    launch_sample(sa, 2 * B, (o.n_grad > o.n_hvp ? o.n_grad : o.n_hvp) / 2, st->stream);
    ncg_theta32_kernel<<<(B * n + 127) / 128, 128, 0, st->stream>>>((const double*)st->theta.ptr,
                                                                     (float*)st->theta32.ptr, B * n);
    RenderBatch rb{};
    rb.theta32 = (const float*)st->theta32.ptr;
    rb.tau = (const float*)st->tau.ptr;
    rb.meta = (const uint2*)st->meta.ptr;
    rb.loss = (float*)st->loss.ptr;
    rb.M = B * st->per_inst;
    rb.n = n;
    rb.per_row = st->per_inst;
    rb.request0 = o.request_base;
    rb.seed = o.seed;
    launch_render_loss(sc, rb, st->stream);
    launch_grad_reduce((const float*)st->w.ptr, (const float*)st->loss.ptr, n, st->per_inst, o.n_grad, B,
                       (double*)st->g.ptr, st->stream);
    NcgArgs a{};
    a.n = n; a.per_inst = st->per_inst; a.Mg = o.n_grad; a.Mh = o.n_hvp;
    a.J = o.ls_iters; a.R = o.recompute; a.T = o.anneal_iters; a.mode = o.residual_mode;
    a.sigma_start = o.sigma_start; a.sigma_end = o.sigma_end; a.tol = o.ls_tol; a.delta = o.trust_radius;
    a.lambda_rel = o.lambda_rel;
    a.tau = (const float*)st->tau.ptr;
    a.invS = (const float*)st->invS.ptr;
    a.loss = (const float*)st->loss.ptr;
    a.g = (const double*)st->g.ptr;
    a.theta = (double*)st->theta.ptr;
    a.d = (double*)st->d.ptr;
    a.r = (double*)st->r.ptr;
    a.rr = (double*)st->rr.ptr;
    a.it = (int32_t*)st->it.ptr;
    a.ls = (int32_t*)st->ls.ptr;
    a.sigma = (double*)st->sigma.ptr;
    a.info = (hr_ncg_info*)st->info.ptr;
    a.tr_q = (double*)st->tr_q.ptr;
    ncg_kernel<<<B, kNcgThreads, 0, st->stream>>>(a);
    ncg_advance_kernel<<<1, 1, 0, st->stream>>>((int32_t*)st->evc.ptr);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "optimiser launch: %s", cudaGetErrorString(e));
    return HR_OK;
}

hr_status launch_eval(hr_ncg_s* st) {
    cudaError_t e;
    if (!st->opts.use_graph) return enqueue_eval(st);
    if (!st->exec) {
        if ((e = cudaStreamBeginCapture(st->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return fail(HR_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
        const hr_status s = enqueue_eval(st);
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
    return HR_OK;
}

}  // namespace

extern "C" {

hr_status hr_ncg_create(hr_scene scene, int32_t B, const double* theta0, const hr_ncg_opts* o, hr_ncg* out) {
    clear_error();
    if (!scene || !theta0 || !o || !out) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    const int n = scene->sc.n;
    if (B < 1 || B > 4096) return fail(HR_ERR_INVALID_ARG, "n_instances must be 1..4096");
    if (n > kMaxN) return fail(HR_ERR_INVALID_ARG, "n > %d", kMaxN);
    if (!(o->sigma_start > 0.0) || !(o->sigma_end > 0.0) || !std::isfinite(o->sigma_start) ||
        !std::isfinite(o->sigma_end))
        return fail(HR_ERR_INVALID_ARG, "sigma_start and sigma_end must be finite and > 0");
    if (o->anneal_iters < 1) return fail(HR_ERR_INVALID_ARG, "anneal_iters must be >= 1");
    if (o->n_grad < 2 || (o->n_grad & 1) || o->n_hvp < 2 || (o->n_hvp & 1) || o->n_hvp > kMaxHvp)
        return fail(HR_ERR_INVALID_ARG, "n_grad, n_hvp must be even and >= 2 (n_hvp <= %d)", kMaxHvp);
    if (o->ls_iters < 1 || o->recompute < 1) return fail(HR_ERR_INVALID_ARG, "ls_iters and recompute must be >= 1");
    if (o->residual_mode != 0 && o->residual_mode != 1) return fail(HR_ERR_INVALID_ARG, "residual_mode must be 0 or 1");
    if (!(o->trust_radius > 0.0) || !(o->lambda_rel >= 0.0) || std::isnan(o->ls_tol))
        return fail(HR_ERR_INVALID_ARG, "bad trust radius, lambda or tolerance");
    hr_ncg_s* st = new hr_ncg_s();
    st->scene = scene; st->B = B; st->n = n; st->opts = *o;
    st->per_inst = o->n_grad + o->n_hvp;
    const size_t Mt = (size_t)B * st->per_inst;
    if (o->stream) st->stream = (cudaStream_t)o->stream;
    else {
        cudaStreamCreateWithFlags(&st->stream, cudaStreamNonBlocking);
        st->own_stream = true;
    }
    cudaError_t e = cudaSuccess;
    const size_t Bn = (size_t)B * n;
    for (auto pr : {std::make_pair(&st->theta, sizeof(double) * Bn), std::make_pair(&st->theta32, sizeof(float) * Bn),
                    std::make_pair(&st->tau, sizeof(float) * Mt * n), std::make_pair(&st->w, sizeof(float) * Mt * n),
                    std::make_pair(&st->invS, sizeof(float) * Mt), std::make_pair(&st->meta, sizeof(uint2) * Mt),
                    std::make_pair(&st->loss, sizeof(float) * Mt),
                    std::make_pair(&st->groups, sizeof(SampleGroup) * 2 * B),
                    std::make_pair(&st->g, sizeof(double) * Bn), std::make_pair(&st->d, sizeof(double) * Bn),
                    std::make_pair(&st->r, sizeof(double) * Bn), std::make_pair(&st->rr, sizeof(double) * B),
                    std::make_pair(&st->it, sizeof(int32_t) * B), std::make_pair(&st->ls, sizeof(int32_t) * B),
                    std::make_pair(&st->sigma, sizeof(double) * B), std::make_pair(&st->info, sizeof(hr_ncg_info) * B),
                    std::make_pair(&st->evc, sizeof(int32_t)), std::make_pair(&st->tr_q, sizeof(double) * Bn)}) {
        if (e == cudaSuccess) e = pr.first->reserve(pr.second);
    }
    if (e != cudaSuccess) {
        hr_ncg_destroy(st);
        return fail(HR_ERR_OOM, "optimiser state: %s", cudaGetErrorString(e));
    }
    std::vector<SampleGroup> groups(2 * B);
    for (int b = 0; b < B; ++b) {
        for (int j = 0; j < 2; ++j) {
            SampleGroup& G = groups[2 * b + j];
            G.m0 = b * st->per_inst + (j == 0 ? 0 : o->n_grad);
            G.P = (j == 0 ? o->n_grad : o->n_hvp) / 2;
            G.lobe = j;
            G.comp_i = -1; G.comp_j = -1;
            G.quantity = j == 0 ? 0 : 3;
            G.sub = (uint32_t)j;
            G.request = o->request_base + (uint32_t)b;
            G.theta_row = b;
            G.pad = 0;
        }
    }
    const double s0 = anneal(o->sigma_start, o->sigma_end, o->anneal_iters, 0);
    std::vector<double> sig(B, s0);
    const int32_t zero = 0;
    if ((e = cudaMemcpy(st->groups.ptr, groups.data(), sizeof(SampleGroup) * groups.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(st->theta.ptr, theta0, sizeof(double) * Bn, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(st->sigma.ptr, sig.data(), sizeof(double) * B, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(st->d.ptr, 0, sizeof(double) * Bn)) != cudaSuccess ||
        (e = cudaMemset(st->r.ptr, 0, sizeof(double) * Bn)) != cudaSuccess ||
        (e = cudaMemset(st->rr.ptr, 0, sizeof(double) * B)) != cudaSuccess ||
        (e = cudaMemset(st->it.ptr, 0, sizeof(int32_t) * B)) != cudaSuccess ||
        (e = cudaMemset(st->ls.ptr, 0, sizeof(int32_t) * B)) != cudaSuccess ||
        (e = cudaMemcpy(st->evc.ptr, &zero, sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess) {
        hr_ncg_destroy(st);
        return fail(HR_ERR_CUDA, "optimiser state upload: %s", cudaGetErrorString(e));
    }
    *out = st;
    return HR_OK;
}

hr_status hr_ncg_destroy(hr_ncg st) {
    if (!st) return HR_OK;
    if (st->stream) cudaStreamSynchronize(st->stream);
    if (st->exec) cudaGraphExecDestroy(st->exec);
    if (st->graph) cudaGraphDestroy(st->graph);
    for (DevBuf* b : {&st->theta, &st->theta32, &st->tau, &st->w, &st->invS, &st->meta, &st->loss, &st->groups,
                      &st->g, &st->d, &st->r, &st->rr, &st->it, &st->ls, &st->sigma, &st->info, &st->evc,
                      &st->tr_q})
        b->release();
    if (st->h_info) cudaFreeHost(st->h_info);
    if (st->own_stream && st->stream) cudaStreamDestroy(st->stream);
    delete st;
    return HR_OK;
}

hr_status hr_ncg_run(hr_scene scene, hr_ncg st, int32_t n_evals, hr_ncg_info* h_info) {
    clear_error();
    if (!scene || !st || st->scene != scene) return fail(HR_ERR_INVALID_ARG, "state does not belong to this scene");
    if (n_evals < 0) return fail(HR_ERR_INVALID_ARG, "n_evals must be >= 0");
    if (st->evals + n_evals > kMaxEvals)
        return fail(HR_ERR_INVALID_ARG, "at most %d evaluations per state", kMaxEvals);
    std::lock_guard<std::mutex> lk(scene->mu);
    cudaError_t e;
    if (h_info && n_evals > st->h_cap) {
        if (st->h_info) { cudaStreamSynchronize(st->stream); cudaFreeHost(st->h_info); st->h_info = nullptr; }
        st->h_cap = 0;
        if ((e = cudaMallocHost((void**)&st->h_info, sizeof(hr_ncg_info) * (size_t)n_evals * st->B)) != cudaSuccess)
            return fail(HR_ERR_OOM, "info buffer: %s", cudaGetErrorString(e));
        st->h_cap = n_evals;
    }
    for (int k = 0; k < n_evals; ++k) {
        const hr_status s = launch_eval(st);
        if (s != HR_OK) return s;
        ++st->evals;
        if (h_info &&
            (e = cudaMemcpyAsync(st->h_info + (size_t)k * st->B, st->info.ptr, sizeof(hr_ncg_info) * st->B,
                                 cudaMemcpyDeviceToHost, st->stream)) != cudaSuccess)
            return fail(HR_ERR_CUDA, "info: %s", cudaGetErrorString(e));
    }
    if ((e = cudaStreamSynchronize(st->stream)) != cudaSuccess)
        return fail(HR_ERR_CUDA, "optimiser: %s", cudaGetErrorString(e));
    if (h_info) memcpy(h_info, st->h_info, sizeof(hr_ncg_info) * (size_t)n_evals * st->B);
    return HR_OK;
}

hr_status hr_ncg_trace(hr_ncg st, double* h_g, double* h_d, double* h_Hd) {
    clear_error();
    if (!st) return fail(HR_ERR_INVALID_ARG, "NULL state");
    const size_t bytes = sizeof(double) * st->B * st->n;
    cudaError_t e = cudaStreamSynchronize(st->stream);
    if (e == cudaSuccess && h_g) e = cudaMemcpy(h_g, st->g.ptr, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_d) e = cudaMemcpy(h_d, st->d.ptr, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_Hd) e = cudaMemcpy(h_Hd, st->tr_q.ptr, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "trace: %s", cudaGetErrorString(e));
    return HR_OK;
}

hr_status hr_ncg_theta(hr_ncg st, double* h_theta) {
    clear_error();
    if (!st || !h_theta) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = cudaStreamSynchronize(st->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(h_theta, st->theta.ptr, sizeof(double) * st->B * st->n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "theta: %s", cudaGetErrorString(e));
    return HR_OK;
}

}  // extern "C"
