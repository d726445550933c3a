// hr_estimate_dev_noalloc: the device-pointer estimate for callers that must
// not allocate device memory while they run.
//
// Its working memory (perturbations, weights, path keys, per-render losses,
// sample-group table, FP32 parameters, sums) is a fixed array in the
// library's own device memory, so the call itself never allocates: no
// cudaMalloc, no cudaFree, no allocating library routine.  The array is
// kScratchBytes (4 MiB) on every GPU that loads the library, held until the
// process exits.  Requests that need more than that are rejected with
// HR_ERR_INVALID_ARG before anything is launched.
#include <cmath>
#include <mutex>

#include "hr.h"
#include "hr_api_internal.h"
#include "hr_device.cuh"
#include "hr_internal.h"

namespace hr {
namespace {

constexpr size_t kScratchBytes = size_t(4) << 20;
constexpr int kMaxDevices = 64;

// In host code this name is only a stand-in for the device array; its device
// address comes from cudaGetSymbolAddress (see scratch_base).
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device with that device current.
hr_status scratch_base(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(HR_ERR_UNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return fail(HR_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return HR_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// The sample-group table, written on the device so that the call needs no
// host staging: group g draws P pairs for element g (element-wise) or from
// the mixture (aggregate).
__global__ void fill_groups_kernel(SampleGroup* groups, int G, int n, int quantity, int strategy, int M,
                                   uint32_t sub, uint32_t request) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    SampleGroup gr;
    gr.m0 = g * M;
    gr.P = M / 2;
    gr.lobe = quantity == HR_GRAD ? 0 : 1;
    gr.quantity = quantity;
    gr.sub = sub + (uint32_t)g;
    gr.request = request;
    gr.theta_row = 0;
    gr.pad = 0;
    if (strategy == HR_AGGREGATE) {
        gr.comp_i = -1; gr.comp_j = -1;
    } else if (strategy == HR_PLAIN) {
        gr.comp_i = -3; gr.comp_j = -3;
    } else if (quantity == HR_GRAD) {
        gr.comp_i = g; gr.comp_j = g;
    } else if (quantity == HR_HVP) {
        gr.comp_i = g; gr.comp_j = -2; gr.quantity = 4;
    } else {
        int r = 0, rem = g;
        while (rem >= n - r) { rem -= n - r; ++r; }
        gr.comp_i = r; gr.comp_j = r + rem;
    }
    groups[g] = gr;
}

__global__ void theta_to_f32_kernel(const double* in, float* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __double2float_rn(in[i]);
}

}  // namespace
}  // namespace hr

using namespace hr;

extern "C" hr_status hr_estimate_dev_noalloc(hr_scene s, int32_t quantity, const double* d_theta, const double* d_v,
                                             const hr_opts* o, double* d_out) {
    clear_error();
    if (!s || !o) return fail(HR_ERR_INVALID_ARG, "scene/opts is NULL");
    if (quantity < HR_GRAD || quantity > HR_HVP) return fail(HR_ERR_INVALID_ARG, "unknown quantity %d", quantity);
    if (!d_theta || !d_out || (quantity == HR_HVP && !d_v)) return fail(HR_ERR_INVALID_ARG, "NULL device pointer");
    // the scene's launch shapes and device pointers are read under its lock,
    // as in hr_estimate_dev (the autotuner and scene teardown take it too)
    std::lock_guard<std::mutex> lk(s->mu);
    const hr_status valid = validate_opts(s, quantity, o);
    if (valid != HR_OK) return valid;
    const DevScene& sc = s->sc;
    const int n = sc.n;
    const int E = n_elements(quantity, n);
    const int G = o->strategy == HR_ELEMENTWISE ? E : 1;
    const int64_t M = o->n_perturb;
    const int64_t Mt = (int64_t)G * M;

    // carve the fixed array: theta32 | groups | tau | weights | keys | losses | sums | scale
    const size_t off_theta = 0;
    const size_t off_groups = off_theta + align256(sizeof(float) * n);
    const size_t off_tau = off_groups + align256(sizeof(SampleGroup) * (size_t)G);
    const size_t off_w = off_tau + align256(sizeof(float) * (size_t)Mt * n);
    const size_t off_meta = off_w + align256(sizeof(float) * (size_t)Mt * E);
    const size_t off_loss = off_meta + align256(sizeof(uint2) * (size_t)Mt);
    const size_t off_flat = off_loss + align256(sizeof(float) * (size_t)Mt);
    const size_t off_scale = off_flat + align256(sizeof(double) * (size_t)E);
    const size_t need = off_scale + align256(sizeof(double) * (size_t)E);
    if (need > kScratchBytes)
        return fail(HR_ERR_INVALID_ARG,
                    "request needs %zu bytes of working memory; this entry point has a fixed %zu-byte array "
                    "(use hr_estimate_dev for larger requests)",
                    need, kScratchBytes);
    unsigned char* base = nullptr;
    const hr_status st = scratch_base(&base);
    if (st != HR_OK) return st;
    cudaStream_t stream = o->stream ? (cudaStream_t)o->stream : s->stream;

    float* theta32 = reinterpret_cast<float*>(base + off_theta);
    SampleGroup* groups = reinterpret_cast<SampleGroup*>(base + off_groups);
    theta_to_f32_kernel<<<(n + 127) / 128, 128, 0, stream>>>(d_theta, theta32, n);
    fill_groups_kernel<<<(G + 127) / 128, 128, 0, stream>>>(groups, G, n, quantity, o->strategy, (int)M, o->sub,
                                                            o->request_id);
    SampleArgs sa{};
    sa.groups = groups;
    sa.n = n;
    sa.E = E;
    sa.sigma = o->sigma;
    const double s2 = o->sigma * o->sigma;
    sa.Zg = std::sqrt(2.0 / M_PI) / o->sigma;
    sa.Zd = 4.0 * std::exp(-0.5) / (std::sqrt(2.0 * M_PI) * s2);
    sa.Zo = sa.Zg * sa.Zg;
    sa.seed = o->seed;
    sa.v = d_v;
    sa.tau = reinterpret_cast<float*>(base + off_tau);
    sa.w = reinterpret_cast<float*>(base + off_w);
    sa.invS = nullptr;
    sa.meta = reinterpret_cast<uint2*>(base + off_meta);
    sa.step = nullptr;
    sa.threads = sc.sample_threads;
    launch_sample(sa, G, (int)(M / 2), stream);

    RenderBatch rb{};
    rb.theta32 = theta32;
    rb.tau = sa.tau;
    rb.meta = sa.meta;
    rb.loss = reinterpret_cast<float*>(base + off_loss);
    rb.M = (int32_t)Mt;
    rb.n = n;
    rb.per_row = (int32_t)Mt;
    rb.request0 = o->request_id;
    rb.seed = o->seed;
    launch_render_loss(sc, rb, stream);

    FinalizeArgs fa{};
    fa.w = sa.w;
    fa.loss = rb.loss;
    fa.E = E;
    fa.n = n;
    fa.pairs2 = (int32_t)M;
    fa.elementwise = o->strategy == HR_ELEMENTWISE;
    fa.hessian = quantity == HR_HESSIAN;
    fa.inv2P = 1.0 / (double)M;
    fa.out_flat = quantity == HR_HESSIAN ? reinterpret_cast<double*>(base + off_flat) : d_out;
    fa.out_scale = reinterpret_cast<double*>(base + off_scale);
    fa.out_full = quantity == HR_HESSIAN ? d_out : nullptr;
    launch_finalize(fa, stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    return HR_OK;
}
