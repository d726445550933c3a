// Autotuner: per scene, times the launch shapes of the render+loss kernel and
// of the sampler on a probe estimate and keeps the fastest.  Every candidate
// computes the same values in the same order (a different register cap,
// warps per CTA or threads per block), so tuning changes speed, never a
// result: estimates before and after tuning are bit-identical.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hr.h"
#include "hr_api_internal.h"
#include "hr_internal.h"

namespace hr {

int render_variant_count(int kind) {
    switch (kind) {
        case HR_SCENE_PTBOX: return 3;     // min resident CTAs per SM 3 / 2 / 4 (register caps 80 / 128 / 64)
        case HR_SCENE_DISC2D: return 3;    // 8 / 4 / 16 warps per CTA, one warp per perturbation
        case HR_SCENE_BOXES2D: return 3;
        default: return 1;                 // mesh and 2D triangles: one CTA shape
    }
}

namespace {

constexpr int kSampleShapes[4] = {32, 64, 128, 16};

// median over `reps` profiled estimates of stage `stage` (0 sampler, 1 render)
hr_status probe(hr_scene_s* s, const double* h_theta, const double* h_v, const hr_opts& o, int stage, int reps,
                float* ms) {
    const int n = s->sc.n;
    std::vector<double> out(n);
    std::vector<float> t;
    for (int r = 0; r <= reps; ++r) {   // the first run warms up
        const hr_status st = run_estimate(s, HR_HVP, h_theta, nullptr, h_v, nullptr, &o, out.data(), nullptr);
        if (st != HR_OK) return st;
        const cudaError_t e0 = cudaEventSynchronize(s->ev[3]);
        float x = 0.0f;
        const cudaError_t e1 = cudaEventElapsedTime(&x, s->ev[stage], s->ev[stage + 1]);
        if (e0 != cudaSuccess || e1 != cudaSuccess) return fail(HR_ERR_CUDA, "tuning events");
        if (r > 0) t.push_back(x);
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return HR_OK;
}

}  // namespace
}  // namespace hr

using namespace hr;

extern "C" {

hr_status hr_set_tuning(hr_scene s, int32_t render_variant, int32_t sample_threads) {
    clear_error();
    if (!s) return fail(HR_ERR_INVALID_ARG, "scene is NULL");
    if (render_variant < 0 || render_variant >= render_variant_count(s->sc.kind))
        return fail(HR_ERR_INVALID_ARG, "render variant %d out of range", render_variant);
    if (sample_threads != 16 && sample_threads != 32 && sample_threads != 64 && sample_threads != 128)
        return fail(HR_ERR_INVALID_ARG, "sample_threads must be 16, 32, 64 or 128");
    std::lock_guard<std::mutex> lk(s->mu);
    s->sc.render_variant = render_variant;
    s->sc.sample_threads = sample_threads;
    return HR_OK;
}

hr_status hr_autotune(hr_scene s, const double* h_theta, int32_t n_probe, hr_tune_info* info) {
    clear_error();
    if (!s || !h_theta) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    if (n_probe < 2 || (n_probe & 1)) return fail(HR_ERR_INVALID_ARG, "n_probe must be even and >= 2");
    std::lock_guard<std::mutex> lk(s->mu);
    for (cudaEvent_t& e : s->ev) {
        if (!e && cudaEventCreate(&e) != cudaSuccess) return fail(HR_ERR_CUDA, "event create");
    }
    const bool was_profiled = s->profile;
    s->profile = true;
    const int n = s->sc.n;
    std::vector<double> v(n, 1.0);
    // a probe that fills the GPU several times over, so that the shapes'
    // occupancy shows in the timings (one render per CTA in the path tracer)
    const int min_probe = 8 * num_sms();
    const int probe_m = n_probe >= min_probe ? n_probe : (min_probe + 1) & ~1;
    hr_opts o{};
    o.sigma = 0.05;
    o.n_perturb = probe_m;
    o.strategy = HR_AGGREGATE;
    o.seed = 0x7E57;
    o.request_id = 0;
    hr_tune_info rep{};
    const int nv = render_variant_count(s->sc.kind);
    rep.n_render_variants = nv;
    rep.n_sample_variants = 4;
    hr_status st = HR_OK;
    int best_v = 0;
    for (int k = 0; k < nv && st == HR_OK; ++k) {
        s->sc.render_variant = k;
        st = probe(s, h_theta, v.data(), o, 1, 3, &rep.render_ms[k]);
        if (st == HR_OK && rep.render_ms[k] < rep.render_ms[best_v]) best_v = k;
    }
    int best_t = 0;
    if (st == HR_OK) s->sc.render_variant = best_v;
    for (int k = 0; k < 4 && st == HR_OK; ++k) {
        s->sc.sample_threads = kSampleShapes[k];
        st = probe(s, h_theta, v.data(), o, 0, 3, &rep.sample_ms[k]);
        if (st == HR_OK && rep.sample_ms[k] < rep.sample_ms[best_t]) best_t = k;
    }
    s->profile = was_profiled;
    s->profile_valid = false;
    if (st != HR_OK) {
        s->sc.render_variant = 0;
        s->sc.sample_threads = 32;
        return st;
    }
    s->sc.render_variant = best_v;
    s->sc.sample_threads = kSampleShapes[best_t];
    rep.render_variant = best_v;
    rep.sample_threads = kSampleShapes[best_t];
    if (info) *info = rep;
    return HR_OK;
}

}  // extern "C"
