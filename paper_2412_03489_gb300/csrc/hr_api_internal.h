// Host-side objects behind the opaque C-ABI handles.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "hr.h"
#include "hr_internal.h"

namespace hr {

hr_status fail(hr_status code, const char* fmt, ...);
void clear_error();
const std::string& last_error();

// device buffer that grows on demand (contents are not preserved)
struct DevBuf {
    void* ptr = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t bytes);
    void release();
};

struct Workspace {
    DevBuf theta32, v, tau, w, meta, loss, flat, scale, full, groups, render_img, render_params;
    DevBuf gb_J, gb_vx, gb_y, gb_vy, gb_out, gb_tmp, gb_hj;
    void release_all() {
        for (DevBuf* b : {&theta32, &v, &tau, &w, &meta, &loss, &flat, &scale, &full, &groups, &render_img,
                          &render_params, &gb_J, &gb_vx, &gb_y, &gb_vy, &gb_out, &gb_tmp, &gb_hj})
            b->release();
    }
};

}  // namespace hr

struct hr_scene_s {
    hr::DevScene sc;
    std::mutex mu;
    cudaStream_t stream = nullptr;
    hr::Workspace ws;
    std::vector<hr::SampleGroup> host_groups;
    bool profile = false;
    bool profile_valid = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace hr {
hr_status optstate_launch_step(hr_optstate st, bool copy_info);
cudaStream_t optstate_stream(hr_optstate st);
int optstate_instances(hr_optstate st);
hr_scene optstate_scene(hr_optstate st);
void optstate_copy_info(hr_optstate st, hr_step_info* out);

// Checks of an estimate's options shared by every estimate entry point:
// sigma > 0, M even and >= 2, a known strategy, pair / perturbation /
// sub-stream counts within range; HR_ERR_INVALID_ARG (with a message)
// otherwise.
int n_elements(int quantity, int n);
hr_status validate_opts(const hr_scene_s* s, int quantity, const hr_opts* o);

hr_status run_hvp_fd(hr_scene_s* s, const double* h_theta, const double* h_v, double eps, const hr_opts* o,
                     double* h_out);
hr_status run_estimate(hr_scene_s* s, int quantity, const double* h_theta, const double* d_theta, const double* h_v,
                       const double* d_v, const hr_opts* o, double* h_out, double* d_out);
}
