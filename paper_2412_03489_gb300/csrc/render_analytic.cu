// Analytic test functions in place of a renderer: f(p) at the FP32 perturbed
// parameters p = RN32(theta32 + tau), evaluated in FP64 and stored as the
// perturbation's FP32 loss.  Their smoothed derivatives have closed forms
// (the Quad task of Sec. 4.1, the 1D hard edge, the negated Gaussian of the
// supplement on positive-definite Hessians), which pins the estimators on the
// GPU without a rendered image.  One thread per perturbation.
#include <cmath>

#include "hr.h"
#include "hr_device.cuh"
#include "hr_internal.h"

namespace hr {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ double analytic_f(int kind, int n, const float* p, const double* A, const double* b, double gs) {
    if (kind == HR_SCENE_STEP1D) return p[0] > 0.0f ? 1.0 : 0.0;
    if (kind == HR_SCENE_NEGGAUSS) {
        double r2 = 0.0;
        for (int i = 0; i < n; ++i) r2 += (double)p[i] * (double)p[i];
        const double s2 = gs * gs;
        return -exp(-0.5 * r2 / s2) / pow(kTwoPi * s2, 0.5 * n);
    }
    // quadratic: 1/2 p^T A p + b^T p
    double f = 0.0;
    for (int i = 0; i < n; ++i) {
        double row = 0.0;
        for (int j = 0; j < n; ++j) row += A[i * n + j] * (double)p[j];
        f += (double)p[i] * (0.5 * row + b[i]);
    }
    return f;
}

__global__ void analytic_loss_kernel(RenderBatch rb, int kind, const double* A, const double* b, double gs) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= rb.M) return;
    const Pert pt = resolve(rb, m);
    float p[64];
    const int n = rb.n;
    for (int i = 0; i < n; ++i) p[i] = __fadd_rn(pt.theta[i], pt.tau[i]);
    *pt.loss = (float)analytic_f(kind, n, p, A, b, gs);
}

__global__ void analytic_image_kernel(const float* params, int kind, int n, const double* A, const double* b,
                                      double gs, float* img) {
    if (threadIdx.x == 0 && blockIdx.x == 0) img[0] = (float)analytic_f(kind, n, params, A, b, gs);
}

}  // namespace

void launch_analytic_loss(const DevScene& sc, const RenderBatch& b, cudaStream_t s) {
    analytic_loss_kernel<<<(b.M + 127) / 128, 128, 0, s>>>(b, sc.kind, sc.qA, sc.qb, sc.gauss_sigma);
}

void launch_analytic_image(const DevScene& sc, const float* params, float* img, cudaStream_t s) {
    analytic_image_kernel<<<1, 32, 0, s>>>(params, sc.kind, sc.n, sc.qA, sc.qb, sc.gauss_sigma, img);
}

}  // namespace hr
