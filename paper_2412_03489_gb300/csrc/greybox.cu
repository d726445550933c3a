// Grey-box differentials (Suppl. "Grey-box differentials"): derivatives of
// f(g(x)) where g is a white-box inner map with a caller-supplied Jacobian J
// (n x n_x) and f the black-box renderer loss.  The black-box part is the
// library's estimate at y = g(x); the compositions J^T g, J^T H J and
// J^T H (J v) run here in FP64.
#include <cstring>

#include "hr.h"
#include "hr_api_internal.h"
#include "hr_internal.h"

namespace {

// out[i] = sum_x J[i][x] v[x]   (one block per row i)
__global__ void jv_kernel(const double* J, const double* v, int n, int nx, double* out) {
    __shared__ double red[256];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) s += J[(size_t)i * nx + x] * v[x];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = red[0];
}

// out[x] = sum_i J[i][x] t[i]
__global__ void jtv_kernel(const double* J, const double* t, int n, int nx, double* out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += J[(size_t)i * nx + x] * t[i];
    out[x] = s;
}

// HJ[i][x] = sum_k H[i][k] J[k][x]
__global__ void hj_kernel(const double* H, const double* J, int n, int nx, double* HJ) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (x >= nx) return;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += H[i * n + k] * J[(size_t)k * nx + x];
    HJ[(size_t)i * nx + x] = s;
}

// out[a][b] = sum_i J[i][a] HJ[i][b]
__global__ void jthj_kernel(const double* J, const double* HJ, int n, int nx, double* out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (b >= nx) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += J[(size_t)i * nx + a] * HJ[(size_t)i * nx + b];
    out[(size_t)a * nx + b] = s;
}

}  // namespace

using namespace hr;

extern "C" hr_status hr_estimate_greybox(hr_scene s, int32_t quantity, const double* h_y, const double* h_J,
                                         int32_t nx, const double* h_vx, const hr_opts* o, double* h_out) {
    clear_error();
    if (!s || !h_y || !h_J || !h_out || !o) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    if (quantity < HR_GRAD || quantity > HR_HVP) return fail(HR_ERR_INVALID_ARG, "unknown quantity %d", quantity);
    if (quantity == HR_HVP && !h_vx) return fail(HR_ERR_INVALID_ARG, "HVP needs v_x");
    if (nx < 1 || nx > (1 << 24) || (quantity == HR_HESSIAN && nx > 4096))
        return fail(HR_ERR_INVALID_ARG, "n_x out of range");
    std::lock_guard<std::mutex> lk(s->mu);
    Workspace& ws = s->ws;
    const int n = s->sc.n;
    cudaStream_t stream = o->stream ? (cudaStream_t)o->stream : s->stream;
    const size_t nout = quantity == HR_HESSIAN ? (size_t)nx * nx : (size_t)nx;
    if (ws.gb_J.reserve(sizeof(double) * (size_t)n * nx) != cudaSuccess ||
        ws.gb_vx.reserve(sizeof(double) * (size_t)nx) != cudaSuccess ||
        ws.gb_y.reserve(sizeof(double) * n) != cudaSuccess || ws.gb_vy.reserve(sizeof(double) * n) != cudaSuccess ||
        ws.gb_out.reserve(sizeof(double) * nout) != cudaSuccess ||
        ws.gb_tmp.reserve(sizeof(double) * (size_t)n * n) != cudaSuccess ||
        (quantity == HR_HESSIAN && ws.gb_hj.reserve(sizeof(double) * (size_t)n * nx) != cudaSuccess))
        return fail(HR_ERR_OOM, "grey-box workspace");
    double* dJ = (double*)ws.gb_J.ptr;
    double* dy = (double*)ws.gb_y.ptr;
    double* dvy = (double*)ws.gb_vy.ptr;
    double* dH = (double*)ws.gb_tmp.ptr;     // black-box estimate: n (grad, HVP) or n x n (Hessian)
    double* dout = (double*)ws.gb_out.ptr;
    cudaError_t e = cudaMemcpyAsync(dJ, h_J, sizeof(double) * (size_t)n * nx, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, h_y, sizeof(double) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && quantity == HR_HVP)
        e = cudaMemcpyAsync(ws.gb_vx.ptr, h_vx, sizeof(double) * nx, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return fail(HR_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    if (quantity == HR_HVP) jv_kernel<<<n, 256, 0, stream>>>(dJ, (const double*)ws.gb_vx.ptr, n, nx, dvy);
    hr_opts o2 = *o;
    o2.stream = stream;
    const hr_status st = run_estimate(s, quantity, nullptr, dy, nullptr, quantity == HR_HVP ? dvy : nullptr, &o2,
                                      nullptr, dH);
    if (st != HR_OK) return st;
    if (quantity == HR_HESSIAN) {
        double* dHJ = (double*)ws.gb_hj.ptr;
        hj_kernel<<<dim3((nx + 127) / 128, n), 128, 0, stream>>>(dH, dJ, n, nx, dHJ);
        jthj_kernel<<<dim3((nx + 127) / 128, nx), 128, 0, stream>>>(dJ, dHJ, n, nx, dout);
    } else {
        jtv_kernel<<<(nx + 127) / 128, 128, 0, stream>>>(dJ, dH, n, nx, dout);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(HR_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpyAsync(h_out, dout, sizeof(double) * nout, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(stream)) != cudaSuccess)
        return fail(HR_ERR_CUDA, "result: %s", cudaGetErrorString(e));
    return HR_OK;
}
