"""Shared parity helpers for the GPU tests.

Tolerance for floating-point estimates (identical samples on both sides):
|gpu_e - oracle_e| <= RTOL * max(|oracle_e|, A_e), with RTOL = 1e-4 and
A_e = 1/(2P) sum_m |w_e(tau_m) f_m| the estimator sum's own magnitude.  The
GPU sums FP32 products of FP32-rounded weights and FP32 losses with Kahan
compensation; the oracle sums FP64.  Per-term relative differences are a few
FP32 ulps (weights rounded once, losses from FP32 pixel sums), so the
difference of the sums is bounded by ~1e-6 A_e, far inside the bound; the
A_e floor only matters for entries that cancel to nearly zero.
"""
import numpy as np

RTOL = 1e-4


def flat_of(quantity, out, n):
    if quantity == "hessian":
        return np.asarray(out)[np.triu_indices(n)]
    return np.asarray(out)


def assert_estimate_close(gpu_flat, ref, rtol=RTOL, what=""):
    gpu_flat = np.asarray(gpu_flat, np.float64)
    err = np.abs(gpu_flat - ref.flat)
    tol = rtol * np.maximum(np.abs(ref.flat), ref.scale)
    assert np.all(err <= tol), f"{what}: gpu {gpu_flat} oracle {ref.flat} scale {ref.scale} err {err}"
    return float(np.max(err / np.maximum(np.abs(ref.flat), 1e-300)))


def assert_losses_close(gpu_losses, ref_losses, rtol, what=""):
    g = np.asarray(gpu_losses, np.float64)
    r = np.asarray(ref_losses, np.float64)
    err = np.abs(g - r)
    ok = err <= rtol * np.maximum(np.abs(r), 1e-12)
    assert np.all(ok), f"{what}: {np.count_nonzero(~ok)} losses differ, worst rel {np.max(err / np.maximum(np.abs(r), 1e-30))}"
