"""Thin ctypes binding of libhr (include/hr.h).

Argument marshalling only: every step of the estimators runs in the CUDA
library.  Functions keep the C names; ``Scene`` and ``OptState`` wrap the
handles and pack the seeded scene dicts of ``workloads`` into the C
descriptor.  There is no fallback: if the library is not built, ``lib()``
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhr.so")

HR_OK = 0
HR_ERR_INVALID_ARG, HR_ERR_OOM, HR_ERR_CUDA, HR_ERR_TIMEOUT, HR_ERR_BUSY, HR_ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
HR_ELEMENTWISE, HR_AGGREGATE, HR_PLAIN = 0, 1, 2
HR_GRAD, HR_HESSIAN, HR_HVP = 0, 1, 2
TAG_PATH, TAG_TARGET = 2, 3

_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)


class hr_scene_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("n_params", ctypes.c_int32), ("theta_target", _f64p), ("target_image", _f32p),
                ("radius", ctypes.c_float),
                ("vertices", _f32p), ("n_vertices", ctypes.c_int32), ("triangles", _i32p),
                ("n_triangles", ctypes.c_int32), ("albedo", ctypes.c_float * 3), ("light", ctypes.c_float * 3),
                ("eye_dist", ctypes.c_float), ("scale", ctypes.c_float),
                ("raw_params", _f32p), ("n_tris", ctypes.c_int32), ("param_index", _i32p),
                ("quad_axis", _i32p), ("quad_geom", _f32p), ("quad_albedo", _f32p), ("sph_center", _f32p),
                ("sph_radius", _f32p), ("sph_albedo", _f32p), ("light_half", ctypes.c_float),
                ("cam_z", ctypes.c_float), ("tan_half", ctypes.c_float), ("pix_scale", ctypes.c_float),
                ("emission", ctypes.c_float * 3), ("spp", ctypes.c_int32), ("target_spp", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("quad_A", _f64p), ("quad_b", _f64p), ("gauss_sigma", ctypes.c_double)]


class hr_opts(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("n_perturb", ctypes.c_int64), ("strategy", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("request_id", ctypes.c_uint32), ("sub", ctypes.c_uint32),
                ("stream", ctypes.c_void_p), ("out_tau", _f32p), ("out_weights", _f32p),
                ("out_losses", _f32p), ("out_scale", _f64p)]


class hr_cg_opts(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("n_grad", ctypes.c_int32), ("n_hvp", ctypes.c_int32),
                ("cg_iters", ctypes.c_int32), ("lambda_rel", ctypes.c_double),
                ("trust_radius", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("request_base", ctypes.c_uint32), ("use_graph", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class hr_step_info(ctypes.Structure):
    _fields_ = [("grad_norm", ctypes.c_double), ("lambda_", ctypes.c_double), ("iters", ctypes.c_int32),
                ("exit_reason", ctypes.c_int32), ("step_norm", ctypes.c_double)]


class hr_ncg_opts(ctypes.Structure):
    _fields_ = [("sigma_start", ctypes.c_double), ("sigma_end", ctypes.c_double), ("anneal_iters", ctypes.c_int32),
                ("n_grad", ctypes.c_int32), ("n_hvp", ctypes.c_int32), ("ls_iters", ctypes.c_int32),
                ("ls_tol", ctypes.c_double), ("recompute", ctypes.c_int32), ("residual_mode", ctypes.c_int32),
                ("trust_radius", ctypes.c_double), ("lambda_rel", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("request_base", ctypes.c_uint32), ("use_graph", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class hr_ncg_info(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int32), ("ls_step", ctypes.c_int32), ("restarted", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("sigma", ctypes.c_double), ("grad_norm", ctypes.c_double),
                ("gd", ctypes.c_double), ("dHd", ctypes.c_double), ("alpha", ctypes.c_double),
                ("step_norm", ctypes.c_double)]


class hr_scene_stats(ctypes.Structure):
    _fields_ = [("mesh_overflow_renders", ctypes.c_int64), ("mesh_renders", ctypes.c_int64),
                ("mesh_survivors", ctypes.c_int64), ("mesh_bin_entries", ctypes.c_int64),
                ("mesh_tiles_with_entries", ctypes.c_int64), ("mesh_raster_steps", ctypes.c_int64),
                ("mesh_tile_height", ctypes.c_int64), ("pt_counted_renders", ctypes.c_int64),
                ("pt_hit_rays", ctypes.c_int64), ("pt_shadow_rays", ctypes.c_int64), ("pt_vertices", ctypes.c_int64),
                ("mesh_walk_all_renders", ctypes.c_int64), ("mesh_redo_renders", ctypes.c_int64),
                ("mesh_compact_slots", ctypes.c_int64)]


class hr_tune_info(ctypes.Structure):
    _fields_ = [("render_variant", ctypes.c_int32), ("sample_threads", ctypes.c_int32),
                ("n_render_variants", ctypes.c_int32), ("n_sample_variants", ctypes.c_int32),
                ("render_ms", ctypes.c_float * 4), ("sample_ms", ctypes.c_float * 4)]


class hr_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_int64), ("max_active", ctypes.c_int32), ("chunk", ctypes.c_int32)]


class hr_queue_opts(ctypes.Structure):
    _fields_ = [("max_requests", ctypes.c_int32), ("idle_budget_us", ctypes.c_int32), ("arena_bytes", ctypes.c_int64)]


class hr_request(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_void_p), ("quantity", ctypes.c_int32), ("h_theta", _f64p), ("h_v", _f64p),
                ("opts", hr_opts), ("optstate", ctypes.c_void_p)]


class hr_request_info(ctypes.Structure):
    _fields_ = [("submit_ms", ctypes.c_double), ("admit_ms", ctypes.c_double), ("done_ms", ctypes.c_double),
                ("status", ctypes.c_int32), ("batches", ctypes.c_int32)]


HR_NEWTON_STEP = 3


class HRError(RuntimeError):
    """A failed call; `status` holds the library's status code."""

    def __init__(self, msg: str, status: int = 0):
        super().__init__(msg)
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Load the in-tree libhr.so; raise if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise HRError(f"libhr is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.hr_create_scene.argtypes = [ctypes.POINTER(hr_scene_desc), ctypes.POINTER(vp)]
        L.hr_destroy_scene.argtypes = [vp]
        L.hr_estimate_grad.argtypes = [vp, _f64p, ctypes.POINTER(hr_opts), _f64p]
        L.hr_estimate_hessian.argtypes = [vp, _f64p, ctypes.POINTER(hr_opts), _f64p]
        L.hr_estimate_hvp.argtypes = [vp, _f64p, _f64p, ctypes.POINTER(hr_opts), _f64p]
        L.hr_estimate_hvp_fd.argtypes = [vp, _f64p, _f64p, ctypes.c_double, ctypes.POINTER(hr_opts), _f64p]
        L.hr_estimate_greybox.argtypes = [vp, ctypes.c_int32, _f64p, _f64p, ctypes.c_int32, _f64p,
                                          ctypes.POINTER(hr_opts), _f64p]
        L.hr_estimate_dev.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.POINTER(hr_opts), vp]
        L.hr_estimate_dev_noalloc.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.POINTER(hr_opts), vp]
        L.hr_render.argtypes = [vp, _f64p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                ctypes.c_uint32, ctypes.c_int32, _f32p]
        L.hr_optstate_create.argtypes = [vp, ctypes.c_int32, _f64p, ctypes.POINTER(hr_cg_opts), ctypes.POINTER(vp)]
        L.hr_optstate_destroy.argtypes = [vp]
        L.hr_newton_cg_step.argtypes = [vp, vp, ctypes.POINTER(hr_step_info)]
        L.hr_optstate_theta.argtypes = [vp, _f64p]
        L.hr_optstate_trace.argtypes = [vp, _f64p, _f64p, _f64p]
        L.hr_ncg_create.argtypes = [vp, ctypes.c_int32, _f64p, ctypes.POINTER(hr_ncg_opts), ctypes.POINTER(vp)]
        L.hr_ncg_destroy.argtypes = [vp]
        L.hr_ncg_run.argtypes = [vp, vp, ctypes.c_int32, ctypes.POINTER(hr_ncg_info)]
        L.hr_ncg_theta.argtypes = [vp, _f64p]
        L.hr_ncg_trace.argtypes = [vp, _f64p, _f64p, _f64p]
        L.hr_scene_get_stats.argtypes = [vp, ctypes.POINTER(hr_scene_stats)]
        L.hr_render_ids.argtypes = [vp, _f64p, ctypes.POINTER(ctypes.c_int32)]
        L.hr_scene_count_work.argtypes = [vp, ctypes.c_int32]
        L.hr_autotune.argtypes = [vp, _f64p, ctypes.c_int32, ctypes.POINTER(hr_tune_info)]
        L.hr_set_tuning.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
        L.hr_profile_enable.argtypes = [vp, ctypes.c_int32]
        L.hr_profile_last.argtypes = [vp, _f32p]
        L.hr_server_create.argtypes = [ctypes.POINTER(hr_server_opts), ctypes.POINTER(vp)]
        L.hr_server_destroy.argtypes = [vp]
        L.hr_server_submit.argtypes = [vp, ctypes.POINTER(hr_request), ctypes.POINTER(ctypes.c_uint64)]
        L.hr_server_wait.argtypes = [vp, ctypes.c_uint64, vp, ctypes.POINTER(hr_request_info), ctypes.c_int32]
        L.hr_queue_create.argtypes = [vp, ctypes.POINTER(hr_queue_opts), ctypes.POINTER(vp)]
        L.hr_queue_submit.argtypes = [vp, ctypes.c_int32, _f64p, _f64p, ctypes.POINTER(hr_opts),
                                      ctypes.POINTER(ctypes.c_uint64)]
        L.hr_queue_wait.argtypes = [vp, ctypes.c_uint64, _f64p, ctypes.c_int32]
        L.hr_queue_submit_many.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, _f64p, _f64p, ctypes.POINTER(hr_opts),
                                           ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32)]
        L.hr_queue_wait_many.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64), _f64p, ctypes.c_int32,
                                         ctypes.c_int32]
        L.hr_queue_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint64)]
        L.hr_queue_destroy.argtypes = [vp]
        L.hr_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
        L.hr_last_error.restype = ctypes.c_size_t
        for name in ("hr_create_scene", "hr_destroy_scene", "hr_estimate_grad", "hr_estimate_hessian",
                     "hr_estimate_hvp", "hr_estimate_hvp_fd", "hr_estimate_greybox", "hr_estimate_dev",
                     "hr_estimate_dev_noalloc",
                     "hr_render", "hr_optstate_create",
                     "hr_optstate_destroy", "hr_newton_cg_step", "hr_optstate_theta", "hr_profile_enable",
                     "hr_profile_last", "hr_server_create", "hr_server_destroy", "hr_server_submit",
                     "hr_server_wait", "hr_ncg_create", "hr_ncg_destroy", "hr_ncg_run", "hr_ncg_theta",
                     "hr_autotune", "hr_set_tuning", "hr_scene_get_stats", "hr_optstate_trace", "hr_ncg_trace", "hr_render_ids", "hr_scene_count_work",
                     "hr_queue_create", "hr_queue_submit", "hr_queue_wait", "hr_queue_status", "hr_queue_destroy",
                     "hr_queue_submit_many", "hr_queue_wait_many"):
            getattr(L, name).restype = ctypes.c_int32
        L.hr_version.restype = ctypes.c_int32
        _lib = L
    return _lib


def hr_last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().hr_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(status: int, what: str = "") -> None:
    if status != HR_OK:
        raise HRError(f"{what} failed with status {status}: {hr_last_error()}", status)


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(t)


# ---------------------------------------------------------------------------
# same-name wrappers of the C entry points
# ---------------------------------------------------------------------------
def hr_create_scene(desc: hr_scene_desc) -> int:
    h = ctypes.c_void_p()
    check(lib().hr_create_scene(ctypes.byref(desc), ctypes.byref(h)), "hr_create_scene")
    return h.value


def hr_destroy_scene(handle: int) -> None:
    check(lib().hr_destroy_scene(handle), "hr_destroy_scene")


def make_opts(sigma, M, strategy, seed, request, sub=0, stream=None, debug=None) -> hr_opts:
    o = hr_opts()
    o.sigma, o.n_perturb, o.strategy = float(sigma), int(M), int(strategy)
    o.seed, o.request_id, o.sub = int(seed), int(request) & 0xFFFFFFFF, int(sub)
    o.stream = stream
    if debug is not None:
        o.out_tau = _ptr(debug.get("tau"), _f32p)
        o.out_weights = _ptr(debug.get("w"), _f32p)
        o.out_losses = _ptr(debug.get("losses"), _f32p)
        o.out_scale = _ptr(debug.get("scale"), _f64p)
    return o


def hr_estimate_grad(handle, theta, opts: hr_opts, out):
    check(lib().hr_estimate_grad(handle, _ptr(theta, _f64p), ctypes.byref(opts), _ptr(out, _f64p)), "hr_estimate_grad")


def hr_estimate_hessian(handle, theta, opts: hr_opts, out):
    check(lib().hr_estimate_hessian(handle, _ptr(theta, _f64p), ctypes.byref(opts), _ptr(out, _f64p)),
          "hr_estimate_hessian")


def hr_estimate_hvp(handle, theta, v, opts: hr_opts, out):
    check(lib().hr_estimate_hvp(handle, _ptr(theta, _f64p), _ptr(v, _f64p), ctypes.byref(opts), _ptr(out, _f64p)),
          "hr_estimate_hvp")


def hr_estimate_hvp_fd(handle, theta, v, eps, opts: hr_opts, out):
    check(lib().hr_estimate_hvp_fd(handle, _ptr(theta, _f64p), _ptr(v, _f64p), float(eps), ctypes.byref(opts),
                                   _ptr(out, _f64p)), "hr_estimate_hvp_fd")


def hr_estimate_greybox(handle, quantity, y, J, vx, opts: hr_opts, out):
    J = np.ascontiguousarray(J, np.float64)
    check(lib().hr_estimate_greybox(handle, int(quantity), _ptr(np.ascontiguousarray(y, np.float64), _f64p),
                                    _ptr(J, _f64p), int(J.shape[1]),
                                    None if vx is None else _ptr(np.ascontiguousarray(vx, np.float64), _f64p),
                                    ctypes.byref(opts), _ptr(out, _f64p)), "hr_estimate_greybox")


def hr_estimate_dev(handle, quantity: int, d_theta: int, d_v, opts: hr_opts, d_out: int):
    check(lib().hr_estimate_dev(handle, quantity, d_theta, d_v, ctypes.byref(opts), d_out), "hr_estimate_dev")


def hr_estimate_dev_noalloc(handle, quantity: int, d_theta: int, d_v, opts: hr_opts, d_out: int):
    check(lib().hr_estimate_dev_noalloc(handle, quantity, d_theta, d_v, ctypes.byref(opts), d_out),
          "hr_estimate_dev_noalloc")


def hr_render(handle, params, seed, request, sub, k, tag, spp, out):
    check(lib().hr_render(handle, _ptr(params, _f64p), seed, request, sub, k, tag, spp, _ptr(out, _f32p)),
          "hr_render")


def hr_render_ids(handle, params, W, H) -> np.ndarray:
    """[H*W] index of the triangle each pixel shows (-1: background)."""
    out = np.zeros(W * H, np.int32)
    p = np.ascontiguousarray(params, np.float64)
    check(lib().hr_render_ids(handle, _ptr(p, _f64p), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
          "hr_render_ids")
    return out


def hr_scene_count_work(handle, on: bool):
    check(lib().hr_scene_count_work(handle, int(on)), "hr_scene_count_work")


def hr_scene_get_stats(handle) -> hr_scene_stats:
    st = hr_scene_stats()
    check(lib().hr_scene_get_stats(handle, ctypes.byref(st)), "hr_scene_get_stats")
    return st


def hr_profile_enable(handle, on: bool):
    check(lib().hr_profile_enable(handle, int(on)), "hr_profile_enable")


def hr_profile_last(handle) -> np.ndarray:
    ms = np.zeros(3, np.float32)
    check(lib().hr_profile_last(handle, _ptr(ms, _f32p)), "hr_profile_last")
    return ms


def hr_optstate_create(handle, n_instances, theta0, opts: hr_cg_opts) -> int:
    h = ctypes.c_void_p()
    check(lib().hr_optstate_create(handle, n_instances, _ptr(theta0, _f64p), ctypes.byref(opts), ctypes.byref(h)),
          "hr_optstate_create")
    return h.value


def hr_newton_cg_step(handle, st, info):
    check(lib().hr_newton_cg_step(handle, st, info), "hr_newton_cg_step")


def hr_optstate_theta(st, out):
    check(lib().hr_optstate_theta(st, _ptr(out, _f64p)), "hr_optstate_theta")


def hr_optstate_trace(st, B, K, n):
    """(g [B][n], p [B][K][n], Hp [B][K][n]) of the state's last step."""
    g, p, hp = np.zeros((B, n)), np.zeros((B, K, n)), np.zeros((B, K, n))
    check(lib().hr_optstate_trace(st, _ptr(g, _f64p), _ptr(p, _f64p), _ptr(hp, _f64p)), "hr_optstate_trace")
    return g, p, hp


def hr_optstate_destroy(st):
    check(lib().hr_optstate_destroy(st), "hr_optstate_destroy")


def hr_autotune(handle, theta, n_probe=1024) -> hr_tune_info:
    info = hr_tune_info()
    th = np.ascontiguousarray(theta, np.float64)
    check(lib().hr_autotune(handle, _ptr(th, _f64p), int(n_probe), ctypes.byref(info)), "hr_autotune")
    return info


def hr_set_tuning(handle, render_variant, sample_threads):
    check(lib().hr_set_tuning(handle, int(render_variant), int(sample_threads)), "hr_set_tuning")


def hr_ncg_create(handle, n_instances, theta0, opts: hr_ncg_opts) -> int:
    h = ctypes.c_void_p()
    check(lib().hr_ncg_create(handle, n_instances, _ptr(theta0, _f64p), ctypes.byref(opts), ctypes.byref(h)),
          "hr_ncg_create")
    return h.value


def hr_ncg_run(handle, st, n_evals, info=None):
    """n_evals evaluations; info: None or a (hr_ncg_info * (n_evals * n_instances)) array."""
    check(lib().hr_ncg_run(handle, st, n_evals, info), "hr_ncg_run")


def hr_ncg_theta(st, out):
    check(lib().hr_ncg_theta(st, _ptr(out, _f64p)), "hr_ncg_theta")


def hr_ncg_trace(st, B, n):
    """(g, d, Hd), each [B][n], of the state's last evaluation."""
    g, d, hd = np.zeros((B, n)), np.zeros((B, n)), np.zeros((B, n))
    check(lib().hr_ncg_trace(st, _ptr(g, _f64p), _ptr(d, _f64p), _ptr(hd, _f64p)), "hr_ncg_trace")
    return g, d, hd


def hr_ncg_destroy(st):
    check(lib().hr_ncg_destroy(st), "hr_ncg_destroy")


# ---------------------------------------------------------------------------
# scene packing
# ---------------------------------------------------------------------------
class Scene:
    """Owns a libhr scene built from a ``workloads`` scene dict."""

    def __init__(self, sc: dict, target_image=None):
        self.sc = sc
        self.n = int(sc["n_params"])
        self.W, self.H, self.C = int(sc["width"]), int(sc["height"]), int(sc["channels"])
        keep = {}
        d = hr_scene_desc()
        d.kind, d.width, d.height, d.n_params = int(sc["kind"]), self.W, self.H, self.n
        if sc.get("theta_target") is not None:
            keep["theta"] = np.ascontiguousarray(sc["theta_target"], np.float64)
            d.theta_target = _ptr(keep["theta"], _f64p)
        if target_image is not None:
            keep["target"] = np.ascontiguousarray(target_image, np.float32)
            d.target_image = _ptr(keep["target"], _f32p)
        kind = int(sc["kind"])
        if kind == wl.SCENE_DISC2D:
            d.radius = float(sc["radius"])
        elif kind == wl.SCENE_BOXES2D:
            d.radius = float(sc["half_size"])
        elif kind == wl.SCENE_REVOLVE3D:
            keep["v"] = np.ascontiguousarray(sc["vertices"], np.float32)
            keep["t"] = np.ascontiguousarray(sc["triangles"], np.int32)
            d.vertices, d.n_vertices = _ptr(keep["v"], _f32p), len(keep["v"])
            d.triangles, d.n_triangles = _ptr(keep["t"], _i32p), len(keep["t"])
            d.albedo[:] = [float(x) for x in sc["albedo"]]
            d.light[:] = [float(x) for x in sc["light"]]
            d.eye_dist, d.scale = float(sc["eye_dist"]), float(sc["scale"])
        elif kind == wl.SCENE_TRIS2D:
            keep["raw"] = np.ascontiguousarray(sc["raw_params"], np.float32)
            keep["idx"] = np.ascontiguousarray(sc["param_index"], np.int32)
            d.raw_params, d.n_tris, d.param_index = _ptr(keep["raw"], _f32p), int(sc["n_tris"]), _ptr(keep["idx"], _i32p)
        elif kind == wl.SCENE_PTBOX:
            keep["qa"] = np.ascontiguousarray(sc["quad_axis"], np.int32)
            for k in ("quad_geom", "quad_albedo", "sph_center", "sph_radius", "sph_albedo"):
                keep[k] = np.ascontiguousarray(sc[k], np.float32)
            d.quad_axis = _ptr(keep["qa"], _i32p)
            d.quad_geom, d.quad_albedo = _ptr(keep["quad_geom"], _f32p), _ptr(keep["quad_albedo"], _f32p)
            d.sph_center, d.sph_radius = _ptr(keep["sph_center"], _f32p), _ptr(keep["sph_radius"], _f32p)
            d.sph_albedo = _ptr(keep["sph_albedo"], _f32p)
            d.light_half, d.cam_z = float(sc["light_half"]), float(sc["cam_z"])
            d.tan_half, d.pix_scale = float(sc["tan_half"]), float(sc["pix_scale"])
            d.emission[:] = [float(x) for x in sc["light_emission"]]
            d.spp, d.target_spp, d.depth = int(sc["spp"]), int(sc["target_spp"]), int(sc.get("depth", 3))
            d.seed = int(sc["seed"])
        elif kind == wl.SCENE_QUADRATIC:
            keep["A"] = np.ascontiguousarray(sc["A"], np.float64)
            keep["b"] = np.ascontiguousarray(sc["b"], np.float64)
            d.quad_A, d.quad_b = _ptr(keep["A"], _f64p), _ptr(keep["b"], _f64p)
        elif kind == wl.SCENE_NEGGAUSS:
            d.gauss_sigma = float(sc["gauss_sigma"])
        self._keep = keep
        self.handle = hr_create_scene(d)

    def close(self):
        if self.handle:
            hr_destroy_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_elements(self, quantity):
        return self.n * (self.n + 1) // 2 if quantity == HR_HESSIAN else self.n

    def estimate(self, quantity, theta, sigma, M, strategy, seed, request, sub=0, v=None, debug=False):
        """One estimate; with debug=True also returns the perturbations,
        weights, per-render losses and the sums' scale A_e."""
        theta = np.ascontiguousarray(theta, np.float64)
        n, E = self.n, self.n_elements(quantity)
        G = E if strategy == HR_ELEMENTWISE else 1
        dbg = None
        if debug:
            Mt = G * M
            dbg = dict(tau=np.zeros((Mt, n), np.float32), w=np.zeros((Mt, E), np.float32),
                       losses=np.zeros(Mt, np.float32), scale=np.zeros(E, np.float64))
        o = make_opts(sigma, M, strategy, seed, request, sub, debug=dbg)
        if quantity == HR_HESSIAN:
            out = np.zeros((n, n), np.float64)
            hr_estimate_hessian(self.handle, theta, o, out)
        elif quantity == HR_GRAD:
            out = np.zeros(n, np.float64)
            hr_estimate_grad(self.handle, theta, o, out)
        else:
            out = np.zeros(n, np.float64)
            hr_estimate_hvp(self.handle, theta, np.ascontiguousarray(v, np.float64), o, out)
        return (out, dbg) if debug else out

    def render(self, params, seed=0, request=0, sub=0, k=0, tag=TAG_PATH, spp=None):
        img = np.zeros(self.W * self.H * self.C, np.float32)
        spp = int(self.sc.get("spp", 1)) if spp is None else spp
        hr_render(self.handle, np.ascontiguousarray(params, np.float64), seed, request, sub, k, tag, spp, img)
        return img


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
def hr_server_create(hbm_budget: int, max_active: int = 32, chunk: int = 0) -> int:
    o = hr_server_opts(int(hbm_budget), int(max_active), int(chunk))
    h = ctypes.c_void_p()
    check(lib().hr_server_create(ctypes.byref(o), ctypes.byref(h)), "hr_server_create")
    return h.value


def hr_server_destroy(srv: int) -> None:
    check(lib().hr_server_destroy(srv), "hr_server_destroy")


def hr_server_submit(srv: int, req: hr_request) -> int:
    t = ctypes.c_uint64()
    check(lib().hr_server_submit(srv, ctypes.byref(req), ctypes.byref(t)), "hr_server_submit")
    return t.value


def hr_server_wait(srv: int, ticket: int, out, info: hr_request_info, timeout_ms: int = 120000) -> None:
    ptr = None if out is None else (out.ctypes.data if isinstance(out, np.ndarray) else ctypes.addressof(out))
    check(lib().hr_server_wait(srv, ticket, ptr, ctypes.byref(info), int(timeout_ms)), "hr_server_wait")


# ---------------------------------------------------------------------------
# persistent queue (disc scenes)
# ---------------------------------------------------------------------------
def hr_queue_create(scene: "Scene", max_requests: int = 1024, idle_budget_us: int = 2000,
                    arena_bytes: int = 256 << 20) -> int:
    o = hr_queue_opts(int(max_requests), int(idle_budget_us), int(arena_bytes))
    h = ctypes.c_void_p()
    check(lib().hr_queue_create(scene.handle, ctypes.byref(o), ctypes.byref(h)), "hr_queue_create")
    return h.value


def hr_queue_submit(q: int, quantity: int, theta, v, opts: hr_opts) -> int:
    """Queue one estimate; raises HRError with status HR_ERR_BUSY when the ring
    or the arena is full (nothing queued)."""
    t = ctypes.c_uint64()
    th = np.ascontiguousarray(theta, np.float64)
    vv = None if v is None else np.ascontiguousarray(v, np.float64)
    check(lib().hr_queue_submit(q, int(quantity), _ptr(th, _f64p), _ptr(vv, _f64p), ctypes.byref(opts),
                                ctypes.byref(t)), "hr_queue_submit")
    return t.value


def hr_queue_wait(q: int, ticket: int, out: np.ndarray, timeout_ms: int = 120000) -> None:
    check(lib().hr_queue_wait(q, int(ticket), _ptr(out, _f64p), int(timeout_ms)), "hr_queue_wait")


def opts_array(sigma, M, strategy, seeds, requests, subs=None):
    """A ctypes array of hr_opts, one per (seed, request[, sub])."""
    arr = (hr_opts * len(seeds))()
    for i, (sd, rq) in enumerate(zip(seeds, requests)):
        o = arr[i]
        o.sigma, o.n_perturb, o.strategy = float(sigma), int(M), int(strategy)
        o.seed, o.request_id = int(sd), int(rq) & 0xFFFFFFFF
        o.sub = 0 if subs is None else int(subs[i])
    return arr


def hr_queue_submit_many(q: int, quantity: int, thetas, vs, opts_array) -> np.ndarray:
    """Queue len(opts_array) estimates (thetas [count][n], vs [count][n] or None,
    opts_array a ctypes array of hr_opts); returns the tickets of those queued
    (fewer than count when the ring or the arena filled up)."""
    count = len(opts_array)
    th = np.ascontiguousarray(thetas, np.float64)
    vv = None if vs is None else np.ascontiguousarray(vs, np.float64)
    tickets = np.zeros(count, np.uint64)
    done = ctypes.c_int32()
    st = lib().hr_queue_submit_many(q, count, int(quantity), _ptr(th, _f64p), _ptr(vv, _f64p), opts_array,
                                    tickets.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ctypes.byref(done))
    if st not in (HR_OK, HR_ERR_BUSY):
        check(st, "hr_queue_submit_many")
    return tickets[:done.value]


def hr_queue_wait_many(q: int, tickets, out: np.ndarray, timeout_ms: int = 120000) -> None:
    """Wait for tickets; out [count][stride] receives their results."""
    t = np.ascontiguousarray(tickets, np.uint64)
    assert out.flags.c_contiguous and out.dtype == np.float64 and out.shape[0] >= len(t)
    stride = int(np.prod(out.shape[1:])) if out.ndim > 1 else 1
    check(lib().hr_queue_wait_many(q, len(t), t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _ptr(out, _f64p),
                                   stride, int(timeout_ms)), "hr_queue_wait_many")


def hr_queue_status(q: int):
    """(kernel status: 1 running, else its exit code; launches so far)."""
    st, n = ctypes.c_int32(), ctypes.c_uint64()
    check(lib().hr_queue_status(q, ctypes.byref(st), ctypes.byref(n)), "hr_queue_status")
    return st.value, n.value


def hr_queue_destroy(q: int) -> None:
    check(lib().hr_queue_destroy(q), "hr_queue_destroy")


def make_request(scene: "Scene", quantity: int, theta=None, v=None, opts: hr_opts = None, optstate=None):
    """Build an hr_request; returns (request, keep-alive arrays)."""
    r = hr_request()
    r.scene = scene.handle
    r.quantity = int(quantity)
    keep = []
    if theta is not None:
        th = np.ascontiguousarray(theta, np.float64)
        keep.append(th)
        r.h_theta = _ptr(th, _f64p)
    if v is not None:
        vv = np.ascontiguousarray(v, np.float64)
        keep.append(vv)
        r.h_v = _ptr(vv, _f64p)
    if opts is not None:
        r.opts = opts
    r.optstate = optstate
    return r, keep
