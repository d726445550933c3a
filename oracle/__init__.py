"""Oracle: plain FP64 CPU restatement of the stochastic Hessian / HVP /
gradient estimator (Wang, Fischer, Ritschel, "Stochastic Gradient Estimation
for Higher-order Differentiable Rendering").

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA path; both sides only share the seeded scene generators in
``paper_2412_03489_gb300.workloads``, which hold none of the method's
arithmetic.

The heavy loops (Philox, lobe samplers, kernel weights, renderers) are in
``oracle.c``; this module assembles estimates with exactly rounded FP64 sums
(math.fsum) and runs the Newton-CG iteration in FP64.

Estimator (Sec. 3.1, Eq. for D fbar as a parameter-space integral): with
fbar(theta) = E f(theta + tau), tau ~ N(0, s^2 I), every derivative is an
integral of a kernel h = c(tau) N(tau) against f(theta + tau); each sample pair
k draws a + leg from the positive lobe and a - leg from the negative lobe, and
   est_e = 1/(2P) sum_m w_e(tau_m) f(theta + tau_m)
over the 2P perturbations m of the request.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_lib = None

_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)


class _RevolveScene(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("nv", ctypes.c_int), ("nt", ctypes.c_int),
                ("verts", _f32p), ("tris", _i32p), ("albedo", ctypes.c_float * 3),
                ("light", ctypes.c_float * 3), ("eye_dist", ctypes.c_float), ("scale", ctypes.c_float)]


class _Tris2dScene(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("n_tris", ctypes.c_int),
                ("n_params", ctypes.c_int), ("raw", _f32p), ("index", _i32p)]


class _PtboxScene(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("quad_axis", _i32p), ("quad_geom", _f32p),
                ("quad_albedo", _f32p), ("sph_center", _f32p), ("sph_radius", _f32p),
                ("sph_albedo", _f32p), ("light_half", ctypes.c_float), ("cam_z", ctypes.c_float),
                ("tan_half", ctypes.c_float), ("pix_scale", ctypes.c_float),
                ("emission", ctypes.c_float * 3), ("emit_all", ctypes.c_int), ("nee", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.or_u01.argtypes = [ctypes.c_uint32]; L.or_u01.restype = ctypes.c_double
        L.or_lambertw.argtypes = [ctypes.c_double, ctypes.c_int]; L.or_lambertw.restype = ctypes.c_double
        L.or_diag_cdf.argtypes = [ctypes.c_double]; L.or_diag_cdf.restype = ctypes.c_double
        L.or_diag_inv_cdf.argtypes = [ctypes.c_double]; L.or_diag_inv_cdf.restype = ctypes.c_double
        for nm in ("or_Zg", "or_Zd", "or_Zo"):
            getattr(L, nm).argtypes = [ctypes.c_double]; getattr(L, nm).restype = ctypes.c_double
        L.or_draw.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64,
                              ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, _f32p, _i32p]
        L.or_draw.restype = ctypes.c_int
        L.or_weights.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _f64p, ctypes.c_int64,
                                 _f32p, ctypes.c_int, ctypes.c_int, _f64p]
        L.or_weights.restype = ctypes.c_int
        L.or_disc_loss.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_float, _f32p, _f32p, _f32p]
        L.or_disc_loss.restype = ctypes.c_double
        L.or_boxes_loss.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, _f32p, _f32p, _f32p]
        L.or_boxes_loss.restype = ctypes.c_double
        L.or_revolve_loss.argtypes = [ctypes.POINTER(_RevolveScene), _f32p, _f32p, _f32p]
        L.or_revolve_loss.restype = ctypes.c_double
        L.or_revolve_render.argtypes = [ctypes.POINTER(_RevolveScene), _f32p, _f32p, _f32p,
                                        ctypes.POINTER(ctypes.c_int32)]
        L.or_revolve_render.restype = ctypes.c_double
        L.or_tris2d_loss.argtypes = [ctypes.POINTER(_Tris2dScene), _f32p, _f32p, _f32p]
        L.or_tris2d_loss.restype = ctypes.c_double
        L.or_ptbox_render.argtypes = [ctypes.POINTER(_PtboxScene), _f32p, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, _f32p, _f64p]
        L.or_ptbox_render.restype = ctypes.c_double
        L.or_ptbox_render_counted.argtypes = [ctypes.POINTER(_PtboxScene), _f32p, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.c_uint32, _f32p, _f64p, ctypes.POINTER(ctypes.c_longlong)]
        L.or_ptbox_render_counted.restype = ctypes.c_double
        L.or_ptbox_intersect.argtypes = [ctypes.POINTER(_PtboxScene), _f32p, _f32p, _f32p, _f32p]
        L.or_ptbox_intersect.restype = ctypes.c_int
        L.or_ptbox_trace.argtypes = [ctypes.POINTER(_PtboxScene), _f32p, _f32p, _f32p, ctypes.c_int,
                                     ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_uint32, _f64p]
        L.or_perturb.argtypes = [ctypes.c_int, _f64p, _f32p, _f32p]
        L.or_draw_hvp_rows.argtypes = [ctypes.c_int, ctypes.c_double, _f64p, ctypes.c_int64, ctypes.c_uint64,
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, _f32p, _i32p]
        L.or_draw_hvp_rows.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


# --------------------------------------------------------------------------
# scalar primitives
# --------------------------------------------------------------------------
def philox(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def u01(x: int) -> float:
    return lib().or_u01(x)


def lambertw(z: float, branch: int) -> float:
    return lib().or_lambertw(z, branch)


def diag_cdf(t: float) -> float:
    return lib().or_diag_cdf(t)


def diag_inv_cdf(c: float) -> float:
    return lib().or_diag_inv_cdf(c)


def Zg(s):
    return lib().or_Zg(s)


def Zd(s):
    return lib().or_Zd(s)


def Zo(s):
    return lib().or_Zo(s)


TAG_SAMPLE, TAG_PATH, TAG_TARGET = 1, 2, 3


def draw(lobe: int, n: int, sigma: float, P: int, seed: int, request: int, sub: int,
         comp_i: int = -1, comp_j: int = -1):
    """tau[2P, n] (FP32; + leg at even rows) and the component of each pair."""
    tau = np.zeros((2 * P, n), np.float32)
    comp = np.zeros(P, np.int32)
    rc = lib().or_draw(lobe, n, sigma, P, seed, request & 0xFFFFFFFF, sub, comp_i, comp_j,
                       _p(tau, _f32p), _p(comp, _i32p))
    assert rc == 0
    return tau, comp


def draw_hvp_rows(n: int, sigma: float, v, P: int, seed: int, request: int, sub: int, row: int):
    """Element-wise HVP pairs for output `row` (component j drawn from the
    |v|-weighted row mixture)."""
    tau = np.zeros((2 * P, n), np.float32)
    comp = np.zeros(P, np.int32)
    vv = np.ascontiguousarray(v, np.float64)
    rc = lib().or_draw_hvp_rows(n, sigma, _p(vv, _f64p), P, seed, request & 0xFFFFFFFF, sub, row,
                                _p(tau, _f32p), _p(comp, _i32p))
    assert rc == 0
    return tau, comp


def weights(quantity: int, n: int, sigma: float, tau: np.ndarray, comp_i: int = -1, comp_j: int = -1,
            v=None) -> np.ndarray:
    M = tau.shape[0]
    E = n * (n + 1) // 2 if quantity == 1 else n
    w = np.zeros((M, E), np.float64)
    vv = None if v is None else np.ascontiguousarray(v, np.float64)
    tau = np.ascontiguousarray(tau, np.float32)
    rc = lib().or_weights(quantity, n, sigma, _p(vv, _f64p), M, _p(tau, _f32p), comp_i, comp_j, _p(w, _f64p))
    assert rc == 0
    return w


def perturb(theta, tau) -> np.ndarray:
    th = np.ascontiguousarray(theta, np.float64)
    tau = np.ascontiguousarray(tau, np.float32)
    p = np.zeros(len(th), np.float32)
    lib().or_perturb(len(th), _p(th, _f64p), _p(tau, _f32p), _p(p, _f32p))
    return p


# --------------------------------------------------------------------------
# renderers
# --------------------------------------------------------------------------
class Renderer:
    n: int

    def loss(self, p: np.ndarray, ctx: dict) -> float:  # pragma: no cover - interface
        raise NotImplementedError


class FunctionRenderer(Renderer):
    """An analytic loss f(p) (test functions: quadratic, step, negated
    Gaussian), evaluated in FP64 at the FP32 perturbed parameters."""

    def __init__(self, f, n):
        self.f, self.n = f, n

    def loss(self, p, ctx):
        return float(self.f(p.astype(np.float64)[None, :])[0])

    def loss_batch(self, P):
        """f at every row of the FP32 perturbed-parameter matrix P."""
        return np.asarray(self.f(P.astype(np.float64)), np.float64)


class DiscRenderer(Renderer):
    def __init__(self, sc: dict, target=None):
        self.W, self.H, self.r, self.n = sc["width"], sc["height"], np.float32(sc["radius"]), 2
        self.target = target if target is not None else self.image(np.asarray(sc["theta_target"], np.float32))

    def image(self, p):
        img = np.zeros(self.W * self.H, np.float32)
        p = np.ascontiguousarray(p, np.float32)
        lib().or_disc_loss(self.W, self.H, self.r, _p(p, _f32p), None, _p(img, _f32p))
        return img

    def loss(self, p, ctx=None):
        p = np.ascontiguousarray(p, np.float32)
        return lib().or_disc_loss(self.W, self.H, self.r, _p(p, _f32p), _p(self.target, _f32p), None)


class BoxesRenderer(Renderer):
    def __init__(self, sc: dict, target=None):
        self.W, self.H, self.h = sc["width"], sc["height"], np.float32(sc["half_size"])
        self.n = sc["n_params"]
        self.K = self.n // 2
        self.target = target if target is not None else self.image(np.asarray(sc["theta_target"], np.float32))

    def image(self, p):
        img = np.zeros(self.W * self.H, np.float32)
        p = np.ascontiguousarray(p, np.float32)
        lib().or_boxes_loss(self.W, self.H, self.K, self.h, _p(p, _f32p), None, _p(img, _f32p))
        return img

    def loss(self, p, ctx=None):
        p = np.ascontiguousarray(p, np.float32)
        return lib().or_boxes_loss(self.W, self.H, self.K, self.h, _p(p, _f32p), _p(self.target, _f32p), None)


class RevolveRenderer(Renderer):
    def __init__(self, sc: dict, target=None):
        self.keep = dict(v=np.ascontiguousarray(sc["vertices"], np.float32),
                         t=np.ascontiguousarray(sc["triangles"], np.int32))
        s = _RevolveScene()
        s.W, s.H = sc["width"], sc["height"]
        s.nv, s.nt = len(self.keep["v"]), len(self.keep["t"])
        s.verts = _p(self.keep["v"], _f32p)
        s.tris = _p(self.keep["t"], _i32p)
        s.albedo[:] = [float(x) for x in sc["albedo"]]
        s.light[:] = [float(x) for x in sc["light"]]
        s.eye_dist, s.scale = float(sc["eye_dist"]), float(sc["scale"])
        self.s, self.n, self.W, self.H = s, 2, sc["width"], sc["height"]
        self.target = target if target is not None else self.image(np.asarray(sc["theta_target"], np.float32))

    def image(self, p):
        img = np.zeros(self.W * self.H * 3, np.float32)
        p = np.ascontiguousarray(p, np.float32)
        lib().or_revolve_loss(ctypes.byref(self.s), _p(p, _f32p), None, _p(img, _f32p))
        return img

    def loss(self, p, ctx=None):
        p = np.ascontiguousarray(p, np.float32)
        return lib().or_revolve_loss(ctypes.byref(self.s), _p(p, _f32p), _p(self.target, _f32p), None)

    def ids(self, p):
        """Index of the triangle each pixel shows (-1: background), [H*W]."""
        out = np.zeros(self.W * self.H, np.int32)
        p = np.ascontiguousarray(p, np.float32)
        lib().or_revolve_render(ctypes.byref(self.s), _p(p, _f32p), None, None,
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        return out


class Tris2dRenderer(Renderer):
    def __init__(self, sc: dict, target=None):
        self.keep = dict(raw=np.ascontiguousarray(sc["raw_params"], np.float32),
                         idx=np.ascontiguousarray(sc["param_index"], np.int32))
        s = _Tris2dScene()
        s.W, s.H, s.n_tris, s.n_params = sc["width"], sc["height"], sc["n_tris"], sc["n_params"]
        s.raw = _p(self.keep["raw"], _f32p)
        s.index = _p(self.keep["idx"], _i32p)
        self.s, self.n, self.W, self.H = s, sc["n_params"], sc["width"], sc["height"]
        self.target = target if target is not None else self.image(np.asarray(sc["theta_target"], np.float32))

    def image(self, p):
        img = np.zeros(self.W * self.H * 3, np.float32)
        p = np.ascontiguousarray(p, np.float32)
        lib().or_tris2d_loss(ctypes.byref(self.s), _p(p, _f32p), None, _p(img, _f32p))
        return img

    def loss(self, p, ctx=None):
        p = np.ascontiguousarray(p, np.float32)
        return lib().or_tris2d_loss(ctypes.byref(self.s), _p(p, _f32p), _p(self.target, _f32p), None)


class PtboxRenderer(Renderer):
    """Path tracer; the path random numbers of a render are those of its pair
    k, sub-stream and request (tag 2); the target uses tag 3, k = 0."""

    def __init__(self, sc: dict, target=None, spp=None, depth=3, emit_all=False, nee=True):
        self.keep = {k: np.ascontiguousarray(sc[k], np.int32 if k == "quad_axis" else np.float32)
                     for k in ("quad_axis", "quad_geom", "quad_albedo", "sph_center", "sph_radius", "sph_albedo")}
        s = _PtboxScene()
        s.W, s.H = sc["width"], sc["height"]
        s.quad_axis = _p(self.keep["quad_axis"], _i32p)
        for k in ("quad_geom", "quad_albedo", "sph_center", "sph_radius", "sph_albedo"):
            setattr(s, k, _p(self.keep[k], _f32p))
        s.light_half, s.cam_z = float(sc["light_half"]), float(sc["cam_z"])
        s.tan_half, s.pix_scale = float(sc["tan_half"]), float(sc["pix_scale"])
        s.emission[:] = [float(x) for x in sc["light_emission"]]
        s.emit_all, s.nee = int(emit_all), int(nee)
        self.s, self.n, self.W, self.H = s, 6, sc["width"], sc["height"]
        self.spp = sc["spp"] if spp is None else spp
        self.depth, self.seed = depth, sc["seed"]
        if target is None:
            target = self.image(np.asarray(sc["theta_target"], np.float32), sc["target_spp"],
                                self.seed, 0, 0, 0, TAG_TARGET).astype(np.float32)
        self.target = np.ascontiguousarray(target, np.float32)

    def image(self, p, spp, seed, request, sub, k, tag):
        img = np.zeros(self.W * self.H * 3, np.float64)
        p = np.ascontiguousarray(p, np.float32)
        lib().or_ptbox_render(ctypes.byref(self.s), _p(p, _f32p), spp, self.depth, seed,
                              request & 0xFFFFFFFF, sub, k, tag, None, _p(img, _f64p))
        return img

    def loss(self, p, ctx):
        p = np.ascontiguousarray(p, np.float32)
        return lib().or_ptbox_render(ctypes.byref(self.s), _p(p, _f32p), self.spp, self.depth, ctx["seed"],
                                     ctx["request"] & 0xFFFFFFFF, ctx["sub"], ctx["k"], TAG_PATH,
                                     _p(self.target, _f32p), None)

    def count_rays(self, p, ctx):
        """(closest-hit rays, shadow rays, shaded vertices) of the loss render
        of perturbation context ctx, as the path tracer traces them."""
        cnt = (ctypes.c_longlong * 3)()
        p = np.ascontiguousarray(p, np.float32)
        lib().or_ptbox_render_counted(ctypes.byref(self.s), _p(p, _f32p), self.spp, self.depth, ctx["seed"],
                                      ctx["request"] & 0xFFFFFFFF, ctx["sub"], ctx["k"], TAG_PATH,
                                      _p(self.target, _f32p), None, cnt)
        return int(cnt[0]), int(cnt[1]), int(cnt[2])

    def intersect(self, p, o, d):
        t = np.zeros(1, np.float32)
        p, o, d = (np.ascontiguousarray(x, np.float32) for x in (p, o, d))
        prim = lib().or_ptbox_intersect(ctypes.byref(self.s), _p(p, _f32p), _p(o, _f32p), _p(d, _f32p),
                                        _p(t, _f32p))
        return prim, float(t[0])

    def trace(self, p, o, d, depth, seed, request, sub, k, tag, idx):
        out = np.zeros(3, np.float64)
        p, o, d = (np.ascontiguousarray(x, np.float32) for x in (p, o, d))
        lib().or_ptbox_trace(ctypes.byref(self.s), _p(p, _f32p), _p(o, _f32p), _p(d, _f32p), depth, seed,
                             request, sub, k, tag, idx, _p(out, _f64p))
        return out


def renderer_for(sc: dict, **kw) -> Renderer:
    from paper_2412_03489_gb300 import workloads as wl
    return {wl.SCENE_DISC2D: DiscRenderer, wl.SCENE_REVOLVE3D: RevolveRenderer,
            wl.SCENE_TRIS2D: Tris2dRenderer, wl.SCENE_PTBOX: PtboxRenderer,
            wl.SCENE_BOXES2D: BoxesRenderer}[sc["kind"]](sc, **kw)


# --------------------------------------------------------------------------
# estimators
# --------------------------------------------------------------------------
QUANTITY = {"grad": 0, "hessian": 1, "hvp": 2}


def estimate_hvp_fd(r: Renderer, theta, v, eps: float, sigma: float, M: int, strategy: str, seed: int,
                    request: int, sub: int = 0):
    """HVP as the central difference of two smoothed-gradient estimates at
    theta +- eps v (Sec. 2, central differences of gradients; Sec. 3.4) with
    common random numbers: both use the same perturbations."""
    theta = np.asarray(theta, np.float64)
    v = np.asarray(v, np.float64)
    gp = estimate(r, "grad", theta + eps * v, sigma, M, strategy, seed, request, sub)
    gm = estimate(r, "grad", theta - eps * v, sigma, M, strategy, seed, request, sub)
    return (gp.flat - gm.flat) / (2.0 * eps), gp, gm


def estimate_greybox(r: Renderer, quantity: str, y, J, sigma, M, strategy, seed, request, sub=0, vx=None):
    """Grey-box derivatives of f(g(x)) (Suppl. "Grey-box differentials"):
    the black-box estimate at y = g(x) composed with the inner Jacobian J:
    J^T g, J^T H J, or J^T H (J v_x)."""
    J = np.asarray(J, np.float64)
    if quantity == "hvp":
        est = estimate(r, "hvp", y, sigma, M, strategy, seed, request, sub, v=J @ np.asarray(vx, np.float64))
        return J.T @ est.value, est
    est = estimate(r, quantity, y, sigma, M, strategy, seed, request, sub)
    if quantity == "grad":
        return J.T @ est.value, est
    return J.T @ est.value @ J, est


def elements(quantity: str, n: int):
    """Unique elements estimated by element-wise importance sampling: the n
    gradient entries, or the upper triangle of the Hessian (symmetry, Sec. 3.3)."""
    if quantity == "grad":
        return [(i, i) for i in range(n)]
    if quantity == "hessian":
        return [(a, b) for a in range(n) for b in range(a, n)]
    raise ValueError("element-wise sampling is defined for grad and hessian")


@dataclass
class Estimate:
    quantity: str
    n: int
    flat: np.ndarray            # E entries (upper triangle for the Hessian)
    scale: np.ndarray           # A_e = 1/(2P) sum |w f|: the sum's own magnitude
    tau: np.ndarray             # [M_total, n] FP32 perturbations in launch order
    w: np.ndarray               # [M_total, E] FP64 weights
    losses: np.ndarray          # [M_total] FP64 losses
    comps: list = field(default_factory=list)

    @property
    def value(self) -> np.ndarray:
        if self.quantity != "hessian":
            return self.flat.copy()
        H = np.zeros((self.n, self.n))
        e = 0
        for a in range(self.n):
            for b in range(a, self.n):
                H[a, b] = H[b, a] = self.flat[e]
                e += 1
        return H


def estimate(r: Renderer, quantity: str, theta, sigma: float, M: int, strategy: str, seed: int,
             request: int, sub: int = 0, v=None, threads: int = 1) -> Estimate:
    """One estimate: M perturbations (renders) for the aggregate strategy, M
    per unique element for element-wise sampling (Tab. 1 render counts).
    threads > 1 runs the per-perturbation renders of renderers without a
    batch form on that many host threads (the C renders release the GIL);
    the losses, and everything computed from them, are the same."""
    n = r.n
    q = QUANTITY[quantity]
    lobe = 0 if quantity == "grad" else 1
    if M < 2 or M % 2:
        raise ValueError("M must be even and >= 2")
    P = M // 2
    if strategy == "aggregate":
        groups = [(-1, -1, sub)]
    elif strategy == "plain":
        groups = [(-3, -1, sub)]
    elif strategy == "elementwise" and quantity == "hvp":
        # one sample set per output row, drawn from the row's |v|-weighted mixture
        groups = [(i, -2, sub + i) for i in range(n)]
    elif strategy == "elementwise":
        groups = [(i, j, sub + e) for e, (i, j) in enumerate(elements(quantity, n))]
    else:
        raise ValueError(strategy)
    taus, ws, ls, comps = [], [], [], []
    for ci, cj, s in groups:
        if cj == -2:
            tau, comp = draw_hvp_rows(n, sigma, v, P, seed, request, s, ci)
            w = weights(3, n, sigma, tau, ci, -1, v)
        else:
            tau, comp = draw(lobe, n, sigma, P, seed, request, s, ci, cj)
            w = weights(q, n, sigma, tau, ci, cj, v)
        if hasattr(r, "loss_batch"):
            # RN32(RN32(theta) + tau) row by row (IEEE single-precision add)
            losses = r.loss_batch(np.asarray(theta, np.float64).astype(np.float32)[None, :] + tau)
        else:
            def one(m, tau=tau, s=s):
                return r.loss(perturb(theta, tau[m]), dict(seed=seed, request=request, sub=s, k=m // 2))
            if threads > 1:
                from concurrent.futures import ThreadPoolExecutor
                with ThreadPoolExecutor(threads) as ex:
                    losses = np.array(list(ex.map(one, range(2 * P))))
            else:
                losses = np.array([one(m) for m in range(2 * P)])
        taus.append(tau); ws.append(w); ls.append(losses); comps.append(comp)
    tau = np.concatenate(taus); w = np.concatenate(ws); losses = np.concatenate(ls)
    E = w.shape[1]
    flat = np.array([math.fsum(w[:, e] * losses) for e in range(E)]) / (2 * P)
    scale = np.array([math.fsum(np.abs(w[:, e] * losses)) for e in range(E)]) / (2 * P)
    return Estimate(quantity, n, flat, scale, tau, w, losses, comps)


# --------------------------------------------------------------------------
# Newton-CG (Sec. 2 "Newton Conjugate Gradient"; trust-region step cap and
# negative-curvature exit from the same section and Suppl. "Positive-Definite
# Hessians")
# --------------------------------------------------------------------------
@dataclass
class StepInfo:
    grad_norm: float
    lam: float
    iters: int
    exit: str
    step_norm: float


def newton_cg_step(r: Renderer, theta, sigma, M_grad, M_hvp, K, lam_rel, delta, seed, request, step,
                   grad_fn=None, hvp_fn=None):
    """One step on (H + lam I) d = -g by linear CG from d = 0 with
    alpha = r.r / p.(H + lam I)p (the quadratic model's exact line step),
    Fletcher-Reeves beta, alpha capped at delta / |p|, each product with
    fresh samples (sub = 64 step + 1 + i; the gradient uses 64 step)."""
    theta = np.asarray(theta, np.float64)
    if grad_fn is None:
        def grad_fn(th):
            return estimate(r, "grad", th, sigma, M_grad, "aggregate", seed, request, sub=64 * step).value
    if hvp_fn is None:
        def hvp_fn(th, i, vec):
            return estimate(r, "hvp", th, sigma, M_hvp, "aggregate", seed, request,
                            sub=64 * step + 1 + i, v=vec).value
    g = grad_fn(theta)
    lam = lam_rel * float(np.linalg.norm(g))
    d = np.zeros_like(theta)
    res = -g
    p = res.copy()
    rr = float(res @ res)
    exit_reason, it = "max_iters", 0
    for i in range(K):
        it = i + 1
        Hp = hvp_fn(theta, i, p) + lam * p
        pHp = float(p @ Hp)
        pn = float(np.linalg.norm(p))
        if pHp <= 0.0 or pn == 0.0:
            if i == 0 and pn > 0.0:
                d = p * (delta / pn)
            exit_reason = "neg_curvature"
            break
        alpha = min(rr / pHp, delta / pn)
        d = d + alpha * p
        res = res - alpha * Hp
        rr_new = float(res @ res)
        if rr_new == 0.0:
            exit_reason = "converged"
            break
        p = res + (rr_new / rr) * p
        rr = rr_new
    return theta + d, StepInfo(float(np.linalg.norm(g)), lam, it, exit_reason, float(np.linalg.norm(d)))


# --------------------------------------------------------------------------
# The published optimiser (Sec. 2 "Newton Conjugate Gradient" with the
# point moved every iteration; Suppl. "Hyperparameters": linear sigma
# annealing, line-search iterations and tolerance, "recompute" period,
# trust region).  Readings:
#  * line search = Newton-Raphson steps along the current direction d, each
#    alpha = -g(x).d / d.H(x)d (Eq. pertubation) at the current point, at most
#    ls_iters steps, ending early once |alpha| |d| <= ls_tol;
#  * |alpha| <= Delta / |d| (trust-region truncation, Sec. 2); where
#    d.H d <= 0 the step goes to that bound in the descent direction;
#  * residual (residual_mode 0) follows the printed recurrence
#    r <- r - alpha (H + lambda I) d at every step; every `recompute` outer
#    iterations it is recomputed from a fresh gradient estimate and the
#    direction restarts, r = d = -g; residual_mode 1 takes r = -g at every
#    outer iteration (nonlinear CG);
#  * Fletcher-Reeves beta = r'.r' / r.r; a direction with r.d <= 0 restarts;
#  * sigma_i = start + (end - start) min(i, T-1) / (T-1) for outer iteration i.
# One evaluation = one line-search step = one gradient estimate (sub 64 e)
# and one aggregate Hessian-vector product (sub 64 e + 1) at the same point.
# --------------------------------------------------------------------------
@dataclass
class NcgOpts:
    sigma_start: float
    sigma_end: float
    anneal_iters: int
    n_grad: int
    n_hvp: int
    ls_iters: int
    ls_tol: float
    recompute: int
    trust_radius: float
    residual_mode: int = 0
    lambda_rel: float = 0.0


def anneal_sigma(start: float, end: float, T: int, i: int) -> float:
    """Linear bandwidth schedule over outer iterations (Suppl. Hyperparameters)."""
    if T <= 1:
        return float(start)
    if i >= T - 1:
        return float(end)
    return float(start) + (float(end) - float(start)) * float(i) / float(T - 1)


@dataclass
class NcgState:
    x: np.ndarray
    d: np.ndarray
    r: np.ndarray
    rr: float = 0.0
    it: int = 0          # outer iteration
    j: int = 0           # line-search step within it
    evals: int = 0
    sigma: float = 0.0


@dataclass
class NcgInfo:
    it: int
    ls_step: int
    restarted: bool
    sigma: float
    grad_norm: float
    gd: float
    dHd: float
    alpha: float
    step_norm: float


def ncg_init(theta0, o: NcgOpts) -> NcgState:
    x = np.asarray(theta0, np.float64).copy()
    z = np.zeros_like(x)
    return NcgState(x=x, d=z.copy(), r=z.copy(), sigma=anneal_sigma(o.sigma_start, o.sigma_end, o.anneal_iters, 0))


def ncg_evaluate(r: Renderer, st: NcgState, o: NcgOpts, seed: int, request: int,
                 grad_fn=None, hvp_fn=None) -> NcgInfo:
    """One evaluation (one line-search step) of the optimiser; updates st."""
    e, sigma = st.evals, st.sigma
    if grad_fn is None:
        def grad_fn(x, s, ev):
            return estimate(r, "grad", x, s, o.n_grad, "aggregate", seed, request, sub=64 * ev).value
    if hvp_fn is None:
        def hvp_fn(x, s, ev, vec):
            return estimate(r, "hvp", x, s, o.n_hvp, "aggregate", seed, request, sub=64 * ev + 1, v=vec).value
    g = np.asarray(grad_fn(st.x, sigma, e), np.float64)
    restarted = False
    if st.j == 0:
        if st.it % o.recompute == 0:
            st.r = -g
            st.d = st.r.copy()
            st.rr = float(st.r @ st.r)
            restarted = True
        else:
            r_new = -g if o.residual_mode == 1 else st.r
            rr_new = float(r_new @ r_new)
            beta = rr_new / st.rr if st.rr > 0.0 else 0.0
            d = r_new + beta * st.d
            if float(r_new @ d) <= 0.0:
                d = r_new.copy()
                restarted = True
            st.r, st.d, st.rr = r_new.copy(), d, rr_new
    lam = o.lambda_rel * float(np.linalg.norm(g))
    q = np.asarray(hvp_fn(st.x, sigma, e, st.d), np.float64) + lam * st.d
    gd = float(g @ st.d)
    dHd = float(st.d @ q)
    dn = float(np.linalg.norm(st.d))
    alpha = 0.0
    if dn > 0.0:
        cap = o.trust_radius / dn
        if dHd > 0.0:
            alpha = -gd / dHd
        elif gd < 0.0:
            alpha = cap
        elif gd > 0.0:
            alpha = -cap
        alpha = min(max(alpha, -cap), cap)
    st.x = st.x + alpha * st.d
    if o.residual_mode == 0:
        st.r = st.r - alpha * q
    info = NcgInfo(st.it, st.j, restarted, sigma, float(np.linalg.norm(g)), gd, dHd, alpha, abs(alpha) * dn)
    st.j += 1
    if st.j >= o.ls_iters or abs(alpha) * dn <= o.ls_tol:
        st.j = 0
        st.it += 1
        st.sigma = anneal_sigma(o.sigma_start, o.sigma_end, o.anneal_iters, st.it)
    st.evals += 1
    return info
