"""Seeded synthetic inputs for the estimator workloads.

This module only builds scene inputs (geometry, albedos, target and query
parameters, HVP directions) from a seed with numpy's PCG64 generator.  It holds
none of the estimator's arithmetic: no perturbation sampling, no kernel
weights, no rendering.  The random numbers the estimator itself draws come from
Philox4x32-10 inside the CUDA path and, independently, inside the oracle.

The scenes stand in for the paper's tasks (Sec. 4.1 "Tasks"): the disc for the
Box2 plateau task, the surface of revolution for Mug, the path-traced box for
Shadow, and the coloured triangles for the Box10/mesh tasks.  The paper's own
assets are not used.

Every scene is a plain dict of numpy arrays plus scalars; `pack_*` helpers in
the binding turn it into the C-ABI scene descriptor.
"""
from __future__ import annotations

import math

import numpy as np

SCENE_DISC2D = 0
SCENE_REVOLVE3D = 1
SCENE_PTBOX = 2
SCENE_TRIS2D = 3
SCENE_BOXES2D = 4
SCENE_QUADRATIC = 5
SCENE_STEP1D = 6
SCENE_NEGGAUSS = 7


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# Disc: 2 params (centre x, y) in [0,1]^2 image coordinates.
# ---------------------------------------------------------------------------
def disc_scene(seed: int = 0xC0, width: int = 64, height: int = 64,
               radius: float = 0.2, query_std: float = 0.1) -> dict:
    g = _rng(seed)
    target = g.uniform(0.3, 0.7, size=2)
    query = target + g.normal(0.0, query_std, size=2)
    return dict(kind=SCENE_DISC2D, width=width, height=height, channels=1,
                n_params=2, radius=np.float32(radius),
                theta_target=target.astype(np.float64),
                theta_query=query.astype(np.float64), sigma=0.05, seed=seed)


# ---------------------------------------------------------------------------
# Squares (Box2 / Box10 plateau tasks): K squares, 2K params (centres).
# ---------------------------------------------------------------------------
def boxes_scene(n_boxes: int = 1, seed: int = 0xB0, width: int = 64, height: int = 64,
                half_size: float = 0.1, query_std: float = 0.15) -> dict:
    g = _rng(seed + n_boxes)
    target = g.uniform(0.2, 0.8, size=2 * n_boxes)
    query = target + g.normal(0.0, query_std, size=2 * n_boxes)
    return dict(kind=SCENE_BOXES2D, width=width, height=height, channels=1, n_params=2 * n_boxes,
                half_size=np.float32(half_size), theta_target=target, theta_query=query,
                sigma=0.05, seed=seed)


# ---------------------------------------------------------------------------
# Analytic test functions (no renderer): the Quad task's quadratic, the 1D
# hard edge, the negated Gaussian.  1 x 1 x 1 "images".
# ---------------------------------------------------------------------------
def quadratic_scene(A=None, b=None, theta=None, sigma: float = 0.1) -> dict:
    A = np.array([[10.0, 7.5], [7.5, 10.0]]) if A is None else np.asarray(A, np.float64)
    n = A.shape[0]
    b = np.zeros(n) if b is None else np.asarray(b, np.float64)
    theta = np.full(n, 0.5) if theta is None else np.asarray(theta, np.float64)
    return dict(kind=SCENE_QUADRATIC, width=1, height=1, channels=1, n_params=n, A=A, b=b,
                theta_target=None, theta_query=theta, sigma=sigma, seed=0)


def step1d_scene(theta: float = 0.03, sigma: float = 0.05) -> dict:
    return dict(kind=SCENE_STEP1D, width=1, height=1, channels=1, n_params=1,
                theta_target=None, theta_query=np.array([theta]), sigma=sigma, seed=0)


def neggauss_scene(gauss_sigma: float = 1.0, theta=(0.7, -0.4), sigma: float = 0.5) -> dict:
    return dict(kind=SCENE_NEGGAUSS, width=1, height=1, channels=1, n_params=len(theta),
                gauss_sigma=gauss_sigma, theta_target=None, theta_query=np.asarray(theta, np.float64),
                sigma=sigma, seed=0)


# ---------------------------------------------------------------------------
# Surface of revolution: 33 rings x 32 slices, 2048 triangles.
# ---------------------------------------------------------------------------
def _catmull_rom(ctrl: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Uniform Catmull-Rom spline through ctrl placed at equally spaced
    heights on [-1, 1]; end points are repeated for the end segments."""
    m = len(ctrl)
    pts = np.concatenate([[ctrl[0]], ctrl, [ctrl[-1]]])
    s = (y + 1.0) * 0.5 * (m - 1)
    seg = np.clip(np.floor(s).astype(int), 0, m - 2)
    u = s - seg
    p0, p1, p2, p3 = pts[seg], pts[seg + 1], pts[seg + 2], pts[seg + 3]
    return 0.5 * (2 * p1 + (-p0 + p2) * u + (2 * p0 - 5 * p1 + 4 * p2 - p3) * u * u
                  + (-p0 + 3 * p1 - 3 * p2 + p3) * u ** 3)


def revolve_mesh(radii: np.ndarray, rings: int = 33, slices: int = 32):
    """Closed surface of revolution about the y axis on y in [-1, 1].

    The profile is the Catmull-Rom spline through `radii` times
    sqrt(1 - y^2), so both ends close at a pole.  Triangles are wound so that
    (v1 - v0) x (v2 - v0) points outward.  Returns (vertices float32 [V,3],
    triangles int32 [T,3]); pole triangles with two equal vertices are kept
    (they have zero area and are culled by the renderer).
    """
    y = -1.0 + 2.0 * np.arange(rings) / (rings - 1)
    rho = _catmull_rom(np.asarray(radii, np.float64), y) * np.sqrt(np.maximum(0.0, 1.0 - y * y))
    phi = 2.0 * math.pi * np.arange(slices) / slices
    verts = np.zeros((rings, slices, 3), np.float64)
    verts[:, :, 0] = rho[:, None] * np.cos(phi)[None, :]
    verts[:, :, 1] = y[:, None]
    verts[:, :, 2] = rho[:, None] * np.sin(phi)[None, :]
    verts = verts.reshape(-1, 3).astype(np.float32)
    tris = []
    for k in range(rings - 1):
        for s in range(slices):
            v00 = k * slices + s
            v01 = k * slices + (s + 1) % slices
            v10 = (k + 1) * slices + s
            v11 = (k + 1) * slices + (s + 1) % slices
            tris.append((v00, v10, v11))
            tris.append((v00, v11, v01))
    return verts, np.asarray(tris, np.int32)


def sheets_mesh(layers: int = 8, grid: int = 8, seed: int = 0xC6, half: float = 1.0):
    """Stacked, slightly tilted square sheets facing the camera (+z), for the
    rasteriser's stress cases: `layers` sheets of grid x grid quads (two
    triangles each), sheet k at depth z_k in [-0.6, 0.6] with seeded
    vertex jitter, so that every pixel is covered by several triangles at
    different depths and every triangle spans many 8x8 tiles.  Triangles are
    wound so that (v1 - v0) x (v2 - v0) points towards +z (front-facing).
    Returns (vertices float32 [V,3], triangles int32 [T,3])."""
    g = _rng(seed)
    verts, tris = [], []
    xs = np.linspace(-half, half, grid + 1)
    for k in range(layers):
        z0 = -0.6 + 1.2 * k / max(1, layers - 1)
        tilt = g.uniform(-0.15, 0.15, size=2)
        base = len(verts)
        for iy in range(grid + 1):
            for ix in range(grid + 1):
                x = xs[ix] + g.uniform(-0.02, 0.02)
                y = xs[iy] + g.uniform(-0.02, 0.02)
                verts.append((x, y, z0 + tilt[0] * x + tilt[1] * y))
        for iy in range(grid):
            for ix in range(grid):
                a = base + iy * (grid + 1) + ix
                b, c, d = a + 1, a + grid + 1, a + grid + 2
                tris.append((a, b, d))
                tris.append((a, d, c))
    return np.asarray(verts, np.float32), np.asarray(tris, np.int32)


def revolve_scene(seed: int = 0xC1, width: int = 256, height: int = 256,
                  fov_deg: float = 30.0, eye_dist: float = 4.0,
                  query_std: float = 0.1) -> dict:
    g = _rng(seed)
    radii = g.uniform(0.3, 0.8, size=8)
    albedo = g.uniform(0.2, 0.9, size=3).astype(np.float32)
    target = g.uniform(-0.4, 0.4, size=2)
    query = target + g.normal(0.0, query_std, size=2)
    verts, tris = revolve_mesh(radii)
    light = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    # pixels per unit of (X/Z) in camera space: (H/2) / tan(fov/2)
    scale = (height / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    return dict(kind=SCENE_REVOLVE3D, width=width, height=height, channels=3,
                n_params=2, vertices=verts, triangles=tris,
                albedo=albedo, light=light.astype(np.float32),
                eye_dist=np.float32(eye_dist), scale=np.float32(scale),
                theta_target=target, theta_query=query, sigma=0.1, seed=seed)


# ---------------------------------------------------------------------------
# Path-traced box: 12 axis-aligned quads (6 walls + a 6-face block), an
# axis-aligned emitting quad (light), 3 spheres.  6 params: light centre xyz,
# sphere-0 centre xyz.
# ---------------------------------------------------------------------------
def _box_quads(lo, hi, inward: bool):
    """Six axis-aligned faces of the box [lo, hi]; each quad is
    (axis, plane, lo_u, lo_v, hi_u, hi_v, normal_sign) with (u, v) the two
    other axes in increasing order.  normal_sign is informative only (the
    renderer faces normals against the incoming ray)."""
    quads = []
    for a in range(3):
        u, v = [x for x in range(3) if x != a]
        for side, plane in ((0, lo[a]), (1, hi[a])):
            sign = (1.0 if side == 0 else -1.0) if inward else (-1.0 if side == 0 else 1.0)
            quads.append((a, plane, lo[u], lo[v], hi[u], hi[v], sign))
    return quads


def ptbox_scene(seed: int = 0xC2, width: int = 128, height: int = 128,
                spp: int = 4, target_spp: int = 64, fov_deg: float = 70.0,
                query_std: float = 0.05) -> dict:
    g = _rng(seed)
    quads = _box_quads((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), inward=True)
    quads += _box_quads((0.2, -1.0, -0.7), (0.7, -0.3, -0.2), inward=False)
    q = np.array([[qq[0], qq[1], qq[2], qq[3], qq[4], qq[5]] for qq in quads], np.float64)
    quad_axis = q[:, 0].astype(np.int32)
    quad_geom = q[:, 1:6].astype(np.float32)            # plane, lo_u, lo_v, hi_u, hi_v
    quad_albedo = g.uniform(0.2, 0.9, size=(12, 3)).astype(np.float32)
    sph_center = np.array([[-0.45, -0.7, -0.3], [0.45, 0.0, -0.5], [-0.5, 0.3, -0.6]], np.float64)
    sph_center[1:] += g.uniform(-0.1, 0.1, size=(2, 3))
    sph_radius = np.array([0.25, 0.2, 0.15], np.float32)
    sph_albedo = g.uniform(0.2, 0.9, size=(3, 3)).astype(np.float32)
    light_target = np.array([0.0, 0.9, 0.0]) + np.array([1, 0, 1]) * g.uniform(-0.2, 0.2, size=3)
    s0_target = sph_center[0] + g.uniform(-0.1, 0.1, size=3)
    target = np.concatenate([light_target, s0_target])
    query = target + g.normal(0.0, query_std, size=6)
    v = g.normal(size=6)
    v /= np.linalg.norm(v)
    tan_half = math.tan(math.radians(fov_deg) / 2.0)
    return dict(kind=SCENE_PTBOX, width=width, height=height, channels=3, n_params=6,
                quad_axis=quad_axis, quad_geom=quad_geom, quad_albedo=quad_albedo,
                sph_center=sph_center.astype(np.float32), sph_radius=sph_radius,
                sph_albedo=sph_albedo, light_half=np.float32(0.25),
                light_emission=np.array([12.0, 12.0, 12.0], np.float32),
                cam_z=np.float32(0.95), tan_half=np.float32(tan_half),
                pix_scale=np.float32(2.0 * tan_half / height),
                spp=spp, target_spp=target_spp,
                theta_target=target, theta_query=query, v=v, sigma=0.05, seed=seed)


# ---------------------------------------------------------------------------
# Coloured triangles: 16 triangles x (x0,y0,x1,y1,x2,y2,r,g,b) = 144 raw
# params; a seeded subset of 64 is optimised.
# ---------------------------------------------------------------------------
def tris2d_scene(seed: int = 0xC3, width: int = 256, height: int = 256,
                 n_tris: int = 16, n_params: int = 64, n_instances: int = 64,
                 init_std: float = 0.03) -> dict:
    g = _rng(seed)
    raw = np.zeros((n_tris, 9), np.float64)
    raw[:, 0:6] = g.uniform(0.05, 0.95, size=(n_tris, 6))
    raw[:, 6:9] = g.uniform(0.1, 0.9, size=(n_tris, 3))
    raw = raw.reshape(-1).astype(np.float32)
    mask = np.sort(g.choice(raw.size, size=n_params, replace=False)).astype(np.int32)
    target = raw[mask].astype(np.float64)
    theta0 = target[None, :] + g.normal(0.0, init_std, size=(n_instances, n_params))
    v = g.normal(size=n_params)
    v /= np.linalg.norm(v)
    return dict(kind=SCENE_TRIS2D, width=width, height=height, channels=3,
                n_params=n_params, n_tris=n_tris, raw_params=raw, param_index=mask,
                theta_target=target, theta_query=theta0[0].copy(), theta_init=theta0,
                v=v, sigma=0.02, seed=seed)


def scaled(scene_fn, **kw) -> dict:
    """Call a scene builder with overrides (small parity sizes)."""
    return scene_fn(**kw)


# ---------------------------------------------------------------------------
# Serving mix: resident scenes of every kind and a seeded request stream with
# Poisson arrivals (parameter dims 2..64, 256..16384 samples, 64^2..512^2).
# ---------------------------------------------------------------------------
def serving_scenes() -> dict:
    return {
        "disc64": disc_scene(),
        "disc512": disc_scene(seed=0xD5, width=512, height=512),
        "revolve128": revolve_scene(seed=0xE1, width=128, height=128),
        "revolve256": revolve_scene(),
        "revolve512": revolve_scene(seed=0xE5, width=512, height=512),
        "pt64": ptbox_scene(seed=0xF2, width=64, height=64, spp=2, target_spp=16),
        "tris128_n64": tris2d_scene(seed=0xA3, width=128, height=128, n_instances=1),
        "tris256_n16": tris2d_scene(seed=0xA4, width=256, height=256, n_params=16, n_instances=1),
    }


# (scene, quantity, strategy, samples); quantity 0 grad, 1 Hessian, 2 HVP,
# 3 Newton-CG step (samples = index of the resident optimizer state);
# strategy 0 element-wise, 1 aggregate
SERVING_KINDS = [
    ("disc64", 1, 0, 1024), ("disc64", 1, 1, 16384), ("disc64", 0, 1, 4096), ("disc512", 1, 1, 256),
    ("revolve128", 1, 1, 2048), ("revolve256", 1, 1, 4096), ("revolve256", 2, 1, 1024), ("revolve512", 1, 1, 256),
    ("pt64", 2, 1, 256), ("tris128_n64", 2, 1, 512), ("tris128_n64", 0, 1, 1024), ("tris256_n16", 2, 1, 256),
    ("tris128_n64", 3, 1, 0), ("tris256_n16", 3, 1, 1),
]


def serving_newton_states(scenes: dict) -> list:
    """Resident Newton-CG states of the serving mix: (scene, instances,
    initial parameters [B][n], sigma, gradient / HVP samples, CG iterations,
    trust radius)."""
    g = _rng(0xC6)
    out = []
    for name, B in (("tris128_n64", 8), ("tris256_n16", 4)):
        sc = scenes[name]
        th0 = np.asarray(sc["theta_target"], np.float64)[None, :] + g.normal(0.0, 0.03, size=(B, sc["n_params"]))
        out.append(dict(scene=name, B=B, theta0=th0, sigma=sc["sigma"], n_grad=32, n_hvp=32, cg_iters=4,
                        trust_radius=0.05))
    return out


def serving_requests(scenes: dict, n_requests: int = 240, rate_hz: float = 1000.0, seed: int = 0xC4) -> list:
    g = _rng(seed)
    t = 0.0
    reqs = []
    for i in range(n_requests):
        t += g.exponential(1.0 / rate_hz)
        name, q, strat, M = SERVING_KINDS[int(g.integers(len(SERVING_KINDS)))]
        sc = scenes[name]
        n = sc["n_params"]
        theta = np.asarray(sc["theta_query"], np.float64) + g.normal(0.0, 0.01, n)
        v = g.normal(size=n) if q == 2 else None
        reqs.append(dict(scene=name, quantity=q, strategy=strat, M=M, theta=theta, v=v,
                         sigma=sc["sigma"], seed=1 + i, request=i, arrival_s=t,
                         state=M if q == 3 else None))
    return reqs
