"""Pins of the oracle's renderers against independent FP64 computations:
a ray cast of the rotated mesh (Moller-Trumbore) for the rasteriser, a
barycentric point-in-triangle test in painter's order for the 2D triangles,
and, for the path tracer, closed-form ray distances, a furnace (every surface
emits E with albedo rho: each pixel is E (1 + rho + ... + rho^(depth-1))) and
direct lighting from the rectangular light against numerical quadrature."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2412_03489_gb300 import workloads as wl


def _rot(a, b):
    ca, sa, cb, sb = math.cos(a), math.sin(a), math.cos(b), math.sin(b)
    Rx = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    return Rx @ Ry


def test_revolve_raster_matches_fp64_ray_cast():
    W = H = 96
    sc = wl.revolve_scene(width=W, height=H)
    sc["scale"] = np.float32((H / 2.0) / math.tan(math.radians(30.0) / 2.0))
    r = O.RevolveRenderer(sc)
    p = np.asarray(sc["theta_query"], np.float32)
    img = r.image(p).reshape(H, W, 3)
    R = _rot(float(p[0]), float(p[1]))
    V = sc["vertices"].astype(np.float64) @ R.T
    T = sc["triangles"]
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    e1, e2 = b - a, c - a
    nrm = np.cross(e1, e2)
    ln = np.linalg.norm(nrm, axis=1)
    ok = ln > 0
    k = float(sc["scale"])
    D = float(sc["eye_dist"])
    eye = np.array([0.0, 0.0, D])
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    dirs = np.stack([(xs - W / 2) / k, -(ys - H / 2) / k, -np.ones_like(xs)], -1).reshape(-1, 3)
    best_t = np.full(len(dirs), np.inf)
    best_i = np.full(len(dirs), -1)
    second = np.full(len(dirs), np.inf)
    margin = np.full(len(dirs), np.inf)       # barycentric margin of the winner
    near_edge = np.zeros(len(dirs), bool)     # any triangle hit within a tiny margin
    for i in np.nonzero(ok)[0]:
        if nrm[i] @ (eye - a[i]) <= 0:        # back face as seen from the eye
            continue
        pv = np.cross(dirs, e2[i])
        det = pv @ e1[i]
        tv = eye - a[i]
        u = (pv @ tv) / det
        qv = np.cross(tv, e1[i])
        v = (dirs @ qv) / det
        t = (qv @ e2[i]) / det
        m = np.minimum(np.minimum(u, v), 1 - u - v)
        near_edge |= np.abs(m) < 2e-3
        hit = (m > 0) & (t > 0)
        upd = hit & (t < best_t)
        second = np.where(upd, best_t, np.where(hit, np.minimum(second, t), second))
        best_t = np.where(upd, t, best_t)
        best_i = np.where(upd, i, best_i)
        margin = np.where(upd, m, margin)
    l = sc["light"].astype(np.float64)
    col = np.zeros((len(dirs), 3))
    hitm = best_i >= 0
    nw = nrm[best_i[hitm]] / ln[best_i[hitm], None]
    col[hitm] = np.maximum(0.0, nw @ l)[:, None] * sc["albedo"].astype(np.float64)[None, :]
    gap = np.where(np.isinf(second), np.inf, second - np.where(np.isinf(best_t), 0.0, best_t))
    safe = ~near_edge & (gap > 1e-3)
    assert safe.mean() > 0.9
    assert hitm.mean() > 0.1                            # the object is on screen
    diff = np.abs(col - img.reshape(-1, 3)).max(1)
    assert np.all(diff[safe] < 1e-5), np.count_nonzero(diff[safe] >= 1e-5)
    # the triangle each pixel shows is the ray cast's nearest hit
    ids = r.ids(p)
    assert np.array_equal(ids[safe], best_i[safe])


def test_revolve_depth_ties_go_to_the_lower_index():
    """A mesh listed twice (the copy's indices shifted by T): copies have the
    same vertices, hence the same FP32 edge functions and depth planes, so
    every covered pixel is an exact depth tie between triangle i and i + T;
    the lower index must win everywhere, giving the single mesh's picture."""
    W = H = 72
    sc = wl.revolve_scene(width=W, height=H)
    sc["vertices"], sc["triangles"] = wl.sheets_mesh(layers=3, grid=4)
    T = len(sc["triangles"])
    dup = dict(sc, triangles=np.concatenate([sc["triangles"], sc["triangles"]]))
    p = np.asarray(sc["theta_query"], np.float32)
    one, two = O.RevolveRenderer(sc).ids(p), O.RevolveRenderer(dup).ids(p)
    assert (one >= 0).mean() > 0.3
    assert np.array_equal(one, two)
    assert two.max() < T


def test_tris2d_raster_matches_fp64_barycentric_painter():
    W = H = 80
    sc = wl.tris2d_scene(width=W, height=H)
    r = O.Tris2dRenderer(sc)
    p = np.asarray(sc["theta_init"][3], np.float32)
    img = r.image(p).reshape(-1, 3)
    raw = sc["raw_params"].astype(np.float64).copy()
    raw[sc["param_index"]] = p.astype(np.float64)
    raw = raw.reshape(-1, 9)
    xs, ys = np.meshgrid((np.arange(W) + 0.5), (np.arange(H) + 0.5))
    P = np.stack([xs.ravel(), ys.ravel()], -1)
    col = np.zeros((W * H, 3))
    unsafe = np.zeros(W * H, bool)
    for t in range(raw.shape[0]):
        A, B, C = (raw[t, 0:2] * [W, H], raw[t, 2:4] * [W, H], raw[t, 4:6] * [W, H])
        den = (B[1] - C[1]) * (A[0] - C[0]) + (C[0] - B[0]) * (A[1] - C[1])
        l1 = ((B[1] - C[1]) * (P[:, 0] - C[0]) + (C[0] - B[0]) * (P[:, 1] - C[1])) / den
        l2 = ((C[1] - A[1]) * (P[:, 0] - C[0]) + (A[0] - C[0]) * (P[:, 1] - C[1])) / den
        m = np.minimum(np.minimum(l1, l2), 1 - l1 - l2)
        unsafe |= np.abs(m) < 1e-4
        col[m > 0] = raw[t, 6:9]
    safe = ~unsafe
    assert safe.mean() > 0.95
    assert np.all(np.abs(col[safe] - img[safe]) < 1e-7)


# ---------------------------------------------------------------------------
# path tracer
# ---------------------------------------------------------------------------
def test_ptbox_ray_distances():
    sc = wl.ptbox_scene(width=16, height=16)
    r = O.PtboxRenderer(sc, target=np.zeros(16 * 16 * 3, np.float32))
    p = np.asarray(sc["theta_target"], np.float32)
    o = np.array([0.0, 0.0, float(sc["cam_z"])], np.float32)
    prim, t = r.intersect(p, o, [0.0, 0.0, -1.0])
    assert prim == 4 and t == pytest.approx(1.0 + float(sc["cam_z"]), abs=1e-6)   # back wall z = -1
    c1 = sc["sph_center"][1].astype(np.float64)
    d = (c1 - o) / np.linalg.norm(c1 - o)
    prim, t = r.intersect(p, o, d)
    assert prim == 14 and t == pytest.approx(np.linalg.norm(c1 - o) - float(sc["sph_radius"][1]), abs=2e-6)
    # straight up from below the light hits the light (index 12) at plane - y
    lo = np.array([p[0], 0.0, p[2]], np.float32)
    prim, t = r.intersect(p, lo, [0.0, 1.0, 0.0])
    assert prim == 12 and t == pytest.approx(float(p[1]), abs=1e-6)
    # sphere 0 follows params 3..5
    c0 = p[3:6].astype(np.float64)
    d = (c0 - o) / np.linalg.norm(c0 - o)
    prim, t = r.intersect(p, o, d)
    assert prim == 13 and t == pytest.approx(np.linalg.norm(c0 - o) - 0.25, abs=2e-6)


def test_ptbox_furnace():
    sc = wl.ptbox_scene(width=24, height=24)
    rho = 0.5
    sc["quad_albedo"] = np.full((12, 3), rho, np.float32)
    sc["sph_albedo"] = np.full((3, 3), rho, np.float32)
    sc["light_emission"] = np.array([1.0, 2.0, 4.0], np.float32)
    r = O.PtboxRenderer(sc, target=np.zeros(24 * 24 * 3, np.float32), emit_all=True, nee=False)
    for depth in (1, 3):
        r.depth = depth
        img = r.image(np.asarray(sc["theta_query"], np.float32), 2, 7, 1, 0, 0, O.TAG_PATH).reshape(-1, 3)
        expect = sum(rho ** kk for kk in range(depth)) * sc["light_emission"].astype(np.float64)
        assert np.allclose(img, expect[None, :], rtol=0, atol=1e-12)


def test_ptbox_direct_lighting_matches_quadrature():
    sc = wl.ptbox_scene(width=8, height=8)
    # move the block and the spheres out of the box so nothing occludes
    g = sc["quad_geom"].copy()
    g[6:, 0] += 10.0
    g[6:, 1:] += 10.0
    sc["quad_geom"] = g
    sc["sph_center"] = sc["sph_center"] + np.float32(10.0)
    rho = np.array([0.3, 0.5, 0.7], np.float32)
    alb = sc["quad_albedo"].copy()
    alb[2] = rho                                   # floor y = -1
    sc["quad_albedo"] = alb
    r = O.PtboxRenderer(sc, target=np.zeros(8 * 8 * 3, np.float32), depth=1)
    p = np.array([0.1, 0.9, -0.2, 5.0, 5.0, 5.0], np.float32)
    x0, z0 = 0.35, 0.15
    o = np.array([x0, -0.99, z0], np.float32)
    N = 20000
    vals = np.array([r.trace(p, o, [0.0, -1.0, 0.0], 1, 3, 1, 0, 0, O.TAG_PATH, i) for i in range(N)])
    # shading point is the floor hit offset by 1e-4 along the normal
    h = float(np.float32(0.9)) - float(np.float32(np.float32(-1.0) + np.float32(1e-4)))
    f = lambda zz, xx: h * h / (h * h + (xx - x0) ** 2 + (zz - z0) ** 2) ** 2
    hl = float(sc["light_half"])
    I, _ = integrate.dblquad(f, 0.1 - hl, 0.1 + hl, -0.2 - hl, -0.2 + hl, epsabs=1e-12, epsrel=1e-10)
    E = sc["light_emission"].astype(np.float64)
    expect = rho.astype(np.float64) / math.pi * E * I
    mean, se = vals.mean(0), vals.std(0, ddof=1) / math.sqrt(N)
    assert np.all(np.abs(mean - expect) < 4 * se + 1e-12), (mean, expect, se)
    assert np.all(vals >= 0)
