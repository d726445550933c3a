"""Pins of the oracle's estimators against closed forms, independent numerical
routes and invariants (none of them re-uses the oracle's formulas):

* quadratic loss: Gaussian smoothing leaves its Hessian unchanged and its
  gradient at theta equal to the true gradient (Quad task of Sec. 4.1);
* 1D hard step: fbar = Phi(theta/s), fbar' = phi/s, fbar'' = -theta/s^3 phi;
* negated Gaussian (Suppl. "Positive-Definite Hessians"): -N(0, s1^2 I)
  smoothed by N(0, s2^2 I) is -N(0, (s1^2 + s2^2) I);
* the disc scene: fbar from the noncentral chi-square CDF, its derivatives by
  a contour integral (divergence theorem), both cross-checked, then the Monte
  Carlo estimates within 4 standard errors; and a 2D Gauss-Hermite brute force;
* invariants: symmetry, HVP = H v on the same samples, render counts (Tab. 1).
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from conftest import read_golden
from paper_2412_03489_gb300 import workloads as wl


def per_pair_stats(est):
    """Estimate and its standard error from the per-pair contributions
    1/2 (w+ f+ + w- f-) of the pairs that carry weight for each element."""
    M, E = est.w.shape
    c = 0.5 * (est.w[0::2] * est.losses[0::2, None] + est.w[1::2] * est.losses[1::2, None])
    used = (np.abs(est.w[0::2]) + np.abs(est.w[1::2])) > 0
    se = np.zeros(E)
    for e in range(E):
        ce = c[used[:, e], e]
        se[e] = ce.std(ddof=1) / math.sqrt(len(ce))
    return se


def upper(H):
    n = H.shape[0]
    return np.array([H[a, b] for a in range(n) for b in range(a, n)])


# ---------------------------------------------------------------------------
# quadratic
# ---------------------------------------------------------------------------
def quad_task():
    a, b, c, h00, h01, h11 = (float(x) for x in read_golden("paper_quad_task.txt")[0])
    f = lambda X: a * X[:, 0] ** 2 + b * X[:, 1] ** 2 + c * X[:, 0] * X[:, 1]
    H = np.array([[h00, h01], [h01, h11]])
    return f, H


@pytest.mark.parametrize("strategy", ["elementwise", "aggregate"])
def test_quad_task_hessian_and_gradient(strategy):
    f, H = quad_task()
    r = O.FunctionRenderer(f, 2)
    theta = np.array([0.8, -0.3])
    for sigma in (0.1, 1.0):
        est = O.estimate(r, "hessian", theta, sigma, 40000, strategy, seed=17, request=3)
        se = per_pair_stats(est)
        assert np.all(np.abs(est.flat - upper(H)) < 4 * se + 1e-12), (est.flat, se)
        g = O.estimate(r, "grad", theta, sigma, 40000, strategy, seed=18, request=3)
        assert np.all(np.abs(g.flat - H @ theta) < 4 * per_pair_stats(g) + 1e-12)
        hv = O.estimate(r, "hvp", theta, sigma, 40000, "aggregate", seed=19, request=3, v=np.array([0.6, 0.8]))
        assert np.all(np.abs(hv.flat - H @ np.array([0.6, 0.8])) < 4 * per_pair_stats(hv) + 1e-12)


def test_random_quadratic_4d_aggregate():
    g = np.random.default_rng(5)
    B = g.normal(size=(4, 4))
    A = B + B.T
    bvec = g.normal(size=4)
    f = lambda X: 0.5 * np.einsum("mi,ij,mj->m", X, A, X) + X @ bvec
    r = O.FunctionRenderer(f, 4)
    theta = g.normal(size=4)
    est = O.estimate(r, "hessian", theta, 0.3, 60000, "aggregate", seed=2, request=9)
    assert np.all(np.abs(est.flat - upper(A)) < 4 * per_pair_stats(est) + 1e-12)
    est = O.estimate(r, "hessian", theta, 0.3, 20000, "elementwise", seed=2, request=9)
    assert np.all(np.abs(est.flat - upper(A)) < 4 * per_pair_stats(est) + 1e-12)
    gr = O.estimate(r, "grad", theta, 0.3, 60000, "aggregate", seed=3, request=9)
    assert np.all(np.abs(gr.flat - (A @ theta + bvec)) < 4 * per_pair_stats(gr) + 1e-12)


# ---------------------------------------------------------------------------
# 1D hard step: the discontinuous case the method exists for (Sec. 3.1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("t", [-1.3, 0.0, 0.7, 2.0])
def test_step_edge(t):
    sigma = 0.2
    theta = np.array([t * sigma])
    r = O.FunctionRenderer(lambda X: (X[:, 0] > 0).astype(np.float64), 1)
    phi = stats.norm.pdf(t)
    est = O.estimate(r, "hessian", theta, sigma, 60000, "elementwise", seed=4, request=1)
    exact2 = -(t * sigma) / sigma ** 3 * phi     # -theta / s^3 phi(theta / s)
    assert abs(est.flat[0] - exact2) < 4 * per_pair_stats(est)[0] + 1e-9
    est = O.estimate(r, "grad", theta, sigma, 60000, "elementwise", seed=5, request=1)
    assert abs(est.flat[0] - phi / sigma) < 4 * per_pair_stats(est)[0] + 1e-9


# ---------------------------------------------------------------------------
# negated Gaussian (non-PSD Hessian)
# ---------------------------------------------------------------------------
def neg_gauss(s):
    def f(X):
        return -np.exp(-0.5 * np.sum(X * X, axis=1) / s ** 2) / (2 * math.pi * s * s)
    return f


def neg_gauss_hessian(theta, s2):
    N = math.exp(-0.5 * theta @ theta / s2) / (2 * math.pi * s2)
    return -N * (np.outer(theta, theta) / s2 ** 2 - np.eye(2) / s2)


@pytest.mark.parametrize("theta", [(0.0, 0.0), (1.5, -0.5), (-2.5, 2.0), (0.4, 0.9)])
def test_negated_gaussian_hessian(theta):
    s1, s2 = 1.0, 0.5
    theta = np.array(theta)
    r = O.FunctionRenderer(neg_gauss(s1), 2)
    est = O.estimate(r, "hessian", theta, s2, 40000, "aggregate", seed=8, request=2)
    exact = neg_gauss_hessian(theta, s1 * s1 + s2 * s2)
    assert np.all(np.abs(est.flat - upper(exact)) < 4 * per_pair_stats(est) + 1e-12)


# ---------------------------------------------------------------------------
# disc scene: closed-form smoothed loss and contour-integral derivatives
# ---------------------------------------------------------------------------
def disc_closed_form(sc, theta, sigma, K=1024):
    W, H, r = sc["width"], sc["height"], float(sc["radius"])
    tgt = O.DiscRenderer(sc).target.astype(np.float64)
    xs = (np.arange(W) + 0.5) / W
    ys = (np.arange(H) + 0.5) / H
    px, py = np.meshgrid(xs, ys)
    px, py, tgt = px.ravel(), py.ravel(), tgt.ravel()
    a = 1.0 - 2.0 * tgt
    # fbar = mean[(1 - 2t) Pr(|p - theta - tau| < r) + t]
    d2 = (px - theta[0]) ** 2 + (py - theta[1]) ** 2
    g = stats.ncx2.cdf(r * r / sigma ** 2, 2, d2 / sigma ** 2)
    fbar = np.mean(a * g + tgt)
    # derivatives by the divergence theorem on each pixel's disc boundary
    phi = 2 * math.pi * np.arange(K) / K
    nx, ny = np.cos(phi), np.sin(phi)
    yx = px[:, None] + r * nx[None, :] - theta[0]
    yy = py[:, None] + r * ny[None, :] - theta[1]
    N = np.exp(-0.5 * (yx ** 2 + yy ** 2) / sigma ** 2) / (2 * math.pi * sigma ** 2)
    dphi = 2 * math.pi / K
    grad = np.array([-(N * nx).sum(1), -(N * ny).sum(1)]) * r * dphi
    Hs = np.zeros((2, 2, len(px)))
    comps = (yx, yy)
    ns = (nx, ny)
    for k in range(2):
        for l in range(2):
            Hs[k, l] = -(comps[k] / sigma ** 2 * N * ns[l][None, :]).sum(1) * r * dphi
    grad = (grad * a).mean(1)
    Hm = (Hs * a).mean(2)
    return fbar, grad, Hm


def test_disc_contour_derivatives_match_finite_differences_of_closed_form():
    sc = wl.disc_scene()
    sigma = sc["sigma"]
    th = np.asarray(sc["theta_query"])
    f0, g, H = disc_closed_form(sc, th, sigma)
    _, _, H2 = disc_closed_form(sc, th, sigma, K=2048)
    assert np.allclose(H, H2, rtol=1e-10, atol=1e-10)          # spectral convergence in K
    assert np.allclose(H, H.T, rtol=1e-8, atol=1e-8)
    h = 1e-4
    fd_g, fd_H = np.zeros(2), np.zeros((2, 2))
    E = np.eye(2)
    for k in range(2):
        fd_g[k] = (disc_closed_form(sc, th + h * E[k], sigma, 8)[0] - disc_closed_form(sc, th - h * E[k], sigma, 8)[0]) / (2 * h)
        fd_H[k] = (disc_closed_form(sc, th + h * E[k], sigma)[1] - disc_closed_form(sc, th - h * E[k], sigma)[1]) / (2 * h)
    assert np.allclose(g, fd_g, rtol=1e-5, atol=1e-6)
    assert np.allclose(H, fd_H, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("strategy", ["elementwise", "aggregate"])
def test_disc_estimates_match_exact_smoothed_derivatives(strategy):
    sc = wl.disc_scene()
    sigma = sc["sigma"]
    th = np.asarray(sc["theta_query"])
    _, g, H = disc_closed_form(sc, th, sigma)
    r = O.DiscRenderer(sc)
    est = O.estimate(r, "hessian", th, sigma, 1 << 14, strategy, seed=21, request=0)
    se = per_pair_stats(est)
    assert np.all(np.abs(est.flat - upper(H)) < 4 * se), (est.flat, upper(H), se)
    gr = O.estimate(r, "grad", th, sigma, 1 << 14, strategy, seed=22, request=0)
    assert np.all(np.abs(gr.flat - g) < 4 * per_pair_stats(gr)), (gr.flat, g)
    hv = O.estimate(r, "hvp", th, sigma, 1 << 14, "aggregate", seed=23, request=0, v=np.array([1.0, -2.0]))
    assert np.all(np.abs(hv.flat - H @ np.array([1.0, -2.0])) < 4 * per_pair_stats(hv))


def test_disc_gauss_hermite_brute_force():
    """2D Gauss-Hermite quadrature of the smoothed-Hessian integral with the
    oracle renderer as the integrand; slow convergence (piecewise-constant f),
    so the check is loose and the error must shrink with the node count."""
    sc = wl.disc_scene()
    sigma = sc["sigma"]
    th = np.asarray(sc["theta_query"])
    _, _, H = disc_closed_form(sc, th, sigma)
    r = O.DiscRenderer(sc)
    errs = []
    for K in (48, 192):
        x, wgt = np.polynomial.hermite.hermgauss(K)
        t = math.sqrt(2) * sigma * x
        acc = np.zeros((2, 2))
        for i in range(K):
            for j in range(K):
                tau = np.array([t[i], t[j]], np.float32)
                fval = r.loss(O.perturb(th, tau))
                c = np.array([[(t[i] ** 2 - sigma ** 2) / sigma ** 4, t[i] * t[j] / sigma ** 4],
                              [t[i] * t[j] / sigma ** 4, (t[j] ** 2 - sigma ** 2) / sigma ** 4]])
                acc += wgt[i] * wgt[j] / math.pi * c * fval
        errs.append(np.abs(acc - H).max())
    scale = np.abs(H).max()
    assert errs[1] < 0.25 * scale
    assert errs[1] < errs[0]


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def test_symmetry_hvp_identity_and_render_counts():
    sc = wl.disc_scene()
    r = O.DiscRenderer(sc)
    th = np.asarray(sc["theta_query"])
    v = np.array([0.3, -1.1])
    Hest = O.estimate(r, "hessian", th, 0.05, 512, "aggregate", seed=1, request=4)
    Hv = O.estimate(r, "hvp", th, 0.05, 512, "aggregate", seed=1, request=4, v=v)
    Hm = Hest.value
    assert np.array_equal(Hm, Hm.T)
    assert np.allclose(Hv.flat, Hm @ v, rtol=1e-12, atol=1e-12 * np.abs(Hest.scale).max())
    assert np.array_equal(Hest.tau, Hv.tau) and np.array_equal(Hest.losses, Hv.losses)
    # Tab. 1: renders per estimate
    n, M = 2, 64
    assert len(O.estimate(r, "hessian", th, 0.05, M, "elementwise", 1, 1).losses) == n * (n + 1) // 2 * M
    assert len(O.estimate(r, "hessian", th, 0.05, M, "aggregate", 1, 1).losses) == M
    assert len(O.estimate(r, "grad", th, 0.05, M, "elementwise", 1, 1).losses) == n * M
    assert len(O.estimate(r, "grad", th, 0.05, M, "aggregate", 1, 1).losses) == M
    assert len(O.estimate(r, "hvp", th, 0.05, M, "aggregate", 1, 1, v=v).losses) == M


def test_aggregate_weights_reduce_to_elementwise_for_one_dimension():
    tau, _ = O.draw(1, 1, 0.3, 100, seed=1, request=1, sub=0)
    w_ais = O.weights(1, 1, 0.3, tau)
    w_is = O.weights(1, 1, 0.3, tau, 0, 0)
    assert np.allclose(w_ais, w_is, rtol=1e-6)


def test_negated_gaussian_error_report():
    """The paper reports a mean Hessian error within 1e-4 over (-3, 3)^2 for 100
    samples without giving s1, s2; this measures ours for s1 = 1, s2 = 0.5 and
    only requires the error to shrink like 1/sqrt(M)."""
    s1, s2 = 1.0, 0.5
    r = O.FunctionRenderer(neg_gauss(s1), 2)
    grid = np.linspace(-2.5, 2.5, 5)
    errs = {}
    for M in (100, 6400):
        e = []
        for a in grid:
            for b in grid:
                th = np.array([a, b])
                est = O.estimate(r, "hessian", th, s2, M, "aggregate", seed=31, request=int(10 * (a + 3) + 100 * (b + 3)))
                e.append(np.abs(est.value - neg_gauss_hessian(th, s1 * s1 + s2 * s2)).mean())
        errs[M] = float(np.mean(e))
    assert errs[6400] < errs[100] / 4


# ---------------------------------------------------------------------------
# HVP forms beyond the aggregate direct kernel
# ---------------------------------------------------------------------------
def test_elementwise_hvp_row_mixture_is_unbiased():
    f, H = quad_task()
    r = O.FunctionRenderer(f, 2)
    theta = np.array([0.3, -0.4])
    v = np.array([0.8, -0.6])
    est = O.estimate(r, "hvp", theta, 0.5, 40000, "elementwise", seed=41, request=5, v=v)
    assert len(est.losses) == 2 * 40000            # Tab. 1: n sample sets for the HVP
    assert np.all(np.abs(est.flat - H @ v) < 4 * per_pair_stats(est) + 1e-12)
    # 4D random quadratic, v with a zero entry (that component is never drawn)
    g = np.random.default_rng(11)
    B = g.normal(size=(4, 4))
    A = B + B.T
    f4 = lambda X: 0.5 * np.einsum("mi,ij,mj->m", X, A, X)
    v4 = np.array([0.5, 0.0, -1.0, 2.0])
    est = O.estimate(O.FunctionRenderer(f4, 4), "hvp", g.normal(size=4), 0.3, 40000, "elementwise", 42, 5, v=v4)
    assert np.all(np.abs(est.flat - A @ v4) < 4 * per_pair_stats(est) + 1e-12)
    assert np.all(est.tau[:, 1] != 0)


def test_elementwise_hvp_on_disc_matches_exact():
    sc = wl.disc_scene()
    th = np.asarray(sc["theta_query"])
    _, _, H = disc_closed_form(sc, th, sc["sigma"])
    v = np.array([1.0, -2.0])
    est = O.estimate(O.DiscRenderer(sc), "hvp", th, sc["sigma"], 1 << 14, "elementwise", 43, 0, v=v)
    assert np.all(np.abs(est.flat - H @ v) < 4 * per_pair_stats(est))


def test_finite_difference_hvp_of_gradients():
    f, H = quad_task()
    r = O.FunctionRenderer(f, 2)
    theta = np.array([0.3, -0.4])
    v = np.array([0.8, -0.6])
    for strat in ("aggregate", "elementwise"):
        hv, gp, gm = O.estimate_hvp_fd(r, theta, v, 1e-2, 0.5, 20000, strat, 44, 6)
        assert np.array_equal(gp.tau, gm.tau)                # common random numbers
        # per-pair differences: for a quadratic the difference has no eps bias
        c = 0.5 * (gp.w[0::2] * (gp.losses[0::2] - gm.losses[0::2])[:, None]
                   + gp.w[1::2] * (gp.losses[1::2] - gm.losses[1::2])[:, None]) / 2e-2
        used = (np.abs(gp.w[0::2]) + np.abs(gp.w[1::2])) > 0
        se = np.array([c[used[:, e], e].std(ddof=1) / math.sqrt(used[:, e].sum()) for e in range(2)])
        assert np.all(np.abs(hv - H @ v) < 4 * se + 1e-9), (strat, hv, H @ v, se)
    # disc: FD of the exact smoothed gradient equals H v up to O(eps^2)
    sc = wl.disc_scene()
    th = np.asarray(sc["theta_query"])
    _, _, Hd = disc_closed_form(sc, th, sc["sigma"])
    vd = np.array([0.6, 0.8])
    hv, gp, gm = O.estimate_hvp_fd(O.DiscRenderer(sc), th, vd, 0.01, sc["sigma"], 1 << 14, "aggregate", 45, 0)
    c = 0.5 * (gp.w[0::2] * (gp.losses[0::2] - gm.losses[0::2])[:, None]
               + gp.w[1::2] * (gp.losses[1::2] - gm.losses[1::2])[:, None]) / 0.02
    se = c.std(axis=0, ddof=1) / math.sqrt(c.shape[0])
    assert np.all(np.abs(hv - Hd @ vd) < 4 * se + 0.02 * np.abs(Hd @ vd).max())


# ---------------------------------------------------------------------------
# plain (no importance sampling) estimator and the squares (Box2/Box10) scene
# ---------------------------------------------------------------------------
def test_plain_sampling_is_unbiased_on_quadratic():
    f, H = quad_task()
    r = O.FunctionRenderer(f, 2)
    theta = np.array([0.3, -0.4])
    est = O.estimate(r, "hessian", theta, 0.5, 40000, "plain", seed=51, request=1)
    assert np.array_equal(est.tau[0::2], -est.tau[1::2])
    assert np.all(np.abs(est.flat - upper(H)) < 4 * per_pair_stats(est) + 1e-12)
    g = O.estimate(r, "grad", theta, 0.5, 40000, "plain", seed=52, request=1)
    assert np.all(np.abs(g.flat - H @ theta) < 4 * per_pair_stats(g) + 1e-12)


def test_boxes_renderer_matches_brute_force_and_box2_variance_ordering():
    sc = wl.boxes_scene(n_boxes=5)
    r = O.BoxesRenderer(sc)
    p = np.asarray(sc["theta_query"], np.float32)
    img = r.image(p).reshape(64, 64)
    xs = (np.arange(64) + 0.5) / 64
    X, Y = np.meshgrid(xs, xs)
    ref = np.zeros((64, 64), bool)
    for k in range(5):
        ref |= (np.abs(X - p[2 * k]) < sc["half_size"]) & (np.abs(Y - p[2 * k + 1]) < sc["half_size"])
    assert np.array_equal(img > 0, ref)
    # Sec. "How much variance is reduced?": element-wise IS <= aggregate << plain,
    # per render, on the Box2 task (diagonal entries)
    b2 = wl.boxes_scene(n_boxes=1)
    rb = O.BoxesRenderer(b2)
    th = np.asarray(b2["theta_target"]) + 0.05
    var = {}
    for strat, M in (("elementwise", 4096), ("aggregate", 3 * 4096), ("plain", 3 * 4096)):
        est = O.estimate(rb, "hessian", th, b2["sigma"], M, strat, 61, 1)
        se = per_pair_stats(est)
        renders = len(est.losses)
        var[strat] = (se ** 2 * renders)[[0, 2]]      # variance per render, diagonal entries
    assert np.all(var["elementwise"] < var["aggregate"])
    assert np.all(var["aggregate"] < var["plain"])


# ---------------------------------------------------------------------------
# grey-box composition (Suppl. "Grey-box differentials")
# ---------------------------------------------------------------------------
def test_greybox_affine_inner_map_is_exact_chain_rule():
    """For an affine inner map y = J x + c the composed Hessian J^T H J and
    gradient J^T grad are the exact derivatives of f(g(x)); with a quadratic
    black box they are unbiased (checked per entry within 4 s.e.)."""
    f, A = quad_task()
    g = np.random.default_rng(21)
    J = g.normal(size=(2, 5))
    x = g.normal(size=5)
    y = J @ x + np.array([0.1, -0.2])
    r = O.FunctionRenderer(f, 2)
    Hx, est = O.estimate_greybox(r, "hessian", y, J, 0.4, 40000, "aggregate", 71, 2)
    c = 0.5 * (est.w[0::2] * est.losses[0::2, None] + est.w[1::2] * est.losses[1::2, None])
    full = np.zeros((c.shape[0], 2, 2))
    full[:, 0, 0], full[:, 0, 1], full[:, 1, 1] = c[:, 0], c[:, 1], c[:, 2]
    full[:, 1, 0] = c[:, 1]
    per = np.einsum("ia,kij,jb->kab", J, full, J)
    se = per.std(axis=0, ddof=1) / math.sqrt(per.shape[0])
    assert np.allclose(per.mean(axis=0), Hx)
    assert np.all(np.abs(Hx - J.T @ A @ J) < 4 * se + 1e-12)
    gx, est = O.estimate_greybox(r, "grad", y, J, 0.4, 40000, "aggregate", 72, 2)
    assert np.allclose(gx, J.T @ est.value)
    vx = g.normal(size=5)
    hvx, est = O.estimate_greybox(r, "hvp", y, J, 0.4, 40000, "aggregate", 73, 2, vx=vx)
    assert np.allclose(hvx, J.T @ est.value)
    cv = 0.5 * (est.w[0::2] * est.losses[0::2, None] + est.w[1::2] * est.losses[1::2, None]) @ J
    sev = cv.std(axis=0, ddof=1) / math.sqrt(cv.shape[0])
    assert np.all(np.abs(hvx - J.T @ A @ J @ vx) < 4 * sev + 1e-12)
