"""Analytic scene kinds on the GPU (HR_SCENE_QUADRATIC / STEP1D / NEGGAUSS):
the same perturbations and estimates as the oracle's function renderer on
identical samples, and estimates that agree with the closed-form smoothed
derivatives within their Monte Carlo error (the Quad task's Hessian, the
1D edge's Gaussian-derivative curves, the negated Gaussian)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2412_03489_gb300 import build as hb
from paper_2412_03489_gb300 import hr
from paper_2412_03489_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

hb.build()


def _f(sc):
    k = sc["kind"]
    if k == wl.SCENE_QUADRATIC:
        A, b = np.asarray(sc["A"]), np.asarray(sc["b"])
        return lambda X: 0.5 * np.einsum("mi,ij,mj->m", X, A, X) + X @ b
    if k == wl.SCENE_STEP1D:
        return lambda X: (X[:, 0] > 0).astype(np.float64)
    s2 = sc["gauss_sigma"] ** 2
    n = sc["n_params"]
    return lambda X: -np.exp(-0.5 * np.sum(X * X, axis=1) / s2) / (2 * math.pi * s2) ** (n / 2)


SCENES = {
    "quad_task": lambda: wl.quadratic_scene(),
    "quad_4d": lambda: wl.quadratic_scene(A=np.array([[4.0, 1, 0, 0.5], [1, 3, 0.2, 0], [0, 0.2, 2, 0.1],
                                                      [0.5, 0, 0.1, 1]]), b=np.array([0.3, -0.2, 0.1, 0.0]),
                                          theta=np.array([0.1, -0.4, 0.2, 0.3])),
    "step1d": lambda: wl.step1d_scene(),
    "neggauss": lambda: wl.neggauss_scene(),
}


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("quantity,strategy", [("hessian", "aggregate"), ("hessian", "elementwise"),
                                               ("grad", "aggregate"), ("hvp", "aggregate")])
def test_matches_oracle_on_identical_samples(name, quantity, strategy):
    sc = SCENES[name]()
    S = hr.Scene(sc)
    th = np.asarray(sc["theta_query"], np.float64)
    n = sc["n_params"]
    v = np.linspace(1.0, -0.5, n)
    q = {"hessian": hr.HR_HESSIAN, "grad": hr.HR_GRAD, "hvp": hr.HR_HVP}[quantity]
    st = hr.HR_AGGREGATE if strategy == "aggregate" else hr.HR_ELEMENTWISE
    M = 256
    out, dbg = S.estimate(q, th, sc["sigma"], M, st, 5, 2, v=v if q == hr.HR_HVP else None, debug=True)
    ref = O.estimate(O.FunctionRenderer(_f(sc), n), quantity, th, sc["sigma"], M, strategy, 5, 2,
                     v=v if q == hr.HR_HVP else None)
    assert np.array_equal(dbg["tau"], ref.tau)
    assert np.allclose(dbg["losses"], ref.losses, rtol=2e-7, atol=1e-12)
    flat = out[np.triu_indices(n)] if q == hr.HR_HESSIAN else out
    assert np.all(np.abs(flat - ref.flat) <= 1e-4 * np.maximum(np.abs(ref.flat), ref.scale)), (flat, ref.flat)
    S.close()


def _mean_se(S, sc, q, st, M, reps, v=None):
    th = np.asarray(sc["theta_query"], np.float64)
    xs = np.array([S.estimate(q, th, sc["sigma"], M, st, 100 + r, r, v=v) for r in range(reps)])
    return xs.mean(axis=0), xs.std(axis=0, ddof=1) / math.sqrt(reps)


def test_quad_task_hessian_and_gradient_closed_form():
    sc = wl.quadratic_scene()
    S = hr.Scene(sc)
    A, th = np.asarray(sc["A"]), np.asarray(sc["theta_query"])
    for st in (hr.HR_AGGREGATE, hr.HR_ELEMENTWISE):
        m, se = _mean_se(S, sc, hr.HR_HESSIAN, st, 1 << 16, 8)
        assert np.all(np.abs(m - A) <= 4 * se + 1e-3), (m, se)
    m, se = _mean_se(S, sc, hr.HR_GRAD, hr.HR_AGGREGATE, 1 << 16, 8)
    assert np.all(np.abs(m - A @ th) <= 4 * se + 1e-3)
    S.close()


def test_step_edge_closed_form():
    sc = wl.step1d_scene()
    S = hr.Scene(sc)
    t, s = float(sc["theta_query"][0]), sc["sigma"]
    phi = math.exp(-0.5 * (t / s) ** 2) / math.sqrt(2 * math.pi)
    g_exact, h_exact = phi / s, -(t / s ** 3) * phi
    m, se = _mean_se(S, sc, hr.HR_GRAD, hr.HR_ELEMENTWISE, 1 << 16, 8)
    assert abs(m[0] - g_exact) <= 4 * se[0] + 1e-6 * abs(g_exact)
    m, se = _mean_se(S, sc, hr.HR_HESSIAN, hr.HR_ELEMENTWISE, 1 << 16, 8)
    assert abs(m[0, 0] - h_exact) <= 4 * se[0, 0] + 1e-6 * abs(h_exact)
    S.close()


def test_negated_gaussian_closed_form():
    sc = wl.neggauss_scene()
    S = hr.Scene(sc)
    th = np.asarray(sc["theta_query"])
    V = sc["gauss_sigma"] ** 2 + sc["sigma"] ** 2
    g = -math.exp(-0.5 * th @ th / V) / (2 * math.pi * V)
    H_exact = g * (np.outer(th, th) / V ** 2 - np.eye(2) / V)
    for st in (hr.HR_AGGREGATE, hr.HR_ELEMENTWISE):
        m, se = _mean_se(S, sc, hr.HR_HESSIAN, st, 1 << 16, 8)
        assert np.all(np.abs(m - H_exact) <= 4 * se + 1e-6), (m, H_exact, se)
    S.close()


def test_analytic_scene_validation():
    bad = wl.quadratic_scene()
    bad["width"] = 4
    with pytest.raises(hr.HRError, match="status -1"):
        hr.Scene(bad)
    bad = wl.neggauss_scene(gauss_sigma=1.0)
    bad["gauss_sigma"] = 0.0
    with pytest.raises(hr.HRError, match="status -1"):
        hr.Scene(bad)
