"""Pins of the oracle's Newton-CG step (Sec. 2 "Newton Conjugate Gradient",
trust-region step cap alpha = min(alpha, Delta / |p|), negative-curvature exit)
with exact derivative oracles injected, and end-to-end on the negated
Gaussian, whose minimum (0, 0) the paper reports reaching from any start in
(-3, 3)^2 (Suppl. "Positive-Definite Hessians")."""
import math

import numpy as np

import oracle as O


def _exact(A, b):
    return (lambda th: A @ th + b), (lambda th, i, v: A @ v)


def test_cg_solves_regularised_newton_system_exactly():
    g = np.random.default_rng(3)
    Bm = g.normal(size=(5, 5))
    A = Bm @ Bm.T + 5 * np.eye(5)
    b = g.normal(size=5)
    th = g.normal(size=5)
    gf, hf = _exact(A, b)
    lam_rel = 1e-3
    new, info = O.newton_cg_step(None, th, 0.1, 0, 0, 10, lam_rel, 1e9, 0, 0, 0, grad_fn=gf, hvp_fn=hf)
    grad = A @ th + b
    lam = lam_rel * np.linalg.norm(grad)
    d = np.linalg.solve(A + lam * np.eye(5), -grad)
    assert np.allclose(new - th, d, rtol=1e-9, atol=1e-12)
    assert info.lam == lam and info.exit in ("max_iters", "converged")


def test_trust_region_caps_each_step_length():
    A = np.diag([1.0, 100.0])
    gf, hf = _exact(A, np.zeros(2))
    th = np.array([10.0, 1.0])
    delta = 0.5
    new, info = O.newton_cg_step(None, th, 0.1, 0, 0, 1, 0.0, delta, 0, 0, 0, grad_fn=gf, hvp_fn=hf)
    assert np.linalg.norm(new - th) <= delta + 1e-12
    # first step is along -g
    gdir = -(A @ th) / np.linalg.norm(A @ th)
    assert np.allclose((new - th) / np.linalg.norm(new - th), gdir)


def test_negative_curvature_exit_moves_along_steepest_descent():
    A = np.diag([-2.0, -1.0])
    gf, hf = _exact(A, np.zeros(2))
    th = np.array([1.0, 0.5])
    new, info = O.newton_cg_step(None, th, 0.1, 0, 0, 5, 0.0, 0.3, 0, 0, 0, grad_fn=gf, hvp_fn=hf)
    assert info.exit == "neg_curvature"
    step = new - th
    assert math.isclose(np.linalg.norm(step), 0.3, rel_tol=1e-12)
    assert step @ (A @ th) < 0


def test_negated_gaussian_newton_cg_finds_minimum():
    s1, s2 = 1.0, 0.5
    f = lambda X: -np.exp(-0.5 * np.sum(X * X, axis=1) / s1 ** 2) / (2 * math.pi * s1 * s1)
    r = O.FunctionRenderer(f, 2)
    for k, start in enumerate([(2.5, -2.0), (-1.0, 2.8), (0.5, 0.5)]):
        th = np.array(start, float)
        tail = []
        for step in range(40):
            th, info = O.newton_cg_step(r, th, s2, 8192, 4096, 4, 1e-3, 0.5, 77, k, step)
            if step >= 30:
                tail.append(th)
        # the iterates settle at the minimum up to the estimator noise
        assert np.linalg.norm(np.mean(tail, axis=0)) < 0.05, (start, tail[-1])
