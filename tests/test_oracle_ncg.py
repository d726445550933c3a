"""Pins of the oracle's published optimiser (Sec. 2 Newton Conjugate Gradient
with the point moved every iteration; Suppl. Hyperparameters: linear sigma
annealing, line-search iterations and tolerance, recompute period, trust
region).  Exact derivatives are injected so that each pin compares against
a closed form: linear CG reaches the exact minimiser of an n-dimensional
quadratic in n iterations, steepest descent (recompute every iteration)
zig-zags with orthogonal gradients, a converged Newton-Raphson line search
leaves the gradient orthogonal to the direction, a concave model steps to
the trust bound."""
import math

import numpy as np
import pytest

import oracle as O


def _quad(n, seed, cond=10.0):
    g = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(g.normal(size=(n, n)))
    A = Q @ np.diag(np.geomspace(1.0, cond, n)) @ Q.T
    b = g.normal(size=n)
    return A, b


def _opts(**kw):
    base = dict(sigma_start=0.1, sigma_end=0.1, anneal_iters=1, n_grad=2, n_hvp=2, ls_iters=1, ls_tol=0.0,
                recompute=1000, trust_radius=1e9, residual_mode=0, lambda_rel=0.0)
    base.update(kw)
    return O.NcgOpts(**base)


def _run(o, x0, gf, hf, n_evals):
    st = O.ncg_init(x0, o)
    infos = [O.ncg_evaluate(None, st, o, 0, 0, grad_fn=gf, hvp_fn=hf) for _ in range(n_evals)]
    return st, infos


@pytest.mark.parametrize("mode", [0, 1])
def test_quadratic_is_linear_cg_exact_in_n_iterations(mode):
    n = 6
    A, b = _quad(n, 1)
    gf = lambda x, s, e: A @ x + b
    hf = lambda x, s, e, v: A @ v
    x0 = np.random.default_rng(2).normal(size=n)
    st, infos = _run(_opts(residual_mode=mode), x0, gf, hf, n)
    x_star = np.linalg.solve(A, -b)
    assert np.allclose(st.x, x_star, rtol=1e-8, atol=1e-9)
    # the printed recurrence keeps r equal to -g(x) on a quadratic
    if mode == 0:
        assert np.allclose(st.r, -(A @ st.x + b), atol=1e-9)
    assert [i.it for i in infos] == list(range(n))
    assert infos[0].restarted and not any(i.restarted for i in infos[1:])


def test_line_search_confirms_exact_step_on_quadratic():
    n = 4
    A, b = _quad(n, 3)
    gf = lambda x, s, e: A @ x + b
    hf = lambda x, s, e, v: A @ v
    st, infos = _run(_opts(ls_iters=3, ls_tol=1e-9), np.zeros(n), gf, hf, 2 * n)
    # the second Newton-Raphson step along each direction finds alpha ~ 0 and ends the search
    assert [i.ls_step for i in infos] == [0, 1] * n
    assert all(abs(i.alpha) * np.linalg.norm(b) < 1e-8 for i in infos[1::2])
    assert np.allclose(st.x, np.linalg.solve(A, -b), rtol=1e-8, atol=1e-9)


def test_recompute_every_iteration_is_steepest_descent():
    A = np.diag([1.0, 10.0])
    b = np.zeros(2)
    gf = lambda x, s, e: A @ x + b
    hf = lambda x, s, e, v: A @ v
    x0 = np.array([10.0, 1.0])
    st, infos = _run(_opts(recompute=1), x0, gf, hf, 6)
    assert all(i.restarted for i in infos)
    # exact line search along -g: successive gradients are orthogonal
    xs = [x0]
    st2 = O.ncg_init(x0, _opts(recompute=1))
    for _ in range(5):
        O.ncg_evaluate(None, st2, _opts(recompute=1), 0, 0, grad_fn=gf, hvp_fn=hf)
        xs.append(st2.x.copy())
    gs = [A @ x for x in xs]
    for g0, g1 in zip(gs, gs[1:]):
        assert abs(g0 @ g1) <= 1e-10 * np.linalg.norm(g0) * np.linalg.norm(g1)
    # and it has not converged (kappa = 10), while conjugate directions reach 0 in two
    assert np.linalg.norm(st.x) > 1e-2
    st_cg, _ = _run(_opts(recompute=2), x0, gf, hf, 2)
    assert np.linalg.norm(st_cg.x) < 1e-10


@pytest.mark.parametrize("x0", [1.0, -1.0])
def test_concave_model_steps_to_trust_bound_downhill(x0):
    gf = lambda x, s, e: -x
    hf = lambda x, s, e, v: -v
    st, infos = _run(_opts(trust_radius=0.3), np.array([x0]), gf, hf, 1)
    assert st.x[0] == x0 + math.copysign(0.3, x0)
    assert infos[0].dHd < 0 and infos[0].step_norm == pytest.approx(0.3, rel=1e-15)


def test_trust_region_truncates_step():
    A = np.diag([1.0, 2.0])
    gf = lambda x, s, e: A @ x
    hf = lambda x, s, e, v: A @ v
    x0 = np.array([3.0, -4.0])
    st, infos = _run(_opts(trust_radius=0.25), x0, gf, hf, 1)
    assert np.linalg.norm(st.x - x0) == pytest.approx(0.25, rel=1e-14)
    assert np.allclose((st.x - x0) / 0.25, -(A @ x0) / np.linalg.norm(A @ x0))


def test_sigma_schedule_and_what_the_estimators_see():
    seen = []

    def gf(x, s, e):
        seen.append(s)
        return x

    hf = lambda x, s, e, v: v
    o = _opts(sigma_start=1.0, sigma_end=0.2, anneal_iters=5, ls_iters=2, ls_tol=-1.0)
    _run(o, np.array([1.0]), gf, hf, 12)
    # two line-search steps per outer iteration; sigma moves per outer iteration
    expect = [1.0, 0.8, 0.6, 0.4, 0.2, 0.2]
    assert seen == pytest.approx([s for s in expect for _ in range(2)], rel=1e-15, abs=1e-15)
    assert O.anneal_sigma(1.0, 0.2, 5, 0) == 1.0 and O.anneal_sigma(1.0, 0.2, 5, 4) == 0.2
    assert O.anneal_sigma(0.3, 0.1, 1, 7) == 0.3


def _convex_nonquadratic(n, seed):
    g = np.random.default_rng(seed)
    Wm = g.normal(size=(2 * n, n)) / math.sqrt(n)
    c = g.normal(size=2 * n)
    # f(x) = sum log cosh(W x - c) + 1/2 |x|^2 / 10
    grad = lambda x: Wm.T @ np.tanh(Wm @ x - c) + 0.1 * x
    hvp = lambda x, v: Wm.T @ ((1.0 - np.tanh(Wm @ x - c) ** 2) * (Wm @ v)) + 0.1 * v
    return grad, hvp


def test_converged_line_search_is_exact_on_nonquadratic():
    n = 5
    grad, hvp = _convex_nonquadratic(n, 4)
    o = _opts(ls_iters=40, ls_tol=1e-13, residual_mode=1, trust_radius=10.0)
    st = O.ncg_init(np.full(n, 2.0), o)
    ends = 0
    while ends < 4:
        info = O.ncg_evaluate(None, st, o, 0, 0, grad_fn=lambda x, s, e: grad(x), hvp_fn=lambda x, s, e, v: hvp(x, v))
        if st.j == 0:
            ends += 1
            g = grad(st.x)
            assert abs(g @ st.d) <= 1e-9 * np.linalg.norm(g) * np.linalg.norm(st.d) + 1e-14


def test_nonlinear_cg_reaches_stationary_point():
    n = 5
    grad, hvp = _convex_nonquadratic(n, 5)
    o = _opts(ls_iters=20, ls_tol=1e-12, residual_mode=1, recompute=n, trust_radius=10.0)
    st, _ = _run(o, np.full(n, -1.5), lambda x, s, e: grad(x), lambda x, s, e, v: hvp(x, v), 200)
    assert np.linalg.norm(grad(st.x)) < 1e-8


def test_stochastic_run_on_disc_scene_approaches_target():
    from paper_2412_03489_gb300 import workloads as wl
    sc = wl.disc_scene()
    r = O.DiscRenderer(sc)
    o = _opts(sigma_start=0.05, sigma_end=0.01, anneal_iters=12, n_grad=256, n_hvp=256, ls_iters=2, ls_tol=1e-3,
              recompute=4, trust_radius=0.05)
    st = O.ncg_init(sc["theta_query"], o)
    err0 = np.linalg.norm(st.x - sc["theta_target"])
    for _ in range(24):
        O.ncg_evaluate(r, st, o, 11, 3)
    assert np.linalg.norm(st.x - sc["theta_target"]) < 0.3 * err0
