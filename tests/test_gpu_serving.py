"""Serving with continuous batching (hr_server_*): every result is the same
alone, in a mix of concurrent requests, and through the plain entry points;
Newton-CG steps through the server match direct steps; budget, validation,
timeouts and shutdown behave as documented."""
import numpy as np
import pytest

from paper_2412_03489_gb300 import build as hb
from paper_2412_03489_gb300 import hr
from paper_2412_03489_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

hb.build()


def scenes():
    return {
        "disc": hr.Scene(wl.disc_scene()),
        "revolve": hr.Scene(wl.revolve_scene(width=96, height=80)),
        "tris": hr.Scene(wl.tris2d_scene(width=64, height=48)),
        "pt": hr.Scene(wl.ptbox_scene(width=24, height=20, spp=2, target_spp=4)),
    }


def request_list(S):
    g = np.random.default_rng(7)
    out = []
    specs = [("disc", hr.HR_HESSIAN, hr.HR_AGGREGATE, 1024), ("disc", hr.HR_GRAD, hr.HR_ELEMENTWISE, 256),
             ("revolve", hr.HR_HESSIAN, hr.HR_AGGREGATE, 600), ("revolve", hr.HR_HESSIAN, hr.HR_ELEMENTWISE, 128),
             ("tris", hr.HR_HVP, hr.HR_AGGREGATE, 64), ("tris", hr.HR_GRAD, hr.HR_AGGREGATE, 96),
             ("pt", hr.HR_HVP, hr.HR_AGGREGATE, 16), ("disc", hr.HR_HVP, hr.HR_AGGREGATE, 5000)]
    for i in range(16):
        name, q, strat, M = specs[i % len(specs)]
        sc = S[name]
        theta = np.asarray(sc.sc["theta_query"], np.float64) + g.normal(0, 0.01, sc.n)
        v = g.normal(size=sc.n) if q == hr.HR_HVP else None
        out.append(dict(scene=sc, q=q, strat=strat, M=M, theta=theta, v=v, seed=100 + i, req=i))
    return out


def submit(srv, spec):
    o = hr.make_opts(spec["scene"].sc["sigma"], spec["M"], spec["strat"], spec["seed"], spec["req"])
    r, keep = hr.make_request(spec["scene"], spec["q"], spec["theta"], spec["v"], o)
    return hr.hr_server_submit(srv, r), keep


def result_shape(spec):
    n = spec["scene"].n
    return (n, n) if spec["q"] == hr.HR_HESSIAN else (n,)


def test_results_identical_alone_in_mix_and_plain():
    S = scenes()
    reqs = request_list(S)
    srv = hr.hr_server_create(64 << 20, max_active=4, chunk=256)
    alone = []
    for spec in reqs:
        t, keep = submit(srv, spec)
        out = np.zeros(result_shape(spec))
        info = hr.hr_request_info()
        hr.hr_server_wait(srv, t, out, info)
        alone.append(out)
    # all at once: more requests than slots, several scenes, chunks interleaved
    tickets = [submit(srv, spec) for spec in reqs]
    mixed, batches = [], []
    for (t, keep), spec in zip(tickets, reqs):
        out = np.zeros(result_shape(spec))
        info = hr.hr_request_info()
        hr.hr_server_wait(srv, t, out, info)
        mixed.append(out)
        batches.append(info.batches)
    hr.hr_server_destroy(srv)
    for a, b in zip(alone, mixed):
        assert np.array_equal(a, b)
    assert max(batches) > 1                       # chunked across several launches
    for spec, a in zip(reqs, alone):
        plain = spec["scene"].estimate(spec["q"], spec["theta"], spec["scene"].sc["sigma"], spec["M"], spec["strat"],
                                       spec["seed"], spec["req"], v=spec["v"])
        assert np.array_equal(a, plain)
    for sc in S.values():
        sc.close()


def test_newton_step_through_server_matches_direct_step():
    sc = wl.tris2d_scene(width=48, height=40, n_instances=2)
    Sd, Ss = hr.Scene(sc), hr.Scene(sc)
    opts = hr.hr_cg_opts()
    opts.sigma, opts.n_grad, opts.n_hvp, opts.cg_iters = sc["sigma"], 16, 8, 3
    opts.lambda_rel, opts.trust_radius, opts.seed, opts.request_base, opts.use_graph = 1e-3, 0.05, 5, 0, 1
    th0 = np.ascontiguousarray(sc["theta_init"][:2], np.float64)
    st_direct = hr.hr_optstate_create(Sd.handle, 2, th0, opts)
    st_served = hr.hr_optstate_create(Ss.handle, 2, th0, opts)
    srv = hr.hr_server_create(16 << 20, max_active=2)
    for _ in range(2):
        info_d = (hr.hr_step_info * 2)()
        hr.hr_newton_cg_step(Sd.handle, st_direct, info_d)
        r, keep = hr.make_request(Ss, hr.HR_NEWTON_STEP, optstate=st_served)
        t = hr.hr_server_submit(srv, r)
        info_s = (hr.hr_step_info * 2)()
        hr.hr_server_wait(srv, t, info_s, hr.hr_request_info())
        for b in range(2):
            assert info_s[b].iters == info_d[b].iters
            assert info_s[b].step_norm == info_d[b].step_norm
    a, b = np.zeros((2, sc["n_params"])), np.zeros((2, sc["n_params"]))
    hr.hr_optstate_theta(st_direct, a)
    hr.hr_optstate_theta(st_served, b)
    assert np.array_equal(a, b)
    hr.hr_server_destroy(srv)
    hr.hr_optstate_destroy(st_direct)
    hr.hr_optstate_destroy(st_served)


def test_overlapping_steps_on_one_state_run_in_order():
    """Two step requests on the same state submitted back to back: the second
    waits for the first, and each returns its own step record."""
    sc = wl.tris2d_scene(width=48, height=40, n_instances=2)
    Sd, Ss = hr.Scene(sc), hr.Scene(sc)
    opts = hr.hr_cg_opts()
    opts.sigma, opts.n_grad, opts.n_hvp, opts.cg_iters = sc["sigma"], 16, 8, 3
    opts.lambda_rel, opts.trust_radius, opts.seed, opts.request_base, opts.use_graph = 1e-3, 0.05, 9, 0, 1
    th0 = np.ascontiguousarray(sc["theta_init"][:2], np.float64)
    st_direct = hr.hr_optstate_create(Sd.handle, 2, th0, opts)
    st_served = hr.hr_optstate_create(Ss.handle, 2, th0, opts)
    direct = []
    for _ in range(3):
        info = (hr.hr_step_info * 2)()
        hr.hr_newton_cg_step(Sd.handle, st_direct, info)
        direct.append([(info[b].iters, info[b].step_norm, info[b].grad_norm) for b in range(2)])
    srv = hr.hr_server_create(16 << 20, max_active=4)
    tickets = []
    for _ in range(3):
        r, keep = hr.make_request(Ss, hr.HR_NEWTON_STEP, optstate=st_served)
        tickets.append((hr.hr_server_submit(srv, r), keep))
    for (t, keep), ref in zip(tickets, direct):
        info = (hr.hr_step_info * 2)()
        hr.hr_server_wait(srv, t, info, hr.hr_request_info())
        assert [(info[b].iters, info[b].step_norm, info[b].grad_norm) for b in range(2)] == ref
    a, b = np.zeros((2, sc["n_params"])), np.zeros((2, sc["n_params"]))
    hr.hr_optstate_theta(st_direct, a)
    hr.hr_optstate_theta(st_served, b)
    assert np.array_equal(a, b)
    hr.hr_server_destroy(srv)
    hr.hr_optstate_destroy(st_direct)
    hr.hr_optstate_destroy(st_served)


def test_budget_validation_timeout_and_shutdown():
    Sd = hr.Scene(wl.disc_scene())
    th = np.asarray(Sd.sc["theta_query"])
    srv = hr.hr_server_create(1 << 20, max_active=1, chunk=64)
    # larger than the whole budget: rejected at submission
    o = hr.make_opts(0.05, 1 << 16, hr.HR_AGGREGATE, 1, 1)
    r, keep = hr.make_request(Sd, hr.HR_HESSIAN, th, None, o)
    with pytest.raises(hr.HRError, match="status -2"):
        hr.hr_server_submit(srv, r)
    # malformed
    o = hr.make_opts(0.05, 3, hr.HR_AGGREGATE, 1, 1)
    r, keep = hr.make_request(Sd, hr.HR_HESSIAN, th, None, o)
    with pytest.raises(hr.HRError, match="status -1"):
        hr.hr_server_submit(srv, r)
    # a queue behind one slot; a zero timeout on the last one times out, then it completes
    o = hr.make_opts(0.05, 8192, hr.HR_AGGREGATE, 1, 1)
    tickets = []
    for i in range(4):
        r, keep = hr.make_request(Sd, hr.HR_HESSIAN, th, None, o)
        tickets.append((hr.hr_server_submit(srv, r), keep))
    out = np.zeros((2, 2))
    with pytest.raises(hr.HRError, match="status -4"):
        hr.hr_server_wait(srv, tickets[-1][0], out, hr.hr_request_info(), timeout_ms=0)
    results = []
    for t, keep in tickets:
        info = hr.hr_request_info()
        hr.hr_server_wait(srv, t, out, info)
        results.append(out.copy())
        assert info.admit_ms >= info.submit_ms and info.done_ms >= info.admit_ms
    assert all(np.array_equal(results[0], x) for x in results)
    # shutdown with queued work returns without hanging
    for i in range(3):
        r, keep = hr.make_request(Sd, hr.HR_HESSIAN, th, None, o)
        hr.hr_server_submit(srv, r)
    hr.hr_server_destroy(srv)
    Sd.close()
