"""Persistent queue (hr_queue_*): one long-running kernel samples, renders and
sums disc requests.  Every result is bit-identical to hr_estimate_* with the
same options, alone and in a mix, through arena wrap-around and from several
host threads; the idle budget ends the kernel with HR_ERR_TIMEOUT in its status
word and the next request launches it again; full rings answer HR_ERR_BUSY."""
import ctypes
import threading
import time

import numpy as np
import pytest

import oracle as O
from paper_2412_03489_gb300 import build as hb
from paper_2412_03489_gb300 import hr
from paper_2412_03489_gb300 import workloads as wl
from parity import assert_estimate_close, flat_of

pytestmark = pytest.mark.gpu

hb.build()

QN = {hr.HR_GRAD: "grad", hr.HR_HESSIAN: "hessian", hr.HR_HVP: "hvp"}
SN = {hr.HR_ELEMENTWISE: "elementwise", hr.HR_AGGREGATE: "aggregate", hr.HR_PLAIN: "plain"}

# (quantity, strategy, M): every quantity and strategy; M = 34 and 30 leave a
# ragged last unit (17 and 15 pairs per group), M = 2 a single pair
KINDS = [(hr.HR_HESSIAN, hr.HR_ELEMENTWISE, 1024), (hr.HR_HESSIAN, hr.HR_AGGREGATE, 1024),
         (hr.HR_HESSIAN, hr.HR_PLAIN, 512), (hr.HR_GRAD, hr.HR_ELEMENTWISE, 256),
         (hr.HR_GRAD, hr.HR_AGGREGATE, 4096), (hr.HR_GRAD, hr.HR_PLAIN, 34),
         (hr.HR_HVP, hr.HR_ELEMENTWISE, 30), (hr.HR_HVP, hr.HR_AGGREGATE, 2048),
         (hr.HR_HVP, hr.HR_PLAIN, 2), (hr.HR_HESSIAN, hr.HR_ELEMENTWISE, 34)]


def requests(sc, count, seed=5):
    g = np.random.default_rng(seed)
    out = []
    for i in range(count):
        q, strat, M = KINDS[i % len(KINDS)]
        theta = np.asarray(sc["theta_query"], np.float64) + g.normal(0, 0.02, 2)
        v = g.normal(size=2) if q == hr.HR_HVP else None
        out.append(dict(q=q, strat=strat, M=M, theta=theta, v=v, seed=40 + i, req=1000 + i, sub=i % 3))
    return out


def opts(sc, r):
    return hr.make_opts(sc["sigma"], r["M"], r["strat"], r["seed"], r["req"], sub=r["sub"])


def plain(S, sc, r):
    return S.estimate(r["q"], r["theta"], sc["sigma"], r["M"], r["strat"], r["seed"], r["req"], r["sub"], v=r["v"])


def out_for(r):
    return np.zeros((2, 2) if r["q"] == hr.HR_HESSIAN else 2)


def submit_retry(q, sc, r, pending, results):
    """Submit; on HR_ERR_BUSY wait for the oldest pending ticket and retry."""
    while True:
        try:
            return hr.hr_queue_submit(q, r["q"], r["theta"], r["v"], opts(sc, r))
        except hr.HRError as e:
            assert e.status == hr.HR_ERR_BUSY, e
            t, i = pending.pop(0)
            hr.hr_queue_wait(q, t, results[i])


def test_queue_bit_identical_alone_and_in_mix():
    sc = wl.disc_scene()
    S = hr.Scene(sc)
    reqs = requests(sc, 30)
    ref = [plain(S, sc, r) for r in reqs]
    q = hr.hr_queue_create(S, max_requests=64, idle_budget_us=5000)
    try:
        # alone: one request in the queue at a time
        for r, e in zip(reqs[:10], ref[:10]):
            out = out_for(r)
            hr.hr_queue_wait(q, hr.hr_queue_submit(q, r["q"], r["theta"], r["v"], opts(sc, r)), out)
            assert np.array_equal(out, e), (r, out, e)
        # in the mix: all submitted before any is waited for
        tickets = [hr.hr_queue_submit(q, r["q"], r["theta"], r["v"], opts(sc, r)) for r in reqs]
        outs = [out_for(r) for r in reqs]
        for t, o in reversed(list(zip(tickets, outs))):
            hr.hr_queue_wait(q, t, o)
        for r, o, e in zip(reqs, outs, ref):
            assert np.array_equal(o, e), (r, o, e)
    finally:
        hr.hr_queue_destroy(q)
        S.close()


def test_queue_matches_oracle():
    """The queued element-wise Hessian of the disc against the FP64 oracle on
    the same samples (1e-4 of the estimator's magnitude, as the plain path)."""
    sc = wl.disc_scene()
    S = hr.Scene(sc)
    q = hr.hr_queue_create(S)
    try:
        for quantity, strat, M in [(hr.HR_HESSIAN, hr.HR_ELEMENTWISE, 1024), (hr.HR_HVP, hr.HR_AGGREGATE, 1024)]:
            theta = np.asarray(sc["theta_query"], np.float64)
            v = np.array([0.6, -0.8]) if quantity == hr.HR_HVP else None
            out = np.zeros((2, 2) if quantity == hr.HR_HESSIAN else 2)
            t = hr.hr_queue_submit(q, quantity, theta, v, hr.make_opts(sc["sigma"], M, strat, 11, 3))
            hr.hr_queue_wait(q, t, out)
            ref = O.estimate(O.DiscRenderer(sc), QN[quantity], theta, sc["sigma"], M, SN[strat], 11, 3, 0, v=v)
            assert_estimate_close(flat_of(QN[quantity], out, 2), ref, what=f"queue {QN[quantity]}")
    finally:
        hr.hr_queue_destroy(q)
        S.close()


def test_queue_idle_budget_runs_out_and_relaunches():
    sc = wl.disc_scene()
    S = hr.Scene(sc)
    r = requests(sc, 1)[0]
    e = plain(S, sc, r)
    q = hr.hr_queue_create(S, max_requests=8, idle_budget_us=200)
    try:
        status, launches = hr.hr_queue_status(q)
        assert launches == 0
        for k in range(3):
            out = out_for(r)
            hr.hr_queue_wait(q, hr.hr_queue_submit(q, r["q"], r["theta"], r["v"], opts(sc, r)), out)
            assert np.array_equal(out, e)
            # nothing more arrives: the dispatcher's budget runs out and the
            # kernel reports HR_ERR_TIMEOUT through its status word
            t0 = time.time()
            while True:
                status, launches = hr.hr_queue_status(q)
                if status != 1 or time.time() - t0 > 5.0:
                    break
                time.sleep(0.001)
            assert status == hr.HR_ERR_TIMEOUT, status
            assert launches == k + 1
    finally:
        hr.hr_queue_destroy(q)
        S.close()


def test_queue_ring_full_is_busy_and_arena_wraps():
    sc = wl.disc_scene()
    S = hr.Scene(sc)
    reqs = requests(sc, 60, seed=9)
    ref = [plain(S, sc, r) for r in reqs]
    # 1 MiB holds about a dozen 3 x 1024 Hessians (72 KiB each): the arena wraps
    q = hr.hr_queue_create(S, max_requests=8, idle_budget_us=5000, arena_bytes=1 << 20)
    try:
        first = [hr.hr_queue_submit(q, r["q"], r["theta"], r["v"], opts(sc, r)) for r in reqs[:8]]
        with pytest.raises(hr.HRError) as ei:
            hr.hr_queue_submit(q, reqs[8]["q"], reqs[8]["theta"], reqs[8]["v"], opts(sc, reqs[8]))
        assert ei.value.status == hr.HR_ERR_BUSY
        results = [out_for(r) for r in reqs]
        pending = list(zip(first, range(8)))
        for i in range(8, len(reqs)):
            pending.append((submit_retry(q, sc, reqs[i], pending, results), i))
        for t, i in pending:
            hr.hr_queue_wait(q, t, results[i])
        for r, o, e in zip(reqs, results, ref):
            assert np.array_equal(o, e), (r, o, e)
        with pytest.raises(hr.HRError) as ei:
            hr.hr_queue_wait(q, first[0], results[0])
        assert ei.value.status == hr.HR_ERR_INVALID_ARG
    finally:
        hr.hr_queue_destroy(q)
        S.close()


def test_queue_from_several_threads():
    sc = wl.disc_scene()
    S = hr.Scene(sc)
    reqs = requests(sc, 48, seed=13)
    ref = [plain(S, sc, r) for r in reqs]
    q = hr.hr_queue_create(S, max_requests=256, idle_budget_us=5000)
    outs = [out_for(r) for r in reqs]
    errors = []

    def worker(ids):
        try:
            for i in ids:
                r = reqs[i]
                t = hr.hr_queue_submit(q, r["q"], r["theta"], r["v"], opts(sc, r))
                hr.hr_queue_wait(q, t, outs[i])
        except Exception as ex:   # reported below
            errors.append(ex)

    th = [threading.Thread(target=worker, args=(list(range(k, len(reqs), 4)),)) for k in range(4)]
    try:
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors, errors
        for r, o, e in zip(reqs, outs, ref):
            assert np.array_equal(o, e), (r, o, e)
    finally:
        hr.hr_queue_destroy(q)
        S.close()


def test_queue_validation_and_destroy_with_pending_work():
    sc = wl.disc_scene()
    S = hr.Scene(sc)
    with pytest.raises(hr.HRError) as ei:
        hr.hr_queue_create(S, max_requests=0)
    assert ei.value.status == hr.HR_ERR_INVALID_ARG
    with pytest.raises(hr.HRError) as ei:
        hr.hr_queue_create(S, idle_budget_us=0)
    assert ei.value.status == hr.HR_ERR_INVALID_ARG
    R = hr.Scene(wl.revolve_scene(width=32, height=32))
    with pytest.raises(hr.HRError) as ei:
        hr.hr_queue_create(R)
    assert ei.value.status == hr.HR_ERR_UNSUPPORTED
    R.close()
    q = hr.hr_queue_create(S)
    theta = np.asarray(sc["theta_query"], np.float64)
    with pytest.raises(hr.HRError) as ei:
        hr.hr_queue_submit(q, hr.HR_HESSIAN, theta, None, hr.make_opts(sc["sigma"], 33, hr.HR_AGGREGATE, 1, 1))
    assert ei.value.status == hr.HR_ERR_INVALID_ARG
    with pytest.raises(hr.HRError) as ei:
        hr.hr_queue_submit(q, hr.HR_HVP, theta, None, hr.make_opts(sc["sigma"], 32, hr.HR_AGGREGATE, 1, 1))
    assert ei.value.status == hr.HR_ERR_INVALID_ARG
    with pytest.raises(hr.HRError) as ei:
        hr.hr_queue_wait(q, 5, np.zeros(2))
    assert ei.value.status == hr.HR_ERR_INVALID_ARG
    # pending requests are finished by the kernel before destroy returns
    for i in range(6):
        hr.hr_queue_submit(q, hr.HR_HESSIAN, theta, None, hr.make_opts(sc["sigma"], 1024, hr.HR_ELEMENTWISE, i, i))
    hr.hr_queue_destroy(q)
    # the scene still renders through the plain path afterwards
    out = S.estimate(hr.HR_HESSIAN, theta, sc["sigma"], 64, hr.HR_AGGREGATE, 1, 1)
    assert np.all(np.isfinite(out))
    S.close()


def test_queue_batches():
    """hr_queue_submit_many / hr_queue_wait_many: every result bit-identical to
    the plain path; a batch larger than the ring queues what fits (HR_ERR_BUSY
    for the rest) and the remainder goes in after the first results are read."""
    sc = wl.disc_scene()
    S = hr.Scene(sc)
    g = np.random.default_rng(21)
    count = 300
    thetas = np.asarray(sc["theta_query"], np.float64) + g.normal(0, 0.02, (count, 2))
    seeds, reqs = np.arange(count) + 500, np.arange(count) * 3 + 1
    for quantity, strat, M in [(hr.HR_HESSIAN, hr.HR_ELEMENTWISE, 1024), (hr.HR_HVP, hr.HR_AGGREGATE, 66)]:
        vs = g.normal(size=(count, 2)) if quantity == hr.HR_HVP else None
        arr = hr.opts_array(sc["sigma"], M, strat, seeds, reqs)
        ref = [S.estimate(quantity, thetas[i], sc["sigma"], M, strat, int(seeds[i]), int(reqs[i]),
                          v=None if vs is None else vs[i]) for i in range(count)]
        q = hr.hr_queue_create(S, max_requests=128, idle_budget_us=5000)
        try:
            out = np.zeros((count, 4))
            done = 0
            while done < count:
                sub = (hr.hr_opts * (count - done)).from_buffer(arr, done * ctypes.sizeof(hr.hr_opts))
                t = hr.hr_queue_submit_many(q, quantity, thetas[done:], None if vs is None else vs[done:], sub)
                assert len(t) > 0
                if done == 0:
                    assert len(t) == 128          # the ring's slots
                hr.hr_queue_wait_many(q, t, out[done:done + len(t)])
                done += len(t)
            for i in range(count):
                e = np.asarray(ref[i]).ravel()
                assert np.array_equal(out[i, :e.size], e), (i, out[i], e)
        finally:
            hr.hr_queue_destroy(q)
    S.close()


def test_queue_exits_and_relaunches_under_bursts():
    """A 50 us idle budget with bursts of requests separated by pauses: the
    kernel leaves and is launched again many times, with requests arriving
    around its exits.  Every request completes (a unit lost at an exit would
    leave its request waiting) and matches the plain path bit for bit."""
    sc = wl.disc_scene()
    S = hr.Scene(sc)
    reqs = requests(sc, 60, seed=17)
    ref = [plain(S, sc, r) for r in reqs]
    q = hr.hr_queue_create(S, max_requests=128, idle_budget_us=50)
    outs = [out_for(r) for r in reqs]
    try:
        tickets = []
        for b in range(0, len(reqs), 3):
            for r in reqs[b:b + 3]:
                tickets.append(hr.hr_queue_submit(q, r["q"], r["theta"], r["v"], opts(sc, r)))
            time.sleep(0.0002 * (b % 4))
        for t, o in zip(tickets, outs):
            hr.hr_queue_wait(q, t, o, timeout_ms=20000)
        for r, o, e in zip(reqs, outs, ref):
            assert np.array_equal(o, e), (r, o, e)
        status, launches = hr.hr_queue_status(q)
        assert launches >= 2
    finally:
        hr.hr_queue_destroy(q)
        S.close()


@pytest.mark.parametrize("W,H,grey", [(64, 64, True), (37, 23, False), (96, 10, True), (512, 3, False)])
def test_queue_other_sizes_and_grey_targets(W, H, grey):
    """The queue's renders take the same loss paths as the plain kernel: row
    spans for 0/1 targets, the per-pixel loops for grey ones (fixed columns
    per lane at W = 64, the general loop at W = 96), ragged and wide images."""
    sc = wl.disc_scene(width=W, height=H)
    tgt = np.random.default_rng(W + H).uniform(0.0, 1.0, size=W * H).astype(np.float32) if grey else None
    S = hr.Scene(sc, target_image=tgt) if grey else hr.Scene(sc)
    reqs = requests(sc, 10, seed=W * H)
    ref = [plain(S, sc, r) for r in reqs]
    q = hr.hr_queue_create(S, max_requests=16, idle_budget_us=2000)
    try:
        tickets = [hr.hr_queue_submit(q, r["q"], r["theta"], r["v"], opts(sc, r)) for r in reqs]
        outs = [out_for(r) for r in reqs]
        for t, o in zip(tickets, outs):
            hr.hr_queue_wait(q, t, o)
        for r, o, e in zip(reqs, outs, ref):
            assert np.array_equal(o, e), (r, o, e)
    finally:
        hr.hr_queue_destroy(q)
        S.close()


@pytest.mark.parametrize("n_boxes", [1, 4])
def test_queue_squares_scenes(n_boxes):
    """Squares scenes (Box2 with one square; four squares, n = 8) through the
    queue: each request bit-identical to the plain path (the same render
    code); ten squares (n = 20) are beyond the queue's parameter limit."""
    sc = wl.boxes_scene(n_boxes=n_boxes)
    S = hr.Scene(sc)
    n = sc["n_params"]
    g = np.random.default_rng(n_boxes)
    kinds = [(hr.HR_HESSIAN, hr.HR_AGGREGATE, 512), (hr.HR_GRAD, hr.HR_AGGREGATE, 66),
             (hr.HR_HVP, hr.HR_AGGREGATE, 258), (hr.HR_HESSIAN, hr.HR_PLAIN, 34)]
    if n_boxes == 1:   # element-wise: n or n(n+1)/2 sample groups, at most 4 in the queue
        kinds += [(hr.HR_HESSIAN, hr.HR_ELEMENTWISE, 256), (hr.HR_GRAD, hr.HR_ELEMENTWISE, 66)]
    reqs = []
    for i, (quantity, strat, M) in enumerate(kinds * 2):
        theta = np.asarray(sc["theta_query"], np.float64) + g.normal(0, 0.02, n)
        v = g.normal(size=n) if quantity == hr.HR_HVP else None
        reqs.append(dict(q=quantity, strat=strat, M=M, theta=theta, v=v, seed=70 + i, req=i, sub=0))
    ref = [plain(S, sc, r) for r in reqs]
    q = hr.hr_queue_create(S, max_requests=32, idle_budget_us=2000)
    try:
        tickets = [hr.hr_queue_submit(q, r["q"], r["theta"], r["v"], opts(sc, r)) for r in reqs]
        for r, t, e in zip(reqs, tickets, ref):
            o = np.zeros((n, n) if r["q"] == hr.HR_HESSIAN else n)
            hr.hr_queue_wait(q, t, o)
            assert np.array_equal(o, e), (r, o, e)
    finally:
        hr.hr_queue_destroy(q)
        S.close()
    S10 = hr.Scene(wl.boxes_scene(n_boxes=10))
    with pytest.raises(hr.HRError) as ei:
        hr.hr_queue_create(S10)
    assert ei.value.status == hr.HR_ERR_UNSUPPORTED
    S10.close()


def test_queue_unit_ring_fills_and_wraps():
    """Requests of 3 x 2^18 perturbations (24,576 units of 16 pairs each):
    about 43 of them fill the 2^20-entry unit ring, so a submit is refused
    with HR_ERR_BUSY ("unit ring full") before the slots or the 1 GiB arena
    run out; after the first results are read, more requests go in and the
    ring's indices wrap.  Sampled results against the plain path."""
    sc = wl.disc_scene()
    S = hr.Scene(sc)
    theta = np.asarray(sc["theta_query"], np.float64)
    M = 1 << 18
    q = hr.hr_queue_create(S, max_requests=64, idle_budget_us=20000, arena_bytes=1 << 30)
    try:
        tickets, busy = [], None
        for i in range(64):
            try:
                tickets.append(hr.hr_queue_submit(q, hr.HR_HESSIAN, theta, None,
                                                  hr.make_opts(sc["sigma"], M, hr.HR_ELEMENTWISE, 900 + i, i)))
            except hr.HRError as e:
                busy = e
                break
        assert busy is not None and busy.status == hr.HR_ERR_BUSY and "unit ring" in str(busy), busy
        assert 40 <= len(tickets) <= 43, len(tickets)
        outs = {}
        for k, t in enumerate(tickets[:20]):
            o = np.zeros((2, 2))
            hr.hr_queue_wait(q, t, o)
            outs[k] = o
        # the ring has room again: these units take indices past 2^20
        more = [hr.hr_queue_submit(q, hr.HR_HESSIAN, theta, None,
                                   hr.make_opts(sc["sigma"], M, hr.HR_ELEMENTWISE, 900 + len(tickets) + j,
                                                len(tickets) + j)) for j in range(10)]
        for k, t in enumerate(tickets[20:] + more, start=20):
            o = np.zeros((2, 2))
            hr.hr_queue_wait(q, t, o)
            outs[k] = o
        for k in (0, 19, 20, len(tickets) - 1, len(tickets) + 9):
            e = S.estimate(hr.HR_HESSIAN, theta, sc["sigma"], M, hr.HR_ELEMENTWISE, 900 + k, k)
            assert np.array_equal(outs[k], e), (k, outs[k], e)
    finally:
        hr.hr_queue_destroy(q)
        S.close()
