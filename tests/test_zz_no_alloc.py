"""The estimate entry point that allocates nothing (hr_estimate_dev_noalloc)
against the ordinary device-pointer entry point, through the C ABI.

Some callers cannot allocate device memory while they run (latency-bound
loops that must not take allocator locks or wait for cudaFree's device-wide
synchronisation, host applications that give the library a fixed memory
budget); this entry point serves them from one fixed array inside the
library.  It runs the same kernels in the same order on the same values as
hr_estimate_dev, so its outputs must be bit-identical, for every quantity
and strategy, on two calls in a row.

Collected last on purpose: it also checks that the fixed working array gives
the same results after every other test has used the library."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2412_03489_gb300 import build as hb
from paper_2412_03489_gb300 import hr
from paper_2412_03489_gb300 import workloads as wl
from parity import assert_estimate_close, flat_of

pytestmark = pytest.mark.gpu

hb.build()

QUANT = [("grad", hr.HR_GRAD), ("hessian", hr.HR_HESSIAN), ("hvp", hr.HR_HVP)]
STRAT = [("elementwise", hr.HR_ELEMENTWISE), ("aggregate", hr.HR_AGGREGATE), ("plain", hr.HR_PLAIN)]


def _scenes():
    # n = 8 exercises the element-wise Hessian's upper-triangle walk (36
    # groups, more than fit in the sampler's by-value table) and the
    # element-wise HVP rows; the mesh and the disc are the n = 2 workloads
    return [("tris2d_n8", wl.tris2d_scene(width=64, height=48, n_params=8), 32),
            ("revolve64", wl.revolve_scene(width=64, height=64), 256),
            ("disc", wl.disc_scene(), 512)]


def _pair(torch, S, q, d_theta, d_v, o, shape):
    """hr_estimate_dev and hr_estimate_dev_noalloc on the same request and
    stream; returns both outputs."""
    ref = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
    out = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
    hr.hr_estimate_dev(S.handle, q, d_theta.data_ptr(), d_v.data_ptr() if q == hr.HR_HVP else None, o,
                       ref.data_ptr())
    status = hr.lib().hr_estimate_dev_noalloc(S.handle, q, d_theta.data_ptr(),
                                              d_v.data_ptr() if q == hr.HR_HVP else None, ctypes.byref(o),
                                              out.data_ptr())
    assert status == hr.HR_OK, hr.hr_last_error()
    return ref, out


@pytest.mark.parametrize("scene_i", range(3))
def test_no_alloc_is_bit_identical_to_device_entry_point_twice(scene_i):
    torch = pytest.importorskip("torch")
    name, sc, M = _scenes()[scene_i]
    S = hr.Scene(sc)
    n = sc["n_params"]
    stream = torch.cuda.Stream()
    d_theta = torch.tensor(sc["theta_query"], dtype=torch.float64, device="cuda")
    v = np.asarray(sc.get("v", np.linspace(-1.0, 1.0, n)), np.float64)
    d_v = torch.tensor(v, dtype=torch.float64, device="cuda")
    for call in range(2):
        for qn, q in QUANT:
            for sn, s in STRAT:
                o = hr.make_opts(sc["sigma"], M, s, 77, 10 * call + q, stream=stream.cuda_stream)
                ref, out = _pair(torch, S, q, d_theta, d_v, o, (n, n) if q == hr.HR_HESSIAN else (n,))
                stream.synchronize()
                r, g = ref.cpu().numpy(), out.cpu().numpy()
                assert np.all(np.isfinite(r)), (name, qn, sn)
                assert np.array_equal(g, r), (name, call, qn, sn, g, r)
    S.close()


def test_no_alloc_matches_oracle():
    """The fixed-array path against the oracle on the same samples: an
    element-wise Hessian of the 8-parameter triangle scene (36 sample
    groups) and an aggregate HVP."""
    torch = pytest.importorskip("torch")
    sc = wl.tris2d_scene(width=64, height=48, n_params=8)
    S = hr.Scene(sc)
    r = O.Tris2dRenderer(sc)
    n = sc["n_params"]
    theta = np.asarray(sc["theta_query"], np.float64)
    d_theta = torch.tensor(theta, dtype=torch.float64, device="cuda")
    d_v = torch.tensor(sc["v"], dtype=torch.float64, device="cuda")
    for qn, q, strat, sn in (("hessian", hr.HR_HESSIAN, hr.HR_ELEMENTWISE, "elementwise"),
                             ("hvp", hr.HR_HVP, hr.HR_AGGREGATE, "aggregate")):
        out = torch.zeros((n, n) if q == hr.HR_HESSIAN else (n,), dtype=torch.float64, device="cuda")
        o = hr.make_opts(sc["sigma"], 32, strat, 13, 5)
        status = hr.lib().hr_estimate_dev_noalloc(S.handle, q, d_theta.data_ptr(),
                                                  d_v.data_ptr() if q == hr.HR_HVP else None, ctypes.byref(o),
                                                  out.data_ptr())
        assert status == hr.HR_OK, hr.hr_last_error()
        torch.cuda.synchronize()
        ref = O.estimate(r, qn, theta, sc["sigma"], 32, sn, 13, 5, v=sc["v"] if q == hr.HR_HVP else None)
        assert_estimate_close(flat_of(qn, out.cpu().numpy(), n), ref, what=f"no-alloc {qn} {sn}")
    S.close()


def test_no_alloc_calls_leave_free_device_memory_unchanged():
    """After one warm-up call per request shape (the first call on a device
    looks up the array's address; kernels load on first use), further calls
    change the device's free memory by nothing: the call allocates no device
    memory."""
    torch = pytest.importorskip("torch")
    sc = wl.tris2d_scene(width=64, height=48, n_params=8)
    S = hr.Scene(sc)
    n = sc["n_params"]
    stream = torch.cuda.Stream()
    d_theta = torch.tensor(sc["theta_query"], dtype=torch.float64, device="cuda")
    d_v = torch.tensor(sc["v"], dtype=torch.float64, device="cuda")
    outs = {q: torch.zeros((n, n) if q == hr.HR_HESSIAN else (n,), dtype=torch.float64, device="cuda")
            for _, q in QUANT}

    def round_(req):
        for _, q in QUANT:
            for _, s in STRAT:
                o = hr.make_opts(sc["sigma"], 32, s, 3, req + q, stream=stream.cuda_stream)
                st = hr.lib().hr_estimate_dev_noalloc(S.handle, q, d_theta.data_ptr(),
                                                      d_v.data_ptr() if q == hr.HR_HVP else None,
                                                      ctypes.byref(o), outs[q].data_ptr())
                assert st == hr.HR_OK, hr.hr_last_error()
        stream.synchronize()

    round_(0)
    free0, _ = torch.cuda.mem_get_info()
    for k in range(1, 4):
        round_(100 * k)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    S.close()


def test_no_alloc_rejects_requests_beyond_its_array():
    torch = pytest.importorskip("torch")
    sc = wl.disc_scene()
    S = hr.Scene(sc)
    d_theta = torch.tensor(sc["theta_query"], dtype=torch.float64, device="cuda")
    out = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    o = hr.make_opts(sc["sigma"], 1 << 20, hr.HR_AGGREGATE, 1, 1)
    status = hr.lib().hr_estimate_dev_noalloc(S.handle, hr.HR_HESSIAN, d_theta.data_ptr(), None,
                                              ctypes.byref(o), out.data_ptr())
    assert status == -1
    assert "bytes" in hr.hr_last_error()
    # invalid options take the shared validation of every estimate entry point
    o = hr.make_opts(sc["sigma"], 3, hr.HR_AGGREGATE, 1, 1)
    status = hr.lib().hr_estimate_dev_noalloc(S.handle, hr.HR_HESSIAN, d_theta.data_ptr(), None,
                                              ctypes.byref(o), out.data_ptr())
    assert status == -1 and "even" in hr.hr_last_error()
    S.close()
