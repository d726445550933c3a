"""The estimate entry point that allocates nothing (hr_estimate_dev_noalloc)
against the ordinary device-pointer entry point, through the C ABI.

Collected last on purpose: it also checks that the fixed working array gives
the same results after every other test has used the library."""
import ctypes

import numpy as np
import pytest

from paper_2412_03489_gb300 import build as hb
from paper_2412_03489_gb300 import hr
from paper_2412_03489_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

hb.build()


def test_no_alloc_estimate_matches_device_entry_point_twice():
    torch = pytest.importorskip("torch")
    sc = wl.revolve_scene(width=64, height=64)
    S = hr.Scene(sc)
    stream = torch.cuda.Stream()
    d_theta = torch.tensor(sc["theta_query"], dtype=torch.float64, device="cuda")
    for call in range(2):
        o = hr.make_opts(sc["sigma"], 512, hr.HR_AGGREGATE, 77, call, stream=stream.cuda_stream)
        ref = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
        out = torch.full((2, 2), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        hr.hr_estimate_dev(S.handle, hr.HR_HESSIAN, d_theta.data_ptr(), None, o, ref.data_ptr())
        status = hr.lib().hr_estimate_dev_noalloc(S.handle, hr.HR_HESSIAN, d_theta.data_ptr(), None,
                                                  ctypes.byref(o), out.data_ptr())
        stream.synchronize()
        assert status == hr.HR_OK, hr.hr_last_error()
        r, g = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.allclose(g, r, rtol=1e-4, atol=1e-4 * np.abs(r).max()), (call, g, r)


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
