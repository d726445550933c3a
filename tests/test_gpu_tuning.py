"""Autotuning of launch shapes (hr_autotune, hr_set_tuning): every render
variant and sampler shape gives bit-identical estimates, the tuner reports a
valid choice with its timings, and out-of-range settings are rejected."""
import numpy as np
import pytest

from paper_2412_03489_gb300 import build as hb
from paper_2412_03489_gb300 import hr
from paper_2412_03489_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

hb.build()

SCENES = {
    "disc": lambda: wl.disc_scene(),
    "boxes": lambda: wl.boxes_scene(n_boxes=3),
    "revolve": lambda: wl.revolve_scene(width=96, height=80),
    "tris": lambda: wl.tris2d_scene(width=64, height=48),
    "pt": lambda: wl.ptbox_scene(width=24, height=20, spp=2, target_spp=4),
}


def _estimates(S, sc):
    th = np.asarray(sc["theta_query"], np.float64)
    v = np.random.default_rng(1).normal(size=S.n)
    q = hr.HR_HVP if S.n > 8 else hr.HR_HESSIAN
    a = S.estimate(q, th, sc["sigma"], 512, hr.HR_AGGREGATE, 21, 3, v=v if q == hr.HR_HVP else None)
    b = S.estimate(hr.HR_GRAD, th, sc["sigma"], 64, hr.HR_ELEMENTWISE, 22, 4)
    return a, b


@pytest.mark.parametrize("name", list(SCENES))
def test_every_launch_shape_gives_identical_results(name):
    sc = SCENES[name]()
    S = hr.Scene(sc)
    ref = _estimates(S, sc)
    info = hr.hr_autotune(S.handle, sc["theta_query"], 256)
    assert 0 <= info.render_variant < info.n_render_variants and info.sample_threads in (16, 32, 64, 128)
    assert all(info.render_ms[k] > 0 for k in range(info.n_render_variants))
    assert all(info.sample_ms[k] > 0 for k in range(info.n_sample_variants))
    tuned = _estimates(S, sc)
    for x, y in zip(ref, tuned):
        assert np.array_equal(x, y)
    for rv in range(info.n_render_variants):
        for t in (16, 32, 64, 128):
            hr.hr_set_tuning(S.handle, rv, t)
            for x, y in zip(ref, _estimates(S, sc)):
                assert np.array_equal(x, y), (rv, t)
    S.close()


def test_out_of_range_settings_are_rejected():
    sc = wl.revolve_scene(width=64, height=64)
    S = hr.Scene(sc)
    for rv, t in ((1, 32), (-1, 32), (0, 48), (0, 256), (0, 8)):
        with pytest.raises(hr.HRError, match="status -1"):
            hr.hr_set_tuning(S.handle, rv, t)
    with pytest.raises(hr.HRError, match="status -1"):
        hr.hr_autotune(S.handle, sc["theta_query"], 3)
    S.close()
