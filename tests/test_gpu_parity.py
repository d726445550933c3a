"""GPU parity: the CUDA path through the C ABI against the oracle on the same
seeded inputs and the same Philox samples.

* perturbations: bit-exact (FP32 equality of every tau);
* disc losses: bit-exact (0/1 pixels, exact integer counts);
* raster images: identical coverage (same FP32 decision sequences), shading
  within FP32 rounding;
* estimates: |gpu - oracle| <= 1e-4 max(|oracle|, A_e) (see tests/parity.py).
"""
import math
import os
from types import SimpleNamespace

import numpy as np
import pytest

import oracle as O
from paper_2412_03489_gb300 import build as hb
from paper_2412_03489_gb300 import hr
from paper_2412_03489_gb300 import workloads as wl
from parity import assert_estimate_close, assert_losses_close, flat_of

pytestmark = pytest.mark.gpu

hb.build()

Q = {"grad": hr.HR_GRAD, "hessian": hr.HR_HESSIAN, "hvp": hr.HR_HVP}
S = {"elementwise": hr.HR_ELEMENTWISE, "aggregate": hr.HR_AGGREGATE}


def run_both(sc, renderer, quantity, M, strategy, seed=11, request=3, sub=0, v=None, theta=None, scene=None):
    theta = np.asarray(sc["theta_query"] if theta is None else theta, np.float64)
    own = scene is None
    Sc = hr.Scene(sc) if own else scene
    out, dbg = Sc.estimate(Q[quantity], theta, sc["sigma"], M, S[strategy], seed, request, sub, v=v, debug=True)
    ref = O.estimate(renderer, quantity, theta, sc["sigma"], M, strategy, seed, request, sub, v=v)
    if own:
        Sc.close()
    return flat_of(quantity, out, sc["n_params"]), dbg, ref


def check_samples(dbg, ref):
    assert dbg["tau"].shape == ref.tau.shape
    mism = np.count_nonzero(dbg["tau"] != ref.tau)
    assert mism == 0, f"{mism} perturbation values differ"
    # weights: FP32 of the FP64 value on both sides; compare to FP32 rounding
    w32 = ref.w.astype(np.float32)
    assert np.allclose(dbg["w"], w32, rtol=2e-7, atol=1e-30 + 2e-7 * np.abs(w32).max())


# ---------------------------------------------------------------------------
# disc (64 x 64, 2 params, sigma 0.05, 1024 samples)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("strategy", ["elementwise", "aggregate"])
@pytest.mark.parametrize("quantity", ["hessian", "grad"])
def test_disc_full_size(quantity, strategy):
    sc = wl.disc_scene()
    flat, dbg, ref = run_both(sc, O.DiscRenderer(sc), quantity, 1024, strategy)
    check_samples(dbg, ref)
    assert np.array_equal(dbg["losses"].astype(np.float64), ref.losses)
    assert_estimate_close(flat, ref, what=f"disc {quantity} {strategy}")
    assert np.allclose(dbg["scale"], ref.scale, rtol=1e-5)


def test_disc_hvp_and_identity():
    sc = wl.disc_scene()
    v = np.array([0.3, -1.2])
    flat, dbg, ref = run_both(sc, O.DiscRenderer(sc), "hvp", 1024, "aggregate", v=v)
    check_samples(dbg, ref)
    assert_estimate_close(flat, ref, what="disc hvp")
    Hflat, _, _ = run_both(sc, O.DiscRenderer(sc), "hessian", 1024, "aggregate")
    H = np.array([[Hflat[0], Hflat[1]], [Hflat[1], Hflat[2]]])
    assert np.allclose(H @ v, flat, rtol=1e-5, atol=1e-5 * np.abs(ref.scale).max())


@pytest.mark.parametrize("W,H,M", [(37, 23, 2), (1, 1, 6), (64, 64, 2), (32, 17, 4), (128, 9, 4), (64, 33, 2),
                                   (256, 5, 2), (512, 3, 2)])
def test_disc_ragged_and_minimum(W, H, M):
    sc = wl.disc_scene(width=W, height=H)
    flat, dbg, ref = run_both(sc, O.DiscRenderer(sc), "hessian", M, "aggregate")
    check_samples(dbg, ref)
    # exact mismatch counts; the loss is count / (W H) rounded once to FP32
    npx = W * H
    assert np.array_equal(np.rint(dbg["losses"].astype(np.float64) * npx), np.rint(ref.losses * npx))
    assert np.all(np.abs(dbg["losses"] - ref.losses) <= np.spacing(np.float32(ref.losses)))
    assert_estimate_close(flat, ref, what="disc ragged")


@pytest.mark.parametrize("W,H,radius,sigma,target", [
    (64, 64, 5.0 / 64.0, 1e-6, "disc"),      # centre on a pixel centre, r a whole number of pixels:
    (64, 64, 0.2, 1e-7, "disc"),             #   boundary pixels within rounding of d^2 = r^2
    (37, 23, 0.2, 0.3, "disc"),              # wide perturbations: discs cut by every image edge
    (100, 50, 0.7, 0.2, "random"),           # spans over word boundaries, arbitrary 0/1 target
    (1024, 3, 0.004, 0.05, "random"),        # sub-pixel radius, 32 words per row
    (33, 40, 1.5, 0.5, "random"),            # discs larger than the image
    (64, 48, 1000.0, 0.05, "far"),           # radius 1000 centred 1000.5 below the top: its edge crosses the image
    (1, 1, 0.2, 0.3, "disc")])
def test_disc_binary_target_spans(W, H, radius, sigma, target):
    """Binary targets take the span path (row intervals of the FP32 pixel test,
    mismatch counts by popcount): every loss equals the oracle's per-pixel
    count, including pixels within rounding of the disc's edge."""
    sc = wl.disc_scene(width=W, height=H, radius=radius)
    sc["sigma"] = sigma
    g = np.random.default_rng(W * 7 + H)
    if sigma < 1e-5:   # theta on a pixel centre
        sc["theta_query"] = np.array([(W // 2 + 0.5) / W, (H // 3 + 0.5) / H])
    if target == "far":
        sc["theta_query"] = np.array([0.5, 1000.5])
    tgt = None
    if target in ("random", "far"):
        tgt = (g.uniform(size=W * H) < 0.4).astype(np.float32)
    Sc = hr.Scene(sc, target_image=tgt) if tgt is not None else hr.Scene(sc)
    ren = O.DiscRenderer(sc, target=tgt) if tgt is not None else O.DiscRenderer(sc)
    flat, dbg, ref = run_both(sc, ren, "hessian", 256, "aggregate", scene=Sc)
    Sc.close()
    check_samples(dbg, ref)
    npx = W * H
    assert np.array_equal(np.rint(dbg["losses"].astype(np.float64) * npx), np.rint(ref.losses * npx))
    assert np.all(np.abs(dbg["losses"] - ref.losses) <= np.spacing(np.float32(ref.losses)))
    assert_estimate_close(flat, ref, what="disc spans")


@pytest.mark.parametrize("W,H", [(64, 21), (96, 10), (128, 7), (512, 3)])
def test_disc_grey_target(W, H):
    """A caller's target image with grey levels (the renderer's own targets are
    0/1, whose sums are exact in any order): every loss within FP32 rounding of
    the oracle's FP64 loss, on both pixel loops (fixed columns per lane for
    W = 64, 128 and 512, the general loop for W = 96)."""
    sc = wl.disc_scene(width=W, height=H)
    tgt = np.random.default_rng(W * 1000 + H).uniform(0.0, 1.0, size=W * H).astype(np.float32)
    Sc = hr.Scene(sc, target_image=tgt)
    flat, dbg, ref = run_both(sc, O.DiscRenderer(sc, target=tgt), "hessian", 64, "aggregate", scene=Sc)
    Sc.close()
    check_samples(dbg, ref)
    assert_losses_close(dbg["losses"], ref.losses, 2e-6, "disc grey-target losses")
    assert_estimate_close(flat, ref, what="disc grey target")


# ---------------------------------------------------------------------------
# surface of revolution (2048 triangles)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("size", [(64, 64), (50, 37), (256, 256)])
def test_revolve_images_match(size):
    W, H = size
    sc = wl.revolve_scene(width=W, height=H)
    Sc = hr.Scene(sc)
    r = O.RevolveRenderer(sc)
    g = np.random.default_rng(1)
    for _ in range(3):
        p = np.asarray(sc["theta_target"]) + g.normal(0, 0.3, 2)
        gi = Sc.render(p).reshape(H, W, 3)
        oi = r.image(p.astype(np.float32)).reshape(H, W, 3)
        assert np.array_equal(gi.sum(-1) > 0, oi.sum(-1) > 0), "coverage differs"
        assert np.allclose(gi, oi, rtol=1e-5, atol=1e-6)
    # target
    tgt = Sc.render(np.asarray(sc["theta_target"]))
    assert np.allclose(tgt, r.target, rtol=1e-5, atol=1e-6)
    Sc.close()


@pytest.mark.parametrize("strategy", ["elementwise", "aggregate"])
def test_revolve_small(strategy):
    sc = wl.revolve_scene(width=72, height=56)
    flat, dbg, ref = run_both(sc, O.RevolveRenderer(sc), "hessian", 128, strategy)
    check_samples(dbg, ref)
    assert_losses_close(dbg["losses"], ref.losses, 2e-5, "revolve losses")
    assert_estimate_close(flat, ref, what=f"revolve {strategy}")


def test_revolve_full_size_bench_configuration():
    """256 x 256, 2048 triangles, sigma 0.1, 4096 aggregate samples: the bench
    workload in its launch configuration, compared in full.  Every render
    runs in the compact layout (two renders per SM, records of the ~900
    surviving triangles only): none is handed to the full layout."""
    sc = wl.revolve_scene()
    Sc = hr.Scene(sc)
    before = hr.hr_scene_get_stats(Sc.handle)
    flat, dbg, ref = run_both(sc, O.RevolveRenderer(sc), "hessian", 4096, "aggregate", seed=2024, request=0, scene=Sc)
    st = hr.hr_scene_get_stats(Sc.handle)
    Sc.close()
    check_samples(dbg, ref)
    assert_losses_close(dbg["losses"], ref.losses, 2e-5, "revolve losses")
    assert_estimate_close(flat, ref, what="revolve full")
    assert st.mesh_compact_slots >= len(sc["triangles"]) // 2
    assert st.mesh_renders - before.mesh_renders == 4096
    assert st.mesh_redo_renders - before.mesh_redo_renders == 0


def _ids_cases():
    sc = wl.revolve_scene()
    g = np.random.default_rng(3)
    yield "bench mesh 256", sc, [np.asarray(sc["theta_query"]) + g.normal(0, 0.1, 2) for _ in range(3)]
    yield "bench mesh 50x37", wl.revolve_scene(width=50, height=37), [np.asarray(sc["theta_target"])]
    for W in (128, 512):
        s2 = _sheets_scene(W)
        yield f"sheets {W}", s2, [np.asarray(s2["theta_query"]) + g.normal(0, 0.2, 2) for _ in range(2)]
    s3 = wl.revolve_scene(width=96, height=96)
    v, t = wl.sheets_mesh(layers=3, grid=4)
    s3["vertices"], s3["triangles"] = v, np.concatenate([t, t])
    yield "duplicated sheets 96", s3, [np.asarray(s3["theta_query"]) + g.normal(0, 0.2, 2) for _ in range(2)]


@pytest.mark.parametrize("case", range(5))
def test_revolve_triangle_indices_bit_exact(case):
    """The rasteriser's decisions, pixel by pixel: the index of the triangle
    each pixel shows equals the oracle's, exactly (both decide coverage and
    depth in FP32 with the same operation sequences).  Cases: the bench mesh
    (8x4 tiles), a ragged size, stacked sheets with the binned raster and with
    the bin-overflow fallback, and a mesh listed twice, where every covered
    pixel is an exact depth tie that the lower index must win."""
    name, sc, params = list(_ids_cases())[case]
    Sc = hr.Scene(sc)
    r = O.RevolveRenderer(sc)
    for p in params:
        gi = hr.hr_render_ids(Sc.handle, p, sc["width"], sc["height"])
        oi = r.ids(np.asarray(p, np.float32))
        assert (oi >= 0).any(), name
        bad = np.count_nonzero(gi != oi)
        assert bad == 0, f"{name}: {bad} pixels differ"
    if name.startswith("duplicated"):
        assert gi.max() < len(sc["triangles"]) // 2
        flat, dbg, ref = run_both(sc, r, "hessian", 32, "aggregate", scene=Sc)
        check_samples(dbg, ref)
        assert_losses_close(dbg["losses"], ref.losses, 2e-5, "duplicated-mesh losses")
        assert_estimate_close(flat, ref, what="duplicated mesh")
    Sc.close()


def _sheets_scene(W):
    sc = wl.revolve_scene(width=W, height=W)
    sc["vertices"], sc["triangles"] = wl.sheets_mesh(layers=8, grid=8)
    return sc


@pytest.mark.parametrize("W,banded", [(128, False), (512, True)])
def test_revolve_stacked_sheets_binned_and_banded(W, banded):
    """Eight stacked, tilted sheets of 128 triangles each: every pixel is
    covered at several depths, and every triangle spans many tiles.  At 128^2
    the tile bins hold about 6,000 entries (one binned pass); at 512^2 more
    than 40,000, beyond the bin capacity, so every render is binned and
    rastered in bands of tile rows.  The scene's counters show which path
    ran.  Both against the oracle: images pixel by pixel (the depth winner
    decides each pixel's shade), then an aggregate Hessian on identical
    samples."""
    sc = _sheets_scene(W)
    _check_mesh_paths(sc, W, W, 16, banded, False)


def test_revolve_tile_row_beyond_capacity_walks_every_triangle():
    """A 512 x 4 image (one row of tiles) in front of 1,000 stacked, tilted
    full-frame sheets (2,000 triangles): the row alone holds more than ten
    times the entries the bins can take, so its tiles walk every triangle.
    Images and an estimate against the oracle."""
    sc = wl.revolve_scene(width=512, height=4)
    sc["vertices"], sc["triangles"] = wl.sheets_mesh(layers=1000, grid=1)
    sc["scale"] = np.float32(1024.0)
    _check_mesh_paths(sc, 512, 4, 8, True, True)


def test_revolve_compact_claims_give_the_same_result_every_time():
    """Compact-layout CTAs claim perturbations by compare-and-swap and steal
    the last ones, so which CTA renders which perturbation changes from run to
    run; each loss depends on its perturbation only, so repeated estimates on
    the same samples are bit-identical, losses included."""
    sc = wl.revolve_scene()
    Sc = hr.Scene(sc)
    theta = np.asarray(sc["theta_query"], np.float64)
    runs = [Sc.estimate(Q["hessian"], theta, sc["sigma"], 4096, S["aggregate"], 2024, 5, 0, debug=True)
            for _ in range(4)]
    st = hr.hr_scene_get_stats(Sc.handle)
    Sc.close()
    assert st.mesh_compact_slots > 0 and st.mesh_redo_renders == 0
    out0, dbg0 = runs[0]
    for out, dbg in runs[1:]:
        assert np.array_equal(dbg["losses"], dbg0["losses"])
        assert np.array_equal(out, out0)


@pytest.mark.parametrize("layers", [9, 16])
def test_revolve_compact_layout_hands_over_what_does_not_fit(layers):
    """Stacked full-frame sheets at 128^2 (every triangle faces the camera).
    With 9 sheets (1,152 triangles) the compact layout has a slot for every
    triangle but not room for the ~6,800 bin entries; with 16 (2,048) the
    survivors outnumber its slots.  Either way every render is handed over
    and rendered again in the full layout: images and an aggregate Hessian
    against the oracle, and the counters show the hand-overs."""
    sc = wl.revolve_scene(width=128, height=128)
    sc["vertices"], sc["triangles"] = wl.sheets_mesh(layers=layers, grid=8)
    Sc = hr.Scene(sc)
    slots = hr.hr_scene_get_stats(Sc.handle).mesh_compact_slots
    Sc.close()
    assert 0 < slots
    assert (slots >= len(sc["triangles"])) == (layers == 9)
    st = _check_mesh_paths(sc, 128, 128, 16, None, False)
    assert st.mesh_redo_renders == 16


def _check_mesh_paths(sc, W, H, M, banded, walked):
    Sc = hr.Scene(sc)
    r = O.RevolveRenderer(sc)
    before = hr.hr_scene_get_stats(Sc.handle)
    g = np.random.default_rng(7)
    for _ in range(3):
        p = np.asarray(sc["theta_query"]) + g.normal(0, 0.2, 2)
        gi = Sc.render(p).reshape(H, W, 3)
        oi = r.image(p.astype(np.float32)).reshape(H, W, 3)
        assert np.array_equal(gi.sum(-1) > 0, oi.sum(-1) > 0), "coverage differs"
        assert np.allclose(gi, oi, rtol=1e-5, atol=1e-6), "a different triangle won some pixel"
    flat, dbg, ref = run_both(sc, r, "hessian", M, "aggregate", scene=Sc)
    check_samples(dbg, ref)
    assert_losses_close(dbg["losses"], ref.losses, 2e-5, "mesh losses")
    assert_estimate_close(flat, ref, what=f"mesh {W}x{H}")
    st = hr.hr_scene_get_stats(Sc.handle)
    Sc.close()
    assert st.mesh_renders - before.mesh_renders == M   # the estimate's renders (images are not counted)
    if banded is not None:
        assert st.mesh_overflow_renders - before.mesh_overflow_renders == (M if banded else 0)
    assert st.mesh_walk_all_renders - before.mesh_walk_all_renders == (M if walked else 0)
    assert st.mesh_bin_entries > 0
    assert (st.mesh_raster_steps > 0) != walked   # binned raster steps are counted; a walk has none
    return st


# ---------------------------------------------------------------------------
# coloured triangles
# ---------------------------------------------------------------------------
def test_tris2d_images_and_small_estimate():
    sc = wl.tris2d_scene(width=80, height=60)
    Sc = hr.Scene(sc)
    r = O.Tris2dRenderer(sc)
    for b in range(3):
        p = sc["theta_init"][b]
        gi = Sc.render(p)
        oi = r.image(p.astype(np.float32))
        assert np.array_equal(gi, oi)
    v = sc["v"]
    flat, dbg, ref = run_both(sc, r, "hvp", 32, "aggregate", v=v, scene=Sc)
    check_samples(dbg, ref)
    assert_losses_close(dbg["losses"], ref.losses, 2e-5, "tris2d losses")
    assert_estimate_close(flat, ref, what="tris2d hvp")
    flat, dbg, ref = run_both(sc, r, "grad", 32, "aggregate", scene=Sc)
    assert_estimate_close(flat, ref, what="tris2d grad")
    Sc.close()


# ---------------------------------------------------------------------------
# path tracer
# ---------------------------------------------------------------------------
def test_ptbox_images_match():
    sc = wl.ptbox_scene(width=24, height=20, spp=2, target_spp=4)
    Sc = hr.Scene(sc)
    r = O.PtboxRenderer(sc)
    p = np.asarray(sc["theta_query"])
    gi = Sc.render(p, seed=5, request=2, sub=1, k=3, tag=hr.TAG_PATH, spp=2)
    oi = r.image(p.astype(np.float32), 2, 5, 2, 1, 3, O.TAG_PATH)
    assert np.allclose(gi, oi, rtol=2e-5, atol=2e-5 * oi.max())
    assert np.allclose(Sc.render(np.asarray(sc["theta_target"]), seed=sc["seed"], tag=hr.TAG_TARGET, spp=4),
                       r.target, rtol=2e-5, atol=2e-5 * r.target.max())
    Sc.close()


@pytest.mark.parametrize("case", ["light_within_margin", "light_above_ceiling", "camera_outside"])
def test_ptbox_wall_cut_fallbacks(case):
    """The closest-hit test skips walls only when that cannot change a result
    (origin inside the box; for shadow rays also the light 1e-3 inside every
    wall plane).  Scenes where those conditions fail take the full tests and
    still match the oracle's brute-force path tracer."""
    sc = wl.ptbox_scene(width=24, height=20, spp=2, target_spp=4)
    p = np.asarray(sc["theta_query"], np.float64).copy()
    if case == "light_within_margin":
        p[1] = 0.9995
    elif case == "light_above_ceiling":
        p[1] = 1.02
    else:
        sc["cam_z"] = np.float32(1.4)
    Sc = hr.Scene(sc)
    r = O.PtboxRenderer(sc)
    gi = Sc.render(p, seed=5, request=2, sub=1, k=3, tag=hr.TAG_PATH, spp=2)
    oi = r.image(p.astype(np.float32), 2, 5, 2, 1, 3, O.TAG_PATH)
    assert np.allclose(gi, oi, rtol=2e-5, atol=2e-5 * max(oi.max(), 1e-6)), case
    Sc.close()


def test_ptbox_hvp_small():
    sc = wl.ptbox_scene(width=20, height=16, spp=2, target_spp=4)
    flat, dbg, ref = run_both(sc, O.PtboxRenderer(sc), "hvp", 16, "aggregate", v=sc["v"])
    check_samples(dbg, ref)
    assert_losses_close(dbg["losses"], ref.losses, 1e-4, "ptbox losses")
    assert_estimate_close(flat, ref, what="ptbox hvp")


def test_ptbox_work_counts_match_oracle_and_leave_results_unchanged():
    """The counting build of the path tracer (used to measure its work per
    render) returns the same losses and estimate as the timed build, and its
    closest-hit rays, shadow rays and shaded vertices equal the oracle path
    tracer's counts on the same perturbations and path random numbers."""
    sc = wl.ptbox_scene(width=24, height=20, spp=2, target_spp=4)
    Sc = hr.Scene(sc)
    theta, v, M = np.asarray(sc["theta_query"]), sc["v"], 16
    out0, dbg0 = Sc.estimate(hr.HR_HVP, theta, sc["sigma"], M, hr.HR_AGGREGATE, 5, 6, 0, v=v, debug=True)
    hr.hr_scene_count_work(Sc.handle, True)
    out1, dbg1 = Sc.estimate(hr.HR_HVP, theta, sc["sigma"], M, hr.HR_AGGREGATE, 5, 6, 0, v=v, debug=True)
    hr.hr_scene_count_work(Sc.handle, False)
    st = hr.hr_scene_get_stats(Sc.handle)
    Sc.close()
    assert np.array_equal(dbg0["losses"], dbg1["losses"]) and np.array_equal(out0, out1)
    r = O.PtboxRenderer(sc)
    tau, _ = O.draw(1, 6, sc["sigma"], M // 2, 5, 6, 0)
    ref = np.zeros(3, np.int64)
    for m in range(M):
        ref += r.count_rays(O.perturb(theta, tau[m]), dict(seed=5, request=6, sub=0, k=m // 2))
    assert st.pt_counted_renders == M
    assert (st.pt_hit_rays, st.pt_shadow_rays, st.pt_vertices) == tuple(int(x) for x in ref)


def _host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def test_ptbox_full_size_bench_configuration_sampled():
    """128 x 128, 4 spp, depth 3, aggregate HVP with 8192 perturbations in the
    launch shape the autotuner picks (the bench workload): every perturbation
    and weight against the oracle's sampler, and 64 renders spread over the
    launch against the oracle's path tracer one by one."""
    sc = wl.ptbox_scene()
    Sc = hr.Scene(sc)
    hr.hr_autotune(Sc.handle, sc["theta_query"], 2048)
    theta, v, M, seed, request = np.asarray(sc["theta_query"]), sc["v"], 8192, 11, 3
    out, dbg = Sc.estimate(hr.HR_HVP, theta, sc["sigma"], M, hr.HR_AGGREGATE, seed, request, 0, v=v, debug=True)
    Sc.close()
    assert np.all(np.isfinite(out))
    tau, _ = O.draw(1, 6, sc["sigma"], M // 2, seed, request, 0)
    w = O.weights(2, 6, sc["sigma"], tau, v=v)
    check_samples(dbg, SimpleNamespace(tau=tau, w=w))
    r = O.PtboxRenderer(sc)
    picks = sorted(set([0, 1, M - 2, M - 1] + np.linspace(2, M - 3, 60).astype(int).tolist()))
    assert len(picks) == 64

    def one(m):
        return r.loss(O.perturb(theta, tau[m]), dict(seed=seed, request=request, sub=0, k=m // 2))
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(_host_threads()) as ex:
        ref = np.array(list(ex.map(one, picks)))
    assert_losses_close(dbg["losses"][picks], ref, 1e-4, "ptbox full-size losses")


def test_ptbox_full_size_estimate_against_oracle_estimate():
    """The path-traced HVP at the bench image size (128 x 128, 4 spp, depth 3,
    the autotuned launch shape) against the oracle's own full estimate of the
    same request: the oracle samples, renders every one of the 256
    perturbations with its own path tracer and sums in FP64."""
    sc = wl.ptbox_scene()
    Sc = hr.Scene(sc)
    hr.hr_autotune(Sc.handle, sc["theta_query"], 2048)
    theta, v = np.asarray(sc["theta_query"]), sc["v"]
    flat, dbg, ref = run_both_threads(sc, O.PtboxRenderer(sc), "hvp", 256, "aggregate", 17, 9, v, Sc)
    Sc.close()
    check_samples(dbg, ref)
    assert_losses_close(dbg["losses"], ref.losses, 1e-4, "ptbox estimate losses")
    assert_estimate_close(flat, ref, what="ptbox full-size hvp against the oracle's estimate")


def run_both_threads(sc, renderer, quantity, M, strategy, seed, request, v, scene):
    theta = np.asarray(sc["theta_query"], np.float64)
    out, dbg = scene.estimate(Q[quantity], theta, sc["sigma"], M, S[strategy], seed, request, 0, v=v, debug=True)
    ref = O.estimate(renderer, quantity, theta, sc["sigma"], M, strategy, seed, request, 0, v=v,
                     threads=_host_threads())
    return flat_of(quantity, out, sc["n_params"]), dbg, ref


# ---------------------------------------------------------------------------
# Newton-CG
# ---------------------------------------------------------------------------
def _check_cg_step(r, sc, th_b, got_b, info_b, g_b, p_b, hp_b, M_g, M_h, K, seed, request, step, what):
    """One instance's Newton-CG step, piece by piece:
    * the gradient estimate and every Hessian-vector product inside the CG
      loop against the oracle's estimate of the same request on the same
      samples, at the GPU's own direction p_i: 1e-4 per entry (the estimate
      tolerance of every other parity test);
    * the FP64 CG recurrence: the oracle's Newton-CG fed with the GPU's
      gradient and products takes the same number of iterations and the
      same step to 1e-9 (FP64 sums in another order);
    * the step against the oracle's Newton-CG on its own estimates within
      1e-3: the CG step is a non-linear function of K products, each within
      1e-4, and a product error e moves the step by up to about
      e |p| / lambda_min(H + lambda I)."""
    sigma = sc["sigma"]
    ref_g = O.estimate(r, "grad", th_b, sigma, M_g, "aggregate", seed, request, sub=64 * step)
    assert_estimate_close(g_b, ref_g, what=f"{what}: gradient")
    for i in range(info_b.iters):
        ref = O.estimate(r, "hvp", th_b, sigma, M_h, "aggregate", seed, request, sub=64 * step + 1 + i, v=p_b[i])
        assert_estimate_close(hp_b[i], ref, what=f"{what}: product {i}")

    def hvp_gpu(th, i, vec):
        assert np.allclose(vec, p_b[i], rtol=1e-12, atol=1e-12 * np.abs(p_b[i]).max()), (what, i)
        return hp_b[i]
    new, inf = O.newton_cg_step(r, th_b, sigma, M_g, M_h, K, 1e-3, 0.05, seed, request, step,
                                grad_fn=lambda th: g_b, hvp_fn=hvp_gpu)
    assert inf.iters == info_b.iters, what
    d_gpu = got_b - th_b
    assert np.allclose(d_gpu, new - th_b, rtol=1e-9, atol=1e-9 * np.linalg.norm(d_gpu)), what
    new_o, inf_o = O.newton_cg_step(r, th_b, sigma, M_g, M_h, K, 1e-3, 0.05, seed, request, step)
    assert inf_o.iters == info_b.iters, what
    d_ref = new_o - th_b
    assert np.allclose(d_gpu, d_ref, rtol=1e-3, atol=1e-4 * np.linalg.norm(d_ref)), what
    assert abs(info_b.grad_norm - inf_o.grad_norm) <= 1e-4 * inf_o.grad_norm, what


@pytest.mark.parametrize("use_graph", [0, 1])
def test_newton_cg_step_matches_oracle(use_graph):
    sc = wl.tris2d_scene(width=48, height=40, n_instances=3)
    Sc = hr.Scene(sc)
    r = O.Tris2dRenderer(sc)
    B, n, K = 3, sc["n_params"], 4
    opts = hr.hr_cg_opts()
    opts.sigma, opts.n_grad, opts.n_hvp, opts.cg_iters = sc["sigma"], 16, 8, K
    opts.lambda_rel, opts.trust_radius, opts.seed, opts.request_base, opts.use_graph = 1e-3, 0.05, 99, 10, use_graph
    th0 = np.ascontiguousarray(sc["theta_init"][:B], np.float64)
    st = hr.hr_optstate_create(Sc.handle, B, th0, opts)
    info = (hr.hr_step_info * B)()
    th = th0.copy()
    for step in range(2):
        hr.hr_newton_cg_step(Sc.handle, st, info)
        got = np.zeros((B, n))
        hr.hr_optstate_theta(st, got)
        g, p, hp = hr.hr_optstate_trace(st, B, K, n)
        for b in range(B):
            _check_cg_step(r, sc, th[b], got[b], info[b], g[b], p[b], hp[b], 16, 8, K, 99, 10 + b, step,
                           f"step {step} instance {b}")
        th = got.copy()            # continue both from the GPU iterate
    hr.hr_optstate_destroy(st)
    Sc.close()


def test_newton_cg_full_size_bench_configuration_sampled():
    """256 x 256, 16 triangles, 64 parameters, 64 instances, 32 gradient and
    10 x 32 HVP renders, graph-captured (the bench workload in its launch
    configuration): one step; for three instances every product inside the
    CG loop, the gradient, the CG recurrence and the step against the
    oracle, which renders every one of their perturbations."""
    sc = wl.tris2d_scene()
    Sc = hr.Scene(sc)
    r = O.Tris2dRenderer(sc)
    B, n, K = 64, sc["n_params"], 10
    opts = hr.hr_cg_opts()
    opts.sigma, opts.n_grad, opts.n_hvp, opts.cg_iters = sc["sigma"], 32, 32, K
    opts.lambda_rel, opts.trust_radius, opts.seed, opts.request_base, opts.use_graph = 1e-3, 0.05, 2024, 0, 1
    th0 = np.ascontiguousarray(sc["theta_init"], np.float64)
    st = hr.hr_optstate_create(Sc.handle, B, th0, opts)
    info = (hr.hr_step_info * B)()
    hr.hr_newton_cg_step(Sc.handle, st, info)
    got = np.zeros((B, n))
    hr.hr_optstate_theta(st, got)
    g, p, hp = hr.hr_optstate_trace(st, B, K, n)
    hr.hr_optstate_destroy(st)
    Sc.close()
    for b in (0, 37, 63):
        _check_cg_step(r, sc, th0[b], got[b], info[b], g[b], p[b], hp[b], 32, 32, K, 2024, b, 0, f"instance {b}")


# ---------------------------------------------------------------------------
# device-pointer entry point and argument validation
# ---------------------------------------------------------------------------
def test_dev_entry_point_matches_host():
    torch = pytest.importorskip("torch")
    sc = wl.disc_scene()
    Sc = hr.Scene(sc)
    theta = np.asarray(sc["theta_query"], np.float64)
    host = Sc.estimate(hr.HR_HESSIAN, theta, sc["sigma"], 256, hr.HR_AGGREGATE, 4, 4)
    d_theta = torch.tensor(theta, dtype=torch.float64, device="cuda")
    d_out = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    o = hr.make_opts(sc["sigma"], 256, hr.HR_AGGREGATE, 4, 4, stream=torch.cuda.current_stream().cuda_stream)
    hr.hr_estimate_dev(Sc.handle, hr.HR_HESSIAN, d_theta.data_ptr(), None, o, d_out.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(d_out.cpu().numpy(), host)
    Sc.close()


def test_invalid_arguments_are_rejected():
    sc = wl.disc_scene()
    Sc = hr.Scene(sc)
    theta = np.asarray(sc["theta_query"], np.float64)
    for M, sigma, strat in [(3, 0.05, 1), (0, 0.05, 1), (64, -1.0, 1), (64, 0.05, 7)]:
        with pytest.raises(hr.HRError):
            Sc.estimate(hr.HR_HESSIAN, theta, sigma, M, strat, 1, 1)
    with pytest.raises(hr.HRError):
        Sc.estimate(hr.HR_HVP, theta, 0.05, 64, 9, 1, 1, v=np.ones(2))
    # the scene still works afterwards
    Sc.estimate(hr.HR_HESSIAN, theta, 0.05, 64, hr.HR_AGGREGATE, 1, 1)
    Sc.close()


def test_mesh_beyond_shared_memory_is_rejected():
    sc = wl.revolve_scene()
    verts, tris = wl.revolve_mesh(np.linspace(0.3, 0.8, 8), rings=41, slices=40)   # 3,200 triangles
    assert len(tris) == 3200
    with pytest.raises(hr.HRError, match="status -6"):
        hr.Scene(dict(sc, vertices=verts, triangles=tris))
    verts, tris = wl.revolve_mesh(np.linspace(0.3, 0.8, 8), rings=65, slices=64)   # 8,192: over the format limit
    with pytest.raises(hr.HRError, match="status -1"):
        hr.Scene(dict(sc, vertices=verts, triangles=tris))


# ---------------------------------------------------------------------------
# HVP forms: element-wise (row mixtures) and central difference of gradients
# ---------------------------------------------------------------------------
def test_elementwise_hvp_disc_and_tris():
    sc = wl.disc_scene()
    flat, dbg, ref = run_both(sc, O.DiscRenderer(sc), "hvp", 1024, "elementwise", v=np.array([0.7, -1.3]))
    check_samples(dbg, ref)
    assert np.array_equal(dbg["losses"].astype(np.float64), ref.losses)
    assert_estimate_close(flat, ref, what="disc hvp elementwise")
    st = wl.tris2d_scene(width=64, height=48, n_params=8)
    v = st["v"].copy()
    v[3] = 0.0
    flat, dbg, ref = run_both(st, O.Tris2dRenderer(st), "hvp", 16, "elementwise", v=v)
    check_samples(dbg, ref)
    assert_estimate_close(flat, ref, what="tris hvp elementwise")


@pytest.mark.parametrize("strategy", ["aggregate", "elementwise"])
def test_fd_hvp_matches_oracle(strategy):
    for sc, r, M in [(wl.disc_scene(), None, 1024), (wl.revolve_scene(width=64, height=48), None, 64)]:
        r = O.renderer_for(sc)
        theta = np.asarray(sc["theta_query"], np.float64)
        v = np.array([0.6, -0.8])
        eps = 0.2 * sc["sigma"]
        S = hr.Scene(sc)
        out = np.zeros(2)
        hr.hr_estimate_hvp_fd(S.handle, theta, v, eps, hr.make_opts(sc["sigma"], M, S_[strategy], 21, 4), out)
        S.close()
        ref, gp, gm = O.estimate_hvp_fd(r, theta, v, eps, sc["sigma"], M, strategy, 21, 4)
        scale = (gp.scale + gm.scale) / (2 * eps)
        assert np.all(np.abs(out - ref) <= 1e-4 * np.maximum(np.abs(ref), scale)), (out, ref, scale)


S_ = {"elementwise": hr.HR_ELEMENTWISE, "aggregate": hr.HR_AGGREGATE}


# ---------------------------------------------------------------------------
# squares (Box2 / Box10) and plain Gaussian sampling
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_boxes", [1, 5])
@pytest.mark.parametrize("strategy", ["elementwise", "aggregate", "plain"])
def test_boxes_parity(n_boxes, strategy):
    sc = wl.boxes_scene(n_boxes=n_boxes)
    S_["plain"] = hr.HR_PLAIN
    S["plain"] = hr.HR_PLAIN
    r = O.BoxesRenderer(sc)
    Sc = hr.Scene(sc)
    assert np.array_equal(Sc.render(sc["theta_query"]), r.image(np.asarray(sc["theta_query"], np.float32)))
    M = 256 if n_boxes == 5 and strategy == "elementwise" else 1024
    for q in ("hessian", "grad", "hvp"):
        v = np.linspace(-1, 1, sc["n_params"]) if q == "hvp" else None
        flat, dbg, ref = run_both(sc, r, q, M, strategy, v=v, scene=Sc)
        check_samples(dbg, ref)
        assert np.array_equal(dbg["losses"].astype(np.float64), ref.losses)
        assert_estimate_close(flat, ref, what=f"boxes{n_boxes} {q} {strategy}")
    Sc.close()


@pytest.mark.parametrize("W,H,n_boxes,half,sigma,target", [
    (64, 64, 1, 5.0 / 64.0, 1e-6, "own"),     # square edges on pixel centres, tiny perturbations
    (37, 23, 3, 0.2, 0.3, "own"),             # wide perturbations: squares cut by the image edges
    (100, 50, 5, 0.15, 0.2, "random"),        # overlapping squares, spans over word boundaries
    (33, 40, 2, 1.5, 0.5, "random"),          # squares larger than the image
    (96, 10, 4, 0.1, 0.1, "grey")])           # a grey target keeps the per-pixel loop
def test_boxes_binary_target_spans(W, H, n_boxes, half, sigma, target):
    """Squares against binary targets take the span path (one exact column
    interval per square, rows by the exact row test, mismatch counts by
    popcount): every loss equals the oracle's per-pixel count; a grey target
    is checked within FP32 rounding."""
    sc = wl.boxes_scene(n_boxes=n_boxes, width=W, height=H, half_size=half)
    sc["sigma"] = sigma
    g = np.random.default_rng(W * 11 + H)
    if sigma < 1e-5:   # centres on pixel centres
        sc["theta_query"] = np.array([(W // 2 + 0.5) / W, (H // 3 + 0.5) / H] * n_boxes)
    tgt = None
    if target == "random":
        tgt = (g.uniform(size=W * H) < 0.4).astype(np.float32)
    elif target == "grey":
        tgt = g.uniform(0.0, 1.0, size=W * H).astype(np.float32)
    Sc = hr.Scene(sc, target_image=tgt) if tgt is not None else hr.Scene(sc)
    ren = O.BoxesRenderer(sc, target=tgt) if tgt is not None else O.BoxesRenderer(sc)
    flat, dbg, ref = run_both(sc, ren, "hessian", 128, "aggregate", scene=Sc)
    Sc.close()
    check_samples(dbg, ref)
    if target == "grey":
        assert_losses_close(dbg["losses"], ref.losses, 2e-6, "boxes grey-target losses")
    else:
        npx = W * H
        assert np.array_equal(np.rint(dbg["losses"].astype(np.float64) * npx), np.rint(ref.losses * npx))
        assert np.all(np.abs(dbg["losses"] - ref.losses) <= np.spacing(np.float32(ref.losses)))
    assert_estimate_close(flat, ref, what="boxes spans")


# ---------------------------------------------------------------------------
# grey-box composition
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("quantity", ["grad", "hessian", "hvp"])
def test_greybox_matches_oracle(quantity):
    sc = wl.disc_scene()
    g = np.random.default_rng(5)
    J = g.normal(size=(2, 7))
    y = np.asarray(sc["theta_query"], np.float64)
    vx = g.normal(size=7) if quantity == "hvp" else None
    S = hr.Scene(sc)
    out = np.zeros((7, 7) if quantity == "hessian" else 7)
    hr.hr_estimate_greybox(S.handle, Q[quantity], y, J, vx, hr.make_opts(sc["sigma"], 1024, hr.HR_AGGREGATE, 9, 2), out)
    S.close()
    ref, est = O.estimate_greybox(O.DiscRenderer(sc), quantity, y, J, sc["sigma"], 1024, "aggregate", 9, 2, vx=vx)
    aJ = np.abs(J)
    if quantity == "hessian":
        Sc = np.zeros((2, 2))
        Sc[np.triu_indices(2)] = est.scale
        Sc = Sc + np.triu(Sc, 1).T
        scale = aJ.T @ Sc @ aJ
    elif quantity == "hvp":
        scale = aJ.T @ (est.scale)
    else:
        scale = aJ.T @ est.scale
    assert np.all(np.abs(out - ref) <= 1e-4 * np.maximum(np.abs(ref), scale)), (out, ref)
