"""GPU frozen-path gradients (robast_trace_grad, through the C ABI) against
the oracle's dual-number gradients and central finite differences.

Tolerances: GPU vs oracle duals 1e-3 relative (FP32 trace) and 1e-8 (FP64);
repeated runs bit-identical;
GPU (FP64) vs oracle central differences (h = 1e-6) 1e-4.  Relative error is
|g - g_ref| / max(|g_ref|, 1e-3 max|g_ref|).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
robast = pytest.importorskip("paper_1508_07803_gb300")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    robast.load()


def _rel(g, ref):
    scale = max(np.max(np.abs(ref)), 1e-300)
    return np.abs(g - ref) / np.maximum(np.abs(ref), 1e-3 * scale)


def _dev(bundle, precision):
    dt = torch.float32 if precision == 32 else torch.float64
    b = bundle if precision == 64 else bundle.rounded_to(np.float32)
    return (torch.from_numpy(b.origins).to("cuda", dt), torch.from_numpy(b.dirs).to("cuda", dt),
            torch.from_numpy(b.wavelengths).to("cuda", dt))


def _gpu(scene, b, objective, precision, **kw):
    geom = robast.build_geometry(scene)
    o, d, w = _dev(b, precision)
    v, g, info = robast.trace_grad(geom, o, d, w, objective=objective, precision=precision, **kw)
    geom.close()
    return v, g.cpu().numpy(), info


@pytest.mark.parametrize("precision,tol", [(64, 1e-8), (32, 1e-3)])
def test_dish_msr_gradient_matches_oracle_duals(precision, tol):
    scene, b = W.lst_workload(4_001, seed=5, angles_deg=(0.0, 1.0))
    v, g, info = _gpu(scene, b, "msr", precision, seed=7)
    ref_b = b if precision == 64 else b.rounded_to(np.float32)
    rv, rg = oracle.objective(scene, ref_b, "msr", seed=7, eps=oracle.default_eps(scene, precision))
    assert v == pytest.approx(rv, rel=1e-9 if precision == 64 else 1e-5)
    assert info["n_untracked"] == 0
    mask = np.abs(rg).sum(axis=1) > 0
    assert mask.sum() > 50
    assert np.max(_rel(g[mask], rg[mask])) < tol


def test_dish_gradient_matches_central_differences():
    scene, b = W.lst_workload(1_500, seed=6, angles_deg=(1.5,))
    _, g, _ = _gpu(scene, b, "msr", 64, seed=8)
    ns = len(scene.surfaces)
    picks = np.argsort(-np.abs(g[:, 0]))[:3]
    for sid in picks:
        for k in (0, 1, 2, 5):
            dp = np.zeros((ns, 16))
            dp[sid, k] = 1e-6
            vp, _ = oracle.objective(scene, b, "msr", seed=8, delta=dp, grad=False)
            vm, _ = oracle.objective(scene, b, "msr", seed=8, delta=-dp, grad=False)
            fd = (vp - vm) / 2e-6
            scale = np.max(np.abs(g))
            assert abs(g[sid, k] - fd) / max(abs(fd), 1e-3 * scale) < 1e-4, (sid, k, g[sid, k], fd)


@pytest.mark.parametrize("precision,tol", [(64, 1e-8), (32, 1e-3)])
def test_cone_soft_ce_gradient_matches_oracle_duals(precision, tol):
    scene = W.cone_scene(n_variants=1, seed=0)
    H = W.cone_heights(1)[0]
    b = W.concat([W.hexagon_bundle(3_001, W.CONE_A_IN, H + W.CONE_WINDOW + 1e-4, math.radians(a), seed=3,
                                   stream=60 + i) for i, a in enumerate((5.0, 20.0, 28.0, 33.0))])
    v, g, _ = _gpu(scene, b, "soft_ce", precision, seed=4, max_bounces=30)
    ref_b = b if precision == 64 else b.rounded_to(np.float32)
    rv, rg = oracle.objective(scene, ref_b, "soft_ce", seed=4, max_bounces=30, eps=oracle.default_eps(scene, precision))
    assert v == pytest.approx(rv, rel=1e-9 if precision == 64 else 1e-4)
    assert np.max(_rel(g[1, 10:16], rg[1, 10:16])) < tol, (g[1, 10:16], rg[1, 10:16])


def test_cone_soft_ce_gradient_does_not_depend_on_the_order():
    """Coherent (origin-cell) order and id order give the same bits: contributions are summed
    in 128-bit fixed point."""
    scene = W.cone_scene(n_variants=1, seed=0)
    H = W.cone_heights(1)[0]
    b = W.concat([W.hexagon_bundle(20_011, W.CONE_A_IN, H + W.CONE_WINDOW + 1e-4, math.radians(a), seed=5,
                                   stream=80 + i) for i, a in enumerate((5.0, 20.0, 28.0, 33.0))])
    runs = [_gpu(scene, b, "soft_ce", 32, seed=4, max_bounces=30, coherent_order=c) for c in (1, -1, 0)]
    for v, g, _ in runs[1:]:
        assert v == runs[0][0]
        assert np.array_equal(g, runs[0][1])


def test_autograd_function_returns_the_launch_gradient():
    scene, b = W.lst_workload(2_000, seed=9, angles_deg=(0.5,))
    F = robast.objective_function()
    params = torch.tensor(robast.scene_params(scene), dtype=torch.float64, requires_grad=True)
    o, d, w = _dev(b, 64)
    val = F.apply(params, scene, o, d, w, dict(objective="msr", precision=64, seed=2))
    (2.0 * val).backward()
    rv, rg = oracle.objective(scene, b, "msr", seed=2)
    assert float(val) == pytest.approx(rv, rel=1e-9)
    got = params.grad.numpy()
    mask = np.abs(rg).sum(axis=1) > 0
    assert np.max(_rel(got[mask], 2.0 * rg[mask])) < 1e-8
    # a central difference along a step matches the gradient's directional derivative
    step = 1e-6 * got / np.max(np.abs(got))
    p0 = robast.scene_params(scene)
    opts = dict(objective="msr", precision=64, seed=2)
    vp = float(F.apply(torch.tensor(p0 + step), scene, o, d, w, opts))
    vm = float(F.apply(torch.tensor(p0 - step), scene, o, d, w, opts))
    pred = 0.5 * np.sum(got * step)
    assert abs((vp - vm) / 2 - pred) < 1e-4 * abs(pred)


def test_batched_dishes_gradient_matches_oracle():
    """Several dishes with different facet counts in one launch: the objective
    is the sum of the dishes' MSRs and each facet's gradient uses its own
    dish's centroid."""
    scene, b, vop, counts = W.dish_batch(n_dishes=3, n_min=60, n_max=120, photons_per_dish=2_000,
                                         angles_deg=(0.0, 1.0))
    geom = robast.build_geometry(scene)
    o, d, w = _dev(b, 64)
    v, g, info = robast.trace_grad(geom, o, d, w, objective="msr", precision=64, seed=3,
                                   variant_of_photon=torch.from_numpy(vop).cuda())
    geom.close()
    rv, rg = oracle.objective(scene, b, "msr", seed=3, variant_of_photon=vop)
    assert v == pytest.approx(rv, rel=1e-9)
    g = g.cpu().numpy()
    mask = np.abs(rg).sum(axis=1) > 0
    assert mask.sum() > 100
    assert np.max(_rel(g[mask], rg[mask])) < 1e-8


def test_param_layout_marks_the_differentiated_slots():
    scene, _ = W.lst_workload(10, seed=0, angles_deg=(0.0,))
    geom = robast.build_geometry(scene)
    lay = robast.param_layout(geom)
    assert len(lay) == len(scene.surfaces) * robast.N_PARAM
    for k, (sid, var, slot, active) in enumerate(lay):
        assert sid == k // robast.N_PARAM and var == 0 and slot == robast.PARAM_SLOTS[k % robast.N_PARAM]
        s = scene.surfaces[sid]
        want = s.role == "mirror" and ((s.shape == "sag" and k % 16 < 10) or (s.shape == "hexcone" and k % 16 >= 10))
        assert active == want, (sid, slot)
    assert sum(a for *_, a in lay) == 10 * sum(1 for s in scene.surfaces if s.role == "mirror" and s.shape == "sag")
    geom.close()
    cone = W.cone_scene(n_variants=3, seed=1)
    geom = robast.build_geometry(cone)
    lay = robast.param_layout(geom)
    assert {v for _, v, _, _ in lay} == {0, 1, 2}
    act = [(sid, slot) for sid, _, slot, a in lay if a]
    assert act and all(cone.surfaces[sid].shape == "hexcone" and slot.startswith("P") for sid, slot in act)
    geom.close()


@pytest.mark.parametrize("precision,tol", [(64, 1e-8), (32, 1e-3)])
def test_two_mirror_gradient_covers_primary_and_secondary(precision, tol):
    """Schwarzschild-Couder-like optics: every detected photon meets a primary and a secondary
    panel; the adjoint sweep gives both their gradients, matching the oracle's duals (which
    carry every differentiable surface of a path) and central differences."""
    scene, b = W.sct_workload(1_500, seed=4, angles_deg=(0.0, 2.0))
    v, g, info = _gpu(scene, b, "msr", precision, seed=5)
    ref_b = b if precision == 64 else b.rounded_to(np.float32)
    rv, rg = oracle.objective(scene, ref_b, "msr", seed=5, eps=oracle.default_eps(scene, precision))
    assert v == pytest.approx(rv, rel=1e-9 if precision == 64 else 1e-5)
    assert info["n_untracked"] == 0
    prim = [i for i, s in enumerate(scene.surfaces) if s.role == "mirror" and s.origin[2] == 0.0]
    sec = [i for i, s in enumerate(scene.surfaces) if s.role == "mirror" and s.origin[2] != 0.0]
    assert np.abs(rg[prim]).sum() > 0 and np.abs(rg[sec]).sum() > 0
    assert np.abs(g[sec]).sum() > 0
    mask = np.abs(rg).sum(axis=1) > 0
    assert np.max(_rel(g[mask], rg[mask])) < tol
    if precision == 64:
        ns = len(scene.surfaces)
        for sid in (max(prim, key=lambda i: abs(g[i, 0])), max(sec, key=lambda i: abs(g[i, 0]))):
            for k, h in ((0, 1e-6), (1, 1e-6)):
                dp = np.zeros((ns, 16))
                dp[sid, k] = h
                vp, _ = oracle.objective(scene, b, "msr", seed=5, delta=dp, grad=False)
                vm, _ = oracle.objective(scene, b, "msr", seed=5, delta=-dp, grad=False)
                fd = (vp - vm) / (2 * h)
                assert abs(g[sid, k] - fd) / max(abs(fd), 1e-3 * np.max(np.abs(g))) < 1e-4, (sid, k, g[sid, k], fd)


def test_gradient_is_bit_identical_from_run_to_run():
    """The sums over photons are fixed point with integer atomics: neither the order in which
    photons finish nor the processing order changes a bit of the value or the gradient."""
    scene, b, vop, _ = W.dish_batch(n_dishes=4, n_min=60, n_max=198, photons_per_dish=50_000)
    geom = robast.build_geometry(scene)
    o, d, w = _dev(b, 32)
    v = torch.from_numpy(vop).cuda()
    runs = [robast.trace_grad(geom, o, d, w, objective="msr", precision=32, seed=1, variant_of_photon=v)
            for _ in range(3)]
    # photons in the coherent (origin-cell) order instead of id order: the same bits too
    runs.append(robast.trace_grad(geom, o, d, w, objective="msr", precision=32, seed=1, variant_of_photon=v,
                                  coherent_order=1))
    geom.close()
    for val, g, _ in runs[1:]:
        assert val == runs[0][0]
        assert torch.equal(g, runs[0][1])
