"""Element-by-element comparison of a GPU trace with the oracle's.

Tolerances (per photon, on the same seeded inputs):
  FP64 trace: status and bounce count identical for every photon; final
      position within 1e-10 x the system focal length; final direction and
      focal-plane coordinates within 1e-10 (direction) / 1e-10 f.
  FP32 trace (the oracle traces the FP32-rounded inputs, with the FP32
      self-intersection epsilon): status identical for >= 99.999% of photons;
      every photon whose status, bounce count or last surface differs must
      have met an aperture / wedge / range edge within 1e-5 (relative) on its
      oracle path; photons whose path is the same have directions within
      max(1e-5, 1e-6 (K - 1)) rad and positions within 1e-6 f x max(1, K - 1), where K is the
      path's conditioning, the sum over its interactions of 1 / |cos(theta)|
      (theta = angle of incidence).  First-order error propagation: every
      interaction rounds the new direction to FP32, that error grows with the
      distance travelled, and a hit at incidence theta stretches it by
      1 / |cos(theta)|; a position error on a curved wall turns the next
      normal, so direction errors accumulate per redirection too.  Telescope
      paths (two or three near-normal interactions, K ~ 2-3) stay at 1e-5 rad
      and 1e-6 to 2e-6 f; concentrator paths with tens of wall reflections, or
      a grazing last hit, get the allowance their geometry implies.
"""
import numpy as np

import oracle
import workloads as W


def to_numpy(out):
    return {k: v.detach().cpu().numpy() for k, v in out.items() if v is not None}


def oracle_for(scene, bundle, precision, seed, first_photon_id=0, max_bounces=100, variant_of_photon=None):
    if precision == 32:
        b = bundle.rounded_to(np.float32)
        eps = oracle.default_eps(scene, 32)
    else:
        b = bundle
        eps = oracle.default_eps(scene, 64)
    return oracle.trace(scene, b, seed=seed, first_photon_id=first_photon_id, max_bounces=max_bounces, eps=eps,
                        variant_of_photon=variant_of_photon)


def compare(gpu, ref, precision, focal_length, label=""):
    g = to_numpy(gpu) if not isinstance(gpu["status"], np.ndarray) else gpu
    n = ref["status"].shape[0]
    f = focal_length
    report = {"n": n}
    if precision == 64:
        bad = np.where(g["status"] != ref["status"])[0]
        assert bad.size == 0, f"{label}: {bad.size} FP64 status mismatches, first ids {bad[:10]}"
        assert np.array_equal(g["bounces"], ref["bounces"]), f"{label}: FP64 bounce counts differ"
        assert np.array_equal(g["last_surface"], ref["last_surface"]), f"{label}: FP64 last surface differs"
        dh = np.abs(g["hit"] - ref["hit"]).max(initial=0.0)
        dd = np.abs(g["dir"] - ref["dir"]).max(initial=0.0)
        df = np.abs(g["focal_xy"] - ref["focal_xy"]).max(initial=0.0)
        report.update(max_dhit=float(dh), max_ddir=float(dd), max_dfocal=float(df))
        assert dh <= 1e-10 * f, f"{label}: FP64 hit error {dh} > 1e-10 f"
        assert dd <= 1e-10, f"{label}: FP64 direction error {dd}"
        assert df <= 1e-10 * f, f"{label}: FP64 focal error {df}"
        return report
    same_status = g["status"] == ref["status"]
    same_path = same_status & (g["bounces"] == ref["bounces"]) & (g["last_surface"] == ref["last_surface"])
    frac = 1.0 - same_status.mean()
    report["status_mismatch_frac"] = float(frac)
    report["path_mismatches"] = int((~same_path).sum())
    assert frac <= 1e-5 or (~same_status).sum() <= 1, f"{label}: FP32 status mismatch fraction {frac}"
    bad = np.where(~same_path)[0]
    if bad.size:
        m = ref["edge_margin"][bad]
        assert np.all(m <= 1e-5), f"{label}: FP32 path mismatch away from any edge: ids {bad[m > 1e-5][:10]}, " \
                                  f"margins {m[m > 1e-5][:10]}"
    ok = same_path
    allow = 1e-6 * f * np.maximum(1.0, ref["cond"] - 1.0)
    eh = np.abs(g["hit"].astype(np.float64) - ref["hit"]).max(axis=0)
    ed = np.abs(g["dir"].astype(np.float64) - ref["dir"]).max(axis=0)
    ef = np.abs(g["focal_xy"].astype(np.float64) - ref["focal_xy"]).max(axis=0)
    det = ok & (ref["status"] == W.DETECTED)
    report.update(max_dhit=float(eh[ok].max(initial=0.0)), max_ddir=float(ed[ok].max(initial=0.0)),
                  max_dfocal=float(ef[det].max(initial=0.0)),
                  max_dhit_over_allowance=float((eh[ok] / allow[ok]).max(initial=0.0)))
    worst = np.argmax(np.where(ok, eh / allow, 0.0))
    assert np.all(eh[ok] <= allow[ok]), \
        f"{label}: FP32 hit error {eh[worst]} > {allow[worst]} (photon {worst}, {ref['bounces'][worst]} bounces)"
    dallow = np.maximum(1e-5, 1e-6 * (ref["cond"] - 1.0))
    worst_d = np.argmax(np.where(ok, ed / dallow, 0.0))
    report["max_ddir_over_allowance"] = float((ed[ok] / dallow[ok]).max(initial=0.0))
    assert np.all(ed[ok] <= dallow[ok]), \
        f"{label}: FP32 direction error {ed[worst_d]} > {dallow[worst_d]} (photon {worst_d}, " \
        f"{ref['bounces'][worst_d]} bounces, K = {ref['cond'][worst_d]:.1f})"
    assert np.all(ef[det] <= allow[det]), f"{label}: FP32 focal error {ef[det].max()}"
    return report
