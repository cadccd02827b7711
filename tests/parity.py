"""Element-by-element comparison of a GPU trace with the oracle's.

Tolerances (per photon, on the same seeded inputs):
  FP64 trace: status, bounce count and last surface identical for every
      photon; final position within 1e-10 x the system focal length f; final
      direction within 1e-10; focal-plane coordinates within 1e-10 f.
  FP32 trace (the oracle traces the FP32-rounded inputs, with the FP32
      self-intersection epsilon): status identical for at least 99.999% of
      photons (at most floor(1e-5 n) mismatches, so none below 1e5 photons);
      every photon whose status, bounce count or last surface differs must
      have met an aperture / wedge / range edge within 1e-5 (relative) on its
      oracle path; every photon whose path is the same has its final position
      within 1e-6 f, its focal-plane coordinates within 1e-6 f and its final
      direction within 1e-5 rad.  These are fixed bounds; the path's
      conditioning K = sum over its interactions of 1 / |cos(incidence)| is
      reported next to the worst photons, never used to widen them.
"""
import numpy as np

import oracle
import workloads as W

POS_REL_FP32 = 1e-6   # x focal length
DIR_FP32 = 1e-5       # rad
STATUS_FRAC_FP32 = 1e-5
EDGE_FP32 = 1e-5


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
    n_status = int((~same_status).sum())
    report["status_mismatches"] = n_status
    report["path_mismatches"] = int((~same_path).sum())
    if "retraced" in g:
        report["retraced_fp64"] = [int(x) for x in np.asarray(g["retraced"]).ravel()]
    assert n_status <= int(STATUS_FRAC_FP32 * n), \
        f"{label}: {n_status} FP32 status mismatches in {n} photons (at most {int(STATUS_FRAC_FP32 * n)})"
    bad = np.where(~same_path)[0]
    if bad.size:
        m = ref["edge_margin"][bad]
        assert np.all(m <= EDGE_FP32), f"{label}: FP32 path mismatch away from any edge: ids {bad[m > EDGE_FP32][:10]}, " \
                                       f"margins {m[m > EDGE_FP32][:10]}"
    ok = same_path
    det = ok & (ref["status"] == W.DETECTED)
    eh = np.abs(g["hit"].astype(np.float64) - ref["hit"]).max(axis=0)
    ed = np.abs(g["dir"].astype(np.float64) - ref["dir"]).max(axis=0)
    ef = np.abs(g["focal_xy"].astype(np.float64) - ref["focal_xy"]).max(axis=0)
    tol_p, tol_d = POS_REL_FP32 * f, DIR_FP32
    report.update(max_dhit_over_f=float(eh[ok].max(initial=0.0) / f), max_ddir=float(ed[ok].max(initial=0.0)),
                  max_dfocal_over_f=float(ef[det].max(initial=0.0) / f))
    worst = int(np.argmax(np.where(ok, eh, -1.0)))
    assert not np.any(eh[ok] > tol_p), \
        f"{label}: FP32 hit error {eh[worst]:.3e} m > {tol_p:.3e} m = 1e-6 f (photon {worst}, " \
        f"{ref['bounces'][worst]} bounces, K = {ref['cond'][worst]:.1f}); {int((eh[ok] > tol_p).sum())} photons over"
    worst_d = int(np.argmax(np.where(ok, ed, -1.0)))
    assert not np.any(ed[ok] > tol_d), \
        f"{label}: FP32 direction error {ed[worst_d]:.3e} rad > 1e-5 rad (photon {worst_d}, " \
        f"{ref['bounces'][worst_d]} bounces, K = {ref['cond'][worst_d]:.1f}); {int((ed[ok] > tol_d).sum())} photons over"
    assert not np.any(ef[det] > tol_p), f"{label}: FP32 focal error {ef[det].max():.3e} m > 1e-6 f"
    return report
