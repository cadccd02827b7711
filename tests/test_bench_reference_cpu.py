"""The benchmark's reference arm (the oracle timed on the host's cores) runs
without a GPU and prints one JSON line with the keys the bench contract needs."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                        "--ref-photons-per-angle", "300"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"]


def test_accuracy_block_of_the_bench_measures_errors_against_the_oracle():
    """The bench's per-form accuracy block: per-photon position / direction errors on the photons
    whose path is the same, status mismatches, and per-window relative errors of R80, effective
    area (detected count) and collection efficiency."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(0)
    n = 2000
    r = {"status": np.ones(n, np.uint8), "bounces": np.full(n, 2, np.uint8), "hit": rng.normal(size=(3, n)),
         "dir": rng.normal(size=(3, n)), "last_surface": np.zeros(n, np.int32),
         "focal_xy": rng.normal(0, 0.01, size=(2, n)), "edge_margin": np.ones(n)}
    g = {k: v.copy() for k, v in r.items() if k != "edge_margin"}
    rep = bench._compare(g, r, 32, 2.0, [(0, 1000), (1000, 1000)])
    assert rep["max_pos_err_over_f"] == 0 and rep["max_dir_err_rad"] == 0 and rep["status_mismatch_frac"] == 0
    assert rep["r80_rel_err_max"] == 0 and rep["a_eff_rel_err_max"] == 0 and rep["ce_rel_err_max"] == 0
    g["hit"][1, 17] += 3e-6       # 1.5e-6 f
    g["dir"][2, 5] -= 2e-5
    g["status"][1500] = 3         # one photon lost in the second window
    g["bounces"][1500] = 1
    r["edge_margin"][1500] = 4e-6
    rep = bench._compare(g, r, 32, 2.0, [(0, 1000), (1000, 1000)])
    assert abs(rep["max_pos_err_over_f"] - 1.5e-6) < 1e-12
    assert abs(rep["max_dir_err_rad"] - 2e-5) < 1e-12
    assert abs(rep["status_mismatch_frac"] - 1 / n) < 1e-15 and rep["path_mismatches"] == 1
    assert rep["path_mismatch_max_edge_margin"] == 4e-6
    assert abs(rep["a_eff_rel_err_max"] - 1 / 1000) < 1e-12 and abs(rep["ce_rel_err_max"] - 1 / 1000) < 1e-12
