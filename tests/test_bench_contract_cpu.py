"""The benchmark's reference arm (the FP64 oracle on the host cores) prints the one JSON line
the benchmark contract asks for; it needs no GPU, so it is checked here on a tiny budget."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                          "--ref-budget-s", "2"], cwd=ROOT, capture_output=True, text=True, timeout=600, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    r = json.loads(lines[0])
    assert r["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in r, key
    assert r["steps"] == 2 and r["warmup"] == 3 and r["value"] > 0
    assert r["unit"] == "images/s" and r["higher_is_better"] is True
    assert r["cpu_baseline"]["kind"] == "oracle" and r["cpu_baseline"]["value"] == r["value"]
    assert r["cpu_baseline"]["cores"] >= 1
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert r["config"]["workload"]


def test_warmup_below_three_is_refused():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "2"],
                         cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode != 0


def test_reference_arm_other_ranks_exit_quietly():
    # under torchrun only rank 0 runs and prints the reference line; the others exit 0 at once
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2",
                          "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_pair_census_classes_on_a_single_unit():
    # one 8 x 4-pixel unit at s = 3 (288 samples, box [-0.1467, 0.1467] x [-0.0667, 0.0667] at
    # 0.04"): subhalos placed at known box distances in units of max(tau, 1) Rs land in the
    # near (< 7), 6-term (< 20), 4-term (< 40) and 3-term classes, each pair counted once; the
    # far-field census moves the unmarked ones to 64 node evaluations
    import numpy as np
    from paper_2606_01547_gb300 import workloads as W
    bench = _bench()
    Rs, tau = 0.002, 5.0
    half = (8 * 3 - 1) / 2 * (0.04 / 3)              # box half-width in x
    rho = [2.0, 10.0, 30.0, 60.0]                     # box distances / (tau Rs)
    cx = np.array([half + r * tau * Rs for r in rho], np.float32)
    sub = np.stack([cx, np.zeros(4, np.float32), np.full(4, Rs, np.float32),
                    np.full(4, 1e-3, np.float32), np.full(4, tau * Rs, np.float32)])
    system = W.LensSystem(W.Grid(8, 4, 3, 0.04), [], sub, ("SERSIC", [1.0, 0.1, 1.0, 0.0, 0.0]))
    c = bench.pair_census(system)
    assert c["pairs"] == 288 * 4 == system.pairs()
    assert all(abs(c["fractions"][k] - 0.25) < 1e-12 for k in ("near", "series6", "series4", "series3"))
    assert abs(c["flops_per_pair"] - sum(bench.FLOPS_BY_FORM.values()) / 4) < 1e-12
    # kappa = 3: 3 x the box's larger half-width is 0.44"; only the 60 tau Rs subhalo (0.60") is
    # that far (the 4-term one sits at 0.30"), and it costs 64 node evaluations, not 288 pairs
    f = bench.pair_census(system, kappa=3.0)
    assert f["interpolated_pairs"] == 288
    assert f["pairs"] == 288 * 3 + 64


def test_pair_census_on_the_benchmark_image_and_the_far_field():
    import numpy as np
    from paper_2606_01547_gb300 import workloads as W
    bench = _bench()
    system = W.substructure_system(3, n_sub=2000, nx=48, s=3, k=0)
    c0 = bench.pair_census(system)
    assert c0["pairs"] == system.pairs()
    assert abs(sum(c0["fractions"].values()) - 1.0) < 1e-12
    assert 15 <= c0["flops_per_pair"] <= 46
    c3, c6 = bench.pair_census(system, 3.0), bench.pair_census(system, 6.0)
    assert 0 < c6["interpolated_pairs"] <= c3["interpolated_pairs"] < system.pairs()
    assert c3["pairs"] < c6["pairs"] < c0["pairs"]
    assert c3["flops"] < c0["flops"]


def test_kernel_hash_ignores_comments_but_not_code():
    # the stored profile traffic is matched to the trace kernel by this hash: a comment edit keeps
    # the capture valid, any change of code invalidates it
    sys.path.insert(0, ROOT)
    import bench
    src = "// header\n__device__ float f(float x) {  /* a\n block */\n  return x * 2.f;  // twice\n}\n\n"
    same = "__device__ float f(float x) {\n  return x * 2.f;   // doubled\n}\n"
    other = "__device__ float f(float x) {\n  return x * 3.f;\n}\n"
    assert bench._code_only(src) == bench._code_only(same)
    assert bench._code_only(src) != bench._code_only(other)
    assert "//" not in bench._code_only(src) and "/*" not in bench._code_only(src)
    assert len(bench.kernel_hash()) == 16
