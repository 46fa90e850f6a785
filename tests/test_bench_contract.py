"""The benchmark script's host side: the reference arm's JSON line (the
oracle timed on the host cores) carries the keys the benchmark contract
names, and the flop counts used for the roofline are the algorithm's."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "cluster300_sp"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"] == "cluster300_sp"
    sys.path.insert(0, ROOT)
    import bench
    # the default workload is the 1000-atom s/p/d cluster
    assert bench.DEFAULT_WORKLOAD == "cluster1000_spd" and bench.WORKLOADS[bench.DEFAULT_WORKLOAD] == 2
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_algorithmic_flop_counts():
    """Per-interaction algorithmic flops (an FMA counts 2) grow with the
    angular momentum like the Hermite work: the distance, T and Boys terms,
    the recurrence for R_tuv (t+u+v <= L) and a dot of nherm(L) terms."""
    sys.path.insert(0, ROOT)
    import bench
    nherm = [1, 4, 10, 20, 35]
    prev = 0
    for L in range(5):
        f = bench.flops_per_interaction(L, "esp")
        # at least the dot product (2 nherm) and the Boys orders (12 (L + 1))
        assert f >= 2 * nherm[L] + 12 * (L + 1)
        assert f > prev
        prev = f
        # the Fock accumulation adds each R_tuv once instead of an FMA with D
        assert bench.flops_per_interaction(L, "fock") == f - nherm[L] - 1
    assert bench.flops_per_interaction(0, "esp") == 32 and bench.flops_per_interaction(1, "esp") == 55


def test_traffic_table_matches_the_roofline_label():
    """The DRAM traffic recorded from an ncu capture is looked up by the label
    the roofline gives its dominant class; a recorded entry must carry that
    exact label, or the bench would report traffic null."""
    sys.path.insert(0, ROOT)
    import bench
    res = {"stats": {"M": 1000, "esp_class_pairs": [0, 10, 0, 0, 0, 0], "fock_class_pairs": [0] * 6},
           "esp_cls": [0.0, 3.0, 0.0, 0.0, 0.0, 0.0], "fock_cls": [0.0] * 6}
    roof = bench._dominant(res, "mixed", 1, packed=True)
    assert ("cluster1000_spd", roof["kernel"]) in bench.NCU_TRAFFIC_BYTES
    for (workload, label), traffic in bench.NCU_TRAFFIC_BYTES.items():
        assert workload in bench.WORKLOADS and traffic > 0 and " class: " in label
