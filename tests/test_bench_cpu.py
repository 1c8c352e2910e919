"""bench.py's reference arm (the FP64 CPU oracle, parallel over pairs) keeps
the JSON-line contract on a small workload; no GPU involved."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny",
                          "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "pairs/s"
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["value"] > 0 and line["value"] == line["cpu_baseline"]["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and "pairs" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("tiny")


def _bench_module():
    import importlib
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        sys.path.insert(0, ROOT)
        return importlib.import_module("bench")
    finally:
        sys.argv = saved


def test_algorithmic_counts_match_the_workload_table():
    """bench.py's algorithmic FP64 flops, mixable flops and input bytes per
    forward pass against the workload table's figures for the two chains
    (C40H81: 2.8e11 / 1.0e11 flops, 21 GB; C160H321: 2.9e12 / 1.0e12 flops,
    177 GB), which were summed from the size distributions independently."""
    bench = _bench_module()
    for name, f64, mix, byts in (("c40h81", 2.8e11, 1.0e11, 21e9),
                                 ("c160h321", 2.9e12, 1.0e12, 177e9)):
        wl = bench.make_workload(name, 0)
        a, b, c = (float(x.sum()) if hasattr(x, "sum") else float(x) for x in bench.flops_bytes(wl))
        assert abs(a / f64 - 1) < 0.05, (name, a)
        assert abs(b / mix - 1) < 0.05, (name, b)
        assert abs(c / byts - 1) < 0.05, (name, c)


def test_traffic_is_reported_only_for_the_captured_kernel():
    """roofline.traffic scales the ncu capture of the same kernel variant and
    precision by algorithmic bytes; any other kernel reports null."""
    import argparse
    bench = _bench_module()
    (variant, cap), = bench.TRAFFIC_CAPTURE.items()
    args = argparse.Namespace(precision=cap["precision"], stream_gb=0, augment_somo=False)
    assert bench.traffic_bytes(args, None, cap["alg_bytes"], variant) == cap["bytes"]
    assert bench.traffic_bytes(args, None, 2 * cap["alg_bytes"], variant) == 2 * cap["bytes"]
    assert bench.traffic_bytes(args, None, cap["alg_bytes"], variant + 1) is None
    args.precision = "fp64"
    assert bench.traffic_bytes(args, None, cap["alg_bytes"], variant) is None
    args.precision, args.stream_gb = cap["precision"], 40
    assert bench.traffic_bytes(args, None, cap["alg_bytes"], variant) is None
