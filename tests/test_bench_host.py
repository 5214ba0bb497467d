"""Host-side pieces of the benchmark: the oracle-geometry window counts the
reference arm extrapolates with (the fine level's cone of a cold 4096^2
metres query against the closed form of Lemma 4), the conv traffic
record's tie to the kernel source, and the reference arm's JSON line."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def test_fine_cone_of_the_benchmark_query_matches_the_closed_form():
    # the decode reads the residual over the query plus a halo of 128 px on
    # each side: 4352^2 px from -128, n = 68 aligned tiles of 64 px per side;
    # a cold query of an aligned n-tile region needs sum_{k<K} (n + 2k + 1)^2
    # windows at window = 2 x stride (Lemma 4)
    st = synth.config2_stack()
    nf, nc = bench.oracle_window_counts(st, 4096)
    n = (4096 + 2 * 128) // 64
    closed = sum((n + 2 * k + 1) ** 2 for k in range(20))
    assert nf == closed == 157540
    assert 0 < nc < nf


def test_traffic_record_is_tied_to_the_conv_source_and_precision():
    rec = json.load(open(os.path.join(ROOT, "profiles", "conv_tc_traffic.json")))
    src = open(os.path.join(ROOT, "paper_2512_08309_gb300", "csrc", "conv_tc.cu"), "rb").read()
    live = rec["source_sha256"] == hashlib.sha256(src).hexdigest()
    got = bench.traffic_record(rec["precision"])
    assert (got is not None) == live
    assert bench.traffic_record("bf16x3" if rec["precision"] != "bf16x3" else "tf32") is None


def test_reference_arm_prints_one_contract_line():
    # the reference arm (the FP64 oracle on the host cores) on a short sample:
    # one JSON line with the keys the measurement contract names, and no
    # import of the library
    import subprocess
    # (run in a child that also checks that the arm never imported the library)
    code = ("import runpy, sys\n"
            "sys.argv = ['bench.py', '--impl', 'reference', '--steps', '2', '--warmup', '1', '--ref-seconds', '0.2']\n"
            "try:\n"
            "    runpy.run_path('bench.py', run_name='__main__')\n"
            "except SystemExit as e:\n"
            "    assert not e.code, e.code\n"
            "assert 'paper_2512_08309_gb300' not in sys.modules, 'the reference arm imported the library'\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "px/s" and d["higher_is_better"] is True
    assert d["ms_per_step"] > 0 and "extrapolated" in d["ms_per_step_kind"]
    assert d["e2e"] == {"value": d["value"], "unit": "px/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["config"]["workload"] and d["dtype"] == "f64" and d["data"] == "synthetic"
