"""Host-side helpers of bench.py: the code-only source hash that ties the committed ncu
summary to the correlation kernel, and the traffic figure it gates."""
import json
import os

import bench

SRC = {
    "xe_tc.cu": 'asm volatile("tcgen05.commit // not a comment");\nint a = 1; // comment\n',
    "xe_ptx.cuh": "/* block\n comment */ int b = 2;\n",
    "xe_internal.h": "constexpr int c = '/';\n",
}


def test_code_of_drops_comments_and_whitespace_keeps_literals():
    assert bench.code_of('x = 1; // c\n/* d\n e */ y  =\t2;') == "x=1;y=2;"
    assert bench.code_of('s = "a // b /* c */";') == 's="a//b/*c*/";'
    assert bench.code_of("c = '/'; // x") == "c='/';"
    assert bench.code_of('s = "q\\"//"; t = 1; // u') == 's="q\\"//";t=1;'


def test_kernel_hash_ignores_comments_and_layout_but_not_code():
    h = bench.kernel_hash(SRC)
    edited = dict(SRC)
    edited["xe_tc.cu"] = ('asm volatile("tcgen05.commit // not a comment");  // other words\n'
                          "int a = 1;\n\n")
    assert bench.kernel_hash(edited) == h
    edited["xe_internal.h"] = "/* new */ constexpr int c = '/' ;"
    assert bench.kernel_hash(edited) == h
    for name, before, after in (("xe_tc.cu", "int a = 1", "int a = 2"),
                                ("xe_tc.cu", "// not a comment", "// changed"),
                                ("xe_ptx.cuh", "int b = 2", "int b = 3")):
        changed = dict(SRC)
        changed[name] = SRC[name].replace(before, after)
        assert bench.kernel_hash(changed) != h, (name, after)


def test_traffic_is_reported_only_for_the_profiled_source(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "tc_kernel_n2048_t32768.json")) as f:
        prof = json.load(f)
    monkeypatch.setattr(bench, "kernel_hash", lambda texts=None: prof["kernel_hash"])
    assert bench.ncu_traffic() == float(prof["dram_bytes_per_launch"])
    assert prof["dram_bytes_per_launch"] == prof["dram_bytes_read"] + prof["dram_bytes_write"]
    monkeypatch.setattr(bench, "kernel_hash", lambda texts=None: "0" * 16)
    assert bench.ncu_traffic() is None


def test_reference_arm_line_has_the_contract_keys():
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3"],
                       cwd=bench.ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0
    assert d["higher_is_better"] is True and d["vs_baseline"] is None and "workload" in d["config"]
    assert set(d["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_main_arm_fails_loudly_without_a_gpu():
    # No CPU fallback: without a CUDA device the benchmark prints no result line and exits
    # with an error.
    import subprocess
    import sys
    torch = __import__("pytest").importorskip("torch")
    if torch.cuda.is_available():
        __import__("pytest").skip("a CUDA device is present")
    r = subprocess.run([sys.executable, "bench.py", "--steps", "3", "--warmup", "3", "--no-stream",
                        "--no-masked", "--no-beams", "--no-corner", "--no-cpu-baseline"],
                       cwd=bench.ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_latency_histogram_buckets():
    from paper_2005_09481_gb300 import serve
    ms = 1_000_000
    lat = [0, 9 * ms, 10 * ms, 19.9 * ms, 45 * ms, 639 * ms, 640 * ms, 5000 * ms]
    h = serve.latency_histogram(lat)
    assert len(h) == len(serve.LATENCY_EDGES_MS)
    assert h == [2, 2, 0, 1, 0, 0, 1, 2]
    assert sum(h) == len(lat)
    assert serve.latency_histogram([]) == [0] * len(serve.LATENCY_EDGES_MS)
