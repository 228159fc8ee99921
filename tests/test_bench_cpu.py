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
