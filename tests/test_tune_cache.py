"""The tuning cache file: tuned plan configurations persist across processes.

CPU tests write entries through the library in one process and read them in another, with
the T bucket, the GPU key and malformed lines covered.  The GPU test autotunes a shape in one
process and checks that a second process takes the configuration from the file without
timing any candidate, and stays exact against the oracle.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(code, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


WRITE = """
import json
from paper_2005_09481_gb300 import xe
xe.tune_cache({path!r})
xe.tune_store("NVIDIA_GB300", 152, [(2048, 16384, 16)], 152, 256, 4)
xe.tune_store("NVIDIA_GB300", 152, [(256, 4096, 2), (512, 8192, 1)], 76, 128, 3)
print(json.dumps("ok"))
"""

READ = """
import json
from paper_2005_09481_gb300 import xe
{setup}
q = lambda g, n, s: xe.tune_lookup(g, n, s)
print(json.dumps([q("NVIDIA_GB300", 152, [(2048, 16384, 16)]),
                  q("NVIDIA_GB300", 152, [(2048, 16000, 16)]),      # same T bucket (256 blocks)
                  q("NVIDIA_GB300", 152, [(2048, 8192, 16)]),       # another bucket
                  q("NVIDIA_GB300", 148, [(2048, 16384, 16)]),      # another SM count
                  q("NVIDIA_B200", 152, [(2048, 16384, 16)]),       # another GPU
                  q("NVIDIA_GB300", 152, [(256, 4096, 2), (512, 8192, 1)]),
                  q("NVIDIA_GB300", 152, [(512, 8192, 1), (256, 4096, 2)])]))   # job order matters
"""


def test_second_process_reads_the_stored_plan(tmp_path):
    path = str(tmp_path / "tune.txt")
    _run(WRITE.format(path=path))
    want = [[152, 256, 4], [152, 256, 4], None, None, None, [76, 128, 3], None]
    assert _run(READ.format(setup=f"xe.tune_cache({path!r})")) == want
    # the environment variable names the same file
    assert _run(READ.format(setup=""), {"XE_TUNE_CACHE": path}) == want
    # without a cache nothing is known
    assert _run(READ.format(setup=""), {"XE_TUNE_CACHE": ""}) == [None] * 7


def test_malformed_lines_are_skipped_and_later_lines_win(tmp_path):
    path = tmp_path / "tune.txt"
    path.write_text("garbage\n"
                    "xe-tune 1 NVIDIA_GB300 152 1 1 2048 256 16 100 152 256 4\n"
                    "xe-tune 1 NVIDIA_GB300 152 1 1 2048 256 16 100 152 300 4\n"       # bad tile width
                    "xe-tune 1 NVIDIA_GB300 152 1 1 2048 256 16 100 152 256 9\n"       # bad schedule
                    "xe-tune 2 NVIDIA_GB300 152 1 1 2048 256 16 100 152 128 1\n"       # unknown version
                    "xe-tune 1 NVIDIA_GB300 152 1 1 2048 256\n"                        # truncated
                    "xe-tune 1 NVIDIA_GB300 152 1 1 2048 256 16 100 100 128 2\n")      # later wins
    got = _run(READ.format(setup=f"xe.tune_cache({str(path)!r})"))
    assert got[0] == [100, 128, 2] and got[1] == [100, 128, 2]


def test_bad_arguments_are_refused():
    from paper_2005_09481_gb300 import xe
    with pytest.raises(xe.XeError):
        xe.tune_store("NVIDIA GB300", 152, [(64, 64, 1)], 152, 256, 1)     # blank in the name
    with pytest.raises(xe.XeError):
        xe.tune_store("NVIDIA_GB300", 152, [(64, 64, 1)], 152, 200, 1)     # tile width
    with pytest.raises(xe.XeError):
        xe.tune_store("NVIDIA_GB300", 152, [(64, 64, 1)], 152, 256, 5)     # schedule


TUNE_GPU = """
import json, torch
from paper_2005_09481_gb300 import synth, xe
import oracle
N, T, C = 640, 4096, 3
h = synth.uniform(N, T, C, seed=5)
xe.set_option("autotune", 1)
out = xe.correlate(torch.from_numpy(h).cuda(), N, T, C)
torch.cuda.synchronize()
xe.device_status()
exact = bool(np.array_equal(out.cpu().numpy(), oracle.correlate_dense(h, N, T, C)))
print(json.dumps({{"stats": xe.tune_stats(), "cfg": xe.last_config(), "exact": exact}}))
""".replace("import json, torch", "import json, torch\nimport numpy as np")


@pytest.mark.gpu
def test_autotuned_plan_is_reused_by_a_new_process(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    path = str(tmp_path / "tune.txt")
    a = _run(TUNE_GPU.format(), {"XE_TUNE_CACHE": path})
    assert a["exact"] and a["stats"][0] > 0 and a["stats"][1] == 0
    assert open(path).read().startswith("xe-tune 1 ")
    b = _run(TUNE_GPU.format(), {"XE_TUNE_CACHE": path})
    assert b["exact"] and b["stats"] == [0, 1]
    assert b["cfg"] == a["cfg"]
