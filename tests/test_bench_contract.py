"""bench.py host logic: the algorithmic bytes per node behind every roofline figure, and the JSON
line of the reference arm (the FP64 oracle on the host cores), which needs no GPU."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("prec,sigma,mode,expected", [
    # 9 loads + 9 stores of the storage type, delta rho read + write in the arithmetic type
    ("f32", False, 0, 18 * 4 + 2 * 4),
    ("f32", True, 0, 92),            # + the stress xx, yy, xy written every step (zz = 0 once)
    ("bf16", False, 0, 18 * 2 + 2 * 4),
    ("bf16", True, 0, 56),
    ("f64", True, 0, 18 * 8 + 2 * 8 + 3 * 8),
    ("f32", True, 1, 92 + 6 * 4),    # mode B: the carried (xx, xy, yy) stress read and written
])
def test_bytes_per_node(prec, sigma, mode, expected):
    assert load_bench().bytes_per_node(prec, sigma, mode) == expected


@pytest.mark.parametrize("prec,scheme,expected", [
    ("f32", "paper", 92),
    ("f32", "generalized_newtonian", 92),          # the same planes (delta rho stays 0)
    # first pass: populations + delta rho read, Sigma^nN (3 planes) written; the step reads Sigma^nN
    ("f32", "stress_divergence", 92 + 9 * 4 + 4 + 3 * 4 + 3 * 4),
    ("f32", "relaxation", 92 + 16),                # the FP64 fluidity read and written
    ("bf16", "relaxation", 56 + 16),
    ("f64", "stress_divergence", 184 + 9 * 8 + 8 + 3 * 8 + 3 * 8),
])
def test_bytes_per_node_of_the_schemes(prec, scheme, expected):
    assert load_bench().bytes_per_node(prec, True, 0, scheme) == expected


def test_stored_traffic_is_tied_to_the_kernel_source():
    b = load_bench()
    assert b.stored_traffic("k_step_march", "no_such_precision", 1) is None
    p = os.path.join(ROOT, "profiles", "k_step_march_f32_traffic.json")
    d = json.load(open(p))
    got = b.stored_traffic("k_step_march", "f32", 2 * d["nodes"])
    if d["kernel_hash"] == b.kernel_hash("k_step_march"):
        assert got == pytest.approx(2 * d["dram_read_bytes"] + 2 * d["dram_write_bytes"])
    else:  # counters taken on another kernel source are not reported
        assert got is None


def test_reference_arm_json_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--ref-crop", "32"], capture_output=True, text=True, cwd=ROOT, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "GLUPS" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["nx"] == 32 and line["config"]["ny"] == 32


def test_kernel_hash_covers_code_not_comments():
    b = load_bench()
    src = "int f(int a) {  // one\n    /* two\n       lines */\n    return a + 1;\n}\n"
    assert b.code_only(src) == b.code_only(src.replace("one", "uno").replace("two", "dos") + "\n// more\n")
    assert b.code_only(src) != b.code_only(src.replace("a + 1", "a + 2"))
