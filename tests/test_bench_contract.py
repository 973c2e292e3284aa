"""The benchmark's CPU-side contract: the reference arm (the binary64 oracle
timed on host cores) prints one JSON line with the keys the measurement
contract asks for, other ranks print nothing, and the kernel-source hash is
stable.  No GPU is needed."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_line():
    r = _run(["--impl", "reference", "--size", "256", "--steps", "2", "--warmup", "3", "--ref-rows", "4"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "workload" in line["config"]


def test_reference_arm_config_matches_gpu_arm():
    # both arms describe the headline workload with the same config object,
    # and by default each host thread gets 8 rows of C per step
    sys.path.insert(0, ROOT)
    import bench
    r = _run(["--impl", "reference", "--size", "192", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["config"] == bench.square_config(192)
    cores = line["cpu_baseline"]["cores"]
    assert line["cpu_baseline"]["sample"].startswith(f"{8 * cores} full rows")


def test_reference_arm_other_ranks_silent():
    r = _run(["--impl", "reference", "--size", "64", "--steps", "1", "--warmup", "3"],
             {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_kernel_hash_stable():
    a = _run(["--print-kernel-hash"])
    b = _run(["--print-kernel-hash"])
    assert a.returncode == 0 and b.returncode == 0
    h = a.stdout.strip()
    assert h == b.stdout.strip() and len(h) >= 16


def test_bench_compiles_and_names_defined():
    # every module-level name the bench refers to exists (a typo in a branch
    # that only runs on a GPU would otherwise surface only there)
    import ast
    import builtins
    src = open(os.path.join(ROOT, "bench.py")).read()
    tree = ast.parse(src)
    defined = set(dir(builtins))
    for node in ast.walk(tree):
        if isinstance(node, (ast.FunctionDef, ast.ClassDef)):
            defined.add(node.name)
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            for al in node.names:
                defined.add((al.asname or al.name).split(".")[0])
        elif isinstance(node, ast.Name) and isinstance(node.ctx, (ast.Store, ast.Del)):
            defined.add(node.id)
        elif isinstance(node, ast.arg):
            defined.add(node.arg)
        elif isinstance(node, ast.ExceptHandler) and node.name:
            defined.add(node.name)
    used = {n.id for n in ast.walk(tree) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
    missing = sorted(used - defined - {"__file__", "__name__"})
    assert not missing, missing
