"""The JSON line of bench.py's reference arm (the CPU oracle on a bounded sample), on CPU: one process, and two
ranks under torchrun (rank 0 alone prints; the other rank exits 0 without work)."""

import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--m", "256", "--n", "2048", "--ref-rows", "128", "--steps", "3", "--warmup", "3"]


def _lines(out: str) -> list[dict]:
    return [json.loads(ln) for ln in out.splitlines() if ln.startswith("{")]


def _check_line(d: dict, n_gpus: int) -> None:
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == n_gpus and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "GCUPS" and d["higher_is_better"] is True
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_line_one_process():
    for variant in ("uniform", "mutated"):
        r = subprocess.run([sys.executable, "bench.py", *ARGS, "--variant", variant], cwd=ROOT, capture_output=True,
                           text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        lines = _lines(r.stdout)
        assert len(lines) == 1
        _check_line(lines[0], 1)
        assert ("substitutions" in lines[0]["config"]["workload"]) == (variant == "mutated")


def test_reference_line_two_ranks_gloo():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    # the launcher's own options would swallow --m / --n: the full-size strings, a sample of 128 rows per step
    args = ["--impl", "reference", "--ref-rows", "128", "--steps", "3", "--warmup", "3", "--gpus", "2"]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", *args]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1  # rank 0 only
    _check_line(lines[0], 2)
