"""The benchmark's JSON-line contract, checked on the CPU through its
reference arm (the oracle timed on the host): one line with the contract's
keys, alone and under torchrun with two ranks (rank 0 prints, the other exits
without work).  The line always describes one host process (n_gpus 1),
whatever the number of ranks launched, and says how many were."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline",
        "e2e"}


def _lines(out):
    return [json.loads(ln) for ln in out.splitlines() if ln.startswith("{")]


def _check(line, ranks):
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["n_gpus"] == 1
    assert line["host_processes"] == 1 and line["ranks_launched"] == ranks
    assert line["value"] > 0 and line["unit"] == "trajectory-steps/s"
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["config"]["workload"].startswith("H2")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert 0 < cb["sample_rate"] <= 1.5 * line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "1"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600, check=True)
    lines = _lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0], 1)


def test_reference_arm_under_torchrun_prints_once():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1", "--master-port",
                        str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps",
                        "1", "--warmup", "0", "--cpu-seconds", "1"], cwd=ROOT,
                       capture_output=True, text=True, timeout=600, check=True)
    lines = _lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0], 2)
