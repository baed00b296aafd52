"""The oracle arm of bench.py (``--impl reference``) on CPU: one JSON line
with the contract's keys, on the sedan workload; under torchrun with two
ranks only rank 0 runs and prints, and both ranks exit 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["bench.py", "--impl", "reference", "--workload", "sedan", "--steps", "1",
        "--warmup", "0"]
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
        "cpu_baseline", "e2e"}

pytestmark = pytest.mark.slow


def _json_lines(out: str):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _check_line(line):
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["vs_baseline"] is None and line["higher_is_better"] is True


def test_reference_arm_single_process():
    r = subprocess.run([sys.executable] + ARGS, cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0])


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + ARGS + ["--gpus", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0])
    assert lines[0]["n_gpus"] == 2


def test_cpu_baseline_leg_reports_all_cores_and_one():
    """bench.py's cpu_baseline leg on a small frame: the oracle's rate on
    all host cores and on one, and the sampled entries' error of a cube
    (here the oracle's own cube, so zero)."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import scenegen as sg
    sc = sg.small_car_scene(ntri=600, M=64, N=4, P=2, Q=2)
    cube = oracle.Frame(sc).adc_full()
    out = bench.cpu_baseline(sc, 0.5, cube)
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] == oracle.num_threads()
    assert out["one_core"]["cores"] == 1 and out["one_core"]["value"] > 0
    assert out["gpu_frame_rel_l2_vs_oracle"] == 0.0
    assert oracle.num_threads() == out["cores"]          # the thread count is restored
