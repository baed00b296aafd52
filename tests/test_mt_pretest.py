"""The FP32 pre-test of the visibility and double-bounce segment tests never
contradicts the FP64 test it stands in front of (CPU only).

The visibility kernel (Sec. 2.2: facet-to-antenna rays) and the
double-bounce leg test run the FP64 Moller-Trumbore test only where an FP32
pre-test with first-order rounding bounds cannot decide; bit-exact
visibility against the oracle rests on the pre-test deciding a miss or a
hit only when the FP64 test would.  ``mt_pretest_check.cpp`` compiles both
functions from ``geom64.cuh`` unchanged as host code and compares them on
1.6M seeded segments, most of them adversarial (through points 1e-13 ..
1e-3 from an edge, ends near the plane, nearly parallel); a plain FP32 test
without the bounds gets many of the same cases wrong, which shows that they
probe the margins.  The same run checks that the FP32 slab test against the
padded, outward-rounded box never drops a segment that hits or grazes the
triangle (the hierarchy traversal may only over-report candidates); with
the pad left out, about four thousand of the 0.8M hitting or grazing
segments are dropped, so the cases reach the pad's scale."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


def test_fp32_pretest_decides_only_what_fp64_decides(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    exe = tmp_path / "mt_check"
    subprocess.run([gxx, "-O2", "-ffp-contract=off", "-std=c++17",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2208_10939_gb300", "csrc"),
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "mt_pretest_check.cpp"),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    m = re.search(r"cases (\d+) violations (\d+) decided (\d+) naive_wrong (\d+) "
                  r"slab_drops (\d+) of (\d+)", r.stdout)
    assert m, r.stdout + r.stderr
    cases, violations, decided, naive_wrong, drops, slab_cases = map(int, m.groups())
    assert violations == 0, r.stdout
    assert drops == 0 and slab_cases > 100_000, r.stdout
    assert r.returncode == 0
    assert cases == 1_600_000 and decided > 100_000
    assert naive_wrong > 10_000
