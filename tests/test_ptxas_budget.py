"""Register and spill budget of the kernels the headline frame times.

Compiles the translation units with the library's own flags plus
``-Xptxas -v`` (nvcc cross-compiles for sm_103a without a GPU) and reads
what ptxas prints per entry function:

* the mixed-path synthesis at 8 and 16 samples per lane runs eight 64-thread
  CTAs per SM, so it must fit 128 registers a thread; it and the other
  kernels of the frame (kinematics rows, visibility, the spectral path, the
  power-of-two range and Doppler passes at the headline's 512 x 256) must
  not spill.
"""
import os
import re
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

from paper_2208_10939_gb300 import _build

pytestmark = pytest.mark.slow

# (translation unit, demangled-name regex, register limit or None)
BUDGET = [
    ("synth.cu", r"synth_mixed_kernel<16, \d+>", 128),
    ("synth.cu", r"synth_mixed_kernel<8, \d+>", 128),
    ("synth.cu", r"kin_coef_kernel\(", None),
    ("synth.cu", r"synth_reduce_kernel\(", None),
    ("spectral.cu", r"synth_spectral_kernel\(", None),
    ("visibility.cu", r"visibility_kernel\(", None),
    ("rdm.cu", r"range_fft_reg_kernel<512>", None),
    ("rdm.cu", r"doppler_sum_tma_kernel<256>", None),
]


def _ptxas_report(src: str, out_dir: str) -> dict:
    """{demangled entry name: (registers, spill store bytes, spill load bytes)}."""
    obj = os.path.join(out_dir, os.path.basename(src) + ".o")
    cmd = [_build.nvcc(), "-c", src, "-o", obj] + _build._flags() + ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    spills, regs, cur = {}, {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Function properties for (\S+)", line) or \
            re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            cur = m.group(1)
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and cur:
            spills[cur] = (int(m.group(1)), int(m.group(2)))
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            regs[cur] = int(m.group(1))
    names = sorted(regs)
    demangled = subprocess.run(["c++filt"] + names, capture_output=True, text=True,
                               check=True).stdout.splitlines()
    return {d: (regs[n],) + spills.get(n, (0, 0)) for n, d in zip(names, demangled)}


@pytest.fixture(scope="module")
def reports(tmp_path_factory):
    if shutil.which("c++filt") is None:
        pytest.skip("c++filt not available")
    try:
        _build.nvcc()
    except RuntimeError as e:
        pytest.skip(str(e))
    out = str(tmp_path_factory.mktemp("ptxas"))
    units = sorted({u for u, _, _ in BUDGET})
    with ThreadPoolExecutor(max_workers=len(units)) as ex:
        res = ex.map(lambda u: _ptxas_report(os.path.join(_build.CSRC, u), out), units)
    return dict(zip(units, res))


@pytest.mark.parametrize("unit,pattern,reg_limit", BUDGET,
                         ids=[p for _, p, _ in BUDGET])
def test_hot_kernels_fit_their_register_budget_without_spills(reports, unit, pattern, reg_limit):
    found = {n: v for n, v in reports[unit].items() if re.search(pattern, n)}
    assert found, f"no entry function matching {pattern} in {unit}"
    for name, (regs, st, ld) in found.items():
        assert st == 0 and ld == 0, f"{name}: {st} bytes spill stores, {ld} loads"
        if reg_limit is not None:
            assert regs <= reg_limit, f"{name}: {regs} registers > {reg_limit}"
