"""CPU checks of the C-ABI boundary: the library builds and loads, exports
every function include/bartsim.h declares, the ctypes mirrors have the C
struct layouts, and the product path fails loudly without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2208_10939_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bartsim.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bart_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_10939_gb300 import _build
    _build.build()
    return pkg.load_library()


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(pkg.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(bart_\w+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, missing
    for name in declared_functions():
        assert getattr(lib, name) is not None


MIRRORS = ["bart_instance", "bart_radar", "bart_stats", "bart_timing", "bart_detect_cfg",
           "bart_point", "bart_tune", "bart_peaks", "bart_dims"]


def test_struct_layouts_match_c(tmp_path):
    """sizeof of every mirrored struct and the offset of every field agree
    between C (gcc on the header) and the ctypes mirrors."""
    lines, expect = [], []
    for name in MIRRORS:
        cls = getattr(pkg, name)
        lines.append(f'printf("%zu\\n", sizeof({name}));')
        expect.append(ctypes.sizeof(cls))
        for field, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({name}, {field}));')
            expect.append(getattr(cls, field).offset)
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "bartsim.h"\n'
                    "int main(void){" + "".join(lines) + "return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                        check=True).stdout.split()))
    assert vals == expect


def test_version_and_error_string(lib):
    assert "sm_103a" in pkg.bart_version()
    assert lib.bart_last_error() is not None


def test_create_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pkg.BartError) as e:
        pkg.bart_create(0)
    assert e.value.code in (pkg.BART_ECUDA, pkg.BART_EINVAL)


def test_null_arguments_are_rejected(lib):
    assert lib.bart_set_stream(None, None) == pkg.BART_EINVAL
    assert lib.bart_sync(None) == pkg.BART_EINVAL
    assert lib.bart_radar_set(None, None) == pkg.BART_EINVAL
    assert b"NULL" in lib.bart_last_error()


def test_alloc_failure_injection_is_armed_and_disarmed_on_the_host(lib):
    assert lib.bart_inject_alloc_failure(-1) == pkg.BART_EINVAL
    assert lib.bart_inject_alloc_failure(3) == pkg.BART_OK
    assert lib.bart_inject_alloc_failure(0) == pkg.BART_OK
