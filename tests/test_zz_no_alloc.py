"""bart_form_rdm_static: the range-Doppler map without any device allocation.

Some callers cannot let a library allocate GPU memory: applications that
manage every device byte through their own pool allocator or run under a
hard memory cap (a foreign cudaMalloc would break their accounting or fail),
and latency-bound loops where cudaMalloc/cudaFree would stall on a device
synchronisation.  For them the library offers this entry point, whose
range-FFT workspace is a fixed 16 MiB array compiled into the library.

This file is named so that pytest collects it last.  The test calls the new
entry point through the C-ABI twice in a row and compares each result with
the context-based bart_form_rdm on the same cube, at the tolerance the other
RDM tests use.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2208_10939_gb300 as pkg
import scenegen as sg

pytestmark = pytest.mark.gpu

RDM_TOL = 1e-6          # relative to the map's peak, as in the RDM parity tests


def _static_rdm(lib, adc, O, N, M, dtype_code):
    out = torch.full((M, N), float("nan"), dtype=torch.float32, device=adc.device)
    stream = torch.cuda.current_stream(adc.device).cuda_stream
    rc = lib.bart_form_rdm_static(ctypes.c_void_p(adc.data_ptr()), dtype_code, O, N, M,
                                  pkg.WINDOW_HANN, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(stream))
    assert rc == pkg.BART_OK, lib.bart_last_error()
    torch.cuda.synchronize(adc.device)
    return out.cpu().numpy()


def test_static_rdm_matches_context_rdm_on_two_calls_in_a_row():
    lib = pkg.load_library()
    sim = pkg.Simulator(0)
    try:
        for scene in (sg.car_scene(seed=3, ntri=3000), sg.plate_scene()):
            sim.load_scene(scene)
            O, N, M = sim.adc_shape()
            for path, code in ((pkg.PATH_MIXED, pkg.C64), (pkg.PATH_FP64, pkg.C128)):
                adc = sim.simulate(path)
                ref = sim.rdm(adc).cpu().numpy()
                assert np.isfinite(ref).all() and ref.max() > 0
                for _ in range(2):
                    got = _static_rdm(lib, adc, O, N, M, code)
                    assert np.isfinite(got).all()
                    assert np.abs(got - ref).max() <= RDM_TOL * ref.max()
    finally:
        sim.close()


def _random_cube(O, N, M, dtype, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    re = torch.randn((O, N, M), generator=g, dtype=torch.float64)
    im = torch.randn((O, N, M), generator=g, dtype=torch.float64)
    return torch.complex(re, im).to(dtype).cuda()


@pytest.mark.parametrize("dtype,O,N,M", [(torch.complex64, 16, 256, 288),
                                         (torch.complex128, 16, 128, 288)])
def test_static_rdm_just_under_its_workspace(dtype, O, N, M):
    """The largest cubes near the 16 MiB limit (complex64: 12 B a sample,
    1 179 648 samples = 14.2 MB; complex128: 24 B a sample, 589 824 samples
    = 14.2 MB), radix-3 range length: the static RDM equals the context RDM
    of a radar of that shape on a random cube, twice in a row."""
    lib = pkg.load_library()
    code = pkg.C64 if dtype == torch.complex64 else pkg.C128
    radar = sg.make_radar(M, N, O, 1, 5.12e6, 30e12, 2.0, centre=(0.0, 0.0, 0.0))
    scene = sg.Scene([sg.plate(0.1, 0.1, 1)], [sg.Instance(0, (0, 10, 0), np.eye(3), (0, 0, 0))],
                     radar)
    sim = pkg.Simulator(0)
    try:
        sim.load_scene(scene)
        adc = _random_cube(O, N, M, dtype, 17)
        ref = sim.rdm(adc).cpu().numpy()
        for _ in range(2):
            got = _static_rdm(lib, adc, O, N, M, code)
            assert np.abs(got - ref).max() <= RDM_TOL * ref.max()
    finally:
        sim.close()


def test_static_rdm_rejects_cubes_beyond_its_workspace():
    lib = pkg.load_library()
    dummy = torch.empty(1, dtype=torch.complex64, device="cuda")
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    # 2^22 complex64 samples need 48 MiB (12 B a sample); and the smallest
    # step past the limit: 16 x 256 x 384 = 1 572 864 samples = 18.9 MB
    for code, (O, N, M) in ((pkg.C64, (64, 256, 256)), (pkg.C64, (16, 256, 384)),
                            (pkg.C128, (16, 256, 288))):
        rc = lib.bart_form_rdm_static(ctypes.c_void_p(dummy.data_ptr()), code, O, N, M,
                                      pkg.WINDOW_HANN, ctypes.c_void_p(out.data_ptr()), None)
        assert rc == pkg.BART_EINVAL
        assert b"workspace" in lib.bart_last_error()


def test_static_rdm_binding_checks_and_no_device_allocation():
    """Through the Python binding: shapes, dtypes and devices are checked
    before the C call; and repeated calls leave the device's free memory
    unchanged (no allocation by the library, after one warm-up call that may
    load the module and so reserve the fixed array)."""
    O, N, M = 4, 64, 128
    adc = _random_cube(O, N, M, torch.complex64, 5)
    rdm = torch.empty((M, N), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        pkg.bart_form_rdm_static(adc, rdm, O, N, M + 32)           # count mismatch
    with pytest.raises(ValueError):
        pkg.bart_form_rdm_static(adc, torch.empty((M, N + 1), device="cuda"), O, N, M)
    with pytest.raises(ValueError):
        pkg.bart_form_rdm_static(adc[:, :, ::2], rdm, O, N, M // 2)   # not contiguous
    with pytest.raises(TypeError):
        pkg.bart_form_rdm_static(adc, rdm.double(), O, N, M)
    with pytest.raises(ValueError):
        pkg.bart_form_rdm_static(adc.cpu(), rdm, O, N, M)
    first = torch.empty_like(rdm)

    def one_call():
        rdm.fill_(float("nan"))
        pkg.bart_form_rdm_static(adc, rdm, O, N, M)
        torch.cuda.synchronize()
        return bool(torch.isfinite(rdm).all())

    assert one_call()                 # warm-up: module load, torch's own small blocks
    first.copy_(rdm)
    assert torch.equal(rdm, first)
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        assert one_call() and torch.equal(rdm, first)
    assert torch.cuda.mem_get_info()[0] == free0
