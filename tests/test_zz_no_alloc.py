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


def test_static_rdm_rejects_cubes_beyond_its_workspace():
    lib = pkg.load_library()
    O, N, M = 64, 256, 256                    # 2^22 complex64 samples = 32 MiB
    dummy = torch.empty(1, dtype=torch.complex64, device="cuda")
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    rc = lib.bart_form_rdm_static(ctypes.c_void_p(dummy.data_ptr()), pkg.C64, O, N, M,
                                  pkg.WINDOW_HANN, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == pkg.BART_EINVAL
    assert b"workspace" in lib.bart_last_error()
