"""Failure detection without a GPU fault.  A device allocation made to fail on
the host (bart_inject_alloc_failure) surfaces as BART_ENOMEM from
bart_simulate_frame with the failing buffer named, whichever allocation of
the frame fails, and the context stays usable afterwards.  A bounded device
wait that expires (an mbarrier nothing completes, by design) surfaces as
BART_ETIMEOUT from bart_sync, and the context stays usable."""
import numpy as np
import pytest
import torch

import paper_2208_10939_gb300 as pkg
import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("path", [pkg.PATH_MIXED, pkg.PATH_FP64])
def test_enomem_propagates_from_every_allocation_of_a_frame(path):
    sc = sg.small_car_scene(ntri=600, M=64, N=4, P=2, Q=2)
    failures = []
    for nth in range(1, 200):
        sim = pkg.Simulator(0)
        try:
            sim.load_scene(sc)                       # uploads allocate before arming
            pkg.bart_inject_alloc_failure(nth)
            try:
                adc = sim.simulate(path)
            except pkg.BartError as e:
                assert e.code == pkg.BART_ENOMEM, e
                assert "injected failure" in str(e)
                failures.append(str(e).split(" for ")[1].split(" failed")[0])
                pkg.bart_inject_alloc_failure(0)
                again = sim.simulate(path)           # the context is still usable
                sim.sync()
                assert torch.isfinite(torch.view_as_real(again)).all()
                continue
            pkg.bart_inject_alloc_failure(0)
            sim.sync()
            assert torch.isfinite(torch.view_as_real(adc)).all()
            break                                    # nth beyond the frame's allocations
        finally:
            pkg.bart_inject_alloc_failure(0)
            sim.close()
    assert len(failures) >= 10, failures
    print(f"path {path}: {len(failures)} allocations, each failure reported: {failures}")


def test_static_rdm_allocates_nothing_even_when_allocation_would_fail():
    O, N, M = 2, 32, 64
    adc = torch.randn((O, N, M), dtype=torch.complex64, device="cuda")
    rdm = torch.empty((M, N), dtype=torch.float32, device="cuda")
    pkg.bart_form_rdm_static(adc, rdm, O, N, M)
    pkg.bart_inject_alloc_failure(1)
    try:
        pkg.bart_form_rdm_static(adc, rdm, O, N, M)   # would fail if it allocated
        torch.cuda.synchronize()
        assert torch.isfinite(rdm).all()
    finally:
        pkg.bart_inject_alloc_failure(0)


def test_bounded_wait_expiry_reports_etimeout_and_the_context_stays_usable():
    """The bounded device waits' expiry path, exercised on purpose: a block
    waits a few thousand polls on an mbarrier that nothing completes (the
    mechanism the TMA-fed Doppler pass uses for its tile copies).  The wait
    ends, bart_sync reports BART_ETIMEOUT once, and the same context then
    forms an RDM that matches the oracle (the TMA Doppler pass included)."""
    import oracle
    sc = sg.small_car_scene(ntri=400, M=64, N=32, P=2, Q=2)
    sim = pkg.Simulator(0)
    try:
        sim.load_scene(sc)
        pkg.bart_selftest_wait_timeout(sim.ctx, 4096)
        with pytest.raises(pkg.BartError) as ei:
            sim.sync()
        assert ei.value.code == pkg.BART_ETIMEOUT, ei.value
        sim.sync()                                   # the status was cleared
        adc = sim.simulate(pkg.PATH_FP64)
        rdm = sim.rdm(adc.to(torch.complex64).contiguous()).cpu().numpy()
        sim.sync()
        ref = oracle.range_doppler_map(adc.cpu().numpy().astype(np.complex64).astype(np.complex128))
        assert np.abs(rdm - ref).max() <= 1e-5 * ref.max()
    finally:
        sim.close()
