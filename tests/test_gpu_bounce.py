"""GPU parity of the double-bounce paths (Sec. 2.2: forward and backward
rays joined through two facets; geometric optics at the first facet,
physical optics at the second): the CUDA path through the C-ABI against the
FP64 oracle.

Bars: the virtual facets (TX, first facet, second facet, side) identical
as a set, their vertices, image sources, velocities and weights equal to
1e-12 (both sides take every decision with one IEEE rounding per operation
in the same order); the FP64 ADC with double bounce <= 1e-9 relative L2,
the mixed and spectral ADC <= 1e-4 (the double-bounce terms are FP64 on
every path); the dihedral's closed form through the C-ABI.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2208_10939_gb300 as pkg
import scenegen as sg

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9
TOL_MIXED = 1e-4


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ground_plate_scene(blocker=False, reverse_ground=False, P=1, Q=2, tdm=False):
    """Two big ground triangles (optionally wound the other way and
    two-sided), a 0.2 m plate 10 m out and 0.5 m up moving toward the
    radar, optionally a small plate across the ground -> plate leg."""
    tris = [[0, 2, 1], [0, 3, 2]] if reverse_ground else [[0, 1, 2], [0, 2, 3]]
    g = sg.Mesh(np.array([[-50, -50, 0], [50, -50, 0], [50, 50, 0], [-50, 50, 0]], float),
                np.array(tris, np.int32), np.ones(2, np.float32), "gnd", two_sided=reverse_ground)
    radar = sg.make_radar(128, 4, P, Q, 5.12e6, 30e12, tx_spacing_wl=2.0,
                          centre=(0.0, 0.0, 1.5), tdm=tdm)
    radar.double_bounce = True
    meshes = [g, sg.plate(0.2, 0.2, 2)]
    insts = [sg.Instance(0, (0, 0, 0), np.eye(3), (0, 0, 0)),
             sg.Instance(1, (0.0, 10.0, 0.5), np.eye(3), (0.0, -5.0, 0.0))]
    if blocker:
        meshes.append(sg.plate(0.4, 0.3, 1))
        rx = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], float)
        insts.append(sg.Instance(2, (0.02, 7.75, 0.05), rx, (0, 0, 0)))
    return sg.Scene(meshes, insts, radar, name="ground_plate")


def fine_ground_scene():
    """A 0.125 m ground grid under the plate: each plate facet is split
    among several ground facets' beams (multi-vertex clips)."""
    s = ground_plate_scene()
    s.meshes[0] = sg.ground(2.0, 16, centre=(0.0, 7.5))
    return s


CASES = {
    "dihedral": lambda: sg.dihedral_scene(range_m=6.0, size=0.1, n=2, speed=-3.0),
    "dihedral_tdm_30deg": lambda: sg.dihedral_scene(range_m=5.0, size=0.12, n=3, alpha_deg=30.0,
                                                    P=2, Q=2, speed=2.0),
    "ground_plate_blocked": lambda: ground_plate_scene(blocker=True),
    "ground_reverse_tdm": lambda: ground_plate_scene(reverse_ground=True, P=2, tdm=True),
    "fine_ground": fine_ground_scene,
    "car_ground": lambda: sg.car_ground_scene(ntri=1500, ground_n=6, M=128, N=4, P=2, Q=2),
    # the bench's ground cells (0.5 m) under a 5000-triangle car: ~19k virtual facets
    "car_ground_fine": lambda: sg.car_ground_scene(ntri=5000, ground_size=12.0, ground_n=24,
                                                   M=128, N=4, P=2, Q=2),
}
_cache = {}


def case(name):
    if name not in _cache:
        sc = CASES[name]()
        fr = oracle.Frame(sc)
        _cache[name] = (sc, fr, fr.adc_full())
    return _cache[name]


@pytest.fixture(scope="module")
def sim():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    s = pkg.Simulator(0)
    yield s
    s.close()


def _sorted(v):
    pab = v["pab"]
    order = np.lexsort((pab[:, 2], pab[:, 1], pab[:, 0]))     # stable: fan order kept
    return {k: a[order] for k, a in v.items()}


@pytest.mark.parametrize("name", list(CASES))
def test_virtual_facets_match_oracle(sim, name):
    sc, fr, _ = case(name)
    sim.load_scene(sc)
    sim.simulate(pkg.PATH_FP64)
    g = _sorted(sim.bounce_facets())
    o = _sorted(fr.bounce)
    assert o["w"].shape[0] > 0
    np.testing.assert_array_equal(g["pab"], o["pab"])
    for k in ("tri", "src", "usrc", "w"):
        scale = max(1.0, float(np.abs(o[k]).max()))
        np.testing.assert_allclose(g[k], o[k], rtol=0, atol=1e-12 * scale, err_msg=k)
    print(f"{name}: {o['w'].shape[0]} virtual facets, "
          f"{len(set(map(tuple, o['pab'][:, :3])))} (TX, a, b) pairs")


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_adc_with_double_bounce_matches_oracle(sim, name):
    sc, fr, ref = case(name)
    sim.load_scene(sc)
    adc, st = sim.simulate(pkg.PATH_FP64, stats=True)
    x = adc.cpu().numpy()
    e = rel_l2(x, ref)
    print(f"{name}: FP64 relL2 {e:.3e}")
    assert e <= TOL_FP64
    # the double-bounce part alone
    bpart = fr.bounce_entries(np.argwhere(np.ones(ref.shape, bool))).reshape(ref.shape)
    assert np.linalg.norm(bpart) > 1e-3 * np.linalg.norm(ref)
    # counters: virtual facets, and records whose second facet the RX sees
    assert st["n_bounce_facets"] == fr.bounce["w"].shape[0]
    r = sc.radar
    pab = fr.bounce["pab"]
    n_rec = 0
    for p in range(r.P):
        for q in range(r.Q):
            sel = pab[:, 0] == p
            want = np.where(pab[sel, 3] > 0, oracle.LIT, oracle.LIT_REV)
            n_rec += int((fr.state[r.P + q, pab[sel, 2]] == want).sum())
    assert st["n_bounce_terms"] == n_rec * r.N * r.M


@pytest.mark.parametrize("name,path", [
    (n, p) for n in ("dihedral", "dihedral_tdm_30deg", "fine_ground", "car_ground",
                     "car_ground_fine")
    for p in (pkg.PATH_MIXED, pkg.PATH_SPECTRAL)] + [("ground_reverse_tdm", pkg.PATH_MIXED)])
def test_fp32_paths_with_double_bounce_match_oracle(sim, name, path):
    sc, fr, ref = case(name)
    sim.load_scene(sc)
    x = sim.simulate(path).cpu().numpy()
    e = rel_l2(x, ref)
    print(f"{name} path {path}: relL2 {e:.3e}")
    assert e <= TOL_MIXED


@pytest.mark.parametrize("name", ["dihedral_tdm_30deg", "fine_ground", "car_ground",
                                  "car_ground_fine"])
@pytest.mark.parametrize("path", [pkg.PATH_MIXED, pkg.PATH_SPECTRAL])
def test_fp32_double_bounce_part_matches_oracle(sim, name, path):
    """The double-bounce part alone (the cube with double bounce minus the
    cube without, the single-bounce part being the same launch sequence in
    both) against the oracle's double-bounce entries: the FP64 records and
    FP32 phasors of the mixed and spectral paths within 1e-4 of that part."""
    sc, fr, ref = case(name)
    bref = fr.bounce_entries(np.argwhere(np.ones(ref.shape, bool))).reshape(ref.shape)
    sim.load_scene(sc)
    on = sim.simulate(path).cpu().numpy().astype(np.complex128)
    sc.radar.double_bounce = False
    try:
        sim.load_scene(sc)
        off = sim.simulate(path).cpu().numpy().astype(np.complex128)
    finally:
        sc.radar.double_bounce = True
    e = rel_l2(on - off, bref)
    print(f"{name} path {path}: double-bounce part relL2 {e:.3e}")
    assert e <= TOL_MIXED


def test_dihedral_closed_form_through_the_c_abi(sim):
    """A 0.1 m dihedral 300 m out on its bisector, monostatic: the
    double-bounce part of every ADC sample (the frame with double bounce
    minus the frame without) has the radar-equation magnitude of the
    cross-section 8 pi A^4 / lambda^2, |x| = sqrt(8 pi) A^2 / ((4 pi)^1.5 R^2)
    at every frequency of the sweep (lambda cancels); the near-field
    curvature across the 0.14 m opening at 300 m is below 1e-3 of it."""
    A, R = 0.1, 300.0
    sc = sg.dihedral_scene(range_m=R, size=A, n=2, P=1, Q=1, M=128, N=2)
    assert np.allclose(sc.radar.tx, sc.radar.rx)
    sim.load_scene(sc)
    on = sim.simulate(pkg.PATH_FP64).cpu().numpy()
    sc.radar.double_bounce = False
    sim.load_scene(sc)
    off = sim.simulate(pkg.PATH_FP64).cpu().numpy()
    db = np.abs(on - off)
    expect = math.sqrt(8 * math.pi) * A ** 2 / ((4 * math.pi) ** 1.5 * R ** 2)
    np.testing.assert_allclose(db, expect, rtol=1e-3)


def test_double_bounce_frames_are_not_graphed_and_stay_correct(sim):
    """With frame graphs on, double-bounce frames run directly (they
    synchronise once to size the virtual facets) and give the same cube."""
    sc, fr, ref = case("car_ground")
    sim.load_scene(sc)
    a = sim.simulate(pkg.PATH_FP64).cpu().numpy()
    pkg.bart_set_graph(sim.ctx, 1)
    try:
        b = sim.simulate(pkg.PATH_FP64).cpu().numpy()
        c = sim.simulate(pkg.PATH_FP64).cpu().numpy()
    finally:
        pkg.bart_set_graph(sim.ctx, 0)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)


def test_double_bounce_rejects_far_field_and_the_adjoint(sim):
    sc = sg.dihedral_scene()
    sc.radar.far_field = True
    with pytest.raises(pkg.BartError):
        sim.load_scene(sc)
    sc.radar.far_field = False
    sim.load_scene(sc)
    shape = sim.adc_shape()
    g = torch.zeros(shape, dtype=torch.complex128, device="cuda:0")
    nv = sum(sc.meshes[i.mesh_id].verts.shape[0] for i in sc.instances)
    gv = torch.empty((nv, 3), dtype=torch.float64, device="cuda:0")
    with pytest.raises(pkg.BartError):
        pkg.bart_simulate_adjoint(sim.ctx, 0.0, g, gv, None)
    sim.sync()


def test_single_bounce_frames_are_unchanged_by_the_new_field(sim):
    """double_bounce off: the cube is the single-bounce one (the field took
    the place of a reserved word)."""
    sc, fr, ref = case("dihedral")
    sc.radar.double_bounce = False
    try:
        sim.load_scene(sc)
        x = sim.simulate(pkg.PATH_FP64).cpu().numpy()
        fr0 = oracle.Frame(sc)
        assert rel_l2(x, fr0.adc_full()) <= TOL_FP64
        assert sim.bounce_facets()["w"].shape[0] == 0
    finally:
        sc.radar.double_bounce = True
