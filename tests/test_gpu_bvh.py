"""The GPU-built hierarchy passes the host-side invariant checker
(diagnostics.check_bvh through bart_get_bvh): the 20k-facet sedan, a
partitioned batch with a one-facet scene (each scene's subtree holds exactly
its own facets), a lone facet, and the sedan on its ground patch.  The
facets the boxes enclose are the world facets the oracle computes for the
frame start."""
import numpy as np
import pytest
import torch

import oracle
import paper_2208_10939_gb300 as pkg
import scenegen as sg
from paper_2208_10939_gb300.diagnostics import check_bvh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    s = pkg.Simulator(0)
    yield s
    s.close()


def _checked(sim, scene_or_scenes, path=pkg.PATH_MIXED):
    if isinstance(scene_or_scenes, list):
        sim.load_scenes(scene_or_scenes)
    else:
        sim.load_scene(scene_or_scenes)
    sim.simulate(path)
    sim.sync()
    h = sim.bvh()
    errs = check_bvh(h["nodes"], h["roots"], h["tri"], h["foff"])
    assert errs == [], errs
    return h


def test_hierarchy_is_unavailable_before_a_frame():
    s = pkg.Simulator(0)
    try:
        s.load_scene(sg.plate_scene(n=2, M=64, N=2))
        with pytest.raises(pkg.BartError) as e:
            s.bvh()
        assert e.value.code == pkg.BART_ESTATE
    finally:
        s.close()


def test_sedan_hierarchy(sim):
    sc = sg.car_scene()
    h = _checked(sim, sc)
    F = h["tri"].shape[0]
    assert h["nodes"].shape[0] == F - 1 and list(h["roots"]) == [0]
    ref, _, _ = oracle.world_facets(sc, float(getattr(sc, "t0", 0.0)))
    np.testing.assert_array_equal(h["tri"], np.asarray(ref, np.float64).reshape(F, 9))


def test_partitioned_batch_hierarchy(sim):
    car = sg.small_car_scene(seed=11, ntri=900, M=64, N=4, P=2, Q=2)
    car2 = sg.small_car_scene(seed=12, ntri=600, M=64, N=4, P=2, Q=2, slant=24.0, speed=-6.0)
    car2.radar = car.radar
    p = sg.plate(0.3, 0.3, 1)
    one = sg.Scene([sg.Mesh(p.verts, p.tris[:1], p.rho[:1], name="one_facet")],
                   [sg.Instance(0, np.array([0.0, 15.0, 1.0]), np.eye(3), np.zeros(3))],
                   car.radar, name="one_facet")
    plate = sg.plate_scene(n=4, M=64, N=4)
    plate.radar = car.radar
    h = _checked(sim, [car, one, car2, plate])
    assert len(h["roots"]) == 4 and h["roots"][1] == ~h["foff"][1]   # the lone facet's leaf


def test_single_facet_hierarchy(sim):
    p = sg.plate(0.3, 0.3, 1)
    sc = sg.Scene([sg.Mesh(p.verts, p.tris[:1], p.rho[:1], name="one_facet")],
                  [sg.Instance(0, np.array([0.0, 15.0, 1.0]), np.eye(3), np.zeros(3))],
                  sg.plate_scene(n=2, M=64, N=2).radar)
    h = _checked(sim, sc, pkg.PATH_FP64)
    assert h["nodes"].shape[0] == 0 and list(h["roots"]) == [~0]


def test_sedan_on_ground_hierarchy(sim):
    _checked(sim, sg.sedan_ground_scene())
