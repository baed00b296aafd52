"""The seeded synthetic workloads have the sizes and structure the design
states (CPU only): triangle counts, arrays, chirp profiles, lanes, speeds,
ranges, and determinism per seed.  The radar profiles follow Table 2's rule
T_c = M / fs + 10 us, with v_max = lambda_c / (4 T_c); the radar height and
the lane centres are Table 1's (tests/golden/table1.json)."""
import json
import os

import numpy as np
import pytest

import scenegen as sg

C0 = sg.C0
TABLE1 = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                     "table1.json")))
LANES = TABLE1["lane_centres_x_m"]


def n_tris(scene) -> int:
    return sum(int(scene.meshes[i.mesh_id].tris.shape[0]) for i in scene.instances)


def spacing(arr) -> np.ndarray:
    a = np.asarray(arr, np.float64).reshape(-1, 3)
    return np.diff(a[:, 0])


def test_plate_workload():
    sc = sg.plate_scene()
    r = sc.radar
    assert n_tris(sc) == 200
    m = sc.meshes[0]
    v = m.verts[m.tris]
    area = 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), axis=1).sum()
    assert area == pytest.approx(1.0, rel=1e-12)
    assert np.allclose(sc.instances[0].pos, (0.0, 20.0, 0.0))
    assert (r.P, r.Q, r.N, r.M) == (1, 4, 64, 128)
    assert (r.slope, r.fs) == (30e12, 5.12e6)
    assert r.Tc == pytest.approx(128 / 5.12e6 + 10e-6, rel=1e-12)
    assert np.allclose(spacing(r.rx), C0 / r.f0 / 2)


def test_moving_sedan_workload():
    sc = sg.car_scene()
    r = sc.radar
    assert abs(n_tris(sc) - 20_000) <= 200
    assert (r.P, r.Q, r.N, r.M) == (3, 4, 128, 256)
    assert (r.slope, r.fs) == (12.5e12, 5.12e6)
    assert r.Tc == pytest.approx(60e-6, rel=1e-12)
    lam0 = C0 / r.f0
    assert np.allclose(spacing(r.tx), 2 * lam0) and np.allclose(spacing(r.rx), lam0 / 2)
    centre = np.asarray(r.tx, np.float64).mean(axis=0)
    assert centre[2] == TABLE1["radar_altitude_m"]
    ins = sc.instances[0]
    los = centre - np.asarray(ins.pos, np.float64)
    assert np.linalg.norm(los) == pytest.approx(30.0, abs=0.05)
    assert ins.pos[0] == pytest.approx(LANES[0])
    v = np.asarray(ins.vel, np.float64)
    assert np.linalg.norm(v) == pytest.approx(10.0, rel=1e-12)
    assert v @ los / np.linalg.norm(los) == pytest.approx(10.0, rel=1e-12)   # toward the radar
    B = r.slope * r.M / r.fs
    lam_c = C0 / (r.f0 + B / 2)
    assert lam_c / (4 * r.Tc) == pytest.approx(16.16, abs=0.01)


def test_intersection_workload():
    sc = sg.intersection_scene()
    r = sc.radar
    assert n_tris(sc) == 1_470_848
    assert (r.P, r.Q, r.N, r.M) == (12, 16, 256, 512)
    assert (r.slope, r.fs) == (12.5e12, 10.24e6)
    lam0 = C0 / r.f0
    assert np.allclose(spacing(r.tx), 8 * lam0) and np.allclose(spacing(r.rx), lam0 / 2)
    assert np.all(np.asarray(r.tx, np.float64)[:, 2] == TABLE1["radar_altitude_m"])
    assert np.diff(LANES) == pytest.approx([TABLE1["lane_width_m"]] * 2)
    names = [sc.meshes[i.mesh_id].name for i in sc.instances]
    ground = [i for i, n in zip(sc.instances, names) if n.startswith("ground")]
    assert len(ground) == 1 and sc.meshes[ground[0].mesh_id].tris.shape[0] == 2 * 158 * 158
    vehicles = [i for i, n in zip(sc.instances, names) if not n.startswith("ground")]
    assert len(vehicles) == 12
    per_class = {"car": 20_000, "suv": 40_000, "bus": 120_000, "truck": 200_000}
    lanes = {}
    for ins in vehicles:
        m = sc.meshes[ins.mesh_id]
        cls = next(c for c in per_class if m.name.startswith(c))
        assert abs(m.tris.shape[0] - per_class[cls]) <= 0.01 * per_class[cls]
        x, y = float(ins.pos[0]), float(ins.pos[1])
        assert min(abs(x - c) for c in LANES) < 1e-12
        assert 10.0 <= y <= 80.0
        assert abs(ins.vel[1]) <= 15.0 and ins.vel[0] == 0.0 and ins.vel[2] == 0.0
        w = (np.asarray(ins.rot, np.float64).reshape(3, 3) @ m.verts.T).T + ins.pos
        lanes.setdefault(x, []).append((w[:, 1].min(), w[:, 1].max()))
    for spans in lanes.values():               # no two vehicles of a lane overlap
        spans.sort()
        assert all(a[1] < b[0] for a, b in zip(spans, spans[1:]))


@pytest.mark.parametrize("index", [0, 1, 7, 4095])
def test_dataset_scene_workload(index):
    sc = sg.batch_scene(index)
    again = sg.batch_scene(index)
    r = sc.radar
    assert 1 <= len(sc.instances) <= 8
    assert 5_000 <= n_tris(sc) <= 200_000
    assert (r.P, r.Q, r.N, r.M) == (3, 4, 128, 256)
    for ins in sc.instances:
        assert float(ins.pos[1]) >= 25.0
        assert min(abs(float(ins.pos[0]) - c) for c in LANES) < 1e-12
        assert -10.0 <= float(ins.vel[1]) <= -0.5               # approaching
    assert n_tris(again) == n_tris(sc)
    for a, b in zip(sc.meshes, again.meshes):
        assert np.array_equal(a.verts, b.verts) and np.array_equal(a.tris, b.tris)
