"""GPU parity of batched scenes (bart_scene_partition): several independent
scenes sharing one radar profile, simulated in one pass, each against the
oracle run on that scene alone.

The batch holds two coarse sedans, an occluder plate placed where it would
shadow the first sedan if scenes leaked into one another, and a scene of a
single facet (a one-leaf hierarchy).
"""
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


def batch_scenes():
    car = sg.small_car_scene(seed=11, ntri=1500, M=128, N=8, P=2, Q=2)
    radar = car.radar
    car2 = sg.small_car_scene(seed=12, ntri=900, M=128, N=8, P=2, Q=2, slant=24.0, speed=-6.0)
    car2.radar = radar
    centre = np.asarray(radar.tx, np.float64).mean(axis=0)
    pos = 0.6 * np.asarray(car.instances[0].pos, np.float64) + 0.4 * centre
    occ = sg.Scene([sg.plate(5.0, 5.0, 16)], [sg.Instance(0, pos, np.eye(3), np.zeros(3))], radar,
                   name="occluder")
    p = sg.plate(0.3, 0.3, 1)
    tri = sg.Mesh(p.verts, p.tris[:1], p.rho[:1], name="one_facet")
    one = sg.Scene([tri], [sg.Instance(0, np.array([0.0, 15.0, 1.0]), np.eye(3), np.zeros(3))],
                   radar, name="one_facet")
    return [car, car2, occ, one]


_cache = {}


def reference():
    if "ref" not in _cache:
        scenes = batch_scenes()
        frames = [oracle.Frame(s) for s in scenes]
        _cache["ref"] = (scenes, frames, [f.adc_full() for f in frames])
    return _cache["ref"]


@pytest.fixture(scope="module")
def sim():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    s = pkg.Simulator(0)
    yield s
    s.close()


def facet_offsets(scenes):
    n = [sum(s.meshes[i.mesh_id].nf for i in s.instances) for s in scenes]
    return np.concatenate([[0], np.cumsum(n)])


def test_batch_visibility_is_per_scene(sim):
    scenes, frames, _ = reference()
    sim.load_scenes(scenes)
    adc, st = sim.simulate(pkg.PATH_FP64, stats=True)
    r = scenes[0].radar
    assert tuple(adc.shape) == (len(scenes), r.P * r.Q, r.N, r.M)
    vis = sim.visibility().cpu().numpy()
    off = facet_offsets(scenes)
    assert vis.shape[1] == off[-1]
    for b, fr in enumerate(frames):
        part = vis[:, off[b]:off[b + 1]]
        diff = np.argwhere(part != fr.state)
        assert diff.size == 0, f"scene {b}: {len(diff)} states differ"
    assert st["n_terms"] == sum(f.n_terms() for f in frames)
    # the occluder does shadow the first sedan when both are one scene
    car, occ = scenes[0], scenes[2]
    both = sg.Scene(car.meshes + occ.meshes,
                    car.instances + [sg.Instance(len(car.meshes), occ.instances[0].pos,
                                                 occ.instances[0].rot, occ.instances[0].vel)],
                    car.radar)
    lit_alone = int((frames[0].state == oracle.LIT).sum())
    lit_both = int((oracle.Frame(both).state[:, :off[1]] == oracle.LIT).sum())
    assert lit_both < 0.5 * lit_alone
    sim.sync()


@pytest.mark.parametrize("path,tol", [(pkg.PATH_FP64, TOL_FP64), (pkg.PATH_MIXED, TOL_MIXED)])
def test_batch_adc_matches_oracle(sim, path, tol):
    scenes, frames, refs = reference()
    sim.load_scenes(scenes)
    adc = sim.simulate(path).cpu().numpy().astype(np.complex128)
    for b, ref in enumerate(refs):
        err = rel_l2(adc[b], ref)
        print(f"batch scene {b} ({scenes[b].name}): path {path} relL2 {err:.3e}")
        assert err <= tol


def test_batch_rdm_matches_oracle(sim):
    scenes, frames, refs = reference()
    sim.load_scenes(scenes)
    adc = sim.simulate(pkg.PATH_FP64)
    rdm = sim.rdm(adc).cpu().numpy()
    assert rdm.shape == (len(scenes), scenes[0].radar.M, scenes[0].radar.N)
    for b, ref in enumerate(refs):
        r_ref = oracle.range_doppler_map(ref)
        assert np.abs(rdm[b] - r_ref).max() <= 1e-6 * r_ref.max()


def test_batch_fp64_equals_single_scene_runs(sim):
    """The FP64 path sums each row in list order, which batching keeps: the
    batched slabs equal the one-scene runs bit for bit."""
    scenes, _, _ = reference()
    sim.load_scenes(scenes)
    batched = sim.simulate(pkg.PATH_FP64).cpu()
    for b, sc in enumerate(scenes):
        sim.load_scene(sc)
        single = sim.simulate(pkg.PATH_FP64).cpu()
        assert torch.equal(batched[b], single), sc.name


def test_frame_host_batched(sim):
    scenes, _, refs = reference()
    sim.load_scenes(scenes)
    r = scenes[0].radar
    host = np.empty((len(scenes), r.M, r.N), np.float32)
    pkg.bart_frame_host(sim.ctx, 0.0, pkg.PATH_FP64, host)
    for b, ref in enumerate(refs):
        r_ref = oracle.range_doppler_map(ref)
        assert np.abs(host[b] - r_ref).max() <= 1e-6 * r_ref.max()


@pytest.mark.parametrize("first", [[1, 2], [0, 3, 2], [0, 0, 2], [0, 5]])
def test_bad_partitions_rejected(sim, first):
    scenes, _, _ = reference()
    sim.load_scene(scenes[0])
    pkg.bart_scene_set(sim.ctx, scenes[0].instances * 2)
    with pytest.raises(pkg.BartError) as e:
        pkg.bart_scene_partition(sim.ctx, first)
    assert e.value.code == pkg.BART_EINVAL


# ---------------------------------------------------------------------------
# frame graphs, synthesis layouts and the autotuner
# ---------------------------------------------------------------------------
def with_t0(scene, t0):
    return sg.Scene(scene.meshes, scene.instances, scene.radar, t0=t0, name=scene.name)


@pytest.mark.parametrize("batched", [False, True])
def test_graph_replay_equals_direct_runs(sim, batched):
    """A recorded frame replays bit for bit what the direct launches
    compute, for the recording t0 and for new ones written into the graph;
    a scene change records anew."""
    scenes, _, _ = reference()
    load = (lambda: sim.load_scenes(scenes)) if batched else (lambda: sim.load_scene(scenes[0]))
    load()
    times = [0.0, 0.05, 0.0, -0.02]
    direct = [sim.simulate(pkg.PATH_MIXED, t0=t).clone() for t in times]
    out = torch.empty_like(direct[0])
    pkg.bart_set_graph(sim.ctx, True)
    try:
        for t, ref in zip(times, direct):
            sim.simulate(pkg.PATH_MIXED, t0=t, out=out)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), t
        sim.load_scene(scenes[1])                     # new configuration: recorded again
        ref2 = None
        pkg.bart_set_graph(sim.ctx, False)
        ref2 = sim.simulate(pkg.PATH_MIXED, t0=0.01).clone()
        pkg.bart_set_graph(sim.ctx, True)
        out2 = torch.empty_like(ref2)
        for _ in range(2):
            sim.simulate(pkg.PATH_MIXED, t0=0.01, out=out2)
            torch.cuda.synchronize()
            assert torch.equal(out2, ref2)
    finally:
        pkg.bart_set_graph(sim.ctx, False)


def test_graph_frame_at_new_t0_matches_oracle(sim):
    scenes, _, _ = reference()
    sc = scenes[0]
    sim.load_scene(sc)
    pkg.bart_set_graph(sim.ctx, True)
    try:
        out = sim.simulate(pkg.PATH_FP64, t0=0.0).clone()      # records
        sim.simulate(pkg.PATH_FP64, t0=0.04, out=out)           # replays with t0 = 0.04
        torch.cuda.synchronize()
    finally:
        pkg.bart_set_graph(sim.ctx, False)
    ref = oracle.Frame(with_t0(sc, 0.04)).adc_full()
    assert rel_l2(out.cpu().numpy(), ref) <= TOL_FP64


@pytest.mark.parametrize("S,tpi", [(16, 8), (16, 64), (8, 8), (8, 512), (0, 0)])
def test_synth_layouts_match_oracle(sim, S, tpi):
    scenes, frames, refs = reference()
    sim.load_scenes(scenes)
    pkg.bart_set_synth_layout(sim.ctx, S, tpi)
    try:
        adc = sim.simulate(pkg.PATH_MIXED).cpu().numpy().astype(np.complex128)
    finally:
        pkg.bart_set_synth_layout(sim.ctx, 0, 0)
    for b, ref in enumerate(refs):
        assert rel_l2(adc[b], ref) <= TOL_MIXED


def test_autotune_keeps_a_valid_fastest_layout(sim):
    scenes, frames, refs = reference()
    sim.load_scenes(scenes)
    adc = torch.empty(sim.adc_shape(), dtype=torch.complex64, device="cuda")
    res = pkg.bart_autotune(sim.ctx, 0.0, adc, reps=2)
    trials = res["trials"]
    assert len(trials) >= 7
    best = res["best"]
    assert best[2] == min(t[2] for t in trials) and best[2] > 0
    assert (best[0], best[1]) in [(t[0], t[1]) for t in trials]
    print("autotune", res)
    out = sim.simulate(pkg.PATH_MIXED).cpu().numpy().astype(np.complex128)
    for b, ref in enumerate(refs):
        assert rel_l2(out[b], ref) <= TOL_MIXED
    pkg.bart_set_synth_layout(sim.ctx, 0, 0)


# ---------------------------------------------------------------------------
# adjoint of the RDM
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 2e-5)])
@pytest.mark.parametrize("O,N,M", [(4, 8, 128), (3, 24, 96), (2, 27, 32)])
def test_rdm_adjoint_matches_oracle(sim, dtype, tol, O, N, M):
    radar = sg.make_radar(M, N, 1, O, 5.12e6, 30e12, 2.0, centre=(0.0, 0.0, 0.0))
    sim.load_scene(sg.Scene([sg.plate(0.1, 0.1, 1)], [sg.Instance(0, np.array([0.0, 5.0, 0.0]),
                                                                  np.eye(3), np.zeros(3))], radar))
    rng = np.random.default_rng(O * 100 + N + M)
    x = rng.normal(size=(O, N, M)) + 1j * rng.normal(size=(O, N, M))
    G = rng.normal(size=(M, N)).astype(np.float32)
    xd = torch.from_numpy(x).cuda().to(dtype)
    gd = torch.from_numpy(G).cuda()
    out = torch.empty_like(xd)
    pkg.bart_rdm_adjoint(sim.ctx, xd, gd, out)
    ref = oracle.rdm_adjoint(xd.cpu().numpy().astype(np.complex128), G.astype(np.float64))
    assert rel_l2(out.cpu().numpy().astype(np.complex128), ref) <= tol


def test_config4_dataset_batch_sampled(sim):
    """Eight seeded dataset scenes (1-8 vehicles, 5k-200k facets each, the
    sedan radar) simulated as one batch: per-scene visibility bit-exact
    against the oracle, and 256 seeded ADC entries per scene on both paths."""
    scenes = [sg.batch_scene(i) for i in range(8)]
    frames = [oracle.Frame(s) for s in scenes]
    sim.load_scenes(scenes)
    off = facet_offsets(scenes)
    r = scenes[0].radar
    rng = np.random.default_rng(44)
    ent = [np.stack([rng.integers(0, r.O, 256), rng.integers(0, r.N, 256),
                     rng.integers(0, r.M, 256)], 1) for _ in scenes]
    refs = [fr.adc_entries(e) for fr, e in zip(frames, ent)]
    for path, tol in ((pkg.PATH_MIXED, TOL_MIXED), (pkg.PATH_FP64, TOL_FP64)):
        adc = sim.simulate(path).cpu().numpy()
        if path == pkg.PATH_MIXED:
            vis = sim.visibility().cpu().numpy()
            for b, fr in enumerate(frames):
                assert np.array_equal(vis[:, off[b]:off[b + 1]], fr.state), b
        for b in range(len(scenes)):
            e = ent[b]
            got = adc[b][e[:, 0], e[:, 1], e[:, 2]].astype(np.complex128)
            err = rel_l2(got, refs[b])
            assert err <= tol, (b, path, err)
        print(f"config4 batch path {path}: worst scene relL2 "
              f"{max(rel_l2(adc[b][e[:, 0], e[:, 1], e[:, 2]].astype(np.complex128), refs[b]) for b, e in enumerate(ent)):.3e}")
        del adc


def test_dataset_runner_resumes_and_matches_oracle(tmp_path):
    """The dataset runner on the GPU: 48 seeded dataset scenes cut into
    batches by a facet budget, interrupted after two batches and resumed;
    every scene's RDM committed once; 8 scenes spread over the batches kept
    as ADC cubes and checked against the oracle (64 entries each, mixed path
    <= 1e-4), and their RDMs equal to the RDMs the library forms from those
    cubes."""
    from paper_2208_10939_gb300 import dataset
    keep = [0, 7, 13, 20, 27, 33, 40, 47]
    gsim = dataset.GpuBatchSimulator(0)
    try:
        st1 = dataset.run_dataset(str(tmp_path), 48, sg.batch_scene, gsim, max_facets=1_200_000,
                                  chunk=16, stop_after_batches=2, keep_adc=keep)
        assert st1["stopped"]
        st2 = dataset.run_dataset(str(tmp_path), 48, sg.batch_scene, gsim, max_facets=1_200_000,
                                  chunk=16, keep_adc=keep)
        assert st1["scenes"] + st2["scenes"] == 48 and st2["skipped"] == st1["scenes"]
        assert st1["batches"] + st2["batches"] >= 4
        adc = {**st1["adc"], **st2["adc"]}
        assert sorted(adc) == keep
        idx, rdm = dataset.load_dataset(str(tmp_path))
        assert list(idx) == list(range(48))
        r = sg.batch_scene(0).radar
        one = pkg.Simulator(0)
        worst = 0.0
        try:
            for i in keep:
                sc = sg.batch_scene(i)
                one.load_scene(sc)
                rd = one.rdm(torch.from_numpy(adc[i]).cuda()).cpu().numpy()
                assert np.abs(rd - rdm[i]).max() <= 1e-5 * rdm[i].max()
                fr = oracle.Frame(sc)
                rng = np.random.default_rng(1000 + i)
                e = np.stack([rng.integers(0, r.O, 64), rng.integers(0, r.N, 64),
                              rng.integers(0, r.M, 64)], 1)
                ref = fr.adc_entries(e)
                err = rel_l2(adc[i][e[:, 0], e[:, 1], e[:, 2]].astype(np.complex128), ref)
                worst = max(worst, err)
                assert err <= TOL_MIXED, (i, err)
        finally:
            one.close()
        print(f"dataset runner: {st1['batches']} + {st2['batches']} batches, worst kept-scene "
              f"relL2 vs oracle {worst:.3e}")
    finally:
        gsim.close()
