#!/usr/bin/env python
"""Throughput benchmark of the BART echo-synthesis hot path on GB300.

Headline workload: the intersection frame -- 12 procedural vehicles (car
20k, SUV 40k, bus 120k, truck 200k triangles; seeded positions 10-80 m,
velocities -15..15 m/s) on a 100 m x 100 m ground of 50k triangles, ~1.47M
facets in all, seen by a 12 TX x 16 RX sparse MIMO FMCW radar (192 virtual
channels), 256 chirps x 512 samples, ADC cube complex64 (201 MB), RDM
512 x 256 FP32.  One step = one whole frame of the hot path: world facets,
LBVH build, BART visibility, FP64 kinematics rows, echo synthesis (mixed
path) and the windowed range-Doppler FFT into the RDM.

Metric: echo terms/s (lit facet x channel x chirp x sample); frames/s, the
spectral (inverse-FFT) path on the same frame, the RDM against HBM, the
moving-sedan frame (20k triangles, 12 channels, 128 x 256), the plain-FP64
path, the differentiable echo and the dataset runner are reported beside
it.  Inputs are resident in HBM when the timed
region starts; the frame's working set (facet records, kinematics rows,
ADC cube) is far larger than L2, which is also flushed (256 MB write)
between timed steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank simulates its own seeded intersection (weak
scaling, replicas: the path needs no collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "echo terms/s (facet x chan x chirp x sample), frames/s; mixed vs FP64 path"
UNIT = "terms/s"
WORKLOAD = ("intersection: 12 vehicles (20k-200k tris) + 50k-tri ground, 12TXx16RX (192 ch), "
            "256 chirps x 512 samples")
SEDAN = "moving sedan 20k tris, 3TXx4RX (12 ch), 128 chirps x 256 samples"
BOUNCE = ("moving sedan 20k tris on a 20 m x 20 m static ground (0.5 m cells, 3200 tris), "
          "3TXx4RX (12 ch), 128 chirps x 256 samples, single + double bounce")
# algorithmic work of one echo term in the mixed path: 3 vertex phases, 3 unit
# phasors, 3 real x complex weighted accumulates and their compensation, about
# 24 FP32 FMA-pipe operations (plus 6 SFU operations when the phasors come from
# sincos); the roofline counts operations of the FMA pipe, whatever their kind
OPS_PER_TERM = 24
# DRAM traffic of one synthesis launch and the FMA-pipe activity, from ncu
# captures of the synthesis kernel on 4 TX x 4 RX cuts of the frame.  A work
# item takes one record chunk of a channel through all its chirps, so a
# (channel, lit facet) record's inputs come from HBM once and from L2 for the
# other chirps: reads grow with those pairs (terms / (N M)), not with the
# terms (16 and 64 chirps read 3.41 and 3.28 GB); the items' partial sums
# grow with the (channel, chirp) rows.  Valid only while the kernel's sources
# hash to the value they had at the capture.
SYNTH_PROFILE = {"sources_sha256_16": "4239e3318de9d32c", "samples_per_lane": 16,
                 "dram_read_bytes_per_channel_facet": 3.277169152e9 / (4 * 50804670464 / (64 * 512)),
                 "dram_write_bytes_per_row": 75.109632e6 / (16 * 64),
                 "fma_pipe_active": 0.686}
SYNTH_SOURCES = ("synth.cu", "bart_internal.cuh", "record_fp64.cuh", "mixed_record.cuh")
# the double-bounce synthesis: 3 centres x (2 accumulates + 4 rotation
# operations) per vertex-form term; ncu figures of its launch on the
# sedan-over-ground frame, valid while its sources hash as at the capture
BOUNCE_OPS_PER_TERM = 18
BOUNCE_SOURCES = ("bounce.cu", "bounce.cuh", "geom64.cuh", "record_fp64.cuh", "bart_internal.cuh")
BOUNCE_PROFILE = {"sources_sha256_16": "0ad733dd979e3494", "fma_pipe_active": 0.324, "fp64_pipe_active": 0.528,
                  "issue_active": 0.523, "warps_active": 0.179}


def synth_sources_hash(sources=SYNTH_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2208_10939_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def synth_profile(samples_per_lane: int):
    """The captured per-term DRAM traffic and FMA-pipe activity, or None when
    the kernel (its sources, or the template instance the layout picks)
    differs from the captured one."""
    if (samples_per_lane != SYNTH_PROFILE["samples_per_lane"]
            or SYNTH_PROFILE["sources_sha256_16"] != synth_sources_hash()):
        return None
    return SYNTH_PROFILE


def layout_samples(M: int, S_req: int) -> int:
    """Samples per lane the mixed synthesis kernel uses for M samples per
    chirp and a layout request (the library's rule, for naming the kernel)."""
    if S_req == 8 and ((M <= 256 and 256 % M == 0) or M % 256 == 0):
        return 8
    if (M <= 512 and 512 % M == 0) or M % 512 == 0:
        return 16
    for S in (8, 4, 2):
        if M % (32 * S) == 0:
            return S
    return 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--sedan-steps", type=int, default=20)
    ap.add_argument("--spectral-steps", type=int, default=5,
                    help="timed frames of the spectral path on the headline frame (0 skips)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dataset-scenes", type=int, default=4096,
                    help="seeded dataset scenes (1-8 vehicles, 5k-200k facets) simulated by the "
                         "batched dataset runner; 0 skips the line")
    ap.add_argument("--dataset-per-scene", type=int, default=256,
                    help="of those, how many are also simulated one per call (per-scene launches)")
    ap.add_argument("--batch-scenes", type=int, default=32,
                    help="small dataset scenes (5k-10k facets) for the batched / graph / "
                         "autotuner comparison (2x this many); 0 skips it")
    ap.add_argument("--batch-size", type=int, default=8)
    ap.add_argument("--adjoint-reps", type=int, default=1,
                    help="timed runs of the perturbed-sedan gradient (0 skips)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the default synthesis layout instead of the autotuned one")
    ap.add_argument("--synth-layout", default=None, metavar="S,T",
                    help="fix the synthesis layout (samples per lane, tiles per item) "
                         "instead of autotuning it")
    ap.add_argument("--workload", default="intersection", choices=["intersection", "sedan"],
                    help="headline frame (the sedan for quick profiling runs)")
    ap.add_argument("--no-sedan", action="store_true", help="skip the moving-sedan lines")
    ap.add_argument("--bounce-steps", type=int, default=5,
                    help="timed frames of the sedan-on-ground double-bounce line (0 skips)")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the peak microbenchmarks (roofline against no measured peak)")
    ap.add_argument("--chirps", type=int, default=0,
                    help="profiling aid: headline frame with this many chirps (0: the workload's)")
    ap.add_argument("--array", default=None, metavar="PxQ",
                    help="profiling aid: headline frame with the first P TX and Q RX")
    ap.add_argument("--no-flush", action="store_true",
                    help="profiling aid: no L2 flush between steps (per-kernel DRAM counters)")
    ap.add_argument("--probe", default=None, choices=["rdm", "adjoint", "bounce"],
                    help="run one stage alone for a profiler capture and print its time: "
                         "the RDM of a seeded 192 x 256 x 512 complex64 cube with the "
                         "intersection radar, the mixed adjoint of the sedan for a "
                         "seeded dL/d(adc), or a mixed-path frame of the sedan on a ground "
                         "patch with double bounce")
    ap.add_argument("--log", default=os.environ.get("BART_RUN_LOG"),
                    help="append the run's record (JSON line plus seeds, clocks, oracle errors, "
                         "grazing counts) to this JSONL file")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _lit_per_channel(fr, r):
    return fr.lit_pairs().sum(axis=1)


def _sample_entries(rng, r, E):
    return np.stack([rng.integers(0, r.O, E), rng.integers(0, r.N, E),
                     rng.integers(0, r.M, E)], 1).astype(np.int32)


def cpu_baseline(scene, seconds: float, adc=None, others=None) -> dict:
    """The FP64 oracle as it stands, on the host cores: echo terms/s of its
    synthesis over a random sample of ADC entries of the same frame (sized
    to ~``seconds`` of work), and the full-frame oracle time extrapolated
    from that rate.  With ``adc`` (the GPU cube of the timed frame, host
    array) the sampled entries also give the frame's error against the
    oracle."""
    import oracle
    t = time.perf_counter()
    fr = oracle.Frame(scene)
    t_vis = time.perf_counter() - t
    r = scene.radar
    per_ch = _lit_per_channel(fr, r)
    rng = np.random.default_rng(12345)
    e = _sample_entries(rng, r, 16)
    t = time.perf_counter()
    fr.adc_entries(e)
    dt = time.perf_counter() - t
    E = max(16, int(16 * seconds / max(dt, 1e-3)))
    e = _sample_entries(rng, r, E)
    terms = int(per_ch[e[:, 0]].sum())
    t = time.perf_counter()
    ref = fr.adc_entries(e)
    dt = time.perf_counter() - t
    rate = terms / dt
    frame_terms = int(per_ch.sum()) * r.N * r.M
    out = {"value": rate, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{E} random ADC entries of the frame ({terms} echo terms, {dt:.1f} s of "
                     f"oracle synthesis); oracle visibility of the frame (its own BVH) took "
                     f"{t_vis:.1f} s, untimed",
           "frame_s_extrapolated": frame_terms / rate + t_vis}
    # the same oracle on one host core, on the first entries of the sample
    # (about a quarter of the sample's time)
    n_all = oracle.num_threads()
    e1 = e[:max(16, E // (4 * max(1, n_all)))]
    oracle.set_threads(1)
    try:
        t = time.perf_counter()
        fr.adc_entries(e1)
        dt1 = time.perf_counter() - t
    finally:
        oracle.set_threads(n_all)
    out["one_core"] = {"value": int(per_ch[e1[:, 0]].sum()) / dt1, "unit": UNIT, "cores": 1,
                       "sample": f"the first {len(e1)} of those entries"}
    if adc is not None:
        got = adc[e[:, 0], e[:, 1], e[:, 2]].astype(np.complex128)
        out["gpu_frame_rel_l2_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        out["gpu_frame_checked_entries"] = int(E)
    for name, cube in (others or {}).items():
        got = cube[e[:, 0], e[:, 1], e[:, 2]].astype(np.complex128)
        out[f"{name}_rel_l2_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return out


def run_reference(args):
    """--impl reference: the oracle, timed on the host cores (rank 0 only),
    on the headline workload: each step a bounded random sample of ADC
    entries of the frame (~4 s of oracle work)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import scenegen as sg
    scene = sg.intersection_scene() if args.workload == "intersection" else sg.car_scene()
    fr = oracle.Frame(scene)
    r = scene.radar
    per_ch = _lit_per_channel(fr, r)
    terms_frame = int(per_ch.sum()) * r.N * r.M
    rng = np.random.default_rng(7)
    e = _sample_entries(rng, r, 16)
    t = time.perf_counter()
    fr.adc_entries(e)
    E = max(16, int(16 * 4.0 / max(time.perf_counter() - t, 1e-3)))
    tot_terms, tot_t = 0, 0.0
    for step in range(args.warmup + args.steps):
        e = _sample_entries(rng, r, E)
        terms = int(per_ch[e[:, 0]].sum())
        t = time.perf_counter()
        fr.adc_entries(e)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            tot_terms += terms
            tot_t += dt
    v = tot_terms / tot_t
    sample = f"{E} random ADC entries per step of the {terms_frame}-term frame"
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": WORKLOAD if args.workload == "intersection" else SEDAN,
                      "path": "FP64 CPU oracle", "seed": 3 if args.workload == "intersection" else 2},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def dataset_batch(pkg, sg, torch, dev, K: int, bsz: int, tri_min: int = 5_000,
                  tri_max: int = 200_000) -> dict:
    """Dataset generation (seeded scenes of 1-8 vehicles, 5k-200k facets,
    radar as the sedan workload): scene-frames per second simulated one
    scene per frame call versus bsz scenes per call (bart_scene_partition),
    each including the instance-table upload, synthesis and RDM, meshes
    resident; then the autotuned layout, and a 4-frame time sequence of one
    batch replayed as a CUDA graph versus direct launches."""
    scenes = [sg.batch_scene(i, tri_min=tri_min, tri_max=tri_max) for i in range(K)]
    sim = pkg.Simulator(dev.index or 0)
    pkg.bart_mesh_clear(sim.ctx)
    placed = []
    for sc in scenes:
        ids = [pkg.bart_mesh_upload(sim.ctx, m.verts, m.tris, m.rho, m.two_sided)
               for m in sc.meshes]
        placed.append([pkg._Placed(ids[i.mesh_id], i) for i in sc.instances])
    radar = scenes[0].radar
    pkg.bart_radar_set(sim.ctx, radar)
    sim.radar = radar
    O, N, M = radar.O, radar.N, radar.M
    facets = [sum(s.meshes[i.mesh_id].nf for i in s.instances) for s in scenes]
    stream = torch.cuda.current_stream(dev)

    def run(groups, out_pool):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for g in groups:
            insts = [x for b in g for x in placed[b]]
            pkg.bart_scene_set(sim.ctx, insts)
            if len(g) > 1:
                first = np.cumsum([0] + [len(placed[b]) for b in g])
                pkg.bart_scene_partition(sim.ctx, first)
            adc, rdm = out_pool[len(g)]
            pkg.bart_simulate_frame(sim.ctx, 0.0, pkg.PATH_MIXED, adc)
            pkg.bart_form_rdm(sim.ctx, adc, rdm)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t, e0.elapsed_time(e1) / 1e3

    pool = {}
    for b in {1, bsz}:
        pool[b] = (torch.empty((b, O, N, M), dtype=torch.complex64, device=dev),
                   torch.empty((b, M, N), dtype=torch.float32, device=dev))
    single = [[i] for i in range(K)]
    batched = [list(range(i, min(K, i + bsz))) for i in range(0, K, bsz)]
    if K % bsz:
        pool[K % bsz] = (torch.empty((K % bsz, O, N, M), dtype=torch.complex64, device=dev),
                         torch.empty((K % bsz, M, N), dtype=torch.float32, device=dev))
    run(single, pool)
    wall1, dev1 = run(single, pool)
    run(batched, pool)
    wallB, devB = run(batched, pool)

    # autotuned synthesis layout on the first batch, kept for all batches
    g0 = batched[0]
    pkg.bart_scene_set(sim.ctx, [x for b in g0 for x in placed[b]])
    pkg.bart_scene_partition(sim.ctx, np.cumsum([0] + [len(placed[b]) for b in g0]))
    tune = pkg.bart_autotune(sim.ctx, 0.0, pool[len(g0)][0], reps=1)
    run(batched, pool)
    wallT, devT = run(batched, pool)

    # a time sequence of one batch: direct launches vs a replayed frame graph
    pkg.bart_scene_set(sim.ctx, [x for b in g0 for x in placed[b]])
    pkg.bart_scene_partition(sim.ctx, np.cumsum([0] + [len(placed[b]) for b in g0]))
    adc, rdm = pool[len(g0)]
    frame_T = N * radar.Tc
    seq = [k * frame_T for k in range(4)]

    def sequence():
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        for t0 in seq:
            pkg.bart_simulate_frame(sim.ctx, t0, pkg.PATH_MIXED, adc)
            pkg.bart_form_rdm(sim.ctx, adc, rdm)
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t

    sequence()
    direct_s = sequence()
    pkg.bart_set_graph(sim.ctx, True)
    sequence()
    graph_s = sequence()
    pkg.bart_set_graph(sim.ctx, False)
    sim.close()
    return {
        "workload": f"{K} seeded dataset scenes (1-8 vehicles, {tri_min // 1000}k-"
                    f"{tri_max // 1000}k facets, "
                    f"mean {int(np.mean(facets))}), radar as the sedan workload, mixed path + RDM",
        "unit": "scene-frames/s",
        "per_scene": {"value": K / wall1, "device_s": dev1, "wall_s": wall1},
        "batched": {"value": K / wallB, "device_s": devB, "wall_s": wallB, "batch_size": bsz},
        "batched_autotuned": {"value": K / wallT, "device_s": devT, "wall_s": wallT,
                              "layout": {"samples_per_lane": tune["best"][0],
                                         "tiles_per_item": tune["best"][1]},
                              "trials": tune["trials"]},
        "sequence_4_frames": {"direct": len(g0) * len(seq) / direct_s,
                              "graph": len(g0) * len(seq) / graph_s},
    }


def dataset_run(pkg, sg, torch, dev, K: int, K_single: int, n_check: int = 8) -> dict:
    """Config 4: K seeded dataset scenes through the batched dataset runner
    (batches cut by a 40M-facet budget, scenes generated ahead in spawned
    worker processes, RDM shards and a resume manifest written to a
    temporary directory): scene-frames/s of the device (frame + RDM per
    batch, CUDA events) and of the whole run; the first K_single scenes
    again one scene per call (per-scene launches); n_check scenes kept as ADC
    cubes and checked against the oracle on sampled entries."""
    import shutil
    from paper_2208_10939_gb300 import dataset
    import oracle
    keep = [int(i) for i in np.linspace(0, K - 1, n_check).round()] if n_check else []
    out = tempfile.mkdtemp(prefix="bart_dataset_")
    gsim = dataset.GpuBatchSimulator(dev.index or 0)
    try:
        workers = max(0, min(15, (os.cpu_count() or 2) - 1))
        st = dataset.run_dataset(out, K, sg.batch_scene, gsim, max_facets=40_000_000,
                                 workers=workers, keep_adc=keep)
        idx, _ = dataset.load_dataset(out)
        assert len(idx) == K
        shutil.rmtree(out, ignore_errors=True)
        out1 = tempfile.mkdtemp(prefix="bart_dataset1_")
        st1 = dataset.run_dataset(out1, K_single, sg.batch_scene, gsim, max_scenes=1,
                                  workers=workers)
        shutil.rmtree(out1, ignore_errors=True)
    finally:
        gsim.close()
    worst, checked = 0.0, 0
    r = sg.batch_scene(0).radar
    for i in keep:
        fr = oracle.Frame(sg.batch_scene(i))
        rng = np.random.default_rng(4000 + i)
        e = _sample_entries(rng, r, 32)
        ref = fr.adc_entries(e)
        got = st["adc"][i][e[:, 0], e[:, 1], e[:, 2]].astype(np.complex128)
        worst = max(worst, float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
        checked += len(e)
    return {"workload": f"{K} seeded dataset scenes (1-8 vehicles, 5k-200k facets, "
                        f"mean {st['facets'] // max(1, st['scenes'])}), 3TXx4RX, 128 x 256, "
                        "mixed path + RDM, RDM shards + resume manifest",
            "unit": "scene-frames/s",
            "batched": {"value": st["scenes"] / st["device_s"], "device_s": st["device_s"],
                        "wall_value": st["scenes"] / st["wall_s"], "wall_s": st["wall_s"],
                        "batches": st["batches"], "facets": st["facets"],
                        "scene_workers": workers},
            "per_scene_launches": {"scenes": st1["scenes"],
                                   "value": st1["scenes"] / st1["device_s"],
                                   "device_s": st1["device_s"],
                                   "wall_value": st1["scenes"] / st1["wall_s"]},
            "oracle_check": {"scenes": keep, "entries": checked, "worst_rel_l2": worst}}


def detect_timing(pkg, torch, sim, adc, stream, reps: int = 10) -> dict:
    """CA-CFAR + angle spectrum + point records (bart_detect) on the timed
    frame's ADC with receiver noise added (20 dB SNR per sample, seed 9):
    device time per call (CUDA events), points found.  A noise-free cube
    would let CFAR pick up the synthesis' rounding floor (paired echoes
    below -100 dB) instead of targets."""
    cfg = pkg.make_detect_cfg(guard_r=2, guard_d=2, train_r=8, train_d=4, pfa=1e-6, angle_bins=512)
    adc = adc.clone()
    pkg.bart_add_noise(sim.ctx, adc, 20.0, 9, 0)
    buf = torch.empty(65536 * pkg.POINT_DTYPE.itemsize, dtype=torch.uint8, device=adc.device)
    n = pkg.bart_detect(sim.ctx, adc, cfg, buf)
    ms = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pkg.bart_detect(sim.ctx, adc, cfg, buf, sync=False)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return {"ms": statistics.median(ms), "points": int(n), "angle_bins": 512,
            "cfar": "guard 2x2, train 8x4, Pfa 1e-6", "snr_db": 20.0}


def adjoint_timing(pkg, sg, torch, dev, reps: int) -> dict:
    """Differentiable echo, the RDM inverse problem: the sedan's RDM as
    target, its copy with 5 mm vertex noise (seed 5) as the variable,
    L = ||RDM(v, rho) - RDM_target||^2 through both adjoints
    (bart_rdm_adjoint, then the echo adjoint) with gradients for the vertex
    positions and the per-facet reflectivities; forward (echo + RDM + loss)
    and backward times (CUDA events), gradient throughput in echo terms per
    second, FP64 and mixed precision (mixed-path forward, the FP32 adjoint
    route), and the mixed gradients' relative L2 distance to the FP64
    ones."""
    from paper_2208_10939_gb300 import autograd as bag
    s = pkg.Simulator(dev.index or 0)
    try:
        sc = sg.car_scene()
        out = {"workload": "sedan 20k tris, RDM target vs 5 mm vertex noise (seed 5), "
                           "L = ||RDM(v, rho) - RDM_target||^2, gradients for vertices and "
                           "reflectivities"}
        grads = {}
        for prec in ("fp64", "mixed"):
            es = bag.EchoScene(s, sc, precision=prec)
            v_true = es.vertex_tensor(sc, dev)
            rho0 = torch.from_numpy(sc.meshes[0].rho.copy()).to(dev)
            with torch.no_grad():
                target = bag.range_doppler_map(bag.echo(v_true, None, es), s).clone()
            rng = np.random.default_rng(5)
            v0 = v_true + torch.from_numpy(0.005 * rng.normal(size=tuple(v_true.shape))).to(dev)
            st = pkg.bart_simulate_frame(s.ctx, 0.0, pkg.PATH_FP64,
                                         torch.empty(s.adc_shape(), dtype=torch.complex128,
                                                     device=dev), stats=True)
            fwd, bwd = [], []
            for rep in range(reps + 1):          # the first pass warms up (allocations)
                verts = v0.clone().requires_grad_(True)
                rho = rho0.clone().requires_grad_(True)
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record()
                rdm = bag.range_doppler_map(bag.echo(verts, rho, es), s)
                loss = (rdm - target).pow(2).sum()
                e1.record()
                loss.backward()
                e2.record()
                e2.synchronize()
                if rep > 0:
                    fwd.append(e0.elapsed_time(e1))
                    bwd.append(e0.elapsed_time(e2) - e0.elapsed_time(e1))
            grads[prec] = (verts.grad.detach().clone(), rho.grad.detach().clone())
            terms = st["n_terms"]
            key = "" if prec == "fp64" else "_mixed"
            out["forward_ms" + key] = min(fwd)
            out["backward_ms" + key] = min(bwd)
            out["backward_over_forward" + key] = min(bwd) / min(fwd)
            out["gradient_terms_per_s" + key] = terms / (min(bwd) / 1e3)
            out["terms"] = terms
            out["parameters"] = int(verts.numel() + rho.numel())
        for i, name in ((0, "vertices"), (1, "reflectivity")):
            out[f"mixed_gradient_rel_l2_vs_fp64_{name}"] = float(
                torch.linalg.norm(grads["mixed"][i] - grads["fp64"][i]) /
                torch.linalg.norm(grads["fp64"][i]))
        return out
    finally:
        s.close()


def measured_hbm_gbs():
    """The measured HBM copy bandwidth of the GB300s, else the
    recipe's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s)"


def measure_peaks(pkg, dev_index: int) -> dict:
    """Measured FP32 FMA-pipe, MUFU and FP64 rates of this GPU (the library's
    own register-only microbenchmarks)."""
    p = pkg.bart_measure_peaks(dev_index, reps=5)
    fp32 = max(p["fp32_fma_per_s"], p["fp32x2_fma_per_s"])
    return {"fp32_fma_pipe_tops": fp32 / 1e12,
            "fp32_scalar_fma_tops": p["fp32_fma_per_s"] / 1e12,
            "fp32x2_fma_tops": p["fp32x2_fma_per_s"] / 1e12,
            "mufu_sincos_per_s": p["sincos_per_s"],
            "fp64_fma_tops": p["fp64_fma_per_s"] / 1e12,
            "sms": p["sms"], "how": "bart_measure_peaks: register-only FMA / f32x2 FMA / "
                                    "__sincosf / FP64 FMA chains, 2048 threads per SM, "
                                    "best of 5 CUDA-event-timed launches"}


def timed_frames(pkg, torch, sim, adc, rdm, flush, stream, steps: int, path: int) -> dict:
    """``steps`` frames (simulate + RDM), L2 flushed before each (unless
    ``flush`` is None); per-step device times (CUDA events on the launching
    stream) and the library's per-stage times."""
    step_ms, synth_ms, rdm_ms, launches, tm = [], [], [], 0, None
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.simulate(path, out=adc)
        sim.rdm(adc, rdm)
        e1.record(stream)
        tm = pkg.bart_get_timing(sim.ctx)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        synth_ms.append(tm["synthesis_ms"])
        rdm_ms.append(tm["rdm_ms"])
        launches += tm["launches"]
    return {"step_ms": step_ms, "synth_ms": synth_ms, "rdm_ms": rdm_ms, "launches": launches,
            "last": tm}


def e2e_run(pkg, torch, sim, scene, path: int, steps: int, job_terms_per_step: float) -> dict:
    """End to end through the public C-ABI with host buffers: every step
    uploads the meshes and instances from pinned host memory, sets the
    radar, simulates the frame, forms the RDM and reads it back
    (bart_frame_host)."""
    import ctypes
    from paper_2208_10939_gb300 import sharding
    L = pkg.load_library()
    r = scene.radar
    hm = [(torch.from_numpy(m.verts).pin_memory(), torch.from_numpy(m.tris).pin_memory(),
           torch.from_numpy(m.rho).pin_memory(), pkg.MESH_TWO_SIDED if m.two_sided else 0)
          for m in scene.meshes]
    h_rdm = torch.empty((r.M, r.N), dtype=torch.float32).pin_memory()
    insts = pkg.make_instances(scene.instances)
    radar_c = pkg.make_radar(r)
    mid = ctypes.c_int32()
    h2d = sum(v.numel() * 8 + t.numel() * 4 + p.numel() * 4 for v, t, p, _ in hm)
    h2d += ctypes.sizeof(insts) + ctypes.sizeof(pkg.bart_radar)

    def step():
        pkg._check(L.bart_mesh_clear(sim.ctx))
        for v, t, p, fl in hm:
            pkg._check(L.bart_mesh_upload(sim.ctx, v.data_ptr(), v.shape[0], t.data_ptr(),
                                          t.shape[0], p.data_ptr(), fl, ctypes.byref(mid)))
        pkg._check(L.bart_scene_set(sim.ctx, ctypes.cast(insts, ctypes.c_void_p), len(insts)))
        pkg._check(L.bart_radar_set(sim.ctx, ctypes.byref(radar_c)))
        pkg._check(L.bart_frame_host(sim.ctx, float(scene.t0), path, h_rdm.data_ptr(), None))

    step()
    sharding.reduce_scalar(0.0)          # barrier-like sync of the ranks
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    e2e_s = sharding.reduce_scalar(time.perf_counter() - t, "max")
    return {"value": job_terms_per_step * steps / e2e_s, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(r.M * r.N * 4),
            "ms_per_step": 1e3 * e2e_s / steps}


def sedan_lines(pkg, sg, torch, dev, args, peaks) -> dict:
    """The moving-sedan frame (config 2): mixed path with the autotuned
    layout, its synthesis roofline, the plain FP64 path on the same frame,
    and the point cloud of the mixed cube with receiver noise."""
    scene = sg.car_scene()
    sim = pkg.Simulator(dev.index or 0)
    try:
        sim.load_scene(scene)
        r = scene.radar
        adc = torch.empty((r.O, r.N, r.M), dtype=torch.complex64, device=dev)
        rdm = torch.empty((r.M, r.N), dtype=torch.float32, device=dev)
        flush = (None if args.no_flush else
                 torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev))
        stream = torch.cuda.current_stream(dev)
        pkg.bart_set_timing(sim.ctx, True)
        _, st = sim.simulate(pkg.PATH_MIXED, out=adc, stats=True)
        terms = st["n_terms"]
        if args.synth_layout:
            S_fix, T_fix = (int(x) for x in args.synth_layout.split(","))
            pkg.bart_set_synth_layout(sim.ctx, S_fix, T_fix)
            tune = {"best": (S_fix, T_fix), "source": "--synth-layout"}
        elif not args.no_autotune:
            tune = pkg.bart_autotune(sim.ctx, 0.0, adc, reps=2)
        else:
            tune = None
        for _ in range(3):
            sim.simulate(pkg.PATH_MIXED, out=adc)
            sim.rdm(adc, rdm)
        sim.sync()
        tf = timed_frames(pkg, torch, sim, adc, rdm, flush, stream, args.sedan_steps,
                          pkg.PATH_MIXED)
        synth_avg = statistics.mean(tf["synth_ms"]) / max(1, tf["last"]["synthesis_launches"])
        out = {"workload": SEDAN, "facets": st["n_facets"], "echo_terms_per_frame": terms,
               "value": terms * len(tf["step_ms"]) / (sum(tf["step_ms"]) / 1e3), "unit": UNIT,
               "ms_per_step": statistics.mean(tf["step_ms"]),
               "frames_per_s": 1e3 / statistics.mean(tf["step_ms"]),
               "synthesis_ms": synth_avg,
               "synthesis_layout": None if tune is None else
               {"samples_per_lane": tune["best"][0], "tiles_per_item": tune["best"][1]},
               "stages_ms_last_step": {k: tf["last"][k] for k in
                                       ("scene_ms", "bvh_ms", "visibility_ms", "kinematics_ms",
                                        "synthesis_ms", "rdm_ms")}}
        if peaks:
            ach = terms * OPS_PER_TERM / (synth_avg / 1e3) / 1e12
            out["roofline_frac_of_measured_fp32"] = ach / peaks["fp32_fma_pipe_tops"]
        # plain FP64 path on the same frame (the parity reference path)
        adc64 = torch.empty((r.O, r.N, r.M), dtype=torch.complex128, device=dev)
        if args.fp64_steps > 0:
            sim.simulate(pkg.PATH_FP64, out=adc64)
            sim.sync()
            t64 = timed_frames(pkg, torch, sim, adc64, rdm, flush, stream, args.fp64_steps,
                               pkg.PATH_FP64)
            out["fp64_path"] = {"value": terms * len(t64["step_ms"]) / (sum(t64["step_ms"]) / 1e3),
                                "unit": UNIT, "ms_per_step": statistics.mean(t64["step_ms"]),
                                "synthesis_ms": statistics.mean(t64["synth_ms"])}
            if peaks:
                out["fp64_path"]["fp64_fma_tops_measured"] = peaks["fp64_fma_tops"]
        del adc64
        out["point_cloud"] = detect_timing(pkg, torch, sim, adc, stream)
        return out
    finally:
        sim.close()


def double_bounce_lines(pkg, sg, torch, dev, args, peaks) -> dict:
    """The sedan on a ground patch with the double-bounce paths (Sec. 2.2,
    two facets): mixed-path frames (simulate + RDM) with and without double
    bounce, the discovery and FP64 synthesis stage times, the virtual facets
    and the double-bounce echo terms."""
    scene = sg.sedan_ground_scene()
    sim = pkg.Simulator(dev.index or 0)
    try:
        r = scene.radar
        adc = torch.empty((r.O, r.N, r.M), dtype=torch.complex64, device=dev)
        rdm = torch.empty((r.M, r.N), dtype=torch.float32, device=dev)
        flush = (None if args.no_flush else
                 torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev))
        stream = torch.cuda.current_stream(dev)
        out = {"workload": BOUNCE}
        for on in (False, True):
            scene.radar.double_bounce = on
            sim.load_scene(scene)
            pkg.bart_set_timing(sim.ctx, True)
            _, st = sim.simulate(pkg.PATH_MIXED, out=adc, stats=True)
            for _ in range(3):
                sim.simulate(pkg.PATH_MIXED, out=adc)
                sim.rdm(adc, rdm)
            sim.sync()
            tf = timed_frames(pkg, torch, sim, adc, rdm, flush, stream, args.bounce_steps,
                              pkg.PATH_MIXED)
            key = "with_double_bounce" if on else "single_bounce_only"
            out[key] = {"ms_per_step": statistics.mean(tf["step_ms"]),
                        "frames_per_s": 1e3 / statistics.mean(tf["step_ms"]),
                        "echo_terms_single_bounce": st["n_terms"]}
            if on:
                dsc, syn = [], []
                for _ in range(args.bounce_steps):
                    sim.simulate(pkg.PATH_MIXED, out=adc)
                    tm = pkg.bart_get_timing(sim.ctx)
                    dsc.append(tm["bounce_discovery_ms"])
                    syn.append(tm["bounce_synthesis_ms"])
                bt = st["n_bounce_terms"]
                syn_s = statistics.median(syn) / 1e3
                if peaks:
                    ach = bt * BOUNCE_OPS_PER_TERM / syn_s / 1e12
                    prof = (BOUNCE_PROFILE if BOUNCE_PROFILE["sources_sha256_16"] ==
                            synth_sources_hash(BOUNCE_SOURCES) else None)
                    out["roofline"] = {
                        "bound": "alu", "kernel": "bounce_synth_f32_kernel<8>",
                        "ops_per_term": BOUNCE_OPS_PER_TERM, "achieved": ach,
                        "peak": peaks["fp32_fma_pipe_tops"], "frac": ach / peaks["fp32_fma_pipe_tops"],
                        "unit": "Top/s (FP32 FMA-pipe operations)",
                        "peak_basis": "measured (bart_measure_peaks)",
                        "ncu": prof,
                        "note": "per-record work (FP64 rows and phases, per-lane start "
                                "phasors) is amortised over 8 samples per lane"}
                out.update({
                    "facets": st["n_facets"], "virtual_facets": st["n_bounce_facets"],
                    "double_bounce_terms_per_frame": bt,
                    "discovery_ms": statistics.median(dsc),
                    "bounce_synthesis_ms": statistics.median(syn),
                    "bounce_synthesis_terms_per_s": bt / (statistics.median(syn) / 1e3),
                    "gpu_launches": tf["launches"]})
                if peaks:
                    out["fp64_fma_tops_measured"] = peaks["fp64_fma_tops"]
        scene.radar.double_bounce = True
        return out
    finally:
        sim.close()


def run_probe(args) -> None:
    """One stage alone (for ncu captures of a representative launch): warm-up
    launches, then ``--steps`` timed ones (CUDA events); prints one JSON
    line."""
    import torch
    import paper_2208_10939_gb300 as pkg
    import scenegen as sg
    dev = torch.device("cuda:0")
    sim = pkg.Simulator(0)
    rng = np.random.default_rng(1)
    try:
        if args.probe == "rdm":
            O, N, M = 192, 256, 512
            radar = sg.make_radar(M, N, 12, 16, 10.24e6, 12.5e12, tx_spacing_wl=8.0)
            pkg.bart_radar_set(sim.ctx, radar)
            cube = torch.complex(torch.from_numpy(rng.normal(size=(O, N, M)).astype(np.float32)),
                                 torch.from_numpy(rng.normal(size=(O, N, M)).astype(np.float32)))
            x = cube.to(dev)
            out = torch.empty((M, N), dtype=torch.float32, device=dev)
            run = lambda: pkg.bart_form_rdm(sim.ctx, x, out)
            what = f"RDM of a {O}x{N}x{M} complex64 cube"
        elif args.probe == "bounce":
            sc = sg.sedan_ground_scene()
            sim.load_scene(sc)
            x = torch.empty(sim.adc_shape(), dtype=torch.complex64, device=dev)
            run = lambda: sim.simulate(pkg.PATH_MIXED, out=x)
            what = "mixed-path frame of the sedan on a ground patch, double bounce on"
        else:
            sc = sg.car_scene()
            sim.load_scene(sc)
            shape = sim.adc_shape()
            G = torch.from_numpy(rng.normal(size=shape) + 1j * rng.normal(size=shape)).to(dev)
            nv = sum(sc.meshes[i.mesh_id].verts.shape[0] for i in sc.instances)
            nf = sum(sc.meshes[i.mesh_id].tris.shape[0] for i in sc.instances)
            gv = torch.empty((nv, 3), dtype=torch.float64, device=dev)
            gr = torch.empty(nf, dtype=torch.float64, device=dev)
            run = lambda: pkg.bart_simulate_adjoint(sim.ctx, 0.0, G, gv, gr, mixed=True)
            what = "mixed adjoint of the sedan (vertex and reflectivity gradients)"
        for _ in range(max(1, args.warmup)):
            run()
        torch.cuda.synchronize()
        ms = []
        for _ in range(max(1, args.steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        print(json.dumps({"probe": args.probe, "what": what, "ms_median": statistics.median(ms),
                          "ms_min": min(ms), "steps": len(ms)}))
    finally:
        sim.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.probe:
        run_probe(args)
        return
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import paper_2208_10939_gb300 as pkg
    from paper_2208_10939_gb300 import sharding
    import scenegen as sg
    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    peaks = None if args.no_peaks else measure_peaks(pkg, local)

    # ---------------- headline frame ----------------
    if args.workload == "intersection":
        seed = 3 + rank
        scene = sg.intersection_scene(seed=seed)
        workload = WORKLOAD
    else:
        seed = 2 + rank
        scene = sg.car_scene(seed=seed)
        workload = SEDAN
    if args.chirps or args.array:
        r0 = scene.radar
        P_, Q_ = ((int(x) for x in args.array.lower().split("x")) if args.array
                  else (r0.P, r0.Q))
        scene.radar = sg.Radar(f0=r0.f0, slope=r0.slope, fs=r0.fs, Tc=r0.Tc, M=r0.M,
                               N=args.chirps or r0.N, tx=r0.tx[:P_], rx=r0.rx[:Q_],
                               intra_chirp_motion=r0.intra_chirp_motion)
        workload += f" (profiling cut: {P_}TXx{Q_}RX, {scene.radar.N} chirps)"
    sim = pkg.Simulator(local)
    sim.load_scene(scene)
    r = scene.radar
    O, N, M = r.O, r.N, r.M
    adc = torch.empty((O, N, M), dtype=torch.complex64, device=dev)
    rdm = torch.empty((M, N), dtype=torch.float32, device=dev)
    flush = (None if args.no_flush else
             torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev))
    pkg.bart_set_timing(sim.ctx, True)
    _, st = sim.simulate(pkg.PATH_MIXED, out=adc, stats=True)
    terms = st["n_terms"]
    layout = None
    if args.synth_layout:
        S_fix, T_fix = (int(x) for x in args.synth_layout.split(","))
        pkg.bart_set_synth_layout(sim.ctx, S_fix, T_fix)
        layout = {"samples_per_lane": S_fix, "tiles_per_item": T_fix, "source": "--synth-layout"}
    elif args.workload == "sedan" and not args.no_autotune:
        tune = pkg.bart_autotune(sim.ctx, 0.0, adc, reps=2)
        layout = {"samples_per_lane": tune["best"][0], "tiles_per_item": tune["best"][1],
                  "source": "bart_autotune"}
    for _ in range(args.warmup):
        sim.simulate(pkg.PATH_MIXED, out=adc)
        sim.rdm(adc, rdm)
    sim.sync()
    stream = torch.cuda.current_stream(dev)
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    tf = timed_frames(pkg, torch, sim, adc, rdm, flush, stream, args.steps, pkg.PATH_MIXED)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    sim.sync()
    last_tm = tf["last"]
    # replicas: whole-job terms over the slowest rank's time
    job = sharding.job_throughput(float(terms) * args.steps, float(sum(tf["step_ms"])) / 1e3)
    total_ms = 1e3 * job["seconds"]
    job_terms_per_step = job["work"] / args.steps
    value = job["per_second"]
    frames = world * args.steps / (total_ms / 1e3)

    # dominant kernel: echo synthesis, average launch duration from CUDA events
    synth_launches = max(1, last_tm["synthesis_launches"])
    synth_avg_ms = statistics.mean(tf["synth_ms"]) / synth_launches
    achieved = terms / synth_launches * OPS_PER_TERM / (synth_avg_ms / 1e3) / 1e12
    S_used = layout_samples(M, 0 if layout is None else layout["samples_per_lane"])
    prof = synth_profile(S_used)
    if peaks:
        peak, peak_basis = peaks["fp32_fma_pipe_tops"], (
            "measured: FP32 FMA-pipe operations/s of this GPU (bart_measure_peaks, the faster "
            "of scalar and packed f32x2 FMA chains)")
    else:
        peak, peak_basis = 152 * 128 * 2.070e9 / 1e12, "nominal: 152 SM x 128 lanes x 2070 MHz"
    roofline = {"bound": "alu", "kernel": f"synth_mixed_kernel<{S_used}, *>",
                "achieved": achieved, "peak": peak, "unit": "Top/s (FP32 FMA-pipe operations)",
                "frac": achieved / peak,
                "traffic": None if prof is None
                else (prof["dram_read_bytes_per_channel_facet"] * terms / (N * M)
                      + prof["dram_write_bytes_per_row"] * O * N) / synth_launches,
                "traffic_unit": "bytes per launch (ncu dram reads of a cut per (channel, lit facet) "
                                "+ writes per (channel, chirp) row)",
                "ops_per_term": OPS_PER_TERM, "launch_ms": synth_avg_ms,
                "ncu_fma_pipe_active": None if prof is None else prof["fma_pipe_active"],
                "peak_basis": peak_basis}

    e2e = e2e_run(pkg, torch, sim, scene, pkg.PATH_MIXED, args.e2e_steps, job_terms_per_step)
    want_host = rank == 0 and world == 1 and not args.no_cpu_baseline
    h_adc = adc.cpu().numpy() if want_host else None
    # the spectral path (inverse-FFT route) on the same frame
    spectral, h_spec = None, None
    if args.spectral_steps > 0 and world == 1:
        sim.simulate(pkg.PATH_SPECTRAL, out=adc)
        sim.sync()
        ts = timed_frames(pkg, torch, sim, adc, rdm, flush, stream, args.spectral_steps,
                          pkg.PATH_SPECTRAL)
        spectral = {"value": terms * len(ts["step_ms"]) / (sum(ts["step_ms"]) / 1e3),
                    "unit": UNIT, "ms_per_step": statistics.mean(ts["step_ms"]),
                    "synthesis_ms": statistics.mean(ts["synth_ms"]),
                    "speedup_vs_mixed_synthesis": statistics.mean(tf["synth_ms"]) /
                    statistics.mean(ts["synth_ms"])}
        if want_host:
            h_spec = adc.cpu().numpy()
    stages = {k: last_tm[k] for k in ("scene_ms", "bvh_ms", "visibility_ms", "kinematics_ms",
                                      "synthesis_ms", "rdm_ms")}
    # the RDM against HBM over the library's RDM stage time: algorithmic bytes
    # of two FFT passes, each reading and writing the complex64 cube (32 B per
    # sample); also the stricter bound of a single pass that reads the cube
    # once and writes the FP32 map (8 B per sample)
    hbm_peak, hbm_basis = measured_hbm_gbs()
    rdm_bytes = O * N * M * 32
    once_bytes = O * N * M * 8 + M * N * 4
    rdm_ms = statistics.median(tf["rdm_ms"]) if tf.get("rdm_ms") else stages["rdm_ms"]
    rdm_line = {"bound": "hbm", "kernels": "range_fft_reg_kernel, doppler_sum_reg_kernel, "
                                          "rdm_sum_kernel",
                "ms": rdm_ms, "algorithmic_bytes": rdm_bytes,
                "bytes_per_sample": 32,
                "achieved": rdm_bytes / (rdm_ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": rdm_bytes / (rdm_ms / 1e3) / 1e9 / hbm_peak,
                "read_once_bytes": once_bytes,
                "read_once_frac": once_bytes / (rdm_ms / 1e3) / 1e9 / hbm_peak,
                "peak_basis": hbm_basis}
    sim.close()
    del adc, rdm, flush
    torch.cuda.empty_cache()

    cpu = None
    if h_adc is not None:
        cpu = cpu_baseline(scene, args.cpu_seconds, h_adc,
                           None if h_spec is None else {"spectral_frame": h_spec})
        if spectral is not None and "spectral_frame_rel_l2_vs_oracle" in cpu:
            spectral["rel_l2_vs_oracle"] = cpu["spectral_frame_rel_l2_vs_oracle"]
        del h_adc, h_spec
    sedan = None
    if world == 1 and not args.no_sedan and args.workload == "intersection":
        sedan = sedan_lines(pkg, sg, torch, dev, args, peaks)
    bounce = None
    if world == 1 and args.bounce_steps > 0:
        bounce = double_bounce_lines(pkg, sg, torch, dev, args, peaks)
    adj = None
    if world == 1 and args.adjoint_reps > 0:
        adj = adjoint_timing(pkg, sg, torch, dev, args.adjoint_reps)
    batch = batch_small = None
    if world == 1 and args.dataset_scenes > 0:
        batch = dataset_run(pkg, sg, torch, dev, args.dataset_scenes,
                            min(args.dataset_per_scene, args.dataset_scenes))
    if world == 1 and args.batch_scenes > 0:
        # small scenes, where per-scene launches leave the GPU under-filled
        batch_small = dataset_batch(pkg, sg, torch, dev, 2 * args.batch_scenes,
                                    2 * args.batch_size, 5_000, 10_000)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "path": "mixed (FP64 phase, FP32 phasors, Kahan)",
                   "adc": "complex64", "rdm": f"{M}x{N} fp32", "facets": st["n_facets"],
                   "echo_terms_per_frame": terms,
                   "l2": "working set larger than L2 (facet records, kinematics rows, ADC "
                         "cube)" + ("" if args.no_flush else
                                    "; also flushed between steps (256 MB write)"),
                   "parallelism": f"replicas x{world}", "seed": seed,
                   "synthesis_layout": layout},
        "frames_per_s": frames,
        "stages_ms_last_step": stages,
        "roofline": roofline,
        "spectral_path": spectral,
        "rdm": rdm_line,
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": tf["launches"],
        "cpu_baseline": cpu,
        "peaks": peaks,
        "grazing_pairs": st["n_grazing"],
        "moving_sedan": sedan,
        "double_bounce": bounce,
        "differentiable_echo": adj,
        "dataset": batch,
        "dataset_batch_small": batch_small,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
        if args.log:
            rec = dict(out)
            rec["run"] = {"time": time.time(), "argv": sys.argv[1:], "seed": seed,
                          "host_cores": os.cpu_count()}
            with open(args.log, "a") as fh:
                fh.write(json.dumps(rec) + "\n")
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
