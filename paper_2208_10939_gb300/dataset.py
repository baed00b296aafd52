"""Batched RDM dataset generation with checkpoint and resume.

The paper builds its classifier's training set from parameter sweeps of
simulated scenes (Sec. 3.4).  This runner simulates many independent scenes
-- scene i from a caller-supplied generator ``make_scene(i)`` -- in batches:
each batch is one partitioned frame (``bart_scene_partition``: one
hierarchy with a subtree per scene, one visibility launch, one persistent
synthesis work queue over all scenes' (scene, channel, chirp group, record
chunk) items) followed by one batched range-Doppler map, so that small
scenes share launches.  Batches are cut by a facet budget (device memory)
and by the library's limit of 65535 (scene, channel) rows.

Outputs under ``out_dir`` (per rank r when several processes share a run):

* ``shard_r<r>_<k>.npy``      float32 [b][M][N]  RDMs of the shard's scenes
* ``shard_r<r>_<k>.idx.npy``  int64 [b]          their scene indices
* ``manifest_r<r>.json``      {"n_scenes", "radar", "done": [...], "shards": [...]}

A shard is written under a temporary name and renamed, then the manifest
is rewritten the same way; a run killed at any point therefore resumes from
its last manifest: scenes listed as done are skipped, and a shard whose
scenes never reached the manifest is written again.

Host scene generation (Python, ~50 ms a scene) runs ahead of the GPU in a
pool of worker processes started with ``spawn`` (a forked child of a CUDA
process is unusable), ``workers`` of them; 0 generates inline.
"""
from __future__ import annotations

import json
import os
import time
from typing import Callable, Iterable, List, Optional

import numpy as np

MAX_ROWS = 65535            # (scene, channel) rows of one partitioned frame


def scene_facets(scene) -> int:
    return int(sum(scene.meshes[i.mesh_id].nf for i in scene.instances))


def owned_scenes(n_scenes: int, rank: int, world: int) -> List[int]:
    """Scene indices of ``rank``: i = rank, rank + world, ... (interleaved,
    so that ranks see the same mix of scene sizes on average)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    return list(range(rank, n_scenes, world))


def _atomic_write_bytes(path: str, data: bytes) -> None:
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "wb") as fh:
        fh.write(data)
        fh.flush()
        os.fsync(fh.fileno())
    os.replace(tmp, path)


def _atomic_save_npy(path: str, arr: np.ndarray) -> None:
    tmp = f"{path}.{os.getpid()}.tmp.npy"
    np.save(tmp, arr)
    os.replace(tmp, path)


class Manifest:
    """The completed scene indices of one rank, persisted atomically."""

    def __init__(self, out_dir: str, rank: int, n_scenes: int, radar_desc: dict):
        self.path = os.path.join(out_dir, f"manifest_r{rank}.json")
        self.rank = rank
        self.n_scenes = n_scenes
        self.radar = radar_desc
        self.done: set = set()
        self.shards: List[str] = []
        if os.path.exists(self.path):
            m = json.load(open(self.path))
            if m.get("n_scenes") != n_scenes or m.get("radar") != radar_desc:
                raise ValueError(f"{self.path} belongs to another run (scene count or radar differ)")
            self.done = set(int(i) for i in m["done"])
            self.shards = list(m["shards"])

    def commit(self, shard: str, indices: Iterable[int]) -> None:
        self.done.update(int(i) for i in indices)
        self.shards.append(shard)
        body = {"n_scenes": self.n_scenes, "radar": self.radar, "rank": self.rank,
                "done": sorted(self.done), "shards": self.shards}
        _atomic_write_bytes(self.path, json.dumps(body).encode())


def plan_batches(facets: List[int], max_facets: int, max_scenes: int) -> List[List[int]]:
    """Consecutive groups of positions 0..len-1 whose facet sums stay within
    ``max_facets`` (a larger single scene forms a batch alone) and whose
    sizes stay within ``max_scenes``."""
    out, cur, tot = [], [], 0
    for p, f in enumerate(facets):
        if cur and (tot + f > max_facets or len(cur) >= max_scenes):
            out.append(cur)
            cur, tot = [], 0
        cur.append(p)
        tot += f
    if cur:
        out.append(cur)
    return out


class GpuBatchSimulator:
    """Simulates a batch of scenes sharing one radar on a CUDA device through
    the C-ABI: meshes and instances uploaded, the partition set, one
    mixed-path frame and one batched RDM; returns the RDMs on the host and the
    device time of the frame + RDM (CUDA events on the context's stream)."""

    def __init__(self, device: int = 0, path: Optional[int] = None):
        import torch
        from . import PATH_MIXED, Simulator
        self.torch = torch
        self.sim = Simulator(device)
        self.dev = torch.device(f"cuda:{device}")
        self.path = PATH_MIXED if path is None else path
        self._bufs = {}

    def close(self) -> None:
        self.sim.close()

    def run(self, scenes, keep_adc: Iterable[int] = ()):
        from . import (bart_form_rdm, bart_mesh_clear, bart_mesh_upload, bart_radar_set,
                       bart_scene_partition, bart_scene_set, bart_simulate_frame, _Placed)
        torch = self.torch
        ctx = self.sim.ctx
        bart_mesh_clear(ctx)
        insts, first = [], [0]
        for sc in scenes:
            ids = [bart_mesh_upload(ctx, m.verts, m.tris, m.rho, getattr(m, "two_sided", False))
                   for m in sc.meshes]
            insts += [_Placed(ids[i.mesh_id], i) for i in sc.instances]
            first.append(len(insts))
        radar = scenes[0].radar
        bart_scene_set(ctx, insts)
        bart_scene_partition(ctx, first)
        bart_radar_set(ctx, radar)
        B, O, N, M = len(scenes), radar.O, radar.N, radar.M
        dtype = torch.complex64 if self.path == 1 else torch.complex128
        need = B * O * N * M
        adc = self._bufs.get("adc")
        if adc is None or adc.numel() < need or adc.dtype != dtype:
            adc = self._bufs["adc"] = torch.empty(need, dtype=dtype, device=self.dev)
        rdm = self._bufs.get("rdm")
        if rdm is None or rdm.numel() < B * M * N:
            rdm = self._bufs["rdm"] = torch.empty(B * M * N, dtype=torch.float32, device=self.dev)
        a = adc[:need].view(B, O, N, M)
        r = rdm[:B * M * N].view(B, M, N)
        stream = torch.cuda.current_stream(self.dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bart_simulate_frame(ctx, float(scenes[0].t0), self.path, a)
        bart_form_rdm(ctx, a, r)
        e1.record(stream)
        out = r.cpu().numpy()
        e1.synchronize()
        kept = {p: a[p].cpu().numpy() for p in keep_adc}
        return out, e0.elapsed_time(e1) / 1e3, kept


def _radar_desc(radar) -> dict:
    return {"f0": float(radar.f0), "slope": float(radar.slope), "fs": float(radar.fs),
            "Tc": float(radar.Tc), "M": int(radar.M), "N": int(radar.N),
            "tx": np.asarray(radar.tx, float).round(12).tolist(),
            "rx": np.asarray(radar.rx, float).round(12).tolist()}


def run_dataset(out_dir: str, n_scenes: int, make_scene: Callable[[int], object], simulator,
                *, max_facets: int = 40_000_000, max_scenes: int = 1024, chunk: int = 256,
                workers: int = 0, rank: int = 0, world: int = 1,
                stop_after_batches: Optional[int] = None,
                keep_adc: Iterable[int] = ()) -> dict:
    """Simulate scenes 0..n_scenes-1 owned by ``rank`` (those not yet done)
    into RDM shards under ``out_dir``.  ``simulator.run(scenes, keep)``
    returns (RDMs [b][M][N], device seconds, {position: ADC}).  Scenes are
    generated ``chunk`` at a time (in ``workers`` spawned processes when
    > 0) and cut into batches by ``plan_batches``.  ``stop_after_batches``
    stops after that many batches of this call (a deliberate interruption,
    for tests); ``keep_adc`` lists scene indices whose ADC cubes are
    returned.  Returns counts and timings of this call."""
    os.makedirs(out_dir, exist_ok=True)
    mine = owned_scenes(n_scenes, rank, world)
    probe = make_scene(mine[0]) if mine else None
    manifest = Manifest(out_dir, rank, n_scenes, _radar_desc(probe.radar) if probe else {})
    todo = [i for i in mine if i not in manifest.done]
    keep = set(int(i) for i in keep_adc)
    rows = probe.radar.O if probe else 1
    max_scenes = max(1, min(max_scenes, MAX_ROWS // rows))
    pool = None
    if workers > 0 and len(todo) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        pool = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    stats = {"scenes": 0, "batches": 0, "facets": 0, "device_s": 0.0, "skipped": len(mine) - len(todo),
             "adc": {}}
    t_start = time.perf_counter()
    shard_no = len(manifest.shards)
    try:
        pending = None
        for c0 in range(0, len(todo), chunk):
            idx = todo[c0:c0 + chunk]
            if pool is None:
                scenes = [make_scene(i) for i in idx]
            else:
                if pending is None:
                    pending = pool.map(make_scene, idx, chunksize=4)
                scenes = list(pending)
                nxt = todo[c0 + chunk:c0 + 2 * chunk]
                pending = pool.map(make_scene, nxt, chunksize=4) if nxt else None
            facets = [scene_facets(s) for s in scenes]
            for grp in plan_batches(facets, max_facets, max_scenes):
                sc = [scenes[p] for p in grp]
                ids = [idx[p] for p in grp]
                kp = [q for q, i in enumerate(ids) if i in keep]
                rdm, dev_s, adc = simulator.run(sc, kp)
                for q, a in adc.items():
                    stats["adc"][ids[q]] = a
                name = f"shard_r{rank}_{shard_no:05d}"
                _atomic_save_npy(os.path.join(out_dir, name + ".idx.npy"),
                                 np.asarray(ids, np.int64))
                _atomic_save_npy(os.path.join(out_dir, name + ".npy"),
                                 np.ascontiguousarray(rdm, np.float32))
                manifest.commit(name, ids)
                shard_no += 1
                stats["scenes"] += len(ids)
                stats["batches"] += 1
                stats["facets"] += int(sum(facets[p] for p in grp))
                stats["device_s"] += dev_s
                if stop_after_batches is not None and stats["batches"] >= stop_after_batches:
                    stats["wall_s"] = time.perf_counter() - t_start
                    stats["stopped"] = True
                    return stats
    finally:
        if pool is not None:
            pool.shutdown(cancel_futures=True)
    stats["wall_s"] = time.perf_counter() - t_start
    stats["stopped"] = False
    return stats


def load_dataset(out_dir: str, rank: Optional[int] = None):
    """(scene indices, RDMs) of every committed shard (of one rank, or all),
    sorted by scene index."""
    idx, rdm = [], []
    for f in sorted(os.listdir(out_dir)):
        if not (f.startswith("manifest_r") and f.endswith(".json")):
            continue
        m = json.load(open(os.path.join(out_dir, f)))
        if rank is not None and m["rank"] != rank:
            continue
        for name in m["shards"]:
            idx.append(np.load(os.path.join(out_dir, name + ".idx.npy")))
            rdm.append(np.load(os.path.join(out_dir, name + ".npy")))
    if not idx:
        return np.zeros(0, np.int64), None
    i = np.concatenate(idx)
    r = np.concatenate(rdm)
    order = np.argsort(i, kind="stable")
    return i[order], r[order]
