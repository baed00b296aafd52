"""Host logic of the batched dataset runner (CPU): batch planning, scene
ownership across ranks, and checkpoint / resume -- a run interrupted after
some batches (and after a shard written but never committed) resumes to
exactly the result of an uninterrupted run.  The GPU is replaced by a fake
simulator with the same interface; the GPU path is tested in
test_gpu_batch.py."""
import os

import numpy as np
import pytest

import scenegen as sg
from paper_2208_10939_gb300 import dataset


def tiny_scene(i: int):
    """A one-facet-pair scene whose range encodes its index."""
    return sg.point_target_scene(10.0 + 0.25 * i, 0.0, M=32, N=2)


class FakeSimulator:
    """Deterministic stand-in for the GPU: RDM of scene b = its range."""

    def __init__(self):
        self.calls = []

    def run(self, scenes, keep=()):
        self.calls.append(len(scenes))
        r = scenes[0].radar
        out = np.stack([np.full((r.M, r.N), s.instances[0].pos[1], np.float32) for s in scenes])
        return out, 1e-3 * len(scenes), {q: np.zeros(1) for q in keep}


def test_plan_batches_respects_budgets():
    f = [5, 5, 5, 20, 1, 1, 1, 1]
    b = dataset.plan_batches(f, max_facets=10, max_scenes=3)
    assert b == [[0, 1], [2], [3], [4, 5, 6], [7]]
    assert sorted(p for g in b for p in g) == list(range(len(f)))


def test_owned_scenes_partition_every_index_once():
    got = sorted(i for r in range(3) for i in dataset.owned_scenes(10, r, 3))
    assert got == list(range(10))
    with pytest.raises(ValueError):
        dataset.owned_scenes(10, 3, 3)


def test_interrupted_run_resumes_to_the_uninterrupted_result(tmp_path):
    n = 23
    full = tmp_path / "full"
    st = dataset.run_dataset(str(full), n, tiny_scene, FakeSimulator(), max_facets=4,
                             max_scenes=8, chunk=10)
    assert st["scenes"] == n and not st["stopped"]
    idx_a, rdm_a = dataset.load_dataset(str(full))
    assert list(idx_a) == list(range(n))

    part = tmp_path / "part"
    st1 = dataset.run_dataset(str(part), n, tiny_scene, FakeSimulator(), max_facets=4,
                              max_scenes=8, chunk=10, stop_after_batches=3)
    assert st1["stopped"] and st1["scenes"] == 6
    # a kill after the next shard was written but before the manifest update
    np.save(part / "shard_r0_00003.npy", np.full((2, 32, 2), -1.0, np.float32))
    np.save(part / "shard_r0_00003.idx.npy", np.array([6, 7]))
    sim = FakeSimulator()
    st2 = dataset.run_dataset(str(part), n, tiny_scene, sim, max_facets=4, max_scenes=8,
                              chunk=10)
    assert st2["skipped"] == 6 and st2["scenes"] == n - 6 and sum(sim.calls) == n - 6
    idx_b, rdm_b = dataset.load_dataset(str(part))
    assert list(idx_b) == list(range(n))
    assert np.array_equal(rdm_a, rdm_b)
    # a third call finds nothing to do
    st3 = dataset.run_dataset(str(part), n, tiny_scene, FakeSimulator(), max_facets=4)
    assert st3["scenes"] == 0 and st3["skipped"] == n


def test_manifest_of_another_run_is_refused(tmp_path):
    dataset.run_dataset(str(tmp_path), 5, tiny_scene, FakeSimulator(), max_facets=4)
    with pytest.raises(ValueError):
        dataset.run_dataset(str(tmp_path), 6, tiny_scene, FakeSimulator(), max_facets=4)


def test_spawned_scene_workers_give_the_same_dataset(tmp_path):
    a, b = tmp_path / "a", tmp_path / "b"
    dataset.run_dataset(str(a), 12, tiny_scene, FakeSimulator(), max_facets=6, chunk=5)
    dataset.run_dataset(str(b), 12, tiny_scene, FakeSimulator(), max_facets=6, chunk=5,
                        workers=2)
    ia, ra = dataset.load_dataset(str(a))
    ib, rb = dataset.load_dataset(str(b))
    assert np.array_equal(ia, ib) and np.array_equal(ra, rb)


def _rank_main(rank, world, out, port):
    import torch.distributed as dist
    from paper_2208_10939_gb300 import sharding
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st = dataset.run_dataset(out, 17, tiny_scene, FakeSimulator(), max_facets=4,
                                 rank=rank, world=world)
        total = sharding.reduce_scalar(st["scenes"], "sum")
        assert total == 17
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_a_dataset_without_overlap(tmp_path):
    import torch.multiprocessing as tmp_mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    tmp_mp.spawn(_rank_main, args=(2, str(tmp_path), port), nprocs=2, join=True)
    idx, rdm = dataset.load_dataset(str(tmp_path))
    assert list(idx) == list(range(17))
    assert np.allclose(rdm[:, 0, 0], [10.0 + 0.25 * i for i in range(17)])
    for r in range(2):
        i_r, _ = dataset.load_dataset(str(tmp_path), rank=r)
        assert list(i_r) == dataset.owned_scenes(17, r, 2)
