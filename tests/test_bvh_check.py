"""CPU tests of the host-side hierarchy checker (diagnostics.check_bvh) on a
hand-built hierarchy: it passes a sound one and names each planted fault --
a box that misses a vertex, a facet under two leaves, a cycle, a child out
of range, a parent slot smaller than its child's boxes, a wrong scene root.
The checker's input format is the C layout of bart_bvh_node (checked here
against gcc's offsets)."""
import os
import subprocess

import numpy as np
import pytest

from paper_2208_10939_gb300.diagnostics import BVH_NODE_DTYPE, check_bvh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# node 0 = (node 1, node 2); node 1 = (~0, node 3); node 3 = (~1, ~2);
# node 2 = (node 4, ~5); node 4 = (~3, ~4).  Scenes: facets 0-2 under node 1,
# facets 3-5 under node 2.
TREE = {0: (1, 2), 1: (~0, 3), 2: (4, ~5), 3: (~1, ~2), 4: (~3, ~4)}


def triangles(seed=1):
    rng = np.random.default_rng(seed)
    base = np.repeat(np.arange(6.0)[:, None], 3, axis=1) * np.array([3.0, 0.5, 0.0])
    return (base[:, None, :] + rng.uniform(-1, 1, size=(6, 3, 3))).reshape(6, 9)


def outward(lo, hi):
    lo32 = lo.astype(np.float32)
    hi32 = hi.astype(np.float32)
    lo32 = np.where(lo32 > lo, np.nextafter(lo32, np.float32(-np.inf)), lo32)
    hi32 = np.where(hi32 < hi, np.nextafter(hi32, np.float32(np.inf)), hi32)
    return lo32, hi32


def build(tri):
    nodes = np.zeros(len(TREE), BVH_NODE_DTYPE)

    def box(c):
        if c < 0:
            v = tri[~c].reshape(3, 3)
            return outward(v.min(axis=0), v.max(axis=0))
        (a0, a1), (b0, b1) = box(TREE[c][0]), box(TREE[c][1])
        return np.minimum(a0, b0), np.maximum(a1, b1)

    for k, (l, r) in TREE.items():
        nodes[k]["left"], nodes[k]["right"] = l, r
        nodes[k]["lmin"], nodes[k]["lmax"] = box(l)
        nodes[k]["rmin"], nodes[k]["rmax"] = box(r)
    return nodes


@pytest.fixture
def sound():
    tri = triangles()
    return build(tri), tri


def test_sound_hierarchy_passes(sound):
    nodes, tri = sound
    assert check_bvh(nodes, [0], tri) == []
    assert check_bvh(nodes, [1, 2], tri, foff=[0, 3, 6]) == []


def test_one_facet(sound):
    _, tri = sound
    assert check_bvh(np.zeros(0, BVH_NODE_DTYPE), [~0], tri[:1]) == []
    assert check_bvh(np.zeros(0, BVH_NODE_DTYPE), [0], tri[:1])


def test_leaf_box_missing_a_vertex(sound):
    nodes, tri = sound
    nodes[3]["lmax"][0] = np.float32(tri[1].reshape(3, 3)[:, 0].max() - 1e-3)
    errs = check_bvh(nodes, [0], tri)
    assert any("misses a vertex" in e for e in errs), errs


def test_facet_under_two_leaves(sound):
    nodes, tri = sound
    nodes[2]["right"] = ~4                        # facet 4 twice, facet 5 never
    errs = check_bvh(nodes, [0], tri)
    assert any("number of leaves other than one" in e for e in errs), errs


def test_cycle(sound):
    nodes, tri = sound
    nodes[4]["left"] = 2                          # node 2 -> node 4 -> node 2
    errs = check_bvh(nodes, [0], tri)
    assert any("parent count" in e for e in errs), errs
    assert any("repeats" in e or "reaches" in e for e in errs), errs


def test_child_out_of_range(sound):
    nodes, tri = sound
    nodes[1]["right"] = 7
    errs = check_bvh(nodes, [0], tri)
    assert any("out of range" in e for e in errs), errs


def test_parent_slot_smaller_than_child(sound):
    nodes, tri = sound
    nodes[0]["rmin"][1] += np.float32(0.25)      # node 2's slot no longer holds its boxes
    errs = check_bvh(nodes, [0], tri)
    assert any("leave its parent's slot" in e for e in errs), errs


def test_wrong_scene_root(sound):
    nodes, tri = sound
    errs = check_bvh(nodes, [3, 2], tri, foff=[0, 3, 6])   # node 3 holds facets 1, 2 only
    assert any("scene 0" in e for e in errs), errs
    assert check_bvh(nodes, [1], tri, foff=[0, 3, 6])      # too few roots


def test_node_record_matches_the_c_layout(tmp_path):
    fields = ["lmin", "left", "lmax", "right", "rmin", "pad0", "rmax", "pad1"]
    prog = tmp_path / "bvh.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "bartsim.h"\n'
                    "int main(void){printf(\"%zu\\n\", sizeof(bart_bvh_node));"
                    + "".join(f'printf("%zu\\n", offsetof(bart_bvh_node, {f}));' for f in fields)
                    + "return 0;}\n")
    exe = tmp_path / "bvh"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                        check=True).stdout.split()))
    assert vals == [BVH_NODE_DTYPE.itemsize] + [BVH_NODE_DTYPE.fields[f][1] for f in fields]
