"""Host-side checks of the library's bounding-volume hierarchy.

The visibility kernel (Sec. 2.2: rays from each facet toward each antenna)
decides occlusion by traversing an LBVH that the GPU builds every frame.  A
wrong hierarchy would not fault: it would silently drop or add occluders.
``check_bvh`` reads the host copy that ``bart_get_bvh`` returns and states
every broken invariant:

* shape: F - 1 internal nodes for F facets, children in range;
* tree: node 0 has no parent, every other internal node and every facet
  leaf has exactly one, and all of them are reachable from node 0 (so there
  is no cycle and no lost subtree);
* boxes: every stored box has min <= max; a leaf's box holds its facet's
  three FP64 vertices; an internal child's two boxes lie inside the slot
  its parent stores for it;
* scenes (a partitioned frame): the subtree under each scene's root holds
  exactly that scene's facets [foff[b], foff[b+1]).

It is plain numpy plus one Python pass over the nodes (about a second per
million facets).
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

BVH_NODE_DTYPE = np.dtype([("lmin", "<f4", (3,)), ("left", "<i4"), ("lmax", "<f4", (3,)),
                           ("right", "<i4"), ("rmin", "<f4", (3,)), ("pad0", "<i4"),
                           ("rmax", "<f4", (3,)), ("pad1", "<i4")])
assert BVH_NODE_DTYPE.itemsize == 64


def _subtree_leaves(left: np.ndarray, right: np.ndarray, root: int, limit: int):
    """Facet ids under ``root`` and the internal nodes visited (None when a
    node repeats or ``limit`` visits pass: not a tree)."""
    if root < 0:
        return [~root], []
    seen_nodes, leaves, stack = [], [], [root]
    while stack:
        k = stack.pop()
        seen_nodes.append(k)
        if len(seen_nodes) > limit:
            return None, None
        for c in (int(left[k]), int(right[k])):
            if c >= 0:
                stack.append(c)
            else:
                leaves.append(~c)
    return leaves, seen_nodes


def check_bvh(nodes: np.ndarray, roots: Sequence[int], tri: np.ndarray,
              foff: Optional[Sequence[int]] = None, max_report: int = 20) -> List[str]:
    """Every broken invariant of the hierarchy (an empty list when sound).

    nodes: ``BVH_NODE_DTYPE`` array (F - 1 internal nodes); roots: the root
    of each scene's subtree (``~facet`` for a one-facet scene); tri: F x 9
    frame-start vertices; foff: S + 1 facet offsets of the scenes (default:
    one scene of all F facets)."""
    tri = np.asarray(tri, np.float64).reshape(-1, 9)
    F = tri.shape[0]
    n = int(nodes.shape[0])
    roots = [int(r) for r in roots]
    foff = [0, F] if foff is None else [int(x) for x in foff]
    errs: List[str] = []

    def report(msg: str, idx) -> None:
        idx = np.asarray(idx).ravel()
        if idx.size:
            errs.append(f"{msg}: {idx.size} case(s), first {idx[:max_report].tolist()}")

    if len(foff) != len(roots) + 1 or foff[0] != 0 or foff[-1] != F:
        errs.append(f"{len(roots)} scene roots do not match the facet offsets {foff[:8]}...")
        return errs
    if n != max(F - 1, 0):
        errs.append(f"{n} internal nodes for {F} facets (expected {max(F - 1, 0)})")
        return errs
    if F == 1:
        if roots != [~0]:
            errs.append(f"one facet: root {roots} (expected [{~0}])")
        return errs

    left = nodes["left"].astype(np.int64)
    right = nodes["right"].astype(np.int64)
    child = np.concatenate([left, right])                  # slot s: node s % n, side s // n
    internal = child >= 0
    out_of_range = np.where(internal, child >= n, ~child >= F)
    report("child index out of range (slot = node + side * n)", np.flatnonzero(out_of_range))
    if out_of_range.any():
        return errs
    parents = np.bincount(child[internal], minlength=n)
    expect = np.ones(n, np.int64)
    expect[0] = 0
    report("internal node with a parent count other than one (node 0: zero)",
           np.flatnonzero(parents != expect))
    leaf_parents = np.bincount(~child[~internal], minlength=F)
    report("facet under a number of leaves other than one", np.flatnonzero(leaf_parents != 1))

    leaves, visited = _subtree_leaves(left, right, 0, n)
    if leaves is None:
        errs.append("a node repeats below node 0 (cycle or shared subtree)")
    elif len(visited) != n or len(leaves) != F:
        errs.append(f"node 0 reaches {len(visited)} of {n} internal nodes and "
                    f"{len(leaves)} of {F} facets")

    smin = np.concatenate([nodes["lmin"], nodes["rmin"]]).astype(np.float64)
    smax = np.concatenate([nodes["lmax"], nodes["rmax"]]).astype(np.float64)
    report("stored box with min > max (slot)", np.flatnonzero((smin > smax).any(axis=1)))
    ls = np.flatnonzero(~internal)
    v = tri[~child[ls]].reshape(-1, 3, 3)                  # (slot, vertex, axis)
    outside = ((v < smin[ls][:, None, :]) | (v > smax[ls][:, None, :])).any(axis=(1, 2))
    report("leaf box that misses a vertex of its facet (slot)", ls[outside])
    cs = np.flatnonzero(internal)
    c = child[cs]
    cmin = np.minimum(nodes["lmin"][c], nodes["rmin"][c]).astype(np.float64)
    cmax = np.maximum(nodes["lmax"][c], nodes["rmax"][c]).astype(np.float64)
    loose = ((cmin < smin[cs]) | (cmax > smax[cs])).any(axis=1)
    report("internal child whose boxes leave its parent's slot (slot)", cs[loose])

    if len(roots) > 1 or foff != [0, F]:
        for b, r in enumerate(roots):
            if r >= n or ~r >= F:
                errs.append(f"scene {b}: root {r} out of range")
                continue
            got, _ = _subtree_leaves(left, right, r, n)
            want = list(range(foff[b], foff[b + 1]))
            if got is None or sorted(got) != want:
                errs.append(f"scene {b}: subtree of root {r} does not hold exactly facets "
                            f"[{foff[b]}, {foff[b + 1]})")
                if len(errs) > max_report:
                    break
    elif roots != [0]:
        errs.append(f"one scene: root {roots} (expected [0])")
    return errs
