"""Leaf lists of octree block forests over the unit cube.

A forest has R root blocks per axis (R^3 roots of edge 1/R).  A block is the key (level, i, j, k): it covers
[i, i+1] x [j, j+1] x [k, k+1] times 1/(R * 2^level).  Refinement splits a block into its 8 children at
level + 1.  These functions only build geometry; the solver receives the final leaf list.
"""
from __future__ import annotations

import math
from typing import Iterable

import numpy as np


def _extent(R: int, level: int) -> float:
    return 1.0 / (R * 2.0 ** level)


def _children(key):
    l, i, j, k = key
    return [(l + 1, 2 * i + a, 2 * j + b, 2 * k + c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]


def _box(R, key):
    l, i, j, k = key
    e = _extent(R, l)
    return np.array([i * e, j * e, k * e]), np.array([(i + 1) * e, (j + 1) * e, (k + 1) * e])


def uniform_leaves(R: int, level: int = 0) -> list[tuple[int, int, int, int]]:
    m = R * 2 ** level
    return [(level, i, j, k) for k in range(m) for j in range(m) for i in range(m)]


def refine_ball(R: int, center, radius: float, max_level: int, open_ball: bool = True):
    """Refine, recursively up to ``max_level``, every block whose closed box meets the ball around ``center``.

    With ``open_ball`` a block is refined when its minimum distance to the centre is < radius, otherwise <= radius.
    """
    c = np.asarray(center, dtype=np.float64)
    out = []
    stack = list(reversed(uniform_leaves(R)))
    while stack:
        key = stack.pop()
        lo, hi = _box(R, key)
        d = math.sqrt(float(np.sum(np.maximum(0.0, np.maximum(lo - c, c - hi)) ** 2)))
        hit = d < radius if open_ball else d <= radius
        if key[0] < max_level and hit:
            stack.extend(reversed(_children(key)))
        else:
            out.append(key)
    return out


def refine_box(R: int, box_lo, box_hi, depth: int, leaves=None):
    """Refine ``depth`` times every leaf whose box overlaps the open box (box_lo, box_hi) with positive volume."""
    lo_b = np.asarray(box_lo, dtype=np.float64)
    hi_b = np.asarray(box_hi, dtype=np.float64)
    cur = list(leaves) if leaves is not None else uniform_leaves(R)
    for _ in range(depth):
        nxt = []
        for key in cur:
            lo, hi = _box(R, key)
            if np.all(lo < hi_b) and np.all(hi > lo_b):
                nxt.extend(_children(key))
            else:
                nxt.append(key)
        cur = nxt
    return cur


def _covering_leaf(leafset, key):
    """The leaf at ``key``'s level or coarser that contains ``key``; None when finer leaves cover it."""
    l, i, j, k = key
    while l >= 0:
        if (l, i, j, k) in leafset:
            return (l, i, j, k)
        l, i, j, k = l - 1, i // 2, j // 2, k // 2
    return None


def balance_2to1(leaves: Iterable, R: int, mode: str = "26"):
    """Refine leaves until any two neighbouring leaves differ by at most one level.

    ``mode`` '26' balances across faces, edges and corners; 'face' across faces only.
    """
    if mode == "26":
        offs = [(a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1) if (a, b, c) != (0, 0, 0)]
    elif mode == "face":
        offs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    else:
        raise ValueError(mode)
    leafset = set(leaves)
    changed = True
    while changed:
        changed = False
        for key in sorted(leafset, key=lambda t: -t[0]):
            if key not in leafset:
                continue
            l, i, j, k = key
            m = R * 2 ** l
            for a, b, c in offs:
                p = (l, i + a, j + b, k + c)
                if not (0 <= p[1] < m and 0 <= p[2] < m and 0 <= p[3] < m):
                    continue
                cov = _covering_leaf(leafset, p)
                if cov is not None and cov[0] < l - 1:
                    leafset.discard(cov)
                    leafset.update(_children(cov))
                    changed = True
    return sorted(leafset, key=lambda t: (t[0], t[3], t[2], t[1]))


def leaves_array(keys, problem: int = 0) -> np.ndarray:
    """Leaf table as int32 rows (problem, level, i, j, k), in the given order."""
    a = np.zeros((len(keys), 5), dtype=np.int32)
    for r, (l, i, j, k) in enumerate(keys):
        a[r] = (problem, l, i, j, k)
    return a


def leaf_keys(leaves: np.ndarray):
    return [tuple(int(v) for v in row[1:5]) for row in np.asarray(leaves)]


def count_cells(leaves, n: int) -> int:
    return len(leaves) * n ** 3


def workload_forest(name: str):
    """(R, n, leaf keys) of the named workload forests.

    'uniform_2x16'    2^3 roots of 16^3 cells (32^3 cells).
    'sphere_2x32'     2^3 roots of 32^3 cells, two levels refined where blocks meet the open ball of radius
                      0.25 around the centre, 26-neighbour 2:1 balance (56 level-1 + 64 level-2 blocks).
    'uniform_8x64'    8^3 roots of 64^3 cells (512^3 cells).
    'sphere_4x32'     4^3 roots of 32^3 cells, sphere-refined two levels as above, 26-neighbour balance.
    Smaller test forests: 'uniform_2x8', 'uniform_2x32', 'sphere_2x8', 'sphere_2x16', 'sphere_2x4'.
    """
    table = {
        "uniform_2x4": (2, 4, "u"), "uniform_2x8": (2, 8, "u"), "uniform_2x16": (2, 16, "u"),
        "uniform_4x16": (4, 16, "u"), "uniform_8x64": (8, 64, "u"), "uniform_4x64": (4, 64, "u"),
        "uniform_2x32": (2, 32, "u"),
        "sphere_2x4": (2, 4, "s"), "sphere_2x8": (2, 8, "s"), "sphere_2x16": (2, 16, "s"),
        "sphere_2x32": (2, 32, "s"), "sphere_4x32": (4, 32, "s"), "sphere_4x8": (4, 8, "s"),
    }
    R, n, kind = table[name]
    if kind == "u":
        keys = uniform_leaves(R)
    else:
        keys = balance_2to1(refine_ball(R, (0.5, 0.5, 0.5), 0.25, 2, open_ball=True), R, "26")
    return R, n, keys


def paper_benchmark_forest(R):
    """The paper's benchmark geometry (Sec. 6) for R^3 root blocks: every root refined once, then the quarter of the
    level-1 blocks with x < 1/2 and y < 1/2 refined once more (22 R^3 leaves; 2:1 balanced by construction).
    Returns leaf keys (level, i, j, k)."""
    keys = []
    m = 2 * R
    for k in range(m):
        for j in range(m):
            for i in range(m):
                if i < R and j < R:
                    keys += [(2, 2 * i + a, 2 * j + b, 2 * k + c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
                else:
                    keys.append((1, i, j, k))
    return keys


def batch_problems(count=256, seed=0, sizes=(16, 32, 64, 128), max_depth=2, box=(0.1, 0.4)):
    """Independent single-root problems: per problem (drawn in this order) the block size n from ``sizes``, the
    refinement depth from {0..max_depth}, box sides U(box) per axis, and the box corner uniform so the box fits;
    blocks meeting the box are refined `depth` times, then 26-neighbour 2:1 balance.

    Returns a list of (n, keys) with keys (level, i, j, k) of a forest with R = 1.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(list(sizes)))
        depth = int(rng.integers(0, max_depth + 1))
        side = rng.uniform(box[0], box[1], size=3)
        lo = rng.uniform(0.0, 1.0 - side)
        keys = balance_2to1(refine_box(1, lo, lo + side, depth), 1, "26")
        out.append((n, keys))
    return out


def batch_leaves(problems):
    """Leaf rows (problem, level, i, j, k) of a batch, problems in order, and the per-problem block sizes."""
    rows = []
    for p, (_, keys) in enumerate(problems):
        rows.extend((p, *key) for key in keys)
    return np.asarray(rows, dtype=np.int32).reshape(-1, 5), np.asarray([n for n, _ in problems], dtype=np.int32)
