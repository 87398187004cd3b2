"""The paper's k-means tree search (section 2.2) for the FP64 oracle: greedy descent of a given
tree and the invariants a hierarchical k = 4 k-means tree satisfies.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: plain numpy.  The tree itself is not
re-derived here (a different rounding order of the Lloyd sums gives a different, equally valid
tree); the oracle checks the structure it is given and repeats the descent in FP64.

Tree arrays (as the library exports them): child [internal, 4] with c >= 0 an internal node,
c <= -2 the leaf -c - 2 and -1 no child; leaf_begin / leaf_end ranges of perm; perm the windows
in leaf order; cent [internal, 4, d] the centroids of a node's children.
"""
from __future__ import annotations

import numpy as np


def descend(tree: dict, Y) -> np.ndarray:
    """Leaf reached by every row of Y [n, d]: from the root, the existing child whose centroid is
    nearest (squared Euclidean distance, the smaller child index on ties), down to a leaf."""
    Y = np.asarray(Y, dtype=np.float64)
    child, cent = tree["child"], tree["cent"].astype(np.float64)
    out = np.empty(len(Y), dtype=np.int64)
    for i, y in enumerate(Y):
        node = 0
        while True:
            best, bc = np.inf, -1
            for k in range(4):
                c = int(child[node, k])
                if c == -1:
                    continue
                dist = float(np.sum((y - cent[node, k]) ** 2))
                if dist < best:
                    best, bc = dist, c
            if bc >= 0:
                node = bc
            else:
                out[i] = -bc - 2
                break
    return out


def subtree_ranges(tree: dict) -> np.ndarray:
    """[internal, 2] range of perm each internal node covers (its leaves are contiguous)."""
    child, lb, le = tree["child"], tree["leaf_begin"], tree["leaf_end"]
    ni = len(child)
    rng = np.full((ni, 2), -1, dtype=np.int64)

    def visit(n):
        lo, hi = None, None
        for k in range(4):
            c = int(child[n, k])
            if c == -1:
                continue
            a, b = (visit(c) if c >= 0 else (int(lb[-c - 2]), int(le[-c - 2])))
            lo = a if lo is None else min(lo, a)
            hi = b if hi is None else max(hi, b)
        rng[n] = (lo, hi)
        return lo, hi

    visit(0)
    return rng


def check_invariants(tree: dict, Y, rel_tol: float = 1e-5):
    """Raises AssertionError unless: perm is a permutation of the windows; the leaves tile it
    without overlap; every internal node's children tile its range in child order; every window
    under a child is, in FP64, nearest to that child's centroid among the node's existing children
    (up to rel_tol, for FP32 near-ties).  Returns the leaf sizes."""
    Y = np.asarray(Y, dtype=np.float64)
    N = len(Y)
    perm, lb, le, child, cent = tree["perm"], tree["leaf_begin"], tree["leaf_end"], tree["child"], tree["cent"]
    assert np.array_equal(np.sort(perm), np.arange(N)), "perm is not a permutation"
    order = np.argsort(lb, kind="stable")
    assert lb[order][0] == 0 and le[order][-1] == N and np.all(lb[order][1:] == le[order][:-1]), "leaves do not tile"
    rng = subtree_ranges(tree)
    for n in range(len(child)):
        pos = rng[n, 0]
        for k in range(4):
            c = int(child[n, k])
            if c == -1:
                continue
            a, b = (rng[c] if c >= 0 else (lb[-c - 2], le[-c - 2]))
            assert a == pos, "children do not tile their parent"
            pos = b
            pts = Y[perm[a:b]]
            ex = [kk for kk in range(4) if child[n, kk] != -1]
            d = np.stack([np.sum((pts - cent[n, kk].astype(np.float64)) ** 2, axis=1) for kk in ex], axis=1)
            mine = d[:, ex.index(k)]
            assert np.all(mine <= d.min(axis=1) * (1 + rel_tol) + 1e-9), "a window is not with its nearest centroid"
        assert pos == rng[n, 1]
    return le - lb
