"""Pins of the oracle's k-means tree checks (section 2.2's search structure) on hand-built trees
whose answers are known: descent to the expected leaves, the invariants holding on a valid tree
and failing on a corrupted one."""
import numpy as np
import pytest

from oracle import kmtree as OT


def _one_level():
    """Root with 4 leaf children, each a pair of nearby 2-D points."""
    Y = np.array([[0, 0], [0, 1], [10, 0], [10, 1], [0, 10], [1, 10], [10, 10], [11, 10]], dtype=float)
    tree = {"child": np.array([[-2, -3, -4, -5]]), "leaf_begin": np.array([0, 2, 4, 6]),
            "leaf_end": np.array([2, 4, 6, 8]), "perm": np.arange(8),
            "cent": np.array([[[0, 0.5], [10, 0.5], [0.5, 10], [10.5, 10]]], dtype=np.float32)}
    return Y, tree


def _two_level():
    """Root -> 4 internal nodes (groups of 4 around the corners of a square of side 100) -> 4
    single-window leaves each."""
    corners = np.array([[0, 0], [100, 0], [0, 100], [100, 100]], dtype=float)
    offs = np.array([[0, 0], [3, 0], [0, 3], [3, 3]], dtype=float)
    Y = np.concatenate([c + offs for c in corners])          # window 4 g + i
    child = np.zeros((5, 4), dtype=np.int64)
    child[0] = [1, 2, 3, 4]
    cent = np.zeros((5, 4, 2), dtype=np.float32)
    cent[0] = corners + 1.5
    lb, le = [], []
    for g in range(4):
        child[g + 1] = [-2 - (4 * g + i) for i in range(4)]
        cent[g + 1] = corners[g] + offs
        for i in range(4):
            lb.append(4 * g + i)
            le.append(4 * g + i + 1)
    tree = {"child": child, "leaf_begin": np.array(lb), "leaf_end": np.array(le), "perm": np.arange(16), "cent": cent}
    return Y, tree


def test_descent_reaches_the_expected_leaves():
    Y, tree = _one_level()
    np.testing.assert_array_equal(OT.descend(tree, [[0.2, 0.1], [9, 9], [1, 9], [10, 2]]), [0, 3, 2, 1])
    Y2, tree2 = _two_level()
    # a point near window 4 g + i reaches leaf 4 g + i; the tie between leaves 0 and 1 at x = 1.5
    # goes to the smaller child index
    q = np.array([[0.4, 0.2], [102.9, 0.1], [0.1, 102.6], [103.5, 103.5], [1.5, 0.0]])
    np.testing.assert_array_equal(OT.descend(tree2, q), [0, 5, 10, 15, 0])


def test_invariants_hold_on_valid_trees():
    for Y, tree in (_one_level(), _two_level()):
        sizes = OT.check_invariants(tree, Y)
        assert sizes.sum() == len(Y)
    np.testing.assert_array_equal(OT.subtree_ranges(_two_level()[1])[1:], [[0, 4], [4, 8], [8, 12], [12, 16]])


def test_invariants_fail_on_corrupted_trees():
    Y, tree = _two_level()
    bad = {k: v.copy() for k, v in tree.items()}
    bad["perm"][[1, 5]] = bad["perm"][[5, 1]]        # windows 1 and 5 swapped between groups
    with pytest.raises(AssertionError):
        OT.check_invariants(bad, Y)
    bad = {k: v.copy() for k, v in tree.items()}
    bad["leaf_end"][3] = 5                            # overlapping leaves
    with pytest.raises(AssertionError):
        OT.check_invariants(bad, Y)
    bad = {k: v.copy() for k, v in tree.items()}
    bad["cent"][0, 0] = [100, 100]                     # a centroid moved away from its windows
    with pytest.raises(AssertionError):
        OT.check_invariants(bad, Y)
