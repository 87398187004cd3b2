"""The paper's k-means tree search (section 2.2; mode "kmtree") on the GPU against the oracle
(`oracle/kmtree.py`): the tree the library builds satisfies the invariants of a k = 4
hierarchical k-means tree over the exemplar windows' PCA coordinates; every query descends to the
leaf the FP64 descent reaches; the result is the exact nearest window of that leaf."""
import numpy as np
import pytest

import oracle
from oracle import kmtree as OT
import pts_inputs as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2006_11851_gb300 as pts  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(DEV)


@pytest.fixture(scope="module")
def tree_index():
    Z = P.synthetic_exemplar(0, 64, 3.0)
    idx = pts.ExemplarIndex(_t(Z), 8, d=24)
    info = pts.build_kmeans_tree(idx, iters=10)
    yield Z, idx, info
    idx.close()


def test_tree_invariants(tree_index):
    Z, idx, info = tree_index
    tree = pts.kmtree_export(idx)
    Y = pts.project_queries(idx, _t(Z), stride=1).cpu().numpy()  # the vectors the tree was built on
    sizes = OT.check_invariants(tree, Y)
    assert info["leaves"] == len(sizes) and info["internal"] == len(tree["child"])
    assert np.mean(sizes < 4) > 0.99
    # rebuilding gives the same tree (the build is deterministic)
    pts.build_kmeans_tree(idx, iters=10)
    again = pts.kmtree_export(idx)
    for k in tree:
        assert np.array_equal(tree[k], again[k]), k


def test_descent_and_leaf_rerank_against_oracle(tree_index):
    Z, idx, _ = tree_index
    X = P.random_patch_init(Z, 128, 128, 8, 3)
    nn, d2 = pts.nn_search(idx, _t(X), 2, "kmtree")
    Q = nn.numel()
    leaves = pts.kmtree_last_leaves(idx, Q)
    tree = pts.kmtree_export(idx)
    Yq = pts.project_queries(idx, _t(X), 2).cpu().numpy()
    assert np.mean(leaves == OT.descend(tree, Yq)) > 0.999  # FP32 near-ties may flip a step
    nn, d2 = nn.cpu().numpy(), d2.cpu().numpy()
    for q in P.sample_indices(11, Q, 400):
        items = tree["perm"][tree["leaf_begin"][leaves[q]]:tree["leaf_end"][leaves[q]]][:32]
        dd = oracle.pair_dist2(X, Z, 8, 2, np.full(len(items), q), items)
        order = np.lexsort((items, dd))
        assert d2[q] == pytest.approx(dd[order[0]], rel=1e-5, abs=1e-6)
        if len(items) == 1 or dd[order[1]] > dd[order[0]] * (1 + 1e-5):
            assert nn[q] == items[order[0]]
