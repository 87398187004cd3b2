"""Pins of the FP64 oracle for the learned cluster proposal (k-means and the MLP)."""
import numpy as np
import pytest

import oracle
import pts_inputs as P


def _params(seed, shapes, scale=0.3):
    din, h1, h2, out = shapes
    g = P.SplitMix64(seed)
    mk = lambda r, c: scale * g.normal(r * c).reshape(r, c)  # noqa: E731
    return {"W1": mk(h1, din), "b1": 0.1 * g.normal(h1), "W2": mk(h2, h1), "b2": 0.1 * g.normal(h2),
            "W3": mk(out, h2), "b3": 0.1 * g.normal(out)}


def test_mlp_gradients_match_central_differences(oracle_lib):
    shapes = (5, 7, 6, 9)
    prm = _params(1, shapes)
    X = P.random_matrix(2, 4, 5)
    y = np.array([0, 8, 3, 3], np.int32)

    def loss(p):
        return oracle.ce_loss(oracle.mlp_forward(X, p)["Z"], y)[0]

    cache = oracle.mlp_forward(X, prm)
    _, Pm = oracle.ce_loss(cache["Z"], y)
    g = oracle.mlp_backward(X, prm, cache, Pm, y)
    h = 1e-6
    for k in prm:
        num = np.zeros_like(prm[k])
        it = np.nditer(prm[k], flags=["multi_index"])
        for _ in it:
            i = it.multi_index
            pp = {kk: v.copy() for kk, v in prm.items()}
            pm = {kk: v.copy() for kk, v in prm.items()}
            pp[k][i] += h
            pm[k][i] -= h
            num[i] = (loss(pp) - loss(pm)) / (2 * h)
        err = np.linalg.norm(g[k] - num) / max(np.linalg.norm(num), 1e-12)
        assert err < 1e-7, (k, err)


def test_cross_entropy_uniform_logits(oracle_lib):
    shapes = (4, 3, 3, 1024)
    prm = {k: np.zeros_like(v) for k, v in _params(3, shapes).items()}
    X = P.random_matrix(4, 6, 4)
    Z = oracle.mlp_forward(X, prm)["Z"]
    loss, Pm = oracle.ce_loss(Z, np.arange(6, dtype=np.int32))
    assert loss == pytest.approx(np.log(1024.0), rel=1e-14)
    np.testing.assert_allclose(Pm, 1.0 / 1024, rtol=1e-14)


def test_gelu_forward_closed_form(oracle_lib):
    # identity weights on one unit: h1 = gelu(x) = x * Phi(x); Phi(0) = 1/2, Phi(-inf) = 0
    prm = {"W1": np.array([[1.0]]), "b1": np.zeros(1), "W2": np.array([[1.0]]), "b2": np.zeros(1),
           "W3": np.array([[1.0]]), "b3": np.zeros(1)}
    X = np.array([[0.0], [2.0], [-30.0]])
    c = oracle.mlp_forward(X, prm)
    assert c["H1"][0, 0] == 0.0
    assert c["H1"][2, 0] == pytest.approx(0.0, abs=1e-150)
    # Phi(2) = 0.977249868051821 (standard normal table value)
    assert c["H1"][1, 0] == pytest.approx(2.0 * 0.977249868051821, rel=1e-12)


def test_kmeans_assign_matches_broadcast_argmin(oracle_lib):
    Y = P.random_matrix(5, 300, 6)
    C = P.random_matrix(6, 17, 6)
    a, cost = oracle.kmeans_assign(Y, C)
    D = ((Y[:, None, :] - C[None, :, :]) ** 2).sum(-1)
    np.testing.assert_array_equal(a, D.argmin(1))
    np.testing.assert_allclose(cost, D.min(1), rtol=1e-13)


def test_kmeans_update_is_member_mean(oracle_lib):
    Y = P.random_matrix(7, 200, 3)
    a = P.random_nn(8, 200, 9)
    C, cnt = oracle.kmeans_update(Y, a, 9)
    for c in range(9):
        m = a == c
        assert cnt[c] == m.sum()
        if m.any():
            np.testing.assert_allclose(C[c], Y[m].mean(0), rtol=1e-13)


def test_kmeans_recovers_separated_blobs(oracle_lib):
    k, per, d = 6, 40, 4
    centers = 20.0 * P.random_matrix(9, k, d)
    Y = np.concatenate([centers[c] + 0.1 * P.random_matrix(10 + c, per, d) for c in range(k)])
    truth = np.repeat(np.arange(k), per)
    u = P.SplitMix64(11).uniform(k)
    C, a, hist = oracle.kmeans(Y, k, u, iters=30)
    # same partition up to relabelling
    for c in range(k):
        assert len(set(a[truth == c])) == 1
    assert len(set(a)) == k
    assert np.all(np.diff(hist) <= 1e-9 * hist[0])


def test_kmeans_pp_picks_distinct_points(oracle_lib):
    Y = P.random_matrix(12, 50, 3)
    u = P.SplitMix64(13).uniform(50)
    C, idx = oracle.kmeans_pp(Y, 50, u)
    assert idx[0] == int(u[0] * 50)
    assert len(set(idx.tolist())) == 50
    np.testing.assert_array_equal(C, Y[idx])


def test_kmeans_empty_clusters_reseed_with_largest_cost_unused_points(oracle_lib):
    """Reading c-17: a cluster left without members takes the point of largest assignment cost
    not yet used in the same update (smallest index on ties), so two empty clusters take the
    two costliest points in cost order.  Hand-built 1-D case: centroids 0, 10, 1000 and 2000 over
    the points 0, 0.1, 10, 10.2 and 50 leave clusters 2 and 3 empty."""
    Y = np.array([[0.0], [0.1], [10.0], [10.2], [50.0]])
    C0 = np.array([[0.0], [10.0], [1000.0], [2000.0]])
    a, cost = oracle.kmeans_assign(Y, C0)
    np.testing.assert_array_equal(a, [0, 0, 1, 1, 1])
    np.testing.assert_allclose(cost, [0.0, 0.01, 0.0, 0.04, 1600.0], rtol=1e-12, atol=1e-15)
    C, cnt = oracle.kmeans_update(Y, a, 4, cost)
    np.testing.assert_array_equal(cnt, [2, 3, 0, 0])
    assert C[0, 0] == pytest.approx(0.05, rel=1e-14)
    assert C[1, 0] == pytest.approx((10.0 + 10.2 + 50.0) / 3, rel=1e-14)
    assert C[2, 0] == 50.0           # largest cost, 1600
    assert C[3, 0] == 10.2           # the next largest unused, 0.04 (not 50 again)
    # equal costs: the smallest index among the unused points
    Y2 = np.array([[0.0], [2.0], [4.0], [6.0]])
    C2 = np.array([[1.0], [5.0], [100.0]])
    a2, cost2 = oracle.kmeans_assign(Y2, C2)
    np.testing.assert_array_equal(a2, [0, 0, 1, 1])
    assert np.all(cost2 == 1.0)
    C2n, cnt2 = oracle.kmeans_update(Y2, a2, 3, cost2)
    assert cnt2[2] == 0 and C2n[2, 0] == 0.0
    # without costs an empty cluster keeps no re-seed (stays at zero in the fresh array)
    C3, _ = oracle.kmeans_update(Y, a, 4)
    assert C3[2, 0] == 0.0 and C3[3, 0] == 0.0


def test_kmeans_duplicate_points_empty_a_cluster_and_lloyd_reseeds(oracle_lib):
    """Two distinct values and k = 3: after k-means++ has taken both, every distance is 0 and its
    third pick lands on a duplicate, whose cluster loses every tie to the lower id and is empty.
    Lloyd then re-seeds it with the unused point of largest cost (all costs 0: the smallest
    index), which here is point 0, a duplicate again -- so the cluster stays empty and the run
    stops when the assignment repeats."""
    Y = np.array([[0.0, 0.0]] * 4 + [[3.0, 4.0]] * 4)
    u = np.array([0.0, 0.5, 0.99])
    Cpp, idx = oracle.kmeans_pp(Y, 3, u)
    assert idx[0] == 0 and Y[idx[1]].tolist() == [3.0, 4.0]
    C, a, hist = oracle.kmeans(Y, 3, u, iters=10)
    np.testing.assert_array_equal(np.bincount(a, minlength=3)[:2], [4, 4])
    assert np.sum(a == 2) == 0
    assert hist[-1] == 0.0
