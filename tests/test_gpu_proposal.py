"""The learned cluster proposal on the GPU against the FP64 oracle and against exact search.

  - tensor-core GEMM of the network: against an FP64 host product (self-test entry point);
  - k-means: same k-means++ uniforms as the oracle, inertia and assignments compared;
  - network gradients: one forward/backward pass against the oracle's FP64 backward on the
    same BF16-rounded weights and inputs (relative Frobenius error per parameter block);
  - search: the proposal never beats exact search, reports exact distances, keeps most exact
    matches, and the synthesis energy stays within 1.01x of exact mode; it is faster.
"""
import time

import numpy as np
import pytest

import oracle
import pts_inputs as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2006_11851_gb300 as pts  # noqa: E402
from paper_2006_11851_gb300.proposal import collect_pairs, subsample  # noqa: E402
from paper_2006_11851_gb300.pyramid import PyramidIndex  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(DEV)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 200, 72), (4096, 256, 1024), (256, 64, 4096)])
def test_gemm_selftest(M, N, K):
    # FP32 accumulation of K exact BF16 products: error relative to sum |terms| ~ K 2^-24
    assert pts.gemm_selftest(M, N, K) < 1e-5 + 2.0 * K * 2.0 ** -24


def test_kmeans_matches_oracle():
    Y = np.concatenate([3.0 * P.random_matrix(20 + c, 1, 16) + P.random_matrix(40 + c, 120, 16) for c in range(40)])
    u = P.SplitMix64(7).uniform(64)
    C_o, a_o, hist = oracle.kmeans(Y.astype(np.float32), 64, u, iters=25)
    C_g, a_g, it = pts.kmeans(_t(Y), 64, u, iters=25)
    a_g = a_g.cpu().numpy()
    inertia_g = ((Y - C_g.cpu().numpy()[a_g]) ** 2).sum()
    inertia_o = ((Y.astype(np.float32).astype(np.float64) - C_o[a_o]) ** 2).sum()
    assert abs(inertia_g / inertia_o - 1) < 1e-4
    assert np.mean(a_g == a_o) > 0.99


def test_kmeans_empty_cluster_reseed_matches_oracle():
    """A hand-found 11-point case whose third Lloyd update leaves cluster 2 empty; the re-seed
    (reading c-17) must take the unused point of largest cost, and two points tie at cost
    1.953125 (exact in FP32), so the smallest index (point 3, not 8) must win.  All coordinates
    are multiples of 1/4, so the GPU's FP32 costs equal the oracle's FP64 ones where it matters."""
    Y = np.array([[0.75, 2.25], [1.75, 3.75], [2.25, 3.25], [2.75, 0.0], [1.0, 1.75], [0.75, 2.25],
                  [1.75, 2.75], [3.25, 3.75], [0.0, 0.5], [2.5, 3.0], [0.0, 2.25]])
    u = np.array([0.2219481468896175, 0.3235902000698858, 0.1342355651416305, 0.7882371723686297])
    C_o, a_o, hist = oracle.kmeans(Y, 4, u, iters=25)
    assert C_o[2].tolist() == [2.75, 0.0]          # the re-seeded centroid is point 3
    C_g, a_g, it = pts.kmeans(_t(Y), 4, u, iters=25)
    np.testing.assert_array_equal(a_g.cpu().numpy(), a_o)
    np.testing.assert_allclose(C_g.cpu().numpy(), C_o, rtol=1e-6)
    assert it == len(hist) - 1


def _mlp_params(seed, C, scale=0.15):
    g = P.SplitMix64(seed)
    shapes = [(256, 64), (256,), (256, 256), (256,), (C, 256), (C,)]
    return [scale * g.normal(int(np.prod(s))).reshape(s) for s in shapes]


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).bfloat16().float().numpy().astype(np.float64)


def test_mlp_gradients_against_oracle():
    C, B = 1024, 64
    blocks = _mlp_params(3, C)
    flat = np.concatenate([b.reshape(-1) for b in blocks]).astype(np.float32)
    X = P.random_matrix(4, B, 64)
    lab = P.random_nn(5, B, C)
    g, loss = pts.mlp_grad(C, _t(flat), _t(X), _t(lab, np.int32))
    g = g.cpu().numpy().astype(np.float64)
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    # oracle on the BF16-rounded weights and inputs the GPU multiplies (biases stay FP32)
    prm = {n: (_bf16(b) if n.startswith("W") else b.astype(np.float32).astype(np.float64)) for n, b in zip(names, blocks)}
    cache = oracle.mlp_forward(_bf16(X), prm)
    loss_o, Pm = oracle.ce_loss(cache["Z"], lab)
    go = oracle.mlp_backward(_bf16(X), prm, cache, Pm, lab)
    assert abs(loss / loss_o - 1) < 1e-2
    o = 0
    for n, b in zip(names, blocks):
        k = b.size
        gg = g[o:o + k].reshape(b.shape)
        o += k
        err = np.linalg.norm(gg - go[n]) / max(np.linalg.norm(go[n]), 1e-30)
        assert err < 2e-2, (n, err)


@pytest.fixture(scope="module")
def trained():
    """Two-level pyramid (64 -> 128 exemplar, windows 16/8, outputs 128/256, d = 64) with a
    proposal of 256 clusters on the fine level, trained on pairs from seeds 0..5."""
    Z = P.synthetic_exemplar(0, 128, 4.0)
    pidx = PyramidIndex(_t(Z), [16, 8], d=64)
    z0 = pidx.exemplars[0].cpu().numpy()
    init = lambda s: _t(P.random_patch_init(z0, 128, 128, 16, s))  # noqa: E731
    y, nn, d2 = collect_pairs(pidx, 1, init, range(6), iters=5)
    y, nn, d2 = subsample(y, nn, d2, 400_000)
    loss = pts.train_proposal(pidx.indices[1], y, nn, d2, n_clusters=256, epochs=6, batch=4096, seed=1)
    yield pidx, init, loss
    pidx.close()


def test_training_reduces_loss(trained):
    _, _, loss = trained
    assert loss[-1] < 0.7 * loss[0]
    assert loss[-1] < np.log(256.0)


def test_fused_inference_matches_gemm_path(trained):
    """The fused inference kernel ranks the same 4 clusters as the training-side GEMMs + top-4."""
    pidx, init, _ = trained
    ix = pidx.indices[1]
    X = init(22)
    pts.synthesize_level(pidx.indices[0], X, 3, mode="exact")
    X = pts.upsample2(X)
    a = pts.proposal_top4(ix, X, 2, fused=True)
    b = pts.proposal_top4(ix, X, 2, fused=False)
    assert torch.equal(a, b)


def test_proposal_search_against_exact(trained):
    pidx, init, _ = trained
    ix = pidx.indices[1]
    X = init(20)
    pts.synthesize_level(pidx.indices[0], X, 5, mode="exact")
    X = pts.upsample2(X)
    pts.synthesize_level(ix, X, 2, mode="exact")  # a mid-synthesis image, as the proposal meets it
    nn_p, d2_p = pts.nn_search(ix, X, 2, "proposal")
    st = ix.search_stats()
    nn_e, d2_e = pts.nn_search(ix, X, 2, "exact")
    nn_p, d2_p, nn_e, d2_e = (t.cpu().numpy() for t in (nn_p, d2_p, nn_e, d2_e))
    assert np.all(d2_p >= d2_e * (1 - 1e-5) - 1e-6)   # never better than exact
    assert np.mean(nn_p == nn_e) > 0.8                  # recall@1
    assert st["fallback_queries"] < 0.5 * st["queries"]
    # distances are the exact distances of the windows returned (oracle, FP64)
    Zf = pidx.exemplars[1].cpu().numpy()
    Xh = X.cpu().numpy()
    sub = P.sample_indices(3, len(nn_p), 256)
    pd = oracle.pair_dist2(Xh, Zf, 8, 2, sub, nn_p[sub])
    np.testing.assert_allclose(d2_p[sub], pd, rtol=1e-5, atol=1e-6)


def test_proposal_energy_and_speed(trained):
    pidx, init, _ = trained
    ix = pidx.indices[1]
    X = init(21)
    pts.synthesize_level(pidx.indices[0], X, 5, mode="exact")
    X = pts.upsample2(X)
    Xe, Xp = X.clone(), X.clone()
    Ee = pts.synthesize_level(ix, Xe, 5, mode="exact")
    Ep = pts.synthesize_level(ix, Xp, 5, mode="proposal")
    # the proposal's output, measured by the exact search, against exact mode's final energy
    _, d2 = pts.nn_search(ix, Xp, 2, "exact")
    assert float(d2.double().sum()) <= 1.01 * Ee[-1], (float(d2.double().sum()), Ee[-1], Ep[-1])
    # what the network buys: E-step time of the proposal against exact search on one image
    def timed(mode):
        pts.nn_search(ix, Xe, 2, mode)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            pts.nn_search(ix, Xe, 2, mode)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / 5
    assert timed("proposal") < timed("exact")


def test_fallback_equals_tensor_core_search():
    """With a fallback threshold near zero every query with a nonzero distance falls back to the
    FP16 tensor-core search over all windows (the listed search); its result must then be the
    "f16" mode's result bit for bit (same candidates, same re-rank)."""
    Z = P.synthetic_exemplar(3, 160, 4.0)
    pidx = PyramidIndex(_t(Z), [16, 8], d=64)
    z0 = pidx.exemplars[0].cpu().numpy()
    init = lambda s: _t(P.random_patch_init(z0, 128, 128, 16, s))  # noqa: E731
    try:
        y, nn, d2 = collect_pairs(pidx, 1, init, range(2), iters=3)
        y, nn, d2 = subsample(y, nn, d2, 100_000)
        pts.train_proposal(pidx.indices[1], y, nn, d2, n_clusters=64, epochs=2, batch=4096, seed=2,
                           fallback_factor=1e-6)
        ix = pidx.indices[1]
        X = init(30)
        pts.synthesize_level(pidx.indices[0], X, 5, mode="exact")
        X = pts.upsample2(X)
        pts.synthesize_level(ix, X, 2, mode="exact")
        nn_p, d2_p = pts.nn_search(ix, X, 2, "proposal")
        st = ix.search_stats()
        nn_f, d2_f = pts.nn_search(ix, X, 2, "f16")
        pos = d2_f > 0
        assert st["fallback_queries"] >= int(pos.sum().item())
        assert torch.equal(d2_p, d2_f)
        assert torch.equal(nn_p[pos], nn_f[pos])
    finally:
        pidx.close()


def test_network_gains_over_the_papers_tree(trained):
    """What the trained network buys over the search it replaces, the k = 4 k-means tree of
    section 2.2 with greedy descent, on the same mid-synthesis image: the share of queries given
    the exact nearest window, and the matched energy against exact search's."""
    pidx, init, _ = trained
    ix = pidx.indices[1]
    pts.build_kmeans_tree(ix, 10)
    X = init(24)
    pts.synthesize_level(pidx.indices[0], X, 5, mode="exact")
    X = pts.upsample2(X)
    pts.synthesize_level(ix, X, 2, mode="exact")
    nn_e, d2_e = pts.nn_search(ix, X, 2, "exact")
    nn_p, d2_p = pts.nn_search(ix, X, 2, "proposal")
    nn_t, d2_t = pts.nn_search(ix, X, 2, "kmtree")
    rec_p = float((nn_p == nn_e).float().mean())
    rec_t = float((nn_t == nn_e).float().mean())
    e_p = float(d2_p.double().sum() / d2_e.double().sum())
    e_t = float(d2_t.double().sum() / d2_e.double().sum())
    print(f"recall@1: proposal {rec_p:.4f}, tree {rec_t:.4f}; matched energy / exact: proposal {e_p:.4f}, "
          f"tree {e_t:.4f}")
    assert rec_p > rec_t + 0.1
    assert e_p < e_t


def test_network_gains_over_brute_force_at_scale():
    """What the trained network buys over the same search without it, the FP16 tensor-core
    search over every exemplar window, where the exemplar is large: 512x512 (N = 255,025
    windows of 8x8), one 512x512 output level, 1,024 clusters trained on four exact-mode EM runs.
    On one mid-synthesis image the proposal's E-step must take less time than the brute-force
    search, and the windows it returns must keep the matched energy within 1.01x of exact
    search's.  (On the benchmark's 256x256 exemplar, 62,001 windows, the brute force is the
    faster of the two: the network, the probe and the fallback cost more than they save.)"""
    from paper_2006_11851_gb300.proposal import train_job_proposal
    Z = _t(P.synthetic_exemplar(0, 512, 4.0))
    ix = pts.ExemplarIndex(Z, 8, d=64)
    try:
        train_job_proposal(ix, Z, 512, 8, [1000 + s for s in range(4)], n_pairs=1_000_000, epochs=6,
                           n_clusters=1024)
        X = _t(P.random_patch_init(Z.cpu().numpy(), 512, 512, 8, 7))
        pts.synthesize_level(ix, X, 2, mode="f16")

        def timed(mode, reps=10):
            pts.nn_search(ix, X, 2, mode)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                nn, d2 = pts.nn_search(ix, X, 2, mode)
            e1.record()
            e1.synchronize()
            return e0.elapsed_time(e1) / reps, d2

        t_f16, d2_f16 = timed("f16")
        t_prop, d2_prop = timed("proposal")
        fallback = ix.search_stats()["fallback_queries"] / ix.search_stats()["queries"]
        _, d2_e = pts.nn_search(ix, X, 2, "exact")
        e_exact = float(d2_e.double().sum())
        ratio_prop = float(d2_prop.double().sum()) / e_exact
        ratio_f16 = float(d2_f16.double().sum()) / e_exact
        print(f"\nN = {ix.N}: E-step FP16 brute force {t_f16:.3f} ms, proposal {t_prop:.3f} ms "
              f"({t_f16 / t_prop:.2f}x), fallback {fallback:.3f}; matched energy / exact: "
              f"proposal {ratio_prop:.5f}, brute force {ratio_f16:.5f}")
        assert t_prop < t_f16
        assert ratio_prop <= 1.01
    finally:
        ix.close()
