"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs are the seeded synthetic exemplars and initialisations of pts_inputs.
Tolerances: NN indices per the tie rule in tests/_util.py; pixels 1e-4
absolute (FP32 path); energies 1e-5 relative per E-step, final energy of an
EM run within 1.001x; eigenvalues 1e-9 relative; PCA projector 1e-6.
"""
import ctypes

import numpy as np
import pytest

import oracle
import pts_inputs as P
from _util import check_nn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2006_11851_gb300 as pts  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


@pytest.fixture(scope="module")
def c1():
    """64x64 exemplar (shrink 3), w = 8, d = 24: the tiny plain-method workload."""
    Z = P.synthetic_exemplar(0, 64, 3.0)
    idx = pts.ExemplarIndex(_t(Z), 8, d=24)
    yield Z, idx
    idx.close()


# --------------------------------------------------------------------------
# pyramid filters
# --------------------------------------------------------------------------
@pytest.mark.parametrize("H,W", [(64, 64), (37, 22), (1, 5)])
def test_downsample_upsample(H, W):
    img = P.SplitMix64(3).uniform(H * W * 3).reshape(H, W, 3).astype(np.float32)
    g = pts.downsample2(_t(img)).cpu().numpy()
    np.testing.assert_allclose(g, oracle.downsample2(img), atol=2e-7)
    g = pts.upsample2(_t(img)).cpu().numpy()
    np.testing.assert_allclose(g, oracle.upsample2(img), atol=2e-7)


# --------------------------------------------------------------------------
# PCA (section 2.2)
# --------------------------------------------------------------------------
def _projector_dist(B1, B2):
    B1 = np.asarray(B1, np.float64)
    B2 = np.asarray(B2, np.float64)
    return np.linalg.norm(B1.T @ B1 - B2.T @ B2)


# d = 92 and 128: the component counts of the tensor-core search (Rayleigh-Ritz beyond 112)
@pytest.mark.parametrize("size,w,d", [(64, 8, 24), (48, 16, 64), (40, 4, 12), (12, 8, 8), (64, 8, 92),
                                      (48, 16, 128)])
def test_pca_fit(size, w, d):
    Z = P.synthetic_exemplar(1, size, 3.0)
    mu_o, B_o, ev_o, _ = oracle.pca_fit(Z, w, d)
    mean, basis, eig, k = pts.pca_fit(_t(Z), w, d)
    assert k == d
    eig = eig.cpu().numpy()
    np.testing.assert_allclose(eig, ev_o[:d], rtol=1e-9, atol=1e-12 * ev_o[0])
    np.testing.assert_allclose(mean.cpu().numpy(), mu_o, atol=1e-6)
    gap = ev_o[d - 1] - ev_o[d] if len(ev_o) > d else ev_o[d - 1]
    if gap > 1e-6 * ev_o[0]:
        # FP32 export of the basis limits the projector to ~1e-6
        assert _projector_dist(basis.cpu().numpy(), B_o) < 1e-5
    Bg = basis.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(Bg @ Bg.T, np.eye(d), atol=1e-5)


@pytest.mark.parametrize("d", [64, 92])
def test_pca_large_window_gram_branch(d):
    """w = 32 (D = 3072) on a 64x64 exemplar: N = 1089 < D."""
    Z = oracle.exemplar_pyramid(P.synthetic_exemplar(0, 256, 4.0), 3)[0].astype(np.float32)
    mu_o, B_o, ev_o, _ = oracle.pca_fit(Z, 32, d)
    mean, basis, eig, k = pts.pca_fit(_t(Z), 32, d)
    np.testing.assert_allclose(eig.cpu().numpy(), ev_o[:d], rtol=1e-9)
    assert _projector_dist(basis.cpu().numpy(), B_o) < 1e-5


def test_pca_variance_fraction():
    Z = P.synthetic_exemplar(2, 48, 3.0)
    _, _, ev_o, _ = oracle.pca_fit(Z, 8, 64)
    # the oracle's full spectrum is min(N, D) values; its sum is the trace
    frac = np.cumsum(ev_o) / ev_o.sum()
    want = int(np.searchsorted(frac, 0.95) + 1)
    _, _, _, k = pts.pca_fit(_t(Z), 8, 0, var_frac=0.95)
    assert k == min(want, 64)


# --------------------------------------------------------------------------
# E-step (Eq. 4), exact mode
# --------------------------------------------------------------------------
def test_nn_search_random_init(c1):
    Z, idx = c1
    X = P.random_patch_init(Z, 128, 128, 8, 0)
    nn, d2 = pts.nn_search(idx, _t(X), 2, "exact")
    nn_o, d2_o = oracle.nn_bruteforce(X, Z, 8, 2)
    check_nn(X, Z, 8, 2, nn.cpu().numpy(), d2.cpu().numpy(), nn_o, d2_o, max_mismatch_frac=0.01)
    st = idx.search_stats()
    assert st["queries"] == 3721


def test_nn_search_along_oracle_trajectory(c1):
    Z, idx = c1
    X0 = P.random_patch_init(Z, 128, 128, 8, 1)
    ref = oracle.synthesize_level(Z, X0, 8, 3, keep_trajectory=True)
    for Xt, nn_o, d2_o, _ in ref["trajectory"]:
        nn, d2 = pts.nn_search(idx, _t(Xt), 2, "exact")
        check_nn(Xt, Z, 8, 2, nn.cpu().numpy(), d2.cpu().numpy(), nn_o, d2_o, max_mismatch_frac=0.01)


@pytest.mark.parametrize("He,Ho,w,d,stride", [
    (10, 20, 8, 8, 2),     # N = 9 < 32 candidates
    (40, 46, 8, 64, 2),    # max d, ragged query count
    (33, 36, 16, 40, 2),   # D = 768
    (24, 29, 5, 10, 1),    # stride 1, odd w
    (30, 40, 8, 20, 4),    # stride 4
])
def test_nn_search_edge_cases(He, Ho, w, d, stride):
    Z = P.synthetic_exemplar(4, He, 3.0)
    X = P.random_patch_init(Z, Ho, Ho, w, 2)
    idx = pts.ExemplarIndex(_t(Z), w, d=d)
    nn, d2 = pts.nn_search(idx, _t(X), stride, "exact")
    nn_o, d2_o = oracle.nn_bruteforce(X, Z, w, stride)
    check_nn(X, Z, w, stride, nn.cpu().numpy(), d2.cpu().numpy(), nn_o, d2_o)
    idx.close()


def test_nn_search_duplicate_windows_tie_smallest_index():
    half = P.synthetic_exemplar(5, 20, 3.0)[:, :14]
    Z = np.ascontiguousarray(np.concatenate([half, half], axis=1))
    X = np.ascontiguousarray(Z[2:14, 4:16])
    idx = pts.ExemplarIndex(_t(Z), 4, d=8)
    nn, d2 = pts.nn_search(idx, _t(X), 2, "exact")
    nn_o, d2_o = oracle.nn_bruteforce(X, Z, 4, 2)
    np.testing.assert_array_equal(nn.cpu().numpy(), nn_o)
    assert np.all(d2.cpu().numpy() == 0.0)
    idx.close()


# --------------------------------------------------------------------------
# IRLS weights / energy (Eqs. 5-8) and M-step (Eq. 8)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("r", [2.0, 0.8])
def test_irls(r):
    d2 = (P.SplitMix64(6).uniform(5000) * 3.0).astype(np.float32)
    d2[:7] = 0.0
    W_o, E_o, _ = oracle.irls(d2, r, 1e-3)
    W, E = pts.irls_weights(_t(d2), r, 1e-3)
    np.testing.assert_allclose(W.cpu().numpy(), W_o, rtol=2e-6)
    assert abs(E.item() / E_o - 1) < 1e-6
    W2, E2 = pts.irls_weights(_t(d2), r, 1e-3)
    assert E2.item() == E.item()  # deterministic reduction


@pytest.mark.parametrize("He,Ho,w,stride,weighted", [
    (64, 128, 8, 2, True), (64, 128, 8, 2, False), (48, 64, 16, 2, True),
    (40, 37, 5, 1, True), (40, 48, 8, 4, True), (70, 96, 32, 2, True)])
def test_m_step(He, Ho, w, stride, weighted):
    Z = P.synthetic_exemplar(7, He, 3.0)
    idx = pts.ExemplarIndex(_t(Z), w, d=4)
    Q = oracle.num_queries(Ho, Ho, w, stride)
    N = oracle.num_exemplar_windows(He, He, w)
    nn = P.random_nn(8, Q, N)
    Wt = P.random_weights(9, Q) if weighted else None
    out = pts.m_step(idx, torch.from_numpy(nn).to(DEV), None if Wt is None else _t(Wt), Ho, Ho, stride)
    ref = oracle.m_step(nn, None if Wt is None else Wt.astype(np.float64), Z, w, Ho, Ho, stride)
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4)
    assert np.abs(out.cpu().numpy() - ref).max() < 2e-6
    idx.close()


# --------------------------------------------------------------------------
# EM (section 2.1): step-wise and end to end
# --------------------------------------------------------------------------
def test_em_stepwise_against_oracle(c1):
    """Each GPU half-step applied to the oracle's own iterate."""
    Z, idx = c1
    X0 = P.random_patch_init(Z, 128, 128, 8, 3)
    ref = oracle.synthesize_level(Z, X0, 8, 4, r=0.8, keep_trajectory=True)
    traj = ref["trajectory"]
    for t in range(len(traj) - 1):
        Xt, nn_o, d2_o, W_o = traj[t]
        _, d2_g = pts.nn_search(idx, _t(Xt), 2, "exact")
        W_g, E_g = pts.irls_weights(d2_g, 0.8, 1e-3)
        assert abs(E_g.item() / ref["E"][t] - 1) < 1e-5
        out = pts.m_step(idx, torch.from_numpy(nn_o).to(DEV), _t(W_o), 128, 128, 2)
        np.testing.assert_allclose(out.cpu().numpy(), traj[t + 1][0], atol=1e-4)


@pytest.mark.parametrize("r", [2.0, 0.8])
def test_synthesize_level_end_to_end(c1, r):
    Z, idx = c1
    X0 = P.random_patch_init(Z, 128, 128, 8, 4)
    xt = _t(X0)
    E = pts.synthesize_level(idx, xt, 5, r=r, mode="exact")
    ref = oracle.synthesize_level(Z, X0, 8, 5, r=r)
    np.testing.assert_allclose(E, ref["E"], rtol=1e-3)
    assert abs(E[-1] / ref["E"][-1] - 1) < 1e-3
    diff = np.abs(xt.cpu().numpy() - ref["X"])
    # pixels agree to FP32 rounding unless a near-tie flipped a match somewhere
    assert np.mean(diff < 1e-4) > 0.99
    if r == 2.0:
        assert np.all(np.diff(E) <= 1e-6 * E[0])


def test_exact_reproduction_gpu(c1):
    Z, idx = c1
    xt = _t(Z)
    E = pts.synthesize_level(idx, xt, 2, r=2.0, mode="exact")
    # FP32 averaging of k equal values can be 1 ulp off at border pixels
    # (covered by fewer than (w/2)^2 windows), so the energy is ~0, not 0
    assert E[0] == 0.0 and np.all(E < 1e-8)
    np.testing.assert_allclose(xt.cpu().numpy(), Z, atol=1e-6)


def test_pyramid_three_levels_small():
    """Coarse-to-fine on a small exemplar: per-level energies against the oracle."""
    from paper_2006_11851_gb300.pyramid import PyramidIndex, synthesize_pyramid
    Z = P.synthetic_exemplar(0, 96, 4.0)
    windows = [8, 8, 8]
    pidx = PyramidIndex(_t(Z), windows, d=16)
    pyr_o = oracle.exemplar_pyramid(Z, 3)
    for zg, zo in zip(pidx.exemplars, pyr_o):
        np.testing.assert_allclose(zg.cpu().numpy(), zo, atol=1e-6)
    X0 = P.random_patch_init(pyr_o[0].astype(np.float32), 48, 48, 8, 0)
    X, E, _ = synthesize_pyramid(pidx, _t(X0), iters=3)
    Xo = X0
    for lev in range(3):
        ref = oracle.synthesize_level(pyr_o[lev].astype(np.float32), Xo, 8, 3)
        assert abs(E[lev][-1] / ref["E"][-1] - 1) < 1e-3
        Xo = oracle.upsample2(ref["X"]) if lev < 2 else ref["X"]
    pidx.close()


# --------------------------------------------------------------------------
# full-size workload, sampled queries
# --------------------------------------------------------------------------
def test_full_size_fine_level_sampled():
    """256x256 exemplar, w = 8, d = 64, 512x512 output: 64,009 queries against
    62,001 windows, in the launch configuration the benchmark times; the
    oracle checks a seeded sample of 2,048 queries."""
    Z = P.synthetic_exemplar(0, 256, 4.0)
    idx = pts.ExemplarIndex(_t(Z), 8, d=64)
    X = P.random_patch_init(Z, 512, 512, 8, 0)
    nn, d2 = pts.nn_search(idx, _t(X), 2, "exact")
    Q = oracle.num_queries(512, 512, 8)
    sub = P.sample_indices(11, Q, 2048)
    nn_o, d2_o = oracle.nn_bruteforce(X, Z, 8, 2, qlist=sub)
    check_nn(X, Z, 8, 2, nn.cpu().numpy()[sub], d2.cpu().numpy()[sub], nn_o, d2_o, qlist=sub)
    st = idx.search_stats()
    assert st["queries"] == Q and st["certified"] + st["range_queries"] == Q
    idx.close()


def _profiled_launches(L, name):
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    assert L.pts_profile_read(name.encode(), ctypes.byref(ms), ctypes.byref(n)) == 0
    return n.value


def test_coarsest_level_exact_all_queries():
    """The benchmark's coarsest level: the 256x256 exemplar down-sampled twice (64x64), w = 32
    (D = 3,072), d = 64, 128x128 output -- all 2,401 queries of the random-patch initialisation
    and of the oracle's next two iterates against its full-dimension FP64 brute force.  Its 64
    components keep under 85% of the variance, so the search skips the PCA pass (nothing
    certified from the 32 best bounds, every query sent to the full-dimension pass), and that
    pass, having few (query block, tile) pairs, is split along the vector (partial sums added in
    fixed order afterwards), which the search statistics report."""
    Z = oracle.exemplar_pyramid(P.synthetic_exemplar(0, 256, 4.0), 3)[0].astype(np.float32)
    idx = pts.ExemplarIndex(_t(Z), 32, d=64)
    assert idx.info["var_retained"] < 0.85
    X0 = P.random_patch_init(Z, 128, 128, 32, 100)
    ref = oracle.synthesize_level(Z, X0, 32, 2, keep_trajectory=True)
    L = pts.lib()
    for Xt, nn_o, d2_o, _ in ref["trajectory"]:
        L.pts_profile_enable(1)
        nn, d2 = pts.nn_search(idx, _t(Xt), 2, "exact")
        torch.cuda.synchronize()
        topk = _profiled_launches(L, "search_topk")
        L.pts_profile_enable(0)
        check_nn(Xt, Z, 32, 2, nn.cpu().numpy(), d2.cpu().numpy(), nn_o, d2_o, max_mismatch_frac=0.01)
        st = idx.search_stats()
        assert st["queries"] == 2401 and st["certified"] == 0 and st["range_queries"] == 2401
        assert topk == 0 and st["full_splits"] > 1, (topk, st)
    idx.close()


# --------------------------------------------------------------------------
# argument errors surface as PtsError, nothing launched
# --------------------------------------------------------------------------
def test_invalid_arguments(c1):
    Z, idx = c1
    with pytest.raises(pts.PtsError):
        pts.nn_search(idx, torch.zeros(127, 128, 3, device=DEV), 2, "exact")  # (Ho - w) odd
    with pytest.raises(pts.PtsError):
        pts.nn_search(idx, torch.zeros(128, 128, 3, device=DEV), 3, "exact")
    with pytest.raises(pts.PtsError):
        pts.ExemplarIndex(_t(Z[:6, :6]), 8)
    with pytest.raises(pts.PtsError):
        pts.pca_fit(_t(Z), 8, 129)
    X = torch.zeros(128, 128, 3, device=DEV)
    Q = idx.num_queries(128, 128, 2)
    nn = torch.zeros(Q, dtype=torch.int32, device=DEV)
    with pytest.raises(pts.PtsError):
        pts.m_step_hist(idx, nn, None, X, 1)          # nbins outside 2..256
    with pytest.raises(pts.PtsError):
        pts.histogram_match(idx, X.clone(), 300)
    with pytest.raises(pts.PtsError):
        pts.synthesize_level(idx, X.clone(), 1, hist_bins=1)
    with pytest.raises(pts.PtsError):
        pts.synthesize_level_converge(idx, X.clone(), -1)
    with pytest.raises(pts.PtsError):
        pts.build_kmeans_tree(idx, 0)                 # Lloyd iterations outside 1..100
    fresh = pts.ExemplarIndex(_t(Z), 8, d=24)
    with pytest.raises(pts.PtsError):
        pts.nn_search(fresh, X, 2, "kmtree")          # no tree built
    with pytest.raises(pts.PtsError):
        pts.nn_search(fresh, X, 2, "proposal")        # no proposal trained
    fresh.close()


def test_tree_on_a_two_window_exemplar():
    """N = 2 windows (fewer than k = 4): the tree is one leaf, so its search is exact."""
    Z = P.synthetic_exemplar(12, 9, 1.0)[:, :8]          # 9 x 8 exemplar, w = 8: windows at y = 0, 1
    idx = pts.ExemplarIndex(_t(Z), 8, d=4)
    info = pts.build_kmeans_tree(idx, 5)
    assert info["leaves"] == 1
    X = P.random_patch_init(Z, 16, 16, 8, 1)
    nn_t, d2_t = pts.nn_search(idx, _t(X), 2, "kmtree")
    nn_e, d2_e = pts.nn_search(idx, _t(X), 2, "exact")
    assert torch.equal(nn_t, nn_e) and torch.equal(d2_t, d2_e)
    idx.close()


def test_index_destroy_returns_device_memory():
    """Building an index, searching it in every mode that allocates workspace (exact, FP16, FP8)
    and destroying it leaves the device's free memory where it was (one warm-up cycle first, so
    the caching allocator and the CUDA context have settled)."""
    Z = P.synthetic_exemplar(4, 96, 3.0)
    X = _t(P.random_patch_init(Z, 192, 192, 8, 1))

    def cycle():
        idx = pts.ExemplarIndex(_t(Z), 8, d=32)
        for mode in ("exact", "f16", "fp8", "f16"):
            pts.nn_search(idx, X, 2, mode)
        idx.close()
        torch.cuda.synchronize()

    cycle()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        cycle()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 8 << 20, (free0 - free1)


@pytest.mark.parametrize("r", [2.0, 0.8])
def test_converge_against_oracle(c1, r):
    """Section 2.1's stopping rule: the GPU loop stops after as many M-steps as the oracle's."""
    Z, idx = c1
    X0 = P.random_patch_init(Z, 96, 96, 8, 6)
    xt = _t(X0)
    E, it = pts.synthesize_level_converge(idx, xt, 30, r=r, mode="exact")
    ref = oracle.synthesize_level_converge(Z, X0, 8, 30, r=r)
    assert it == ref["iters"], (it, ref["iters"])
    np.testing.assert_allclose(E, ref["E"], rtol=1e-3)
    diff = np.abs(xt.cpu().numpy() - ref["X"])
    assert np.mean(diff < 1e-4) > 0.99


def test_converge_reproduces_exemplar_in_one_step(c1):
    """Seeded with the exemplar the windows repeat after one M-step.  (FP32 averaging of equal
    values can be 1 ulp off at border pixels, so the second energy is ~0, not 0.)"""
    Z, idx = c1
    xt = _t(Z)
    E, it = pts.synthesize_level_converge(idx, xt, 10, r=2.0, mode="exact")
    assert it == 1 and E[0] == 0.0 and E[1] < 1e-8
    np.testing.assert_allclose(xt.cpu().numpy(), Z, atol=1e-6)


def test_exact_bound_components_change_the_route_not_the_result():
    """The exact search's PCA bound with the index's first d components (the default, followed by
    the d_fast bound on the queries it leaves uncertified), with its d_fast components alone, or
    with the first d alone: every route returns the certified nearest windows of Eq. 4, bit for bit the same, and the
    larger bound certifies at least as many queries from the 32 best bounds."""
    Z = P.synthetic_exemplar(0, 128, 4.0)
    idx = pts.ExemplarIndex(_t(Z), 8, d=32)
    X = _t(P.random_patch_init(Z, 256, 256, 8, 3))
    assert idx.info["exact_dims"] == 32
    nn_d, d2_d = pts.nn_search(idx, X, 2, "exact")
    st_d = idx.search_stats()
    idx.set_exact_bound(True)
    assert idx.info["exact_dims"] == idx.info["d_fast"] > 32
    nn_f, d2_f = pts.nn_search(idx, X, 2, "exact")
    st_f = idx.search_stats()
    assert torch.equal(nn_f, nn_d) and torch.equal(d2_f, d2_d)
    assert st_f["certified"] >= st_d["certified"], (st_f, st_d)
    # the default route runs the second bound (d_fast components) on the first bound's
    # uncertified queries before the full-dimension pass
    assert st_d["second_queries"] == st_d["range_queries"] > 0, st_d
    assert st_d["full_queries"] == st_d["range_queries"] - st_d["second_certified"], st_d
    assert st_d["full_queries"] < st_d["range_queries"], st_d
    # the first d components alone: no second bound, every uncertified query takes the full pass
    idx.set_exact_bound(2)
    assert idx.info["exact_dims"] == 32
    nn_2, d2_2 = pts.nn_search(idx, X, 2, "exact")
    st_2 = idx.search_stats()
    assert torch.equal(nn_2, nn_d) and torch.equal(d2_2, d2_d)
    assert st_2["second_queries"] == 0 and st_2["full_queries"] == st_2["range_queries"], st_2
    assert st_2["certified"] == st_d["certified"], (st_2, st_d)
    Q = idx.num_queries(256, 256, 2)
    sub = P.sample_indices(13, Q, 256)
    Xh = X.cpu().numpy()
    nn_o, d2_o = oracle.nn_bruteforce(Xh, Z, 8, 2, qlist=sub)
    check_nn(Xh, Z, 8, 2, nn_f.cpu().numpy()[sub], d2_f.cpu().numpy()[sub], nn_o, d2_o, qlist=sub)
    idx.close()


@pytest.mark.parametrize("He,Ho,w,d,stride", [(64, 128, 8, 24, 2), (48, 64, 16, 64, 2), (40, 52, 8, 32, 4),
                                              (30, 37, 5, 12, 1)])
def test_project_queries_against_oracle(He, Ho, w, d, stride):
    """Query projection y_q = B^T (x_q - mu) (section 2.2) on its own, against the oracle's FP64
    projection onto its FP64 basis.  Eigenvectors are defined up to sign, so coordinates are
    compared in absolute value, for components separated from their neighbours by a gap; the
    squared norm of all d coordinates is compared as it is (it does not depend on the basis
    chosen inside the subspace).  FP32 path: 1e-4 relative to the largest window norm."""
    Z = P.synthetic_exemplar(9, He, 3.0)
    X = P.random_patch_init(Z, Ho, Ho, w, 4)
    idx = pts.ExemplarIndex(_t(Z), w, d=d)
    y = pts.project_queries(idx, _t(X), stride).cpu().numpy().astype(np.float64)
    mu, B, ev, _ = oracle.pca_fit(Z, w, d)
    yo, uo, _ = oracle.project(X, w, stride, mu, B)
    assert y.shape == yo.shape
    scale = np.sqrt(uo.max())
    gap = np.minimum(np.abs(np.diff(ev[:d + 1], prepend=np.inf))[:d], np.abs(np.diff(ev[:d + 1]))[:d])
    ok = gap > 1e-4 * ev[0]
    assert ok.sum() >= d // 2
    np.testing.assert_allclose(np.abs(y[:, ok]), np.abs(yo[:, ok]), atol=1e-4 * scale)
    np.testing.assert_allclose((y ** 2).sum(1), (yo ** 2).sum(1), atol=1e-4 * scale ** 2)
    idx.close()
