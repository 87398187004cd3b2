"""The scale map (section 1, Eqs. 1-3) and the RGBS synthesis of section 3 on the GPU, against the
oracle (oracle/scale.py and the 4-channel C oracle).

Bit for bit (FP64 both sides, each operation rounded on its own): the map, its resampling, the
bins of the scale-guided initialisation and the pixel each output pixel copies, the RGBS image.
With tolerances (FP32 path): the PCA of RGBS windows (eigenvalues 1e-9 relative, projector
1e-5), the exact search's tie rule of tests/_util.py, the M-step's colours (1e-4 absolute, the
scale channel untouched bit for bit), EM energies (1e-3 relative) on one level and coarse to fine.
"""
import numpy as np
import pytest

import oracle
import oracle.scale as osc
import pts_inputs as P
from _util import check_nn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2006_11851_gb300 as pts  # noqa: E402

DEV = torch.device("cuda:0")
ANGLES = [(0.0, 0.0), (30.0, 18.0), (60.0, 60.0), (60.0, 20.0), (45.0, 90.0), (60.0, 0.0), (89.0, 45.0)]


def _t(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(DEV)


@pytest.mark.parametrize("h,w", [(64, 64), (37, 50), (9, 14), (3, 2)])
@pytest.mark.parametrize("slant,tilt", ANGLES)
def test_scale_map_bitwise(h, w, slant, tilt):
    S = pts.scale_map(h, w, slant, tilt).cpu().numpy()
    np.testing.assert_array_equal(S, osc.scale_map(h, w, slant, tilt))


def test_scale_map_refusals():
    with pytest.raises(pts.PtsError):
        pts.scale_map(8, 8, 90.0, 0.0)          # slant outside [0, 90)
    with pytest.raises(pts.PtsError):
        pts.scale_map(8, 8, 30.0, 91.0)         # tilt outside [0, 90]
    with pytest.raises(pts.PtsError):
        pts.scale_map(1, 2, 30.0, 0.0)          # Y_delta = 0 at tilt 0 on one row
    with pytest.raises(ValueError):
        osc.scale_map(1, 2, 30.0, 0.0)          # the oracle refuses the same map


@pytest.mark.parametrize("He,We,Ho,Wo", [(64, 64, 128, 128), (37, 50, 80, 61), (5, 7, 5, 7), (16, 16, 9, 3)])
def test_scale_resample_bitwise(He, We, Ho, Wo):
    S = osc.scale_map(He, We, 60.0, 20.0)
    got = pts.scale_resample(_t(S, np.float64), Ho, Wo).cpu().numpy()
    np.testing.assert_array_equal(got, osc.resample(S, Ho, Wo))


@pytest.mark.parametrize("He,Ho,nbins,slant,tilt", [(48, 96, 64, 60.0, 20.0), (40, 72, 7, 30.0, 18.0),
                                                    (32, 40, 1, 60.0, 60.0), (16, 48, 200, 60.0, 0.0),
                                                    (24, 24, 16, 0.0, 0.0)])
def test_scale_guided_init_bitwise(He, Ho, nbins, slant, tilt):
    """Same bins, same copied pixel for every output pixel: including empty bins (tilt 0 makes
    the map constant along rows, so 200 bins over 16 rows leave most empty) and a flat plane
    (slant 0: every pixel in bin 0)."""
    Z = P.synthetic_exemplar(3, He, 3.0)
    S_z = osc.scale_map(He, He, slant, tilt)
    S_x = osc.resample(S_z, Ho, Ho)
    u = P.uniform_field(5, Ho, Ho)
    X0_o, src_o = osc.scale_guided_init(Z, S_z, S_x, u, nbins)
    X0, src = pts.scale_guided_init(_t(Z), _t(S_z, np.float64), _t(S_x, np.float64), _t(u, np.float64), nbins)
    np.testing.assert_array_equal(src.cpu().numpy(), src_o)
    np.testing.assert_array_equal(X0.cpu().numpy(), X0_o.astype(np.float32))


def test_rgbs_images_bitwise():
    Z = P.synthetic_exemplar(4, 30, 3.0)
    S = osc.scale_map(30, 30, 60.0, 20.0)
    for lam in (1.0, 0.37):
        Z4 = pts.rgbs(_t(Z), _t(S, np.float64), lam)
        np.testing.assert_array_equal(Z4.cpu().numpy(), osc.rgbs(Z, S, lam).astype(np.float32))
        np.testing.assert_array_equal(pts.rgb_of(Z4).cpu().numpy(), Z)


def _rgbs_pair(He, Ho, w, seed=0, slant=60.0, tilt=20.0, lam=1.0):
    """An RGBS exemplar and an RGBS output initialised from same-scale pixels (float32)."""
    Z = P.synthetic_exemplar(seed, He, 4.0)
    S_z = osc.scale_map(He, He, slant, tilt)
    S_x = osc.resample(S_z, Ho, Ho)
    X0, _ = osc.scale_guided_init(Z, S_z, S_x, P.uniform_field(seed + 1, Ho, Ho), 64)
    Z4 = osc.rgbs(Z, S_z, lam).astype(np.float32)
    X4 = osc.rgbs(X0, S_x, lam).astype(np.float32)
    return Z4, X4


@pytest.mark.parametrize("size,w,d", [(40, 8, 24), (32, 16, 64), (48, 8, 100)])
def test_pca_fit_rgbs(size, w, d):
    Z4, _ = _rgbs_pair(size, size, w, seed=2)
    mu_o, B_o, ev_o, _ = oracle.pca_fit(Z4, w, d)
    mean, basis, eig, k = pts.pca_fit(_t(Z4), w, d)
    assert k == d
    np.testing.assert_allclose(eig.cpu().numpy(), ev_o[:d], rtol=1e-9, atol=1e-12 * ev_o[0])
    np.testing.assert_allclose(mean.cpu().numpy(), mu_o, atol=1e-6)
    gap = ev_o[d - 1] - ev_o[d]
    if gap > 1e-6 * ev_o[0]:
        Bg = basis.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(Bg.T @ Bg - B_o.T @ B_o) < 1e-5


@pytest.mark.parametrize("He,Ho,w,d,stride", [(48, 96, 8, 32, 2), (36, 48, 16, 64, 2), (30, 37, 5, 12, 1),
                                              (40, 48, 8, 20, 4)])
def test_nn_search_rgbs_exact(He, Ho, w, d, stride):
    Z4, X4 = _rgbs_pair(He, Ho, w, seed=6)
    idx = pts.ExemplarIndex(_t(Z4), w, d=d)
    assert idx.C == 4 and idx.D == 4 * w * w
    nn, d2 = pts.nn_search(idx, _t(X4), stride, "exact")
    nn_o, d2_o = oracle.nn_bruteforce(X4, Z4, w, stride)
    check_nn(X4, Z4, w, stride, nn.cpu().numpy(), d2.cpu().numpy(), nn_o, d2_o)
    # the FP16 tensor-core search: the exact distance of the window it returns, never below exact
    nn_f, d2_f = pts.nn_search(idx, _t(X4), stride, "f16")
    q = np.arange(len(nn_o))
    pd = oracle.pair_dist2(X4, Z4, w, stride, q, nn_f.cpu().numpy())
    np.testing.assert_allclose(d2_f.cpu().numpy(), pd, rtol=1e-5, atol=1e-6)
    assert np.all(pd >= d2_o * (1 - 1e-12) - 1e-12)
    idx.close()


def test_rgbs_index_rejects_rgb_images_and_histograms():
    Z4, X4 = _rgbs_pair(32, 40, 8)
    idx = pts.ExemplarIndex(_t(Z4), 8, d=16)
    with pytest.raises(ValueError):
        pts.nn_search(idx, _t(X4[:, :, :3]), 2, "exact")
    nn = torch.zeros(idx.num_queries(40, 40, 2), dtype=torch.int32, device=DEV)
    with pytest.raises(ValueError):
        pts.m_step_hist(idx, nn, None, _t(X4), 8)          # refused by the binding
    with pytest.raises(pts.PtsError, match="RGB index"):
        pts.synthesize_level(idx, _t(X4), 1, hist_bins=8)  # refused by the library
    idx.close()


@pytest.mark.parametrize("He,Ho,w,stride,weighted", [(48, 96, 8, 2, True), (40, 48, 16, 2, False),
                                                     (30, 37, 5, 1, True)])
def test_m_step_rgbs_keeps_the_scale_channel(He, Ho, w, stride, weighted):
    Z4, X4 = _rgbs_pair(He, Ho, w, seed=8)
    idx = pts.ExemplarIndex(_t(Z4), w, d=4)
    Q = oracle.num_queries(Ho, Ho, w, stride)
    nn = P.random_nn(9, Q, oracle.num_exemplar_windows(He, He, w))
    Wt = P.random_weights(10, Q) if weighted else None
    out = _t(X4)
    pts.m_step(idx, torch.from_numpy(nn).to(DEV), None if Wt is None else _t(Wt), Ho, Ho, stride, out=out)
    got = out.cpu().numpy()
    ref = oracle.m_step(nn, None if Wt is None else Wt.astype(np.float64), Z4, w, Ho, Ho, stride)
    np.testing.assert_allclose(got[:, :, :3], ref[:, :, :3], atol=1e-4)
    assert np.abs(got[:, :, :3] - ref[:, :, :3]).max() < 2e-6
    np.testing.assert_array_equal(got[:, :, 3], X4[:, :, 3])
    idx.close()


@pytest.mark.parametrize("r", [2.0, 0.8])
def test_synthesize_level_rgbs_against_oracle(r):
    Z4, X4 = _rgbs_pair(48, 96, 8, seed=11)
    idx = pts.ExemplarIndex(_t(Z4), 8, d=32)
    xt = _t(X4)
    E = pts.synthesize_level(idx, xt, 4, r=r, mode="exact")
    ref = osc.synthesize_level_rgbs(Z4, X4, 8, 4, r=r)
    np.testing.assert_allclose(E, ref["E"], rtol=1e-3)
    got = xt.cpu().numpy()
    np.testing.assert_array_equal(got[:, :, 3], X4[:, :, 3])
    assert np.mean(np.abs(got - ref["X"]) < 1e-4) > 0.99
    idx.close()


def test_synthesize_pyramid_rgbs_against_oracle():
    """The whole method of section 3 coarse to fine: 96x96 exemplar, 3 levels, windows 8/8/8,
    outputs 48/96/192, slant 60 and tilt 20 degrees.  Per-level final energies within 1e-3 of the
    oracle's (the GPU's exemplar pyramid is FP32, the oracle's FP64) and the colour image close."""
    Z = P.synthetic_exemplar(0, 96, 4.0)
    u = P.uniform_field(2, 48, 48)
    X, E = pts.synthesize_pyramid_rgbs(_t(Z), 60.0, 20.0, 192, 192, [8, 8, 8], 3, _t(u, np.float64), d=24)
    Xo, Eo = osc.synthesize_pyramid_rgbs(Z, 60.0, 20.0, 192, 192, [8, 8, 8], 3, u)
    for lev in range(3):
        assert abs(E[lev][-1] / Eo[lev][-1] - 1) < 1e-3, (lev, E[lev], Eo[lev])
    assert np.mean(np.abs(X.cpu().numpy() - Xo) < 1e-3) > 0.98
