"""Histogram matching on the GPU (section 3, Eq. 9; final matching of section 4) against the
FP64 oracle (`oracle/histogram.py`):

  - the M-step with the weights of Eq. 9 on random matches and weights (several strides and bin
    counts, a ragged image) within 2e-5 of the oracle;
  - with equal histograms (current image = exemplar) it is the plain M-step bit for bit;
  - final matching within 1e-4 of the oracle, and the identity on the exemplar itself;
  - a full pyramid with hist_bins ends with the oracle's matching of its last level's image;
  - a smooth source matched to the exemplar carries the exemplar's histogram.
"""
import numpy as np
import pytest

import oracle
from oracle import histogram as OH
import pts_inputs as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2006_11851_gb300 as pts  # noqa: E402
from paper_2006_11851_gb300.pyramid import PyramidIndex, synthesize_pyramid  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(DEV)


@pytest.mark.parametrize("He,Ho,Wo,w,stride,nbins", [(48, 64, 64, 8, 2, 32), (40, 58, 70, 8, 2, 7),
                                                     (32, 48, 48, 16, 4, 64), (24, 30, 30, 4, 1, 16)])
def test_m_step_hist_against_oracle(He, Ho, Wo, w, stride, nbins):
    Z = P.synthetic_exemplar(5, He, 3.0)
    idx = pts.ExemplarIndex(_t(Z), w, d=8)
    X = P.random_patch_init(Z, Ho, Wo, w, 2)
    Q = oracle.num_queries(Ho, Wo, w, stride)
    N = oracle.num_exemplar_windows(He, He, w)
    rng = np.random.default_rng(3)
    nn = rng.integers(0, N, Q).astype(np.int32)
    Wt = (rng.random(Q) + 0.5).astype(np.float32)
    got = pts.m_step_hist(idx, _t(nn, np.int32), _t(Wt), _t(X), nbins, stride=stride).cpu().numpy()
    ref = OH.m_step_hist(nn, Wt.astype(np.float64), Z, X, w, stride, nbins)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5)
    idx.close()


def test_m_step_hist_equal_histograms_is_plain_m_step():
    Z = P.synthetic_exemplar(6, 48, 3.0)
    idx = pts.ExemplarIndex(_t(Z), 8, d=8)
    Q = oracle.num_queries(48, 48, 8, 2)
    rng = np.random.default_rng(4)
    nn = _t(rng.integers(0, oracle.num_exemplar_windows(48, 48, 8), Q), np.int32)
    Wt = _t(rng.random(Q) + 0.5)
    a = pts.m_step_hist(idx, nn, Wt, _t(Z), 32)
    b = pts.m_step(idx, nn, Wt, 48, 48)
    assert torch.equal(a, b)
    idx.close()


@pytest.mark.parametrize("nbins", [8, 32, 100])
def test_histogram_match_against_oracle(nbins):
    Z = P.synthetic_exemplar(7, 64, 3.0)
    idx = pts.ExemplarIndex(_t(Z), 8, d=8)
    img = np.random.default_rng(nbins).beta(2.0, 3.0, (96, 80, 3)).astype(np.float32)
    got = pts.histogram_match(idx, _t(img), nbins).cpu().numpy()
    ref = OH.histogram_match(img, Z, nbins)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-4)
    same = pts.histogram_match(idx, _t(Z), nbins).cpu().numpy()
    np.testing.assert_allclose(same, np.clip(Z, 0, 1), rtol=0, atol=1e-5)
    idx.close()


def test_pyramid_with_histogram_weights_and_final_matching():
    """The whole procedure: Eq. 9 M-steps on every level, then the final matching, which must be
    the oracle's matching of the image the last level produced."""
    Z = P.synthetic_exemplar(8, 128, 4.0)
    pidx = PyramidIndex(_t(Z), [16, 8], d=32)
    z0 = pidx.exemplars[0].cpu().numpy()
    X0 = _t(P.random_patch_init(z0, 128, 128, 16, 5))
    X, E, imgs = synthesize_pyramid(pidx, X0, iters=3, mode="exact", keep_levels=True, hist_bins=32)
    assert np.all(np.isfinite(E))
    ref = OH.histogram_match(imgs[-1].cpu().numpy(), pidx.exemplars[-1].cpu().numpy(), 32)
    np.testing.assert_allclose(X.cpu().numpy(), ref, rtol=0, atol=1e-4)
    pidx.close()


def test_smooth_source_lands_on_exemplar_histogram():
    """For a source whose values spread smoothly inside each bin, the piecewise-linear CDFs are
    accurate and the matched image carries the exemplar's histogram (a peaky source would not:
    every copy of one value maps to one value)."""
    Z = P.synthetic_exemplar(9, 96, 3.0)
    idx = pts.ExemplarIndex(_t(Z), 8, d=8)
    img = np.random.default_rng(1).beta(2.0, 2.0, (256, 256, 3)).astype(np.float32)
    out = pts.histogram_match(idx, _t(img), 32).cpu().numpy()
    hx, hz = OH.histograms(out, 32), OH.histograms(Z, 32)
    assert np.abs(hx - hz).sum(axis=1).max() < 0.05
    idx.close()
