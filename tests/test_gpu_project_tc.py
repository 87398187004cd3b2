"""The FP16 search's query rows (y, r, 1, 1, 1, 0, ...) from the tensor-core projection (section
2.2: y = B^T (x - mu), r = sqrt(max(0, ||x - mu||^2 - ||y||^2))), against the oracle's FP64
projection onto the index's own basis and mean, and against the FP32 SIMT projection.

Tolerances, from the arithmetic.  The tensor-core route splits every value into FP16 high and low
parts (22 significant bits together) and accumulates u_hi b_hi + u_lo b_hi + u_hi b_lo in FP32, so
a coordinate before its FP16 rounding is within e = 2^-17 ||u|| of the exact one (the dropped
u_lo b_lo is about 2^-22 |u| |b| per term, the FP32 accumulation of 3 D products a few 2^-24
||u||; 2^-17 leaves a wide margin; tests/test_split_arith.py checks the split's arithmetic).
Rounding to FP16 adds at most 2^-11 of the value, or 2^-25 below the normal range.  A dropped
split term (about 2^-12.8 ||u|| / sqrt(D) per coordinate, several times the bound at the largest
of the coordinates), a wrong basis row or a misplaced element fails the bound.  ||u||^2 is an FP32 sum of D positive terms: within
(D + 4) 2^-24 of itself.  The residual's square is a difference of two sums that each carry
errors near 2^-12 ||u||^2 at most, then rounded to FP16 (2^-10 relative in the square)."""
import numpy as np
import pytest

import oracle
import pts_inputs as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2006_11851_gb300 as pts  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def _images(He, Ho, w, C, seed):
    Z = P.synthetic_exemplar(seed, He, 3.0)
    X = P.random_patch_init(Z, Ho, Ho, w, seed + 1)
    if C == 4:  # RGBS: a scale map as the fourth channel of both images
        s = np.linspace(0.2, 1.0, He, dtype=np.float32)[:, None, None] * np.ones((He, He, 1), np.float32)
        Z = np.ascontiguousarray(np.concatenate([Z, s], axis=2))
        sx = np.linspace(1.0, 0.3, Ho, dtype=np.float32)[None, :, None] * np.ones((Ho, Ho, 1), np.float32)
        X = np.ascontiguousarray(np.concatenate([X, sx], axis=2))
    return Z, X


@pytest.mark.parametrize("He,Ho,w,stride,C", [
    (64, 128, 8, 2, 3),   # D = 192 (6 chunks), Q = 3,721: 30 blocks of 128, the last ragged
    (24, 29, 5, 1, 3),    # D = 75: 8-element groups straddle window rows and the vector's end
    (33, 36, 16, 2, 3),   # D = 768 (24 chunks), Q = 121: one ragged block
    (30, 40, 8, 4, 3),    # stride 4
    (40, 52, 8, 2, 4),    # RGBS, D = 256
])
def test_query_rows_against_oracle_and_simt(He, Ho, w, stride, C):
    Z, X = _images(He, Ho, w, C, 3)
    idx = pts.ExemplarIndex(_t(Z), w, d=16)
    d = idx.info["d_fast"]
    rows, norm = pts.query_rows_f16(idx, _t(X), stride, tensor_cores=True)
    rows_s, norm_s = pts.query_rows_f16(idx, _t(X), stride, tensor_cores=False)
    mean, basis = pts.index_pca(idx)
    y64, un64, rs64 = oracle.project(X, w, stride, mean.cpu().numpy(), basis.cpu().numpy())
    h = rows.float().cpu().numpy().astype(np.float64)
    hs = rows_s.float().cpu().numpy().astype(np.float64)
    nrm = norm.cpu().numpy().astype(np.float64)
    Q, K = h.shape
    D = C * w * w
    assert Q == len(un64) and K == (d + 4 + 15) // 16 * 16 and y64.shape == (Q, d)
    # the three norm-slot ones and the zero padding, exactly
    assert np.all(h[:, d + 1:d + 4] == 1.0) and np.all(h[:, d + 4:] == 0.0)
    # coordinates
    un_ = np.sqrt(un64)[:, None]
    err = np.abs(h[:, :d] - y64)
    bound = 2.0 ** -11 * np.abs(y64) + 2.0 ** -17 * un_ * (1 + 2.0 ** -11) + 2.0 ** -25
    assert np.all(err <= bound), (err / bound).max()
    # ||u||^2 and the residual
    assert np.all(np.abs(nrm - un64) <= (D + 4) * 2.0 ** -24 * un64 + 1e-30)
    r2 = h[:, d] ** 2
    assert np.all(np.abs(r2 - rs64 ** 2) <= 2.0 ** -10 * r2 + 2.0 ** -11 * un64), \
        (np.abs(r2 - rs64 ** 2) / (2.0 ** -10 * r2 + 2.0 ** -11 * un64)).max()
    # the SIMT projection's rows: the same values up to each route's own error before rounding
    diff = np.abs(h[:, :d] - hs[:, :d])
    assert np.all(diff <= 2.0 ** -10 * np.maximum(np.abs(h[:, :d]), np.abs(hs[:, :d])) + 2.0 ** -16 * un_ + 2.0 ** -24)
    frac = float((diff > 0).mean())
    print(f"\nD = {D}: {frac:.2e} of the coordinates differ from the SIMT route's (each by its rounding)")
    assert frac < 0.02
    np.testing.assert_allclose(nrm, norm_s.cpu().numpy(), rtol=2 * (D + 4) * 2.0 ** -24, atol=1e-30)
    idx.close()


def test_f16_search_through_the_tensor_core_projection():
    """The FP16 search, its query rows from the tensor-core projection, against the oracle: the
    FP32 distance of every window it returns is never below the nearest one's, and the total
    stays within 1% of the oracle's (the mode's energy criterion); the fraction of queries that
    get the oracle's own window is printed."""
    Z = P.synthetic_exemplar(0, 96, 4.0)
    X = P.random_patch_init(Z, 160, 160, 8, 2)
    idx = pts.ExemplarIndex(_t(Z), 8, d=32)
    nn_f, d2_f = pts.nn_search(idx, _t(X), 2, "f16")
    nn_o, d2_o = oracle.nn_bruteforce(X, Z, 8, 2)
    d2f = d2_f.cpu().numpy().astype(np.float64)
    assert np.all(d2f >= d2_o * (1 - 1e-5) - 1e-6)
    assert float(d2f.sum()) <= 1.01 * float(d2_o.sum())
    agree = float((nn_f.cpu().numpy() == nn_o).mean())
    print(f"\nFP16 search: {agree:.4f} of the queries get the oracle's nearest window")
    idx.close()
