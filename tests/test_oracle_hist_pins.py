"""Pins of the oracle's histogram matching (section 3, Eq. 9; final matching of section 4) against
what the mathematics fixes: brute-force counting, the reduction to the plain M-step when the two
histograms agree, a two-colour case whose Eq. 9 divisors are worked out by hand, the identity
of matching an image to itself, a closed-form matching (uniform on [0, 1] onto uniform on
[0, 1/2] is v -> v/2), and monotonicity."""
import numpy as np
import pytest

import oracle
from oracle import histogram as OH
import pts_inputs as P


def test_counts_match_brute_force():
    rng = np.random.default_rng(0)
    img = rng.random((7, 9, 3)).astype(np.float32)
    img[0, 0] = [0.0, 1.0, 0.5]          # both ends of the range
    img[1, 1] = [-0.2, 1.3, 0.25]        # clamped values
    nb = 8
    expect = np.zeros((3, nb), dtype=np.int64)
    for y in range(7):
        for x in range(9):
            for j in range(3):
                v = min(max(float(img[y, x, j]), 0.0), 1.0)
                expect[j, min(int(np.floor(v * nb)), nb - 1)] += 1
    np.testing.assert_array_equal(OH.histogram_counts(img, nb), expect)
    np.testing.assert_allclose(OH.histograms(img, nb).sum(axis=1), 1.0)


@pytest.mark.parametrize("w,stride", [(4, 2), (8, 2), (4, 1)])
def test_equal_histograms_reduce_to_plain_m_step(w, stride):
    """X_cur = Z: H_x = H_z, every divisor is 1 and Eq. 9 leaves the weights as they are."""
    Z = P.synthetic_exemplar(1, 32, 2.0)
    Ho = Wo = 32
    Q = oracle.num_queries(Ho, Wo, w, stride)
    N = oracle.num_exemplar_windows(32, 32, w)
    rng = np.random.default_rng(1)
    nn = rng.integers(0, N, Q).astype(np.int32)
    Wt = rng.random(Q) + 0.5
    a = OH.m_step_hist(nn, Wt, Z, Z, w, stride, 16)
    b = oracle.m_step(nn, Wt, Z, w, Ho, Wo, stride, X_prev=Z)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


def test_two_colour_case_by_hand():
    """Exemplar: left half colour A = 0.1, right half B = 0.9 (all channels), so H_z gives each
    colour's bin 1/2 in every channel.  Current image: all A, so H_x gives A's bin 1.  Eq. 9:
    divisor(A) = 1 + 3 * (1 - 1/2) = 2.5, divisor(B) = 1 + 3 * max(0, 0 - 1/2) = 1."""
    A, B = 0.1, 0.9
    Z = np.full((8, 8, 3), A)
    Z[:, 4:] = B
    X = np.full((8, 8, 3), A)
    w, stride = 4, 2
    rng = np.random.default_rng(2)
    Q = oracle.num_queries(8, 8, w, stride)
    ex = 8 - w + 1
    nn = rng.integers(0, ex * ex, Q)
    Wt = rng.random(Q) + 0.5
    got = OH.m_step_hist(nn, Wt, Z, X, w, stride, 8)
    div = {A: 2.5, B: 1.0}
    qn = (8 - w) // stride + 1
    for y in range(8):
        for x in range(8):
            num = den = 0.0
            for p in range(Q):
                py, px = (p // qn) * stride, (p % qn) * stride
                if py <= y < py + w and px <= x < px + w:
                    c = Z[nn[p] // ex + y - py, nn[p] % ex + x - px, 0]
                    wp = Wt[p] / div[c]
                    num += wp * c
                    den += wp
            assert got[y, x, 0] == pytest.approx(num / den, abs=1e-12)
            assert got[y, x, 1] == pytest.approx(num / den, abs=1e-12)


def test_match_to_itself_is_identity():
    Z = P.synthetic_exemplar(2, 48, 3.0)
    out = OH.histogram_match(Z, Z, 32)
    np.testing.assert_allclose(out, np.clip(Z, 0, 1), rtol=0, atol=1e-9)


@pytest.mark.parametrize("nbins", [8, 32])
def test_uniform_onto_half_range_is_halving(nbins):
    """Values spread evenly over [0, 1] (the same count in every bin), matched to values spread
    evenly over [0, 1/2): F_x(v) = v, F_z^-1(u) = u / 2."""
    n = 64 * nbins
    v = (np.arange(n) + 0.5) / n
    img = np.stack([v, v[::-1], v], axis=-1).reshape(n, 1, 3)
    z = (np.arange(n) + 0.5) / (2 * n)
    Z = np.stack([z, z, z], axis=-1).reshape(n, 1, 3)
    out = OH.histogram_match(img, Z, nbins)
    np.testing.assert_allclose(out, img / 2, rtol=0, atol=1e-12)


def test_matching_is_monotone_per_channel():
    rng = np.random.default_rng(3)
    img = rng.beta(2, 5, (40, 40, 3))
    Z = P.synthetic_exemplar(3, 40, 3.0)
    out = OH.histogram_match(img, Z, 32)
    for j in range(3):
        order = np.argsort(img[..., j].ravel(), kind="stable")
        assert np.all(np.diff(out[..., j].ravel()[order]) >= -1e-12)
