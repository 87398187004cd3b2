"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each one checks it against an
independent computation (pure-Python enumeration, LAPACK, a least-squares
solve of the explicit normal equations), a closed form, an invariant, or a
value the paper prints.  A dropped term, a wrong sign, a transposed index or
a wrong window offset in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import pts_inputs as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_img(seed, H, W):
    return P.SplitMix64(seed).uniform(H * W * 3).reshape(H, W, 3)


def _windows(img, w, stride):
    """Materialised window vectors, element order (dy, dx, c), test-side code."""
    H, W, _ = img.shape
    out = []
    for y0 in range(0, H - w + 1, stride):
        for x0 in range(0, W - w + 1, stride):
            out.append(img[y0:y0 + w, x0:x0 + w, :].reshape(-1))
    return np.array(out)


# --------------------------------------------------------------------------
# E-step (Eq. 4)
# --------------------------------------------------------------------------
def test_nn_matches_pure_python_enumeration(oracle_lib):
    Z = _rand_img(1, 12, 12)
    X = _rand_img(2, 16, 16)
    w, s = 4, 2
    nn, d2 = oracle.nn_bruteforce(X, Z, w, s)
    qx = (16 - w) // s + 1
    ex = 12 - w + 1
    for q in range(len(nn)):
        y0, x0 = (q // qx) * s, (q % qx) * s
        best, bn = math.inf, -1
        for n in range(ex * ex):
            ey, exx = divmod(n, ex)
            acc = 0.0
            for dy in range(w):
                for dx in range(w):
                    for c in range(3):
                        t = X[y0 + dy, x0 + dx, c] - Z[ey + dy, exx + dx, c]
                        acc += t * t
            if acc < best:
                best, bn = acc, n
        assert nn[q] == bn
        assert d2[q] == best


def test_nn_tie_goes_to_smallest_index(oracle_lib):
    # exemplar made of two identical halves: every window in the right half
    # duplicates one in the left half, so each query has >= 2 minimisers
    half = _rand_img(3, 10, 6)
    Z = np.concatenate([half, half], axis=1)
    X = Z[0:6, 0:6].copy()
    nn, d2 = oracle.nn_bruteforce(X, Z, 4, 2)
    ex = Z.shape[1] - 4 + 1
    for q, n in enumerate(nn):
        y0, x0 = divmod(q, 2)
        assert d2[q] == 0.0
        assert n == (2 * y0) * ex + 2 * x0  # left copy, not the right one


def test_translation_special_case(oracle_lib):
    """An output equal to an exemplar crop at an even offset matches the window
    at the same offset with distance 0 (windows are unique under noise)."""
    Z = P.synthetic_exemplar(5, 48, 3.0).astype(np.float64)
    oy, ox, Ho, w = 6, 10, 24, 8
    X = Z[oy:oy + Ho, ox:ox + Ho].copy()
    nn, d2 = oracle.nn_bruteforce(X, Z, w, 2)
    qx = (Ho - w) // 2 + 1
    ex = 48 - w + 1
    q = np.arange(len(nn))
    expect = (oy + 2 * (q // qx)) * ex + (ox + 2 * (q % qx))
    np.testing.assert_array_equal(nn, expect)
    assert np.all(d2 == 0.0)


def test_subset_queries_equal_full(oracle_lib):
    Z = _rand_img(7, 14, 14)
    X = _rand_img(8, 20, 20)
    nn, d2 = oracle.nn_bruteforce(X, Z, 6, 2)
    sub = np.array([0, 3, 17, len(nn) - 1])
    nn_s, d2_s = oracle.nn_bruteforce(X, Z, 6, 2, qlist=sub)
    np.testing.assert_array_equal(nn_s, nn[sub])
    np.testing.assert_array_equal(d2_s, d2[sub])
    pd = oracle.pair_dist2(X, Z, 6, 2, sub, nn[sub])
    np.testing.assert_array_equal(pd, d2[sub])


# --------------------------------------------------------------------------
# PCA (section 2.2)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("He,w", [(20, 4), (14, 6)])  # N >= D and N < D (Gram branch)
def test_pca_against_lapack(oracle_lib, He, w):
    Z = P.synthetic_exemplar(9, He, 3.0).astype(np.float64)
    V = _windows(Z, w, 1)
    N, D = V.shape
    d = min(8, N - 1)
    mu, B, ev, sweeps = oracle.pca_fit(Z, w, d)
    assert sweeps > 0
    np.testing.assert_allclose(mu, V.mean(axis=0), rtol=0, atol=1e-14)
    U = V - V.mean(axis=0)
    C = U.T @ U / N
    lam, vec = np.linalg.eigh(C)
    lam, vec = lam[::-1], vec[:, ::-1]
    k = min(N, D)
    np.testing.assert_allclose(ev[:d], lam[:d], rtol=1e-10, atol=1e-14 * lam[0])
    assert abs(ev.sum() - np.trace(C)) <= 1e-12 * np.trace(C)
    np.testing.assert_allclose(B @ B.T, np.eye(d), atol=1e-12)
    # projector onto the top-d subspace (eigenvector signs do not matter)
    P_or = B.T @ B
    P_la = vec[:, :d] @ vec[:, :d].T
    gap = lam[d - 1] - lam[d]
    assert gap > 1e-6 * lam[0]
    assert np.linalg.norm(P_or - P_la) < 1e-9
    # each basis vector is an eigenvector: C b = lambda b
    for j in range(d):
        np.testing.assert_allclose(C @ B[j], ev[j] * B[j], atol=1e-11 * lam[0])
    assert k == len(ev)


def test_jacobi_recovers_planted_spectrum(oracle_lib):
    rng = P.SplitMix64(11)
    n = 9
    lam = np.array([5.0, 3.0, 3.0 - 1e-7, 1.0, 0.5, 0.25, 1e-3, 0.0, -2.0])
    v = rng.normal(n)
    H = np.eye(n) - 2.0 * np.outer(v, v) / (v @ v)  # Householder reflector
    A = H @ np.diag(lam) @ H.T
    ev, V, sweeps = oracle.jacobi_eigh(A)
    np.testing.assert_allclose(ev, np.sort(lam)[::-1], atol=1e-14 * 5)
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(V @ np.diag(ev) @ V.T, A, atol=1e-13)


def test_projection_pythagoras_and_explicit(oracle_lib):
    Z = P.synthetic_exemplar(12, 24, 3.0).astype(np.float64)
    X = _rand_img(13, 20, 20)
    w, d = 4, 6
    mu, B, _, _ = oracle.pca_fit(Z, w, d)
    y, un, rs = oracle.project(X, w, 2, mu, B)
    U = _windows(X, w, 2) - mu
    np.testing.assert_allclose(y, U @ B.T, atol=1e-13)
    np.testing.assert_allclose(un, (U * U).sum(1), rtol=1e-13)
    np.testing.assert_allclose(rs ** 2 + (y * y).sum(1), un, rtol=1e-12)
    lst = np.array([4, 0, 9])
    y2, _, r2 = oracle.project(X, w, 2, mu, B, lst)
    np.testing.assert_array_equal(y2, y[lst])
    np.testing.assert_array_equal(r2, rs[lst])


# --------------------------------------------------------------------------
# IRLS (Eqs. 5-8)
# --------------------------------------------------------------------------
def test_irls_identity_eq6(oracle_lib):
    d2 = P.SplitMix64(14).uniform(200) * 4.0 + 0.01
    r = 0.8
    W, er, ed = oracle.irls(d2, r, delta=1e-3)
    # Eq. 6/8: sum W_p ||x_p - z_p||^2 equals the robust energy of Eq. 5
    assert abs((W * d2).sum() - er) <= 1e-12 * er
    assert er == pytest.approx(ed, rel=1e-15)
    assert er == pytest.approx((d2 ** (r / 2)).sum(), rel=1e-13)
    W2, e2, e2d = oracle.irls(d2, 2.0)
    assert np.all(W2 == 1.0) and e2 == pytest.approx(d2.sum(), rel=1e-14) and e2d == e2


def test_irls_delta_branch_continuous(oracle_lib):
    r, delta = 0.8, 0.1
    eps = 1e-9
    d2 = np.array([(delta - eps) ** 2, (delta + eps) ** 2, 0.0])
    W, _, _ = oracle.irls(d2, r, delta)
    assert W[0] == pytest.approx(delta ** (r - 2), rel=1e-14)
    assert W[2] == pytest.approx(delta ** (r - 2), rel=1e-14)
    _, _, lo = oracle.irls(d2[:1], r, delta)
    _, _, hi = oracle.irls(d2[1:2], r, delta)
    assert abs(hi - lo) < 1e-7
    _, _, z = oracle.irls(d2[2:], r, delta)
    assert z == pytest.approx(delta ** r * (1 - r / 2), rel=1e-13)


# --------------------------------------------------------------------------
# M-step (Eq. 8 minimiser) and the paper's neighbourhood count
# --------------------------------------------------------------------------
def test_m_step_equals_weighted_least_squares(oracle_lib):
    Z = _rand_img(15, 10, 10)
    Ho = Wo = 12
    w, s = 4, 2
    Q = oracle.num_queries(Ho, Wo, w, s)
    N = oracle.num_exemplar_windows(10, 10, w)
    nn = P.random_nn(16, Q, N)
    Wt = P.random_weights(17, Q).astype(np.float64)
    X = oracle.m_step(nn, Wt, Z, w, Ho, Wo, s)
    # explicit: minimise sum_p W_p ||S_p x - z_p||^2 over x (per channel)
    qx = (Wo - w) // s + 1
    ex = 10 - w + 1
    rows, rhs = [], []
    for p in range(Q):
        y0, x0 = (p // qx) * s, (p % qx) * s
        ey, exx = divmod(int(nn[p]), ex)
        for dy in range(w):
            for dx in range(w):
                r = np.zeros(Ho * Wo)
                r[(y0 + dy) * Wo + (x0 + dx)] = math.sqrt(Wt[p])
                rows.append(r)
                rhs.append(math.sqrt(Wt[p]) * Z[ey + dy, exx + dx])
    A = np.array(rows)
    Bm = np.array(rhs)
    sol, *_ = np.linalg.lstsq(A, Bm, rcond=None)
    np.testing.assert_allclose(X.reshape(-1, 3), sol, atol=1e-12)


def test_paper_neighbourhood_count(oracle_lib):
    """Section 2.2 worked example: with 8x8 neighbourhoods every pixel lies in
    4x4 = 16 windows (on the 2x2 patch grid), so with all windows matched to
    one exemplar window and unit weights an interior pixel is the mean of the
    16 window entries sharing its row/column parity."""
    with open(os.path.join(GOLDEN, "paper_values.json")) as f:
        pv = json.load(f)
    w = pv["window_width_example"]["value"]
    cover = pv["windows_per_pixel_8x8"]["value"]
    Z = _rand_img(18, 12, 12)
    Ho = Wo = 24
    Q = oracle.num_queries(Ho, Wo, w, 2)
    n0 = 7
    X = oracle.m_step(np.full(Q, n0, np.int32), None, Z, w, Ho, Wo, 2)
    ey, ex_ = divmod(n0, 12 - w + 1)
    win = Z[ey:ey + w, ex_:ex_ + w]
    for y in range(w, Ho - w):
        for x in range(w, Wo - w):
            sub = win[(y % 2)::2, (x % 2)::2]
            assert sub.shape[0] * sub.shape[1] == cover
            np.testing.assert_allclose(X[y, x], sub.reshape(-1, 3).mean(0), atol=1e-14)


# --------------------------------------------------------------------------
# EM behaviour: monotone energy, exact reproduction
# --------------------------------------------------------------------------
def test_energy_never_rises_r2(oracle_lib):
    Z = P.synthetic_exemplar(19, 32, 3.0)
    X0 = P.random_patch_init(Z, 40, 40, 8, 1)
    res = oracle.synthesize_level(Z, X0, 8, 5, r=2.0, f32_io=False)
    E = res["E"]
    assert np.all(np.diff(E) <= 1e-12 * E[0])
    assert E[-1] < E[0]


def test_energy_never_rises_robust_r08(oracle_lib):
    Z = P.synthetic_exemplar(20, 32, 3.0)
    X0 = P.random_patch_init(Z, 40, 40, 8, 2)
    res = oracle.synthesize_level(Z, X0, 8, 5, r=0.8, delta=1e-3, f32_io=False)
    Ed = res["E_delta"]
    assert np.all(np.diff(Ed) <= 1e-12 * Ed[0])


def test_exact_reproduction(oracle_lib):
    """Output seeded with the exemplar: every query has a zero-distance match,
    the M-step returns the exemplar bit for bit and the energy is 0."""
    Z = P.synthetic_exemplar(21, 32, 3.0)
    res = oracle.synthesize_level(Z, Z, 8, 3, r=2.0, keep_trajectory=True)
    assert np.all(res["E"] == 0.0)
    assert np.array_equal(res["X"], Z.astype(np.float64))
    # also a crop whose origin lies on the stride grid
    C = Z[4:28, 2:26]
    res = oracle.synthesize_level(Z, C, 8, 2, r=2.0)
    assert np.all(res["E"] == 0.0) and np.array_equal(res["X"], C.astype(np.float64))


# --------------------------------------------------------------------------
# pyramid (section 2.1 coarse-to-fine)
# --------------------------------------------------------------------------
def test_downsample_preserves_constants_and_ramps(oracle_lib):
    H = W = 16
    const = np.full((H, W, 3), 0.37)
    np.testing.assert_allclose(oracle.downsample2(const), 0.37, atol=1e-15)
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    ramp = np.stack([xx, yy, 2 * xx - yy], -1)
    out = oracle.downsample2(ramp)
    # the symmetric binomial kernel reproduces linear functions away from borders
    for y in range(1, 7):
        for x in range(1, 7):
            np.testing.assert_allclose(out[y, x], [2 * x, 2 * y, 4 * x - 2 * y], atol=1e-12)
    # binomial weights: an impulse spreads as outer([1,4,6,4,1])/256
    imp = np.zeros((H, W, 3))
    imp[8, 8] = 1.0
    o = oracle.downsample2(imp)
    assert o[4, 4, 0] == pytest.approx(36 / 256)
    assert o[4, 5, 0] == pytest.approx(6 / 256)
    assert o[3, 5, 0] == pytest.approx(1 / 256)


@pytest.mark.parametrize("H", [8, 9])
def test_downsample_border_mirrors_without_edge_repeat(oracle_lib, H):
    """Reading c-9 of section 2.1's coarse-to-fine step at the border: index -1 maps to 1 and H to
    H-2 (the edge sample is not repeated).  Hand-computed taps of the 1-D binomial [1 4 6 4 1]/16
    for an impulse on the first and on the last row, even and odd H: an edge-repeating or clamping
    border gives 10/16 or 11/16 at the first output row instead of 6/16, and moves the weights of
    the last row."""
    W = 6
    top = np.zeros((H, W, 3))
    top[0] = 1.0                     # impulse on row 0 (constant along x, so only the rows count)
    o = oracle.downsample2(top)
    assert o.shape == ((H + 1) // 2, (W + 1) // 2, 3)
    # out row 0 reads rows -2..2 -> 2 1 0 1 2: row 0 only at the centre tap
    assert o[0, 1, 0] == pytest.approx(6 / 16, abs=1e-15)
    # out row 1 reads rows 0..4: row 0 at the first tap
    assert o[1, 1, 0] == pytest.approx(1 / 16, abs=1e-15)
    assert np.all(o[2:] == 0.0)
    bot = np.zeros((H, W, 3))
    bot[H - 1] = 1.0                 # impulse on the last row
    o = oracle.downsample2(bot)
    if H == 8:
        # out row 3 reads rows 4 5 6 7 8 -> 4 5 6 7 6: row 7 at the fourth tap only
        assert o[3, 1, 0] == pytest.approx(4 / 16, abs=1e-15)
        assert o[2, 1, 0] == 0.0     # rows 2..6
    else:
        # out row 4 reads rows 6 7 8 9 10 -> 6 7 8 7 6: row 8 at the centre tap only
        assert o[4, 1, 0] == pytest.approx(6 / 16, abs=1e-15)
        # out row 3 reads rows 4..8: row 8 at the last tap
        assert o[3, 1, 0] == pytest.approx(1 / 16, abs=1e-15)
    # the corner of a 2-D impulse: both directions at the centre tap
    cor = np.zeros((H, H, 3))
    cor[0, 0] = 1.0
    assert oracle.downsample2(cor)[0, 0, 2] == pytest.approx(36 / 256, abs=1e-15)
    cor[0, 0] = 0.0
    cor[H - 1, H - 1] = 1.0
    want = (4 / 16) ** 2 if H == 8 else (6 / 16) ** 2
    last = (H + 1) // 2 - 1
    assert oracle.downsample2(cor)[last, last, 1] == pytest.approx(want, abs=1e-15)


def test_upsample_bilinear(oracle_lib):
    H = W = 6
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    ramp = np.stack([xx, yy, xx + yy], -1)
    out = oracle.upsample2(ramp)
    for Y in range(1, 2 * H - 1):
        for X in range(1, 2 * W - 1):
            sy, sx = (Y + 0.5) / 2 - 0.5, (X + 0.5) / 2 - 0.5
            np.testing.assert_allclose(out[Y, X], [sx, sy, sx + sy], atol=1e-12)
    assert out[0, 0, 0] == 0.0 and out[-1, -1, 1] == H - 1  # clamped corners


# --------------------------------------------------------------------------
# input generator frozen
# --------------------------------------------------------------------------
def test_generator_golden_hashes():
    with open(os.path.join(GOLDEN, "generator_hashes.json")) as f:
        g = json.load(f)
    for key, digest in g.items():
        seed, size, shrink = key.split("_")
        img = P.synthetic_exemplar(int(seed), int(size), float(shrink))
        assert P.array_digest(img) == digest, key


# --------------------------------------------------------------------------
# stopping rule of section 2.1: iterate until {z_p} no longer changes
# --------------------------------------------------------------------------
def test_converge_stops_at_once_on_the_exemplar(oracle_lib):
    """Seeded with the exemplar: the first search matches every window to itself, the M-step
    returns the exemplar, the second search repeats the first: one M-step, energy 0."""
    Z = P.synthetic_exemplar(22, 32, 3.0)
    res = oracle.synthesize_level_converge(Z, Z, 8, 10, r=0.8)
    assert res["iters"] == 1
    assert np.all(res["E"] == 0.0) and len(res["E"]) == 2


def test_converged_image_is_a_fixed_point(oracle_lib):
    """r = 2 (all weights 1): when two consecutive searches return the same windows, one more
    iteration of the plain EM loop returns the image unchanged, a fixed point of the E- and
    M-steps.  (For r < 2 the IRLS weights still move with the image, so only the windows are fixed.)"""
    Z = P.synthetic_exemplar(23, 32, 3.0)
    X0 = P.random_patch_init(Z, 40, 40, 8, 3)
    res = oracle.synthesize_level_converge(Z, X0, 8, 40, r=2.0)
    assert 1 <= res["iters"] < 40
    again = oracle.synthesize_level(Z, res["X"], 8, 1, r=2.0)
    np.testing.assert_array_equal(again["X"], res["X"])


def test_converge_robust_energy_never_rises(oracle_lib):
    """r = 0.8: the delta-form energy, which Eq. 8 majorises, never rises until the rule stops."""
    Z = P.synthetic_exemplar(23, 32, 3.0)
    X0 = P.random_patch_init(Z, 40, 40, 8, 5)
    res = oracle.synthesize_level_converge(Z, X0, 8, 40, r=0.8, f32_io=False)
    assert 1 <= res["iters"] <= 40
    assert np.all(np.diff(res["E_delta"]) <= 1e-12 * res["E_delta"][0])


def test_converge_respects_the_iteration_cap(oracle_lib):
    Z = P.synthetic_exemplar(24, 32, 3.0)
    X0 = P.random_patch_init(Z, 40, 40, 8, 4)
    res = oracle.synthesize_level_converge(Z, X0, 8, 1, r=0.8)
    assert res["iters"] == 1 and len(res["E"]) == 2
    res0 = oracle.synthesize_level_converge(Z, X0, 8, 0, r=0.8)
    assert res0["iters"] == 0 and len(res0["E"]) == 1
