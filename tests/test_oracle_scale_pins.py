"""Pins of the oracle's scale map (Methodology section 1, Eqs. 1-3) and of its use in synthesis
(section 3: the scale map as a fourth channel, resampling to the output size, the scale-guided
initialisation), against closed forms, the geometry the paper states, and independent numpy
brute force on small inputs.  Each is chosen so that a plausible slip fails it: a swapped sin
and cos, a top-left origin instead of the bottom-left one, integer halves, Eq. 3's printed
Y_max kept as the leading term, a channel stride left at 3, a guide channel that drifts."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import pts_inputs as P
from oracle import scale as OS

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.json")
PAPER = json.load(open(GOLDEN))
FIG_ANGLES = [tuple(a) for a in PAPER["scale_map_angles_deg"]["value"]]


# ---------------------------------------------------------------------------
# Eq. 1
# ---------------------------------------------------------------------------
def test_eq1_closed_forms():
    assert OS.scale_range(0.0) == (1.0, 1.0, 0.0)
    s_max, s_min, s_d = OS.scale_range(60.0)
    assert s_max == pytest.approx(2.0, rel=1e-15) and s_min == pytest.approx(0.5, rel=1e-15)
    assert s_d == pytest.approx(1.5, rel=1e-15)
    s_max, s_min, _ = OS.scale_range(30.0)
    assert s_max == pytest.approx(2.0 / math.sqrt(3.0), rel=1e-15)
    assert s_min == pytest.approx(math.sqrt(3.0) / 2.0, rel=1e-15)
    for sigma in (5.0, 30.0, 45.0, 60.0, 80.0):
        s_max, s_min, s_d = OS.scale_range(sigma)
        assert s_max * s_min == pytest.approx(1.0, rel=1e-14)     # reciprocal pair
        assert s_d > 0.0
    # a plane whose texels shrink by a factor k from bottom to top has S_max / S_min = k
    k = 4.0
    s_max, s_min, _ = OS.scale_range(math.degrees(math.acos(1.0 / math.sqrt(k))))
    assert s_max / s_min == pytest.approx(k, rel=1e-14)
    with pytest.raises(ValueError):
        OS.scale_range(90.0)


# ---------------------------------------------------------------------------
# Eq. 2
# ---------------------------------------------------------------------------
def test_eq2_closed_forms():
    h, w = 64, 96
    y_max, y_min, y_d = OS.y_range(h, w, 0.0)                 # tilt 0: only the height counts
    assert (y_max, y_min, y_d) == (h / 2 - 1, -(h / 2 - 1), h - 2)
    y_max, _, _ = OS.y_range(h, w, 90.0)                      # tilt 90: only the width counts
    assert y_max == pytest.approx(w / 2 - 1, abs=1e-12)
    y_max, _, _ = OS.y_range(h, w, 45.0)
    assert y_max == pytest.approx((w / 2 - 1 + h / 2 - 1) / math.sqrt(2.0), rel=1e-15)
    # real halves: an odd width gives a half-integer range
    assert OS.y_range(9, 7, 90.0)[0] == pytest.approx(2.5, abs=1e-12)
    with pytest.raises(ValueError):
        OS.y_range(h, w, 120.0)


# ---------------------------------------------------------------------------
# Eq. 3
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("sigma,tau", FIG_ANGLES + [(45.0, 0.0), (45.0, 90.0), (10.0, 33.0)])
@pytest.mark.parametrize("h,w", [(64, 64), (37, 52)])
def test_eq3_endpoints_and_orientation(sigma, tau, h, w):
    S = OS.scale_map(h, w, sigma, tau)
    s_max, s_min, _ = OS.scale_range(sigma)
    # pixel (1, 1) (bottom-left origin) projects to Y_min and carries S_max; the top-right pixel
    # projects to Y_max and carries S_min.  In array rows, p(y) = 1 is row h - 2.
    assert S[h - 2, 1] == pytest.approx(s_max, rel=1e-12)
    assert S[0, w - 1] == pytest.approx(s_min, rel=1e-12)
    # the largest scale is at the origin (bottom-left corner), the smallest at the top-right
    if 0.0 < tau < 90.0:
        assert np.unravel_index(np.argmax(S), S.shape) == (h - 1, 0)
        assert np.unravel_index(np.argmin(S), S.shape) == (0, w - 1)
    assert S.max() >= s_max and S.min() == pytest.approx(s_min, rel=1e-12)


def test_eq3_flat_plane_has_unit_scale():
    for tau in (0.0, 18.0, 60.0, 90.0):
        assert np.array_equal(OS.scale_map(20, 30, 0.0, tau), np.ones((20, 30)))


def test_eq3_level_sets_follow_the_tilt():
    h, w, sigma = 40, 48, 50.0
    # an affine map: all second differences vanish
    S = OS.scale_map(h, w, sigma, 27.0)
    assert np.abs(np.diff(S, 2, axis=0)).max() < 1e-12 and np.abs(np.diff(S, 2, axis=1)).max() < 1e-12
    assert np.abs(np.diff(np.diff(S, axis=0), axis=1)).max() < 1e-12
    # tilt 0: the scale changes only with height, shrinking towards the top rows
    S0 = OS.scale_map(h, w, sigma, 0.0)
    assert np.abs(S0 - S0[:, :1]).max() < 1e-12
    assert np.all(np.diff(S0[:, 0]) > 0)                         # row index grows downwards
    # tilt 90: only with the column, shrinking to the right
    S90 = OS.scale_map(h, w, sigma, 90.0)
    assert np.abs(S90 - S90[:1, :]).max() < 1e-12
    assert np.all(np.diff(S90[0, :]) < 0)
    # tilt 45: constant along the direction (+1 in x, -1 in y up) = down-right in the array
    S45 = OS.scale_map(h, w, sigma, 45.0)
    assert np.abs(S45[:-1, :-1] - S45[1:, 1:]).max() < 1e-12
    # a larger slant gives a steeper map with the same level sets
    S_lo, S_hi = OS.scale_map(h, w, 20.0, 27.0), OS.scale_map(h, w, 60.0, 27.0)
    assert np.ptp(S_hi) > np.ptp(S_lo)
    assert np.array_equal(np.argsort(S_lo, axis=None, kind="stable"), np.argsort(S_hi, axis=None, kind="stable"))


def test_eq3_rejects_a_degenerate_extent():
    with pytest.raises(ValueError):
        OS.scale_map(2, 2, 30.0, 45.0)
    with pytest.raises(ValueError):
        OS.scale_map(2, 50, 30.0, 0.0)


# ---------------------------------------------------------------------------
# resampling to the output size (section 3, step 2)
# ---------------------------------------------------------------------------
def test_resample_identity_and_corners():
    S = OS.scale_map(17, 23, 40.0, 18.0)
    assert np.array_equal(OS.resample(S, 17, 23), S)
    R = OS.resample(S, 41, 30)
    for (a, b), (c, d) in [((0, 0), (0, 0)), ((0, -1), (0, -1)), ((-1, 0), (-1, 0)), ((-1, -1), (-1, -1))]:
        assert R[a, b] == pytest.approx(S[c, d], rel=1e-14)


def test_resample_of_an_affine_map_is_exact():
    """Bilinear interpolation reproduces an affine function exactly, so resampling the (affine)
    scale map must equal the affine function fitted to three exemplar pixels, evaluated at the
    corner-aligned source coordinates."""
    He, We, Ho, Wo = 31, 45, 64, 50
    S = OS.scale_map(He, We, 60.0, 60.0)
    a = S[0, 0]
    gx = S[0, 1] - S[0, 0]                 # per column
    gy = S[1, 0] - S[0, 0]                 # per row
    R = OS.resample(S, Ho, Wo)
    yy, xx = np.mgrid[0:Ho, 0:Wo].astype(np.float64)
    expect = a + gx * xx * (We - 1) / (Wo - 1) + gy * yy * (He - 1) / (Ho - 1)
    assert np.abs(R - expect).max() < 1e-12


# ---------------------------------------------------------------------------
# scale-guided initialisation (section 3, step 3)
# ---------------------------------------------------------------------------
def _init_bruteforce(Z, S_z, S_x, u, nbins):
    """The same reading, written differently: sort exemplar pixels by bin (stable), find each
    output pixel's bin range with searchsorted, widening to the nearest filled bin."""
    lo, hi = S_z.min(), S_z.max()
    bz = OS.scale_bins(S_z, lo, hi, nbins).ravel()
    order = np.argsort(bz, kind="stable")
    sorted_b = bz[order]
    src = []
    for b, uu in zip(OS.scale_bins(S_x, lo, hi, nbins).ravel(), u.ravel()):
        for dist in range(nbins):
            cands = [c for c in (b - dist, b + dist) if 0 <= c < nbins]
            ranges = [(np.searchsorted(sorted_b, c, "left"), np.searchsorted(sorted_b, c, "right")) for c in cands]
            ranges = [r for r in ranges if r[1] > r[0]]
            if ranges:
                i0, i1 = ranges[0]
                src.append(order[i0 + min(int(uu * (i1 - i0)), i1 - i0 - 1)])
                break
    return np.array(src).reshape(S_x.shape)


def test_init_copies_pixels_of_the_same_scale():
    He, Ho, nbins = 48, 80, 32
    Z = P.synthetic_exemplar(4, He, 4.0).astype(np.float64)
    sigma = math.degrees(math.acos(0.5))                   # S_max / S_min = 4, the exemplar's shrink
    S_z = OS.scale_map(He, He, sigma, 0.0)
    S_x = OS.resample(S_z, Ho, Ho)
    u = P.uniform_field(1, Ho, Ho)
    X0, src = OS.scale_guided_init(Z, S_z, S_x, u, nbins)
    lo, hi = S_z.min(), S_z.max()
    bz = OS.scale_bins(S_z, lo, hi, nbins).ravel()
    bx = OS.scale_bins(S_x, lo, hi, nbins)
    assert np.array_equal(bz[src], bx)                     # every bin is filled at tilt 0
    assert np.array_equal(X0, Z.reshape(-1, 3)[src.ravel()].reshape(Ho, Ho, 3))
    # tilt 0: the scale is a function of height only, so a pixel at a given fraction of the
    # output height copies from the same fraction of the exemplar height, within one bin
    rows_src = src // He
    frac_x = np.arange(Ho)[:, None] / (Ho - 1)
    assert np.abs(rows_src / (He - 1) - frac_x).max() <= 1.0 / nbins + 1.0 / (He - 1)
    assert np.array_equal(src, _init_bruteforce(Z, S_z, S_x, u, nbins))


def test_init_on_a_flat_plane_is_uniform_over_the_exemplar():
    He, Ho = 12, 20
    Z = P.synthetic_exemplar(2, He, 2.0).astype(np.float64)
    S_z = OS.scale_map(He, He, 0.0, 0.0)
    u = P.uniform_field(3, Ho, Ho)
    _, src = OS.scale_guided_init(Z, S_z, OS.resample(S_z, Ho, Ho), u, nbins=16)
    assert np.array_equal(src, np.floor(u * He * He).astype(np.int64))


def test_init_borrows_the_nearest_filled_bin():
    # exemplar scales fill bins 0 and 3 of 4 only; output pixels in bins 1 and 2 borrow from
    # 0 and 3 respectively (bin 1 is nearer to 0, bin 2 to 3), a tie would go to the lower bin
    S_z = np.array([[1.0, 1.0], [4.0, 4.0]])
    Z = np.arange(12, dtype=np.float64).reshape(2, 2, 3)
    S_x = np.array([[1.0, 1.9], [3.2, 4.0]])
    u = np.array([[0.0, 0.99], [0.0, 0.5]])
    _, src = OS.scale_guided_init(Z, S_z, S_x, u, nbins=4)
    assert src.tolist() == [[0, 1], [2, 3]]
    S_z3 = np.array([[1.0, 4.0], [4.0, 4.0]])              # bins 0 and 3 again
    _, src = OS.scale_guided_init(Z, S_z3, np.array([[2.5, 2.5], [2.5, 2.5]]), np.zeros((2, 2)), nbins=2)
    # 2 bins: 2.5 -> bin 1 (filled by pixels 1, 2, 3)
    assert src.tolist() == [[1, 1], [1, 1]]
    S_z5 = np.array([[0.0, 0.0, 4.0, 4.0, 4.0]])
    _, src = OS.scale_guided_init(np.zeros((1, 5, 3)), S_z5, np.array([[2.0, 2.0]]), np.array([[0.0, 0.6]]), nbins=5)
    assert src.tolist() == [[0, 1]]                        # bin 2 is 2 from bins 0 and 4: the lower wins


# ---------------------------------------------------------------------------
# RGBS windows (sections 2.2 and 3) through the channel-general oracle
# ---------------------------------------------------------------------------
def _windows(img, w, stride):
    v = np.lib.stride_tricks.sliding_window_view(img, (w, w), axis=(0, 1))   # [y, x, C, w, w]
    v = v[::stride, ::stride].transpose(0, 1, 3, 4, 2)                        # [y, x, w, w, C]
    return v.reshape(-1, w * w * img.shape[2])


def test_rgbs_dimension_is_the_papers():
    w = PAPER["window_width_example"]["value"]
    Z4 = OS.rgbs(np.zeros((12, 12, 3)), np.ones((12, 12)))
    assert O.window_mean(Z4, w).shape == (PAPER["pca_dims_rgbs_8x8"]["input_dim"],)


def test_rgbs_search_matches_numpy_bruteforce():
    rng = np.random.default_rng(11)
    He, Ho, w = 14, 12, 4
    Z4 = OS.rgbs(rng.random((He, He, 3)), OS.scale_map(He, He, 45.0, 30.0))
    X4 = OS.rgbs(rng.random((Ho, Ho, 3)), OS.resample(OS.scale_map(He, He, 45.0, 30.0), Ho, Ho))
    nn, d2 = O.nn_bruteforce(X4, Z4, w, 2)
    Vq, Vz = _windows(X4, w, 2), _windows(Z4, w, 1)
    D2 = ((Vq[:, None, :] - Vz[None, :, :]) ** 2).sum(-1)
    assert np.array_equal(nn, D2.argmin(1))
    assert np.abs(d2 - D2.min(1)).max() < 1e-12
    q = np.arange(len(nn))
    n = (q * 7) % len(Vz)
    assert np.abs(O.pair_dist2(X4, Z4, w, 2, q, n) - D2[q, n]).max() < 1e-12


def test_zero_scale_weight_leaves_the_rgb_search_unchanged():
    rng = np.random.default_rng(12)
    Z, X = rng.random((16, 16, 3)), rng.random((14, 14, 3))
    S = OS.scale_map(16, 16, 60.0, 20.0)
    nn3, d3 = O.nn_bruteforce(X, Z, 4, 2)
    nn4, d4 = O.nn_bruteforce(OS.rgbs(X, np.ones((14, 14)), 0.0), OS.rgbs(Z, S, 0.0), 4, 2)
    assert np.array_equal(nn3, nn4) and np.array_equal(d3, d4)


def test_rgbs_self_match_and_m_step_fixed_point():
    rng = np.random.default_rng(13)
    H, w = 14, 4
    Z4 = OS.rgbs(rng.random((H, H, 3)), OS.scale_map(H, H, 30.0, 18.0))
    nn, d2 = O.nn_bruteforce(Z4, Z4, w, 2)
    qy, qx = O.grid(H, H, w, 2)
    own = np.array([(2 * (q // qx)) * (H - w + 1) + 2 * (q % qx) for q in range(qy * qx)])
    assert np.array_equal(nn, own) and np.all(d2 == 0.0)
    X = O.m_step(own, np.linspace(0.5, 2.0, len(own)), Z4, w, H, H, 2)
    assert np.abs(X - Z4).max() < 1e-15


def test_rgbs_pca_against_numpy():
    rng = np.random.default_rng(14)
    Z4 = OS.rgbs(rng.random((13, 15, 3)), OS.scale_map(13, 15, 50.0, 70.0), 0.5)
    w = 3
    V = _windows(Z4, w, 1)
    mu, B, ev, _ = O.pca_fit(Z4, w, 10)
    assert np.abs(mu - V.mean(0)).max() < 1e-14
    cov = np.cov(V.T, bias=True)
    assert ev.sum() == pytest.approx(np.trace(cov), rel=1e-12)
    assert np.abs(B @ B.T - np.eye(10)).max() < 1e-12
    assert np.abs(ev[:10] - np.sort(np.linalg.eigvalsh(cov))[::-1][:10]).max() < 1e-12


def test_resize_filters_act_per_channel():
    rng = np.random.default_rng(15)
    img = rng.random((11, 9, 3))
    S = OS.scale_map(11, 9, 30.0, 18.0)
    for f in (O.downsample2, O.upsample2):
        a = f(OS.rgbs(img, S))
        assert np.array_equal(a[..., :3], f(img))
        assert np.array_equal(a[..., 3], f(np.repeat(S[..., None], 3, axis=2))[..., 0])


# ---------------------------------------------------------------------------
# EM on RGBS images (section 3, step 4)
# ---------------------------------------------------------------------------
def _rgbs_case(lam):
    He, Ho, w = 24, 28, 4
    sigma = math.degrees(math.acos(0.5))
    Z = P.synthetic_exemplar(6, He, 4.0).astype(np.float64)
    S_z = OS.scale_map(He, He, sigma, 0.0)
    S_x = OS.resample(S_z, Ho, Ho)
    X0 = P.random_patch_init(Z.astype(np.float32), Ho, Ho, w, seed=2).astype(np.float64)
    return OS.rgbs(Z, S_z, lam), OS.rgbs(X0, S_x, lam), S_z, S_x, w


def test_rgbs_em_keeps_the_guide_and_lowers_the_energy():
    Z4, X4, _, _, w = _rgbs_case(1.0)
    out = OS.synthesize_level_rgbs(Z4, X4, w, iters=4)
    assert np.array_equal(out["X"][..., 3], X4[..., 3].astype(np.float32).astype(np.float64))
    E = out["E"]
    assert np.all(np.diff(E) <= 1e-6 * E[0])


def test_scale_channel_pulls_matches_to_the_right_scale():
    """With the scale channel the matched exemplar windows sit at the output window's scale;
    without it (weight 0) they need not.  Measured on the windows' top-left pixels."""
    errs = {}
    for lam in (0.0, 4.0):
        Z4, X4, S_z, S_x, w = _rgbs_case(lam)
        out = OS.synthesize_level_rgbs(Z4, X4, w, iters=3)
        nn, _ = O.nn_bruteforce(out["X"], Z4, w, 2)
        qy, qx = O.grid(*S_x.shape, w, 2)
        ex = S_z.shape[1] - w + 1
        q = np.arange(qy * qx)
        errs[lam] = np.abs(S_z[nn // ex, nn % ex] - S_x[2 * (q // qx), 2 * (q % qx)]).mean()
    assert errs[4.0] < 0.5 * errs[0.0]


def test_rgbs_pca_dimension_is_in_the_papers_range():
    """Section 2.2: 95% of the variance of 8 x 8 RGBS neighbourhoods (256 dimensions) is kept by
    about 20-45 PCA components.  Checked qualitatively, as the paper's photographs are not
    available: on the synthetic 128² exemplar (three seeds, the scale map of its own slant at
    tilt 0) the oracle needs 30-31 components, and the colour channels alone (192 dimensions)
    need far more, since the smooth scale channel carries much of the variance."""
    lo, hi = PAPER["pca_dims_rgbs_8x8"]["value"]
    frac = PAPER["pca_variance_kept"]["value"]
    sigma = math.degrees(math.acos(0.5))
    for seed in (0, 1, 2):
        Z = P.synthetic_exemplar(seed, 128, 4.0).astype(np.float64)
        d95 = {}
        for name, img in (("rgbs", OS.rgbs(Z, OS.scale_map(128, 128, sigma, 0.0))), ("rgb", Z)):
            _, _, ev, _ = O.pca_fit(img, 8, 1)
            d95[name] = int(np.searchsorted(np.cumsum(ev) / ev.sum(), frac) + 1)
        assert lo <= d95["rgbs"] <= hi, (seed, d95)
        assert d95["rgb"] > 2 * d95["rgbs"], (seed, d95)


def test_rgbs_pyramid_keeps_each_levels_map_and_lowers_the_energy():
    """Coarse to fine on RGBS images: each level's scale channel is that level's resampled map
    (checked through the final level), the energy never rises within a level (r = 2), and the
    perspective survives: rows of the output match exemplar windows of the same scale."""
    sigma = math.degrees(math.acos(0.5))
    Z = P.synthetic_exemplar(8, 48, 4.0).astype(np.float64)
    u = P.uniform_field(5, 24, 24)
    X, energies = OS.synthesize_pyramid_rgbs(Z, sigma, 0.0, 48, 48, [8, 4], 3, u)
    assert X.shape == (48, 48, 3) and len(energies) == 2
    for E in energies:
        assert np.all(np.diff(E) <= 1e-6 * E[0])
    S_z = OS.scale_map(48, 48, sigma, 0.0)
    S_x = OS.resample(S_z, 48, 48)
    X4 = OS.rgbs(X, S_x)
    nn, _ = O.nn_bruteforce(X4, OS.rgbs(Z, S_z), 4, 2)
    qy, qx = O.grid(48, 48, 4, 2)
    rows = nn // (48 - 4 + 1)
    want = 2 * (np.arange(qy * qx) // qx)
    assert np.abs(rows - want).mean() < 4.0       # within a texel's height of the same scale
    with pytest.raises(ValueError, match="double"):     # 24 up-sampled is 48, not 49
        OS.synthesize_pyramid_rgbs(Z, sigma, 0.0, 49, 49, [8, 4], 1, u)
