"""The paper's scale map (Methodology section 1, Eqs. 1-3) and its use in synthesis (section 3):
the scale map as a fourth channel beside R, G and B, the resampling of the map to the output
size, and the initial output filled from exemplar pixels of the same scale.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: plain numpy in FP64, written from the
definitions.  Readings where the paper is silent or garbled:

* Image-plane coordinates (section 1): the origin is the bottom-left pixel, so array row r (row
  0 at the top, as everywhere in this library) has p(y) = h - 1 - r, and column c has p(x) = c.
  w / 2 and h / 2 are real divisions.
* Eq. 3's leading term is printed as Y_max; it is read as S_max.  Only that makes S a scale:
  S(p) = S_max where p(Y_proj) = Y_min and S_min where p(Y_proj) = Y_max, and S = 1 everywhere
  for a fronto-parallel plane (sigma = 0).  With real halves Y_min is reached at pixel (1, 1)
  and Y_max at the top-right pixel (w - 1, h - 1); the bottom row and the left column lie just
  beyond the range and carry scales slightly above S_max.
* Angles: sigma in [0, 90) degrees, tau in [0, 90] degrees.  Section 1 mirrors or flips the
  exemplar until its largest texel sits at the origin, which is what makes sin(tau) and
  cos(tau) non-negative in Eq. 2; the map is undefined when Y_delta = 0 (a 2 x 2 image, or
  one that is 2 pixels long along the projected axis).
* Resampling to the output size (section 3, step 2): bilinear, corner-aligned, so that the
  output map spans the exemplar's range of scales: output pixel (xo, yo) reads the exemplar
  map at ((We - 1) xo / (Wo - 1), (He - 1) yo / (Ho - 1)).
* Scale-guided initialisation (section 3, step 3): "the same scale" is taken as the same bin
  of `nbins` equal-width bins spanning the exemplar map's range [lo, hi], with
  bin(s) = min(floor((s - lo) / (hi - lo) * nbins), nbins - 1), clamped to [0, nbins - 1];
  for hi = lo every pixel is in bin 0.  Output pixel o takes the colour of the exemplar pixel
  floor(u_o * m) of its bin's m pixels in raster order, u_o in [0, 1) a given uniform; an
  empty bin borrows the nearest non-empty bin (the lower one on a tie).
* RGBS vectors (sections 2.2 and 3): the fourth channel is lam * S, lam = 1 unless stated.  In
  the output the fourth channel is the resampled map and stays fixed: the M-step updates R, G
  and B, so the search matches appearance and scale while the map keeps guiding it.
"""
from __future__ import annotations

import math

import numpy as np

from . import irls, m_step, nn_bruteforce


def scale_range(sigma_deg: float) -> tuple[float, float, float]:
    """Eq. 1: (S_max, S_min, S_delta) = (1 / cos sigma, cos sigma, S_max - S_min)."""
    if not 0.0 <= sigma_deg < 90.0:
        raise ValueError("slant must lie in [0, 90) degrees")
    c = math.cos(math.radians(sigma_deg))
    s_max, s_min = 1.0 / c, c
    return s_max, s_min, s_max - s_min


def y_range(h: int, w: int, tau_deg: float) -> tuple[float, float, float]:
    """Eq. 2: (Y_max, Y_min, Y_delta) of the projected image-plane Y coordinate."""
    if not 0.0 <= tau_deg <= 90.0:
        raise ValueError("tilt must lie in [0, 90] degrees")
    t = math.radians(tau_deg)
    y_max = (w - 1 - w / 2.0) * math.sin(t) + (h - 1 - h / 2.0) * math.cos(t)
    y_min = -y_max
    return y_max, y_min, y_max - y_min


def projected_y(h: int, w: int, tau_deg: float) -> np.ndarray:
    """Eq. 3, first line: p(Y_proj) of every pixel, as an h x w array (row 0 at the top)."""
    t = math.radians(tau_deg)
    px = np.arange(w, dtype=np.float64)[None, :]
    py = (h - 1 - np.arange(h, dtype=np.float64))[:, None]   # bottom-left origin
    return (px - w / 2.0) * math.sin(t) + (py - h / 2.0) * math.cos(t)


def scale_map(h: int, w: int, sigma_deg: float, tau_deg: float) -> np.ndarray:
    """Eq. 3: the local scale S(p) of every pixel of an h x w image (row 0 at the top)."""
    s_max, _, s_delta = scale_range(sigma_deg)
    _, y_min, y_delta = y_range(h, w, tau_deg)
    if not y_delta > 0.0:
        raise ValueError("Y_delta = 0: the image has no extent along the projected axis")
    return s_max - (projected_y(h, w, tau_deg) - y_min) * s_delta / y_delta


def resample(S, Ho: int, Wo: int) -> np.ndarray:
    """Section 3, step 2: the map S (He x We) resampled bilinearly to Ho x Wo, corner-aligned."""
    S = np.asarray(S, dtype=np.float64)
    He, We = S.shape
    if Ho < 2 or Wo < 2 or He < 2 or We < 2:
        raise ValueError("resampling needs at least 2 x 2 pixels on both sides")
    out = np.empty((Ho, Wo))
    for yo in range(Ho):
        sy = (He - 1) * yo / (Ho - 1)
        y0 = min(int(math.floor(sy)), He - 2)
        fy = sy - y0
        for xo in range(Wo):
            sx = (We - 1) * xo / (Wo - 1)
            x0 = min(int(math.floor(sx)), We - 2)
            fx = sx - x0
            out[yo, xo] = ((1 - fy) * ((1 - fx) * S[y0, x0] + fx * S[y0, x0 + 1])
                           + fy * ((1 - fx) * S[y0 + 1, x0] + fx * S[y0 + 1, x0 + 1]))
    return out


def scale_bins(S, lo: float, hi: float, nbins: int) -> np.ndarray:
    """Bin of every scale value: nbins equal-width bins over [lo, hi], clamped at both ends."""
    S = np.asarray(S, dtype=np.float64)
    if hi <= lo:
        return np.zeros(S.shape, dtype=np.int64)
    b = np.floor((S - lo) / (hi - lo) * nbins).astype(np.int64)
    return np.clip(b, 0, nbins - 1)


def scale_guided_init(Z, S_z, S_x, u, nbins: int = 64) -> tuple[np.ndarray, np.ndarray]:
    """Section 3, step 3: the initial output (Ho x Wo x C) and, per output pixel, the raster index
    of the exemplar pixel it copies.  S_z (He x We) is the exemplar's map, S_x (Ho x Wo) the
    output's, u (Ho x Wo) uniforms in [0, 1)."""
    Z = np.asarray(Z, dtype=np.float64)
    S_z = np.asarray(S_z, dtype=np.float64)
    S_x = np.asarray(S_x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    He, We = S_z.shape
    Ho, Wo = S_x.shape
    if Z.shape[:2] != (He, We) or u.shape != (Ho, Wo) or nbins < 1:
        raise ValueError("shape mismatch")
    lo, hi = float(S_z.min()), float(S_z.max())
    bz = scale_bins(S_z, lo, hi, nbins).ravel()
    members = [np.flatnonzero(bz == b) for b in range(nbins)]     # raster order within a bin
    # the bin each bin borrows from: itself if non-empty, else the nearest non-empty one
    filled = [b for b in range(nbins) if len(members[b])]
    source_bin = [min(filled, key=lambda f: (abs(f - b), f)) for b in range(nbins)]
    bx = scale_bins(S_x, lo, hi, nbins)
    src = np.empty((Ho, Wo), dtype=np.int64)
    for yo in range(Ho):
        for xo in range(Wo):
            m = members[source_bin[bx[yo, xo]]]
            k = min(int(math.floor(u[yo, xo] * len(m))), len(m) - 1)
            src[yo, xo] = m[k]
    X0 = Z.reshape(He * We, -1)[src.ravel()].reshape(Ho, Wo, Z.shape[2])
    return X0, src


def rgbs(img, S, lam: float = 1.0) -> np.ndarray:
    """Sections 2.2 and 3: the H x W x 4 image whose fourth channel is lam * S beside R, G, B."""
    img = np.asarray(img, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    if img.ndim != 3 or img.shape[2] != 3 or S.shape != img.shape[:2]:
        raise ValueError("expected an H x W x 3 image and an H x W scale map")
    return np.concatenate([img, lam * S[:, :, None]], axis=2)


def synthesize_level_rgbs(Z4, X4, w: int, iters: int, r: float = 2.0, delta: float = 1e-3, stride: int = 2,
                          nthreads: int = 0, f32_io: bool = True):
    """EM iterations (section 2.1: search phase, then optimization phase) on RGBS images: the
    search compares full 4-channel windows (D = 4 w^2); the M-step averages all four channels
    of the matched windows and the output's fourth channel is then put back to its fixed map.
    Same schedule and float32 rounding points as the 3-channel ``synthesize_level``; returns a
    dict with X (Ho x Wo x 4), E (iters + 1 energies of Eq. 4 over the 4-channel windows) and
    E_delta."""
    Z4 = np.asarray(Z4, dtype=np.float64)
    X = np.asarray(X4, dtype=np.float64).copy()
    if Z4.ndim != 3 or Z4.shape[2] != 4 or X.ndim != 3 or X.shape[2] != 4:
        raise ValueError("expected H x W x 4 exemplar and output")
    if f32_io:
        X = X.astype(np.float32).astype(np.float64)
    guide = X[:, :, 3].copy()
    Ho, Wo, _ = X.shape
    E, Ed = [], []
    for it in range(iters + 1):
        if f32_io:
            X = X.astype(np.float32).astype(np.float64)
        nn, d2 = nn_bruteforce(X, Z4, w, stride, nthreads=nthreads)
        W, er, ed = irls(d2, r, delta)
        if f32_io:
            W = W.astype(np.float32).astype(np.float64)
        E.append(er)
        Ed.append(ed)
        if it == iters:
            break
        X = m_step(nn, W, Z4, w, Ho, Wo, stride, X_prev=X)
        X[:, :, 3] = guide
    return {"X": X, "E": np.array(E), "E_delta": np.array(Ed)}


def synthesize_pyramid_rgbs(Z, sigma_deg: float, tau_deg: float, Ho: int, Wo: int, windows, iters: int, u,
                            lam: float = 1.0, nbins: int = 64, r: float = 2.0, delta: float = 1e-3,
                            stride: int = 2, nthreads: int = 0):
    """The whole method of section 3 on RGBS images, coarse to fine (section 2.1's pyramid): at
    every level the exemplar's scale map (Eqs. 1-3 at that level's size) and its resampling to the
    level's output size; the coarsest output initialised from exemplar pixels of the same scale
    (u: uniforms of the coarsest output's shape), each finer one from the coarser result's colours
    up-sampled by 2; then the EM iterations of synthesize_level_rgbs.  Z (He x We x 3) is the
    finest exemplar, (Ho, Wo) the finest output size, windows the window width per level (coarsest
    first).  Returns the final colour image (Ho x Wo x 3) and the per-level energy arrays."""
    from . import exemplar_pyramid, upsample2

    levels = len(windows)
    pyr = exemplar_pyramid(Z, levels)
    X, energies = None, []
    for lev, w in enumerate(windows):
        Zl = pyr[lev]
        He, We = Zl.shape[:2]
        h, wd = Ho >> (levels - 1 - lev), Wo >> (levels - 1 - lev)
        S_z = scale_map(He, We, sigma_deg, tau_deg)
        S_x = resample(S_z, h, wd)
        if X is None:
            X0, _ = scale_guided_init(Zl, S_z, S_x, u, nbins)
        else:
            X0 = upsample2(X[:, :, :3])
            if X0.shape[:2] != (h, wd):
                raise ValueError("level sizes must double from one level to the next")
        out = synthesize_level_rgbs(rgbs(Zl, S_z, lam), rgbs(X0, S_x, lam), w, iters, r, delta, stride, nthreads)
        X = out["X"]
        energies.append(out["E"])
    return X[:, :, :3], energies
