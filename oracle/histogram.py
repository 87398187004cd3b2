"""Histogram matching (section 3, Eq. 9, and the last step of the synthesis procedure, section 4)
for the FP64 oracle.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: plain numpy, FP64 except where a float
decides an integer.  The bin of a channel value is taken in float32 (clamped to [0, 1], times the
bin count, floored, capped at the last bin), as the CUDA kernels take it, so both sides bin every
value alike.

Readings (the passage is ambiguous):
  - one histogram per colour channel j, so the sum of Eq. 9 runs over the three channels (the text
    calls k the number of bins while j indexes histograms); each histogram has ``nbins`` equal
    bins over [0, 1] and holds fractions of the image's pixels;
  - H_x is taken from the image the E-step matched (the image entering the M-step), H_z from the
    exemplar;
  - the weight of Eq. 9 applies to every exemplar pixel a matched window contributes to the pixel
    average of Eq. 8, and that pixel's colour picks the bins.  The weight is therefore per
    (window, pixel), and each pixel is normalised by its own sum of weights.
  - Final histogram matching maps each channel through F_z^-1(F_x(v)), both CDFs piecewise linear
    inside the bins (values spread evenly within a bin).
"""
from __future__ import annotations

import numpy as np


def channel_bins(v, nbins: int) -> np.ndarray:
    """Bin index of each channel value, decided in float32."""
    v32 = np.clip(np.asarray(v, dtype=np.float32), np.float32(0.0), np.float32(1.0))
    b = np.floor(v32 * np.float32(nbins)).astype(np.int64)
    return np.minimum(b, nbins - 1)


def histogram_counts(img, nbins: int) -> np.ndarray:
    """[3, nbins] pixel counts per channel and bin."""
    px = np.asarray(img).reshape(-1, 3)
    return np.stack([np.bincount(channel_bins(px[:, j], nbins), minlength=nbins) for j in range(3)])


def histograms(img, nbins: int) -> np.ndarray:
    """[3, nbins] fractions of the image's pixels per channel and bin."""
    n = np.asarray(img).reshape(-1, 3).shape[0]
    return histogram_counts(img, nbins) / float(n)


def weight_divisor(colors, Hx, Hz) -> np.ndarray:
    """1 + sum_j max[0, Hx_j(b_j(c)) - Hz_j(b_j(c))] for each colour c (last axis of `colors`)."""
    nbins = Hx.shape[1]
    c = np.asarray(colors, dtype=np.float64).reshape(-1, 3)
    s = np.ones(c.shape[0])
    for j in range(3):
        b = channel_bins(c[:, j], nbins)
        s += np.maximum(0.0, Hx[j, b] - Hz[j, b])
    return s.reshape(np.asarray(colors).shape[:-1])


def m_step_hist(nn, Wt, Z, X_cur, w: int, stride: int, nbins: int) -> np.ndarray:
    """The M-step (Eq. 8 minimised over x) with the weights of Eq. 9:
    x_i = sum_{p covers i} W_pi z_{n(p)}[i - p] / sum_{p covers i} W_pi,
    W_pi = w_p / (1 + sum_j max[0, H_x,j(b_j(c)) - H_z,j(b_j(c))]), c = z_{n(p)}[i - p].
    Pixels no window covers keep their value in X_cur."""
    Z = np.asarray(Z, dtype=np.float64)
    Xc = np.asarray(X_cur, dtype=np.float64)
    Ho, Wo, _ = Xc.shape
    He, We, _ = Z.shape
    qy_n, qx_n = (Ho - w) // stride + 1, (Wo - w) // stride + 1
    ex = We - w + 1
    Hx, Hz = histograms(Xc, nbins), histograms(Z, nbins)
    nn = np.asarray(nn, dtype=np.int64).reshape(qy_n, qx_n)
    W = np.ones((qy_n, qx_n)) if Wt is None else np.asarray(Wt, dtype=np.float64).reshape(qy_n, qx_n)
    ey, exx = nn // ex, nn % ex
    qy = (np.arange(qy_n) * stride)[:, None]
    qx = (np.arange(qx_n) * stride)[None, :]
    num = np.zeros((Ho, Wo, 3))
    den = np.zeros((Ho, Wo))
    for dy in range(w):
        for dx in range(w):
            col = Z[ey + dy, exx + dx]  # [qy_n, qx_n, 3]: what window p contributes at offset (dy, dx)
            wp = W / weight_divisor(col, Hx, Hz)
            np.add.at(num, (qy + dy, qx + dx), wp[..., None] * col)
            np.add.at(den, (qy + dy, qx + dx), wp)
    X = Xc.copy()
    cov = den > 0
    X[cov] = num[cov] / den[cov][:, None]
    return X


def histogram_match(img, Z, nbins: int) -> np.ndarray:
    """Each channel v -> F_z^-1(F_x(v)).  F(v) = C[b] + (v nbins - b) h[b] for v in bin b, with h the
    fractions and C[m] = h[0] + ... + h[m-1] (integer counts summed, then divided);
    F_z^-1(u) = (m + (u - C_z[m]) / h_z[m]) / nbins for the bin m with C_z[m] <= u < C_z[m+1]
    (never an empty one), and 1 once u reaches C_z[nbins]."""
    img = np.asarray(img, dtype=np.float64)
    nx = img.reshape(-1, 3).shape[0]
    nz = np.asarray(Z).reshape(-1, 3).shape[0]
    cx_cnt, cz_cnt = histogram_counts(img, nbins), histogram_counts(Z, nbins)
    out = img.copy()
    for j in range(3):
        hx, hz = cx_cnt[j] / nx, cz_cnt[j] / nz
        Cx = np.concatenate([[0], np.cumsum(cx_cnt[j])]) / nx
        Cz = np.concatenate([[0], np.cumsum(cz_cnt[j])]) / nz
        v = np.clip(img[..., j], 0.0, 1.0)
        b = channel_bins(img[..., j], nbins)
        u = Cx[b] + (v * nbins - b) * hx[b]
        m = np.searchsorted(Cz[1:], u, side="right")  # edges C_z[1..] at or below u
        inside = m < nbins
        mm = np.minimum(m, nbins - 1)
        res = np.ones_like(u)
        res[inside] = (mm[inside] + (u[inside] - Cz[mm[inside]]) / hz[mm[inside]]) / nbins
        out[..., j] = res
    return out
