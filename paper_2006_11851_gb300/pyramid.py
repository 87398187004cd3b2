"""Coarse-to-fine synthesis (section 2.1: a coarse result, up-sampled by
interpolation, initialises the next level).  Sequencing of C-ABI calls only:
the exemplar pyramid, the per-level EM and the up-sampling all run in libpts.
"""
from __future__ import annotations

import numpy as np
import torch

from ._binding import (ExemplarIndex, downsample2, histogram_match, rgb_of, rgbs, scale_guided_init, scale_map,
                       scale_resample, synthesize_level, synthesize_level_async, synthesize_level_converge,
                       upsample2)

# The paper's preferred schedule (section 2.1): the robust energy of Eq. 5 with r = 0.8, IRLS
# weights max(d, delta)^(r-2) (Eq. 7), iterated at every level until the searched windows repeat.
ROBUST_R = 0.8
ROBUST_MAX_ITERS = 30


class PyramidIndex:
    """One exemplar index per level, coarsest first.

    `windows[l]` is the window width used at level l; the exemplar of level l
    is the finest exemplar down-sampled (levels - 1 - l) times on the GPU.
    """

    def __init__(self, exemplar: torch.Tensor, windows: list[int], d: int = 64,
                 var_frac: float = 0.95, d_fast: int = 0):
        self.levels = len(windows)
        pyr = [exemplar.contiguous()]
        for _ in range(self.levels - 1):
            pyr.append(downsample2(pyr[-1]))
        self.exemplars = pyr[::-1]
        self.windows = list(windows)
        self.indices = [ExemplarIndex(z, w, d=min(d, 3 * w * w), var_frac=var_frac, d_fast=d_fast)
                        for z, w in zip(self.exemplars, windows)]

    def close(self):
        for ix in self.indices:
            ix.close()


def synthesize_pyramid(pidx: PyramidIndex, init_coarse: torch.Tensor, iters: int = 5,
                       r: float = 2.0, delta: float = 1e-3, mode="exact", stride: int = 2,
                       keep_levels: bool = False, hist_bins: int = 0, schedule: str = "fixed"):
    """Runs every level in place, coarse to fine.

    mode is one search mode for every level or a list with one per level.
    hist_bins > 0 runs the M-steps with the histogram weights of Eq. 9 and ends
    with the final histogram matching of the result to the finest exemplar
    (section 4).  Returns (final image, energies [levels, iters + 1], per-level
    images if keep_levels).  init_coarse is the initial image of level 0.

    schedule "fixed" runs `iters` EM iterations per level with the given r;
    "robust" is section 2.1's own schedule: r = 0.8 and, at every level, EM
    until the searched windows repeat (at most `iters` M-steps when iters > 0,
    else 30); its energies are then a list of per-level arrays of varying
    length (energy of the iterate entering each iteration, then the result's).
    """
    X = init_coarse.contiguous()
    imgs = []
    modes = list(mode) if isinstance(mode, (list, tuple)) else [mode] * pidx.levels
    if schedule == "robust":
        energies = []
        cap = iters if iters > 0 else ROBUST_MAX_ITERS
        for lev, ix in enumerate(pidx.indices):
            E, _ = synthesize_level_converge(ix, X, cap, r=ROBUST_R, delta=delta, mode=modes[lev], stride=stride,
                                             hist_bins=hist_bins)
            energies.append(E)
            if keep_levels:
                imgs.append(X.clone())
            if lev + 1 < pidx.levels:
                X = upsample2(X)
        if hist_bins:
            histogram_match(pidx.indices[-1], X, hist_bins)
        return X, energies, imgs
    if schedule != "fixed":
        raise ValueError("schedule must be 'fixed' or 'robust'")
    if hist_bins:
        energies = np.zeros((pidx.levels, iters + 1))
    else:  # the levels are queued back to back; one synchronisation at the end
        E = torch.empty(pidx.levels, iters + 1, device=X.device, dtype=torch.float64)
    for lev, ix in enumerate(pidx.indices):
        if hist_bins:
            energies[lev] = synthesize_level(ix, X, iters, r=r, delta=delta, mode=modes[lev], stride=stride,
                                             hist_bins=hist_bins)
        else:
            synthesize_level_async(ix, X, iters, r=r, delta=delta, mode=modes[lev], stride=stride, energy=E[lev])
        if keep_levels:
            imgs.append(X.clone())
        if lev + 1 < pidx.levels:
            X = upsample2(X)
    if hist_bins:
        histogram_match(pidx.indices[-1], X, hist_bins)
    else:
        energies = E.cpu().numpy()
        for ix in pidx.indices:
            ix.device_status()  # a kernel's error surfaces here
    return X, energies, imgs


def synthesize_pyramid_rgbs(exemplar: torch.Tensor, slant_deg: float, tilt_deg: float, Ho: int, Wo: int,
                            windows: list[int], iters: int, u: torch.Tensor, lam: float = 1.0, nbins: int = 64,
                            r: float = 2.0, delta: float = 1e-3, stride: int = 2, d: int = 64, mode="exact",
                            d_fast: int = 0):
    """The method of section 3 on RGBS images, coarse to fine (section 2.1's pyramid).

    Per level: the exemplar's scale map (Eqs. 1-3 at the level's size) and its resampling to the
    level's output size; the coarsest output filled from exemplar pixels of the same scale (u:
    float64 uniforms of the coarsest output's shape), each finer one from the coarser result's
    colours up-sampled by 2; then `iters` EM iterations on the 4-channel images (the fourth
    channel lam S, fixed in the output) with an RGBS index of the level.  exemplar is the finest
    H x W x 3 exemplar, (Ho, Wo) the finest output size, windows the window width per level
    (coarsest first).  Returns (colour image Ho x Wo x 3, per-level energies)."""
    levels = len(windows)
    pyr = [exemplar.contiguous()]
    for _ in range(levels - 1):
        pyr.append(downsample2(pyr[-1]))
    pyr = pyr[::-1]
    X, energies = None, []
    modes = list(mode) if isinstance(mode, (list, tuple)) else [mode] * levels
    for lev, w in enumerate(windows):
        Zl = pyr[lev]
        He, We = Zl.shape[0], Zl.shape[1]
        h, wd = Ho >> (levels - 1 - lev), Wo >> (levels - 1 - lev)
        S_z = scale_map(He, We, slant_deg, tilt_deg, device=Zl.device)
        S_x = scale_resample(S_z, h, wd)
        if X is None:
            X0, _ = scale_guided_init(Zl, S_z, S_x, u, nbins)
        else:
            X0 = upsample2(rgb_of(X))
            if tuple(X0.shape[:2]) != (h, wd):
                raise ValueError("level sizes must double from one level to the next")
        ix = ExemplarIndex(rgbs(Zl, S_z, lam), w, d=min(d, 4 * w * w), d_fast=d_fast)
        X = rgbs(X0, S_x, lam)
        energies.append(synthesize_level(ix, X, iters, r=r, delta=delta, mode=modes[lev], stride=stride))
        ix.close()
    return rgb_of(X), energies
