"""Coarse-to-fine synthesis (section 2.1: a coarse result, up-sampled by
interpolation, initialises the next level).  Sequencing of C-ABI calls only:
the exemplar pyramid, the per-level EM and the up-sampling all run in libpts.
"""
from __future__ import annotations

import numpy as np
import torch

from ._binding import (ExemplarIndex, downsample2, histogram_match, synthesize_level, synthesize_level_async,
                       upsample2)


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
                       keep_levels: bool = False, hist_bins: int = 0):
    """Runs every level in place, coarse to fine.

    mode is one search mode for every level or a list with one per level.
    hist_bins > 0 runs the M-steps with the histogram weights of Eq. 9 and ends
    with the final histogram matching of the result to the finest exemplar
    (section 4).  Returns (final image, energies [levels, iters + 1], per-level
    images if keep_levels).  init_coarse is the initial image of level 0.
    """
    X = init_coarse.contiguous()
    imgs = []
    modes = list(mode) if isinstance(mode, (list, tuple)) else [mode] * pidx.levels
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
