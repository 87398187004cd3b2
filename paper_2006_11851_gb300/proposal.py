"""Training pairs for the learned cluster proposal, and its training (sequencing of C-ABI calls).

Pairs are (query PCA coordinates, exact nearest window) from the search phases of exact-mode
synthesis runs: for every training seed the coarse-to-fine synthesis runs in exact mode, and at
the level that gets the proposal each E-step's queries are recorded before the optimization
phase updates the image.
"""
from __future__ import annotations

import numpy as np
import torch

import pts_inputs as P

from ._binding import irls_weights, m_step, nn_search, project_queries, synthesize_level, train_proposal, upsample2
from .pyramid import PyramidIndex


def collect_pairs(pidx: PyramidIndex, level: int, init_fn, seeds, iters: int = 5, r: float = 2.0,
                  stride: int = 2, keep_every: int = 1, coarse_mode="exact"):
    """(y [n, d], nn [n], d2 [n]) gathered at `level` over the synthesis runs of `seeds`.

    init_fn(seed) returns the level-0 initial image (torch, on the device).  Levels below
    `level` run synthesize_level in `coarse_mode`; at `level` every E-step (iters + 1 of them)
    is recorded, keeping every `keep_every`-th query.
    """
    ys, nns, d2s = [], [], []
    for s in seeds:
        X = init_fn(s)
        for lev in range(level):
            synthesize_level(pidx.indices[lev], X, iters, r=r, mode=coarse_mode, stride=stride)
            X = upsample2(X)
        ix = pidx.indices[level]
        Ho, Wo, _ = X.shape
        for t in range(iters + 1):
            y = project_queries(ix, X, stride)
            nn, d2 = nn_search(ix, X, stride, "exact")
            ys.append(y[::keep_every].clone())
            nns.append(nn[::keep_every].clone())
            d2s.append(d2[::keep_every].clone())
            if t == iters:
                break
            W, _ = irls_weights(d2, r)
            X = m_step(ix, nn, W, Ho, Wo, stride, out=X)
    return torch.cat(ys).contiguous(), torch.cat(nns).contiguous(), torch.cat(d2s).contiguous()


def subsample(y, nn, d2, n_max: int, seed: int = 0):
    """Seeded subsample of at most n_max pairs (sorted indices)."""
    n = y.shape[0]
    if n <= n_max:
        return y, nn, d2
    keep = torch.from_numpy(P.sample_indices(seed, n, n_max).astype(np.int64)).to(y.device)
    return y[keep].contiguous(), nn[keep].contiguous(), d2[keep].contiguous()


def random_patch_init_fn(pidx: PyramidIndex):
    """init_fn for collect_pairs: random exemplar patches of the coarsest level (host input)."""
    z0 = pidx.exemplars[0].cpu().numpy()
    w = pidx.windows[0]

    def fn(seed, Ho=None):
        H = Ho or 2 * z0.shape[0]
        return torch.from_numpy(P.random_patch_init(z0, H, H, w, seed)).to(pidx.exemplars[0].device)

    return fn


def train_level_proposal(pidx: PyramidIndex, level: int, seeds, iters: int = 5, n_pairs: int = 2_000_000,
                         init_fn=None, **params):
    """Collect pairs over `seeds`, subsample to n_pairs and train the proposal of `level`."""
    init_fn = init_fn or random_patch_init_fn(pidx)
    y, nn, d2 = collect_pairs(pidx, level, init_fn, seeds, iters)
    y, nn, d2 = subsample(y, nn, d2, n_pairs, seed=12345)
    loss = train_proposal(pidx.indices[level], y, nn, d2, **params)
    return loss, y.shape[0]


def train_job_proposal(ix, exemplar: torch.Tensor, Ho: int, w: int, seeds, iters: int = 5, n_pairs: int = 500_000,
                       r: float = 2.0, stride: int = 2, **params):
    """Train the proposal of a single-level index on (query, exact nearest window) pairs from its
    own exact-mode EM runs: one run per seed from random exemplar patches (Ho x Ho output).
    Returns the per-epoch loss."""
    ys, nns, d2s = [], [], []
    z = exemplar.cpu().numpy()
    for s in seeds:
        X = torch.from_numpy(P.random_patch_init(z, Ho, Ho, w, s)).to(exemplar.device)
        for t in range(iters + 1):
            ys.append(project_queries(ix, X, stride).clone())
            nn, d2 = nn_search(ix, X, stride, "exact")
            nns.append(nn.clone())
            d2s.append(d2.clone())
            if t == iters:
                break
            W, _ = irls_weights(d2, r)
            X = m_step(ix, nn, W, Ho, Ho, stride, out=X)
    y, nn, d2 = subsample(torch.cat(ys).contiguous(), torch.cat(nns).contiguous(), torch.cat(d2s).contiguous(),
                          n_pairs, seed=54321)
    params.setdefault("n_clusters", min(1024, max(4, ix.N // 64)))
    return train_proposal(ix, y, nn, d2, **params)
