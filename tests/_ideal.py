"""The tensor-core search's candidate rule evaluated in FP64 (test support).

The FP16 search keeps, per query and per column half of every 256-window tile (windows whose
index mod 256 is below or above 128), the 8 groups of 8 consecutive windows with the smallest
minimum score (ties to the smaller group), and re-ranks the 32 smallest scores among those
groups' windows in full dimension.  Evaluated with the oracle's FP64 PCA bound
LB(q, n) = ||y_q - y_n||^2 + (r_q - r_n)^2 in place of the FP16 scores, the misses that remain
are those of the rule itself, not of its arithmetic; the GPU's mismatch rate is tested against
this rate plus an allowance for FP16 rounding.  With fp16_operands the scores are instead formed
from the operands rounded to FP16 as the search stores them (query (y, r), exemplar -2 (y, r)),
their products summed in FP64, plus the exemplar norm: the rule with FP16 operand rounding alone.
"""
import numpy as np

import oracle

TILE, HALF, GROUP, KEEP, TOPK = 256, 128, 8, 8, 32


def group_rule_mismatch(X, Z, w, d, qs, nn_o, stride=2, chunk=128, fp16_operands=False):
    """Boolean per sampled query q in qs: the rule's window differs from the oracle's nn_o."""
    mu, B, _, _ = oracle.pca_fit(Z, w, d)
    ye, _, re = oracle.project(Z, w, 1, mu, B)
    yq, _, rq = oracle.project(X, w, stride, mu, B)
    qs = np.asarray(qs)
    yq, rq = yq[qs], rq[qs]
    N = len(ye)
    T = -(-N // TILE)
    ng = HALF // GROUP                                   # groups per tile half
    ne = (ye ** 2).sum(1)
    gid = np.arange(T)[:, None, None] * (TILE // GROUP) + np.arange(2)[None, :, None] * ng \
        + np.arange(ng)[None, None, :]                   # [tile, half, group] -> global group id
    miss = np.zeros(len(qs), dtype=bool)
    if fp16_operands:
        f16 = lambda v: v.astype(np.float16).astype(np.float64)  # noqa: E731
        E16 = f16(-2.0 * np.concatenate([ye, re[:, None]], 1))
        Q16 = f16(np.concatenate([yq, rq[:, None]], 1))
        nrm = ne + re ** 2
    for a in range(0, len(qs), chunk):
        b = min(len(qs), a + chunk)
        if fp16_operands:
            lb = nrm[None, :] + Q16[a:b] @ E16.T
        else:
            lb = (yq[a:b] ** 2).sum(1)[:, None] + ne[None, :] - 2.0 * (yq[a:b] @ ye.T) \
                + (rq[a:b, None] - re[None, :]) ** 2
        lbp = np.full((b - a, T * TILE), np.inf)
        lbp[:, :N] = lb
        gmin = lbp.reshape(b - a, T, 2, ng, GROUP).min(-1)
        for i in range(b - a):
            cand = []
            for h in range(2):
                gm = gmin[i, :, h, :].reshape(-1)
                gi = gid[:, h, :].reshape(-1)
                for g in gi[np.lexsort((gi, gm))[:KEEP]]:
                    cand.extend(range(g * GROUP, min(N, g * GROUP + GROUP)))
            cand = np.asarray(cand)
            top = cand[np.lexsort((cand, lbp[i, cand]))[:TOPK]]
            dd = oracle.pair_dist2(X, Z, w, stride, np.full(len(top), qs[a + i]), top)
            miss[a + i] = top[np.lexsort((top, dd))[0]] != nn_o[a + i]
    return miss
