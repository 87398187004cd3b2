"""The robust schedule of section 2.1 (Eq. 5 with r = 0.8, IRLS weights max(d, delta)^(r - 2) of
Eq. 7, EM at each level until the searched windows repeat) on the plain-method workload at
scale, as a function of delta (the paper gives none; Eq. 7 is infinite at d = 0).

    python -m paper_2006_11851_gb300.delta_study [--seeds 4] [--deltas 1e-4,1e-3,...]

Per delta and seed: the M-steps each level took to stop (the cap counts as a stop), the final
image's energies measured by the certified exact search -- Eq. 4 (sum of d^2) and Eq. 5 at
r = 0.8 (sum of d^0.8, the energy the schedule minimises) -- and their ratios to those of the
image the fixed schedule (r = 2, 5 iterations per level, the benchmark's) reaches from the same
initialisation.  Search modes per level
as the benchmark's default (exact on the coarsest level, FP16 tensor cores on the others) unless
--modes names others.
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

from . import nn_search
from .pyramid import PyramidIndex, synthesize_pyramid

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import pts_inputs as P  # noqa: E402

WINDOWS, OUTPUTS, LEVEL_MODES = [32, 16, 8], [128, 256, 512], ["exact", "f16", "f16"]


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=4)
    ap.add_argument("--deltas", default="1e-4,1e-3,1e-2,3e-2,1e-1")
    ap.add_argument("--max-iters", type=int, default=30)
    ap.add_argument("--modes", default=",".join(LEVEL_MODES), help="search mode per level, coarse to fine")
    args = ap.parse_args()
    modes = args.modes.split(",")
    dev = torch.device("cuda", torch.cuda.current_device())
    Z = P.synthetic_exemplar(0, 256, 4.0)
    pidx = PyramidIndex(torch.from_numpy(Z).to(dev), WINDOWS, d=64)
    z0 = pidx.exemplars[0].cpu().numpy()

    def init(seed):
        return torch.from_numpy(P.random_patch_init(z0, OUTPUTS[0], OUTPUTS[0], WINDOWS[0], 500 + seed)).to(dev)

    def final_energy(X):
        _, d2 = nn_search(pidx.indices[-1], X, 2, "exact")
        d2 = d2.double().clamp_min(0.0)
        return float(d2.sum()), float(d2.pow(0.4).sum())

    base = []
    for s in range(args.seeds):
        X, _, _ = synthesize_pyramid(pidx, init(s), iters=5, r=2.0, mode=modes)
        base.append(final_energy(X))
    rows = []
    for delta in [float(x) for x in args.deltas.split(",")]:
        its, r2, r08, secs = [], [], [], 0.0
        for s in range(args.seeds):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            X, E, _ = synthesize_pyramid(pidx, init(s), iters=args.max_iters, delta=delta, mode=modes,
                                         schedule="robust")
            torch.cuda.synchronize()
            secs += time.perf_counter() - t0
            its.append([len(e) - 1 for e in E])
            e2, e08 = final_energy(X)
            r2.append(e2 / base[s][0])
            r08.append(e08 / base[s][1])
        rows.append({"delta": delta, "m_steps_per_level": np.mean(its, axis=0).tolist(),
                     "capped_levels": int(np.sum(np.array(its) >= args.max_iters)),
                     "eq4_energy_ratio_vs_fixed_r2": {"mean": float(np.mean(r2)), "max": float(np.max(r2))},
                     "eq5_r08_energy_ratio_vs_fixed_r2": {"mean": float(np.mean(r08)), "max": float(np.max(r08))},
                     "seconds_per_synthesis": secs / args.seeds})
    print(json.dumps({"workload": "exemplar 256x256 (shrink 4), windows 32/16/8, outputs 128/256/512, PCA 64, "
                                  f"modes {'/'.join(modes)}; robust schedule r = 0.8 with the stopping rule",
                      "seeds": args.seeds, "max_iters": args.max_iters,
                      "fixed_r2_final_energies_eq4_eq5": base,
                      "rows": rows}))
    pidx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
