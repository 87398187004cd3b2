"""Runs E-steps of one level of the benchmark workload, for profiling a kernel in isolation,
or (--pyramid) whole coarse-to-fine syntheses with a search mode per level.

    python -m paper_2006_11851_gb300.profile_case --level 2 --mode exact --steps 2
    python -m paper_2006_11851_gb300.profile_case --pyramid --modes exact,f16,f16 --steps 2
    python -m paper_2006_11851_gb300.profile_case --big 4096 --steps 3 [--hist 32]
    python -m paper_2006_11851_gb300.profile_case --rgbs --modes exact,f16,f16 --steps 2
    python -m paper_2006_11851_gb300.profile_case --level 2 --mode proposal --steps 3
    python -m paper_2006_11851_gb300.profile_case --level 0 --mode exact_tc --steps 3

--big H projects (d = 64) and averages (M-step) one H x H output against the finest level's
index (256x256 exemplar, w = 8), so that the working set is far above the L2 cache: a uniform
random image and uniform random matches with weights in [0.5, 1.5).

--rgbs runs the RGBS method of section 3 coarse to fine on the same workload (scale map of the
synthetic exemplar's geometry, slant 60 degrees, tilt 0; scale-guided initialisation).

--mode proposal first trains the level's proposal as the benchmark does, on a smaller budget
(4 training seeds, 500,000 pairs, 4 epochs, 1024 clusters), then times its searches.

Levels follow the 3-level workload (256x256 exemplar, shrink 4; windows 32/16/8; outputs
128/256/512, d = 64).  The output image is a seeded random-patch initialisation.  Prints the
per-E-step device time of each step.
"""
from __future__ import annotations

import argparse
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import paper_2006_11851_gb300 as pts  # noqa: E402
import pts_inputs as P  # noqa: E402

LEVELS = [(64, 32, 128), (128, 16, 256), (256, 8, 512)]  # (exemplar, window, output)


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--level", type=int, default=2)
    ap.add_argument("--mode", default="exact")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--d", type=int, default=64)
    ap.add_argument("--pyramid", action="store_true")
    ap.add_argument("--modes", default="exact,f16,f16")
    ap.add_argument("--big", type=int, default=0)
    ap.add_argument("--rgbs", action="store_true")
    ap.add_argument("--hist", type=int, default=0, help="with --big: also time the Eq. 9 M-step and the final "
                                                        "histogram matching with this many bins")
    args = ap.parse_args()
    if args.pyramid:
        return run_pyramid(args)
    if args.big:
        return run_big(args)
    if args.rgbs:
        return run_rgbs(args)
    He, w, Ho = LEVELS[args.level]
    dev = torch.device("cuda:0")
    Z = P.synthetic_exemplar(0, 256, 4.0)
    z = torch.from_numpy(Z).to(dev)
    for _ in range(2 - args.level):
        z = pts.downsample2(z)
    idx = pts.ExemplarIndex(z.contiguous(), w, d=args.d)
    if args.mode == "proposal":
        from paper_2006_11851_gb300.proposal import train_job_proposal
        train_job_proposal(idx, z.contiguous(), Ho, w, [1000 + t for t in range(4)], n_pairs=500_000, epochs=4,
                           n_clusters=1024)
    X = torch.from_numpy(P.random_patch_init(z.cpu().numpy(), Ho, Ho, w, 0)).to(dev)
    for s in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pts.nn_search(idx, X, 2, args.mode)
        e1.record()
        e1.synchronize()
        print(f"step {s}: {e0.elapsed_time(e1):.3f} ms  {idx.search_stats()}")
    idx.close()
    return 0


def run_pyramid(args) -> int:
    from paper_2006_11851_gb300.pyramid import PyramidIndex, synthesize_pyramid
    dev = torch.device("cuda:0")
    Z = P.synthetic_exemplar(0, 256, 4.0)
    pidx = PyramidIndex(torch.from_numpy(Z).to(dev), [w for _, w, _ in LEVELS], d=args.d)
    z0 = pidx.exemplars[0].cpu().numpy()
    modes = args.modes.split(",")
    for s in range(args.steps):
        x0 = torch.from_numpy(P.random_patch_init(z0, LEVELS[0][2], LEVELS[0][2], LEVELS[0][1], s)).to(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, E, _ = synthesize_pyramid(pidx, x0, iters=5, mode=modes)
        e1.record()
        e1.synchronize()
        print(f"synthesis {s}: {e0.elapsed_time(e1):.3f} ms  final energies {E[:, -1]}")
    pidx.close()
    return 0


def run_rgbs(args) -> int:
    dev = torch.device("cuda:0")
    Z = torch.from_numpy(P.synthetic_exemplar(0, 256, 4.0)).to(dev)
    modes = args.modes.split(",")
    for s in range(args.steps):
        u = torch.from_numpy(P.uniform_field(s, LEVELS[0][2], LEVELS[0][2])).to(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, E = pts.synthesize_pyramid_rgbs(Z, 60.0, 0.0, LEVELS[2][2], LEVELS[2][2], [w for _, w, _ in LEVELS], 5, u,
                                           d=args.d, mode=modes)
        e1.record()
        e1.synchronize()
        print(f"rgbs synthesis {s}: {e0.elapsed_time(e1):.3f} ms  final energies {[e[-1] for e in E]}")
    return 0


def run_big(args) -> int:
    dev = torch.device("cuda:0")
    z = torch.from_numpy(P.synthetic_exemplar(0, 256, 4.0)).to(dev)
    idx = pts.ExemplarIndex(z, 8, d=args.d)
    H = args.big
    g = torch.Generator().manual_seed(0)
    X = torch.rand(H, H, 3, generator=g).to(dev)
    Q = idx.num_queries(H, H, 2)
    nn = torch.randint(0, idx.info["N"], (Q,), generator=g, dtype=torch.int32).to(dev)
    wts = (torch.rand(Q, generator=g) + 0.5).to(dev)
    out = torch.empty(H, H, 3, device=dev)
    da = idx.info["da"]
    for s in range(args.steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        pts.project_queries(idx, X, 2)
        ev[1].record()
        pts.m_step(idx, nn, wts, H, H, 2, out)
        ev[2].record()
        ev[2].synchronize()
        tp, tm = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        # compulsory bytes: projection reads the image and writes Q x da coordinates + 2 floats;
        # the M-step reads Q matches and weights and writes the image
        bp = H * H * 12 + Q * (da + 2) * 4
        bm = Q * 8 + H * H * 12
        msg = (f"step {s}: project {tp:.3f} ms ({bp / tp / 1e6:.0f} GB/s, "
               f"{2.0 * idx.info['D'] * idx.info['d'] * Q / tp / 1e9:.1f} TFLOP/s)  "
               f"m_step {tm:.3f} ms ({bm / tm / 1e6:.0f} GB/s)  Q={Q}")
        if args.hist:
            out2 = torch.empty_like(out)
            eh = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            eh[0].record()
            pts.m_step_hist(idx, nn, wts, X, args.hist, out=out2)
            eh[1].record()
            pts.histogram_match(idx, out2, args.hist)
            eh[2].record()
            eh[2].synchronize()
            msg += (f"  m_step_hist {eh[0].elapsed_time(eh[1]):.3f} ms  "
                    f"histogram_match {eh[1].elapsed_time(eh[2]):.3f} ms")
        print(msg)
    idx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
