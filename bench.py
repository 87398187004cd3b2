#!/usr/bin/env python
"""Benchmark: E-step queries/s of the energy-optimisation texture synthesis.

Workload (the plain method at scale): seeded synthetic 256x256 exemplar
(perspective shrink 4x), 3-level Gaussian pyramid with windows 32/16/8 and
outputs 128/256/512, PCA to 64 dims, 2x2-patch query stride, 5 EM iterations
per level plus the final search phase.  One step = one full coarse-to-fine
synthesis from a fresh random-patch initialisation (one init seed per step);
the per-level exemplar indices are built once, before timing.

  value  E-step queries of the whole step / device time of the step, inputs
         resident in HBM, L2 flushed between steps (a 256 MB write).
  e2e    the same through the public Python API with the initial image in
         pinned host memory and the final image read back every step.

Search modes per level (--mode): exact (certified FP32, the baseline the ratio
is taken against), f16 (FP16 tensor-core PCA-space search + exact FP32 re-rank
on every level), f16c (the coarsest level exact, the finer two f16), f16x
(default: as f16c, the coarsest level's exact windows found through the
certified full-dimension FP16 GEMM, exact_tc), proposal (the learned cluster
proposal on the finest level, f16 on the middle one, exact_tc on the coarsest;
the network is trained before timing).  Every run
also times exact mode on the same seeds and reports the final exact energy of
both; --also names a further mode timed in the same run and reported under
other_modes (default proposal).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload's queries (E-step only).  Multi-GPU runs are independent replicas
(weak scaling): the method has no exchange between GPUs for this workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "E-step queries/s at final energy ≤1.01× exact vs exact FP32 search, same GB300"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0

WORKLOAD = {
    "workload": "plain method at scale: exemplar 256x256 (shrink 4x), 3-level pyramid, "
                "windows 32/16/8, outputs 128/256/512, PCA 64 (exact-mode bound; the tensor-core search "
                "ranks by d_fast = 124 components), stride 2, 5 EM iterations/level",
    "exemplar": 256, "shrink": 4.0, "levels": 3, "windows": [32, 16, 8], "outputs": [128, 256, 512],
    "d": 64, "iters": 5, "r": 2.0, "stride": 2,
}


def level_sizes(cfg=WORKLOAD):
    out = []
    for lev, (w, Ho) in enumerate(zip(cfg["windows"], cfg["outputs"])):
        He = cfg["exemplar"] >> (cfg["levels"] - 1 - lev)
        N = (He - w + 1) ** 2
        Q = ((Ho - w) // cfg["stride"] + 1) ** 2
        out.append({"He": He, "w": w, "Ho": Ho, "N": N, "Q": Q, "D": 3 * w * w})
    return out


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest x over the ranks of the process group (x itself without one)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Units processed by all ranks (each the same share: weak scaling) per second of the slowest."""
    return units_per_rank * world / (max_ms / 1000.0)


def queries_per_step(cfg=WORKLOAD):
    return sum(l["Q"] for l in level_sizes(cfg)) * (cfg["iters"] + 1)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self._t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded samples of the workload's E-step queries)
# ---------------------------------------------------------------------------
def oracle_inputs(cfg=WORKLOAD):
    import oracle
    import pts_inputs as P
    Z = P.synthetic_exemplar(0, cfg["exemplar"], cfg["shrink"])
    pyr = [p.astype(np.float32) for p in oracle.exemplar_pyramid(Z, cfg["levels"])]
    imgs = [P.random_patch_init(pyr[l], L["Ho"], L["Ho"], L["w"], 100 + l) for l, L in enumerate(level_sizes(cfg))]
    return pyr, imgs


def oracle_sample_rate(n_per_level, cfg=WORKLOAD, seed=0):
    """(queries/s of the oracle E-step over the workload's query mix, threads,
    queries timed, seconds)."""
    import oracle
    import pts_inputs as P
    pyr, imgs = oracle_inputs(cfg)
    threads = oracle.threads()
    t_per_q, timed, total = [], 0, 0.0
    for lev, L in enumerate(level_sizes(cfg)):
        k = n_per_level[lev]
        sub = P.sample_indices(seed * 10 + lev, L["Q"], k)
        t0 = time.perf_counter()
        oracle.nn_bruteforce(imgs[lev], pyr[lev], L["w"], cfg["stride"], qlist=sub)
        dt = time.perf_counter() - t0
        t_per_q.append(dt / len(sub))
        timed += len(sub)
        total += dt
    per_step_s = sum(L["Q"] * (cfg["iters"] + 1) * t for L, t in zip(level_sizes(cfg), t_per_q))
    return queries_per_step(cfg) / per_step_s, threads, timed, total


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    sizes = level_sizes()
    per = [max(8, int(round(1200 * L["Q"] / sizes[-1]["Q"]))) for L in sizes]  # ~ workload mix
    for i in range(args.warmup):
        oracle_sample_rate(per, seed=1000 + i)
    rates, secs, qs = [], 0.0, 0
    for i in range(args.steps):
        r, threads, n, dt = oracle_sample_rate(per, seed=i)
        rates.append(r)
        secs += dt
        qs += n
    value = float(np.mean(rates))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(WORKLOAD, l2="cpu run (no GPU)"),
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads, "kind": "oracle",
                         "sample": f"{per} queries per level per step (levels coarse to fine), "
                                   "full-dimension FP64 brute force, rate weighted by the workload's query mix"},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
LEVEL_MODES = {
    "exact": ["exact", "exact", "exact"],
    "f16": ["f16", "f16", "f16"],
    # the coarsest level (1,089 windows of 3,072 dimensions, where 64 PCA components keep only
    # 76% of the variance) searched exactly, the two finer levels on the FP16 tensor cores
    "f16c": ["exact", "f16", "f16"],
    # as f16c, the coarsest level's exact windows found through the full-dimension FP16 GEMM and
    # its certificate (the same windows as exact mode, FP32 pass for what it cannot certify)
    "f16x": ["exact_tc", "f16", "f16"],
    "fp8c": ["exact", "fp8", "fp8"],
    # the learned proposal on the finest level (the proposal trained there), the middle level on
    # the FP16 tensor-core brute force, the coarsest exact (as f16x)
    "proposal": ["exact_tc", "f16", "proposal"],
    # the paper's own search on the finest level (k = 4 k-means tree, greedy descent), for comparison
    "kmtree": ["exact", "f16", "kmtree"],
}
PCA_PASS_MIN_VAR = 0.85  # the exact search skips its PCA pass below this retained variance
PEAK_FP32_TFLOPS = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12


# DRAM bytes (read + write) of one fine-level k_search_tc launch (Q = 64,009, N = 62,001) from the
# ncu capture summarised in profiles/k_search_tc_fine_level_512_f16.md; reported only while the
# search source file is unchanged (the digest below is of that file with the profiled kernel; any
# later edit of the file, even of host code, turns the figure off until it is checked again).
TC_TRAFFIC_BYTES = 32.898e6 + 0.178e6
TC_TRAFFIC_SHA256 = "a4a8bd7ba3c5c2f33560f6021880a94a5ffe716cd532e785dec0ac42bfefc049"


def _tc_traffic():
    import hashlib
    with open(os.path.join(ROOT, "paper_2006_11851_gb300", "csrc", "search_tc.cu"), "rb") as f:
        return TC_TRAFFIC_BYTES if hashlib.sha256(f.read()).hexdigest() == TC_TRAFFIC_SHA256 else None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return m.get("bf16_tflops"), m.get("bf16_tflops_sustained"), "measured (MEASURED_PEAKS.json)"
    except (OSError, ValueError):
        return 1900.0, 1700.0, "fallback"


def exact_route_counts(pts, pidx, x0, cfg):
    """One exact-mode synthesis of the workload replayed search by search (the same calls
    synthesize_level makes: search, IRLS weights, M-step; a last search), returning per level,
    summed over the level's searches: the queries the full-dimension pass took, the queries the
    first PCA bound did not certify (the second bound's queries when it runs), those certified by
    the first bound and all queries."""
    X = x0.clone()
    rng, second, cert, allq = [], [], [], []
    for lev, ix in enumerate(pidx.indices):
        r = s2 = c = a = 0
        for t in range(cfg["iters"] + 1):
            nn, d2 = pts.nn_search(ix, X, cfg["stride"], "exact")
            st = ix.search_stats()
            r, c, a = r + st["full_queries"], c + st["certified"], a + st["queries"]
            s2 += st["second_queries"]
            if t < cfg["iters"]:
                wts, _ = pts.irls_weights(d2, cfg["r"], 1e-3)
                H, W, _ = X.shape
                X = pts.m_step(ix, nn, wts, H, W, cfg["stride"])
        rng.append(r)
        second.append(s2)
        cert.append(c)
        allq.append(a)
        if lev + 1 < pidx.levels:
            X = pts.upsample2(X)
    return {"range_queries": rng, "second_bound_queries": second, "certified": cert, "queries": allq}


PRECISION_FORM = {
    "workload": "precision form: exemplar 512x512 (shrink 4x), output 1024x1024, window 16x16 (D = 768), "
                "PCA 64 (exact-mode bound; the tensor-core searches rank by d_fast = 124 components), stride 2, "
                "one level, 5 EM iterations + final search",
    "exemplar": 512, "shrink": 4.0, "w": 16, "Ho": 1024, "d": 64, "iters": 5, "r": 2.0, "stride": 2,
}


def time_proposal_large(pts, P, dev, stream, flush, steps, warmup):
    """The learned proposal against the FP16 brute-force search it replaces, on a large exemplar:
    512x512 (shrink 4x), windows 8x8 (N = 255,025), one 512x512 output level, d = 64; the network
    (1,024 clusters) trained on four exact-mode EM runs (seeds disjoint from the timed one).  Each
    timed E-step searches one mid-synthesis image (two FP16 EM iterations from a random-patch
    initialisation) after an L2 flush; energies measured by the certified exact search."""
    import torch
    from paper_2006_11851_gb300.proposal import train_job_proposal
    Z = torch.from_numpy(P.synthetic_exemplar(0, 512, 4.0)).to(dev)
    idx = pts.ExemplarIndex(Z, 8, d=64)
    t0 = time.perf_counter()
    train_job_proposal(idx, Z, 512, 8, [1000 + s for s in range(4)], n_pairs=1_000_000, epochs=6, n_clusters=1024)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    X = torch.from_numpy(P.random_patch_init(Z.cpu().numpy(), 512, 512, 8, 7)).to(dev)
    pts.synthesize_level(idx, X, 2, mode="f16")
    Q = idx.num_queries(512, 512, 2)
    out = {"workload": "exemplar 512x512 (shrink 4x), windows 8x8 (N = 255,025), output 512x512 (Q = 64,009), "
                       "d = 64, 1,024 clusters trained on 4 exact-mode EM runs, one mid-synthesis image",
           "N": idx.N, "Q": Q, "proposal_train_s": train_s}
    _, d2e = pts.nn_search(idx, X, 2, "exact")
    e_exact = float(d2e.double().sum())
    for mode in ("f16", "proposal"):
        for _ in range(warmup):
            pts.nn_search(idx, X, 2, mode)
        ms = 0.0
        for _ in range(steps):
            flush.zero_()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            _, d2 = pts.nn_search(idx, X, 2, mode)
            ev1.record(stream)
            ev1.synchronize()
            ms += ev0.elapsed_time(ev1)
        out[mode] = {"value": Q * steps / (ms / 1000.0), "unit": "queries/s", "ms_per_estep": ms / steps,
                     "matched_energy_vs_exact": float(d2.double().sum()) / e_exact}
        if mode == "proposal":
            st = idx.search_stats()
            out[mode]["fallback_fraction"] = st["fallback_queries"] / max(1, st["queries"])
    out["proposal_vs_f16"] = out["proposal"]["value"] / out["f16"]["value"]
    idx.close()
    return out


def time_precision_form(pts, P, L, dev, stream, flush, steps, warmup, bf16_burst, peak_src):
    """queries/s of every search mode on the precision-form workload (one level), the FP16/FP8
    search's tensor roofline, and each mode's final energy (measured by the certified exact
    search) against exact mode's on the same seeds."""
    import ctypes

    import torch
    cfg = PRECISION_FORM
    Z = P.synthetic_exemplar(0, cfg["exemplar"], cfg["shrink"])
    t0 = time.perf_counter()
    idx = pts.ExemplarIndex(torch.from_numpy(Z).to(dev), cfg["w"], d=cfg["d"])
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    Ho, w, it = cfg["Ho"], cfg["w"], cfg["iters"] + 1
    Q, N, dfast = idx.num_queries(Ho, Ho, cfg["stride"]), idx.info["N"], idx.info["d_fast"]
    res = {"config": dict(cfg, N=N, Q=Q, d_fast=dfast, index_build_s=build_s,
                          l2="flushed between steps (256 MB write)"), "modes": {}}

    def init(seed):
        return torch.from_numpy(P.random_patch_init(Z, Ho, Ho, w, seed)).to(dev)

    def run(mode, x):
        pts.synthesize_level_async(idx, x, cfg["iters"], r=cfg["r"], mode=mode, stride=cfg["stride"])

    finals = {}
    for mode in ("f16", "fp8", "exact"):
        n, nw = (steps, warmup) if mode != "exact" else (1, 1)
        for i in range(nw):
            run(mode, init(i))
        xs = [init(warmup + i) for i in range(n)]
        torch.cuda.synchronize()
        ms = 0.0
        for x in xs:
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run(mode, x)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        idx.device_status()
        entry = {"value": Q * it * n / (ms / 1000.0), "unit": "queries/s", "ms_per_step": ms / n, "steps": n}
        if mode != "exact":
            x = init(warmup)
            L.pts_profile_enable(1)
            run(mode, x)
            torch.cuda.synchronize()
            tms, cnt = ctypes.c_double(), ctypes.c_longlong()
            L.pts_profile_read(b"search_tc", ctypes.byref(tms), ctypes.byref(cnt))
            L.pts_profile_enable(0)
            pk = bf16_burst * (2.0 if mode == "fp8" else 1.0)
            ach = 2.0 * (dfast + 1) * N * Q * it / (tms.value / 1000.0) / 1e12
            entry["roofline"] = {"kernel": "k_search_tc" + ("<FP8>" if mode == "fp8" else ""), "bound": "tensor",
                                 "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                                 "launches": int(cnt.value),
                                 "note": f"2(d_fast+1) flops per (query, window) pair, d_fast = {dfast}; peak = "
                                         f"{'2 x ' if mode == 'fp8' else ''}BF16 burst, {peak_src}"}
        fin = []
        for x in xs:
            _, d2 = pts.nn_search(idx, x, cfg["stride"], "exact")
            fin.append(float(d2.double().sum()))
        finals[mode] = fin
        res["modes"][mode] = entry
    for mode in ("f16", "fp8"):
        k = len(finals["exact"])
        ratios = [a / b for a, b in zip(finals[mode][:k], finals["exact"])]
        res["modes"][mode]["final_energy_ratio_vs_exact"] = max(ratios)
        res["modes"][mode]["speedup_vs_exact"] = res["modes"][mode]["value"] / res["modes"]["exact"]["value"]
    idx.close()
    return res


BATCHED_FORM = {
    "workload": "batched form: 64 independent single-level jobs in one CUDA graph, exemplars 128-512 px "
                "square (shrink 4, generator seeds 0-63), outputs 256-1024 px square, windows 8x8 (even jobs) "
                "and 16x16 (odd jobs), PCA 32/48/64, FP16 tensor-core search + FP32 re-rank, 5 EM iterations + "
                "final search per job, exemplar split per job shape picked by the autotuner",
    "jobs": 64, "iters": 5, "mode": "f16",
}


def time_batched(dev, stream, flush, steps, warmup):
    """queries/s and EM iterations/s of one graph replay of the 64-job batch."""
    import torch
    from paper_2006_11851_gb300.batched import Batch, job_specs
    cfg = BATCHED_FORM
    specs = job_specs(cfg["jobs"])
    t0 = time.perf_counter()
    b = Batch(specs, mode=cfg["mode"], iters=cfg["iters"], n_streams=8)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    for _ in range(warmup):
        b.reset()
        b.run()
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(steps):
        b.reset()
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run()
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    for ix in b.indices:
        ix.device_status()
    q = b.queries()
    out = {"config": dict(cfg, index_build_and_autotune_s=build_s, queries_per_run=q,
                          launches_per_run=b.launches_per_run, autotuned_parts=b.parts.tolist()),
           "value": q * steps / (ms / 1000.0), "unit": "queries/s", "ms_per_run": ms / steps, "runs": steps,
           "em_iterations_per_s": len(b.indices) * cfg["iters"] * steps / (ms / 1000.0)}
    b.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="f16x", choices=list(LEVEL_MODES))
    ap.add_argument("--also", default="proposal", choices=[""] + list(LEVEL_MODES),
                    help="a second mode timed in the same run, reported under other_modes")
    ap.add_argument("--train-seeds", type=int, default=16)
    ap.add_argument("--train-pairs", type=int, default=2_000_000)
    ap.add_argument("--clusters", type=int, default=1024)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=0, help="queries per level for the CPU baseline")
    ap.add_argument("--d-fast", type=int, default=0, help="PCA dimensions of the tensor-core search (0 = library default)")
    ap.add_argument("--no-robust", action="store_true", help="skip the robust-schedule timing (other_configs)")
    ap.add_argument("--no-proposal-large", action="store_true",
                    help="skip the learned proposal against the FP16 brute force on a 512x512 exemplar")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched form: 64 uneven jobs in one CUDA graph (other_configs)")
    ap.add_argument("--no-precision-form", action="store_true",
                    help="skip the 512x512 -> 1024x1024, w = 16 precision-form timing (other_configs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import ctypes

    import torch

    import paper_2006_11851_gb300 as pts
    from paper_2006_11851_gb300.proposal import train_level_proposal
    from paper_2006_11851_gb300.pyramid import PyramidIndex, synthesize_pyramid
    import pts_inputs as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = pts.lib()

    cfg = WORKLOAD
    sizes = level_sizes(cfg)
    modes = LEVEL_MODES[args.mode]
    Z = P.synthetic_exemplar(0, cfg["exemplar"], cfg["shrink"])
    t0 = time.perf_counter()
    pidx = PyramidIndex(torch.from_numpy(Z).to(dev), cfg["windows"], d=cfg["d"], d_fast=args.d_fast)
    torch.cuda.synchronize()
    index_build_s = time.perf_counter() - t0
    z0 = pidx.exemplars[0].cpu().numpy()
    Hc, wc = sizes[0]["Ho"], sizes[0]["w"]

    def init_dev(seed):
        return torch.from_numpy(P.random_patch_init(z0, Hc, Hc, wc, seed)).to(dev)

    train_s, n_pairs, train_loss = 0.0, 0, []
    also = args.also if args.also and args.also != args.mode else ""
    need = modes + (LEVEL_MODES[also] if also else [])
    if "proposal" in need:
        # training seeds 1000.. are disjoint from the timed seeds 0..(warmup + steps)
        t0 = time.perf_counter()
        loss, n_pairs = train_level_proposal(pidx, need.index("proposal") % cfg["levels"],
                                             [1000 + s for s in range(args.train_seeds)], iters=cfg["iters"],
                                             n_pairs=args.train_pairs, init_fn=init_dev, n_clusters=args.clusters,
                                             epochs=args.epochs, seed=7)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        train_loss = [float(x) for x in loss]

    if "kmtree" in need:
        pts.build_kmeans_tree(pidx.indices[need.index("kmtree") % cfg["levels"]], 10)
        torch.cuda.synchronize()

    n_total = args.warmup + args.steps
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(x0, mode_list):
        X, E, _ = synthesize_pyramid(pidx, x0, iters=cfg["iters"], r=cfg["r"], mode=mode_list)
        return X, E

    def exact_energy(X):
        _, d2 = pts.nn_search(pidx.indices[-1], X, cfg["stride"], "exact")
        return float(d2.double().sum())

    def timed_run(mode_list, profile):
        for i in range(args.warmup):
            step(init_dev(i), mode_list)
        work = [init_dev(args.warmup + i) for i in range(args.steps)]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        launches0 = L.pts_launch_count()
        if profile:
            L.pts_profile_enable(1)
        times, finals = [], []
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.zero_()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                X, _ = step(work[i], mode_list)
                ev1.record(stream)
                ev1.synchronize()
                times.append(ev0.elapsed_time(ev1))
                finals.append(X)
        torch.cuda.synchronize()
        launches = L.pts_launch_count() - launches0
        last_stats = pidx.indices[-1].search_stats()  # the finest level's last search phase
        kern = {}
        if profile:
            for name in ("search_topk", "search_full", "search_tc", "search_tc_list", "search_tcf", "rerank",
                         "project", "m_step", "brute", "irls", "mlp", "probe"):
                ms, n = ctypes.c_double(), ctypes.c_longlong()
                L.pts_profile_read(name.encode(), ctypes.byref(ms), ctypes.byref(n))
                if n.value:
                    kern[name] = {"ms_per_step": ms.value / args.steps, "launches_per_step": n.value / args.steps}
            L.pts_profile_enable(0)
        total_ms = max_over_ranks(sum(times), dist, dev)
        energies = [exact_energy(X) for X in finals]
        timed_run.last_stats = last_stats
        return total_ms, launches, kern, energies, clk.summary()

    # `value` from a pass with the library's per-kernel event recording off; the kernel shares and
    # the roofline's kernel time from a second, profiled pass over the same seeds
    total_ms, launches, _, energies, clocks = timed_run(modes, False)
    prof_ms, _, kern, _, _ = timed_run(modes, True)
    qps = whole_job_rate(queries_per_step(cfg) * args.steps, world, total_ms)
    if args.mode == "exact":
        ex_ms, ex_energies = total_ms, energies
    else:
        ex_ms, _, _, ex_energies, _ = timed_run(LEVEL_MODES["exact"], False)
    _, _, ex_kern, _, _ = timed_run(LEVEL_MODES["exact"], True)
    exact_qps = whole_job_rate(queries_per_step(cfg) * args.steps, world, ex_ms)
    ratios = [e / x for e, x in zip(energies, ex_energies)]
    other = {}
    if also:
        a_ms, _, _, a_energies, _ = timed_run(LEVEL_MODES[also], False)
        a_stats = timed_run.last_stats
        a_qps = whole_job_rate(queries_per_step(cfg) * args.steps, world, a_ms)
        a_ratios = [e / x for e, x in zip(a_energies, ex_energies)]
        other[also] = {"level_modes": LEVEL_MODES[also], "value": a_qps, "ms_per_step": a_ms / args.steps,
                       "speedup_vs_exact": a_qps / exact_qps,
                       "final_energy_ratio_vs_exact": {"max": max(a_ratios), "mean": float(np.mean(a_ratios)),
                                                       "within_1.01": bool(max(a_ratios) <= 1.01)}}
        if "proposal" in LEVEL_MODES[also]:
            other[also]["fallback_fraction_last_search"] = a_stats["fallback_queries"] / max(1, a_stats["queries"])

    # ---- end to end through the public API with host buffers ----
    inits = [P.random_patch_init(z0, Hc, Hc, wc, args.warmup + i) for i in range(args.steps)]
    pinned = [torch.from_numpy(x).pin_memory() for x in inits]
    out_host = torch.empty(sizes[-1]["Ho"], sizes[-1]["Ho"], 3, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_ms = 0.0
    for i in range(args.steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        x0 = pinned[i].to(dev, non_blocking=True)
        X, _ = step(x0, modes)
        out_host.copy_(X, non_blocking=True)
        ev1.record(stream)
        ev1.synchronize()
        e2e_ms += ev0.elapsed_time(ev1)
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    e2e_qps = whole_job_rate(queries_per_step(cfg) * args.steps, world, e2e_ms)

    # ---- the exact FP32 arm against the FP32 SIMT pipe (FMA rate measured here, this GPU) ----
    fma_tf, _ = pts.fp32_fma_peak()
    it = cfg["iters"] + 1
    pca_levels = [(l, ix.info) for l, ix in zip(sizes, pidx.indices) if ix.info["exact_var"] >= PCA_PASS_MIN_VAR]
    # queries the full-dimension pass took per step: one untimed exact step replayed search by
    # search through the public API, reading each search's statistics
    route = exact_route_counts(pts, pidx, init_dev(args.warmup), cfg)
    full_fl = sum(2.0 * l["D"] * l["N"] * n for l, n in zip(sizes, route["range_queries"]))
    pca_fl = sum(2.0 * (inf["exact_dims"] + 1) * l["N"] * l["Q"] * it for l, inf in pca_levels)
    # the second bound (d_fast components) on the first bound's uncertified queries, same class
    pca_fl += sum(2.0 * (inf["d_fast"] + 1) * l["N"] * n
                  for l, inf, n in zip(sizes, [ix.info for ix in pidx.indices], route["second_bound_queries"]))
    ex_roofs = {}
    if "search_topk" in ex_kern and pca_levels:
        ach = pca_fl / (ex_kern["search_topk"]["ms_per_step"] / 1000.0) / 1e12
        ex_roofs["search_topk"] = {
            "kernel": "k_search_pca (FP32 SIMT PCA-space bound GEMM + top-32)", "bound": "alu", "achieved": ach,
            "peak": fma_tf, "unit": "TFLOP/s", "frac": ach / fma_tf,
            "note": "algorithmic 2(k+1) flops per (query, window) pair at the levels that run the PCA pass "
                    f"(k = {[inf['exact_dims'] for _, inf in pca_levels]} bound components); peak = FP32 FMA probe "
                    "measured in this run "
                    f"(nominal {PEAK_FP32_TFLOPS:.1f} = 152 SMs x 128 lanes x 2 x 2070 MHz)"}
    if "search_full" in ex_kern and full_fl > 0:
        ach = full_fl / (ex_kern["search_full"]["ms_per_step"] / 1000.0) / 1e12
        ex_roofs["search_full"] = {
            "kernel": "k_search_full (FP32 SIMT full-dimension GEMM + top-32)", "bound": "alu", "achieved": ach,
            "peak": fma_tf, "unit": "TFLOP/s", "frac": ach / fma_tf,
            "note": "algorithmic 2D flops per (listed query, window) pair, listed queries per step "
                    f"{route['range_queries']} (coarse to fine); peak = FP32 FMA probe measured in this run"}
    ex_dom = max((k for k in ex_roofs), key=lambda k: ex_kern[k]["ms_per_step"], default=None)
    ex_roof = dict(ex_roofs[ex_dom]) if ex_dom else {"kernel": None, "bound": "alu", "achieved": None,
                                                      "peak": fma_tf, "unit": "TFLOP/s", "frac": None}
    ex_roof["others"] = {k: v for k, v in ex_roofs.items() if k != ex_dom}

    # ---- roofline of the dominant kernel of this mode ----
    bf16_burst, bf16_sust, peak_src = _peaks()
    dom = max(kern, key=lambda k: kern[k]["ms_per_step"]) if kern else None
    roof = {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None}
    it = cfg["iters"] + 1
    if dom == "search_tc":
        dfs = [ix.info["d_fast"] for ix in pidx.indices]
        fl = sum(2.0 * (df + 1) * l["N"] * l["Q"] * it for l, m, df in zip(sizes, modes, dfs) if m in ("f16", "fp8"))
        ach = fl / (kern[dom]["ms_per_step"] / 1000.0) / 1e12
        if "fp8" in modes:
            # dense FP8 runs at twice the BF16 rate (nominal 4.5 vs 2.25 PFLOP/s)
            pk = 2.0 * bf16_burst
            roof.update(bound="tensor", achieved=ach, peak=pk, unit="TFLOP/s", frac=ach / pk,
                        kernel="k_search_tc<FP8> (E4M3 tcgen05 PCA-space GEMM + top-32)",
                        note=f"algorithmic 2(d_fast+1) flops per pair, d_fast={dfs}; peak = 2 x BF16 burst "
                             f"({peak_src}) x the nominal FP8/BF16 ratio")
        else:
            roof.update(bound="tensor", achieved=ach, peak=bf16_burst, unit="TFLOP/s", frac=ach / bf16_burst,
                        kernel="k_search_tc (FP16 tcgen05 PCA-space GEMM + top-32)", traffic=_tc_traffic(),
                        note=f"algorithmic 2(d_fast+1) flops per (query, window) pair, d_fast={dfs}; peak = BF16 "
                             f"burst (dense FP16 has the BF16 rate; a step lasts milliseconds), {peak_src}; "
                             "traffic = DRAM bytes of one fine-level launch (ncu), the algorithmic operand bytes "
                             "being 32.3 MB")
    elif dom in ex_roofs and args.mode == "exact":
        roof.update(ex_roofs[dom], traffic=None)
    elif dom == "search_full" and all(m != "exact" or ix.info["exact_var"] < PCA_PASS_MIN_VAR
                                      for m, ix in zip(modes, pidx.indices)):
        # exact levels without a PCA pass send every query to the full-dimension pass, and the
        # other modes never reach it: the work is 2 D flops per (query, window) pair there
        fl = sum(2.0 * 3 * l["w"] ** 2 * l["N"] * l["Q"] * it for l, m in zip(sizes, modes) if m == "exact")
        ach = fl / (kern[dom]["ms_per_step"] / 1000.0) / 1e12
        roof.update(bound="alu", achieved=ach, peak=fma_tf, unit="TFLOP/s", frac=ach / fma_tf,
                    kernel="k_search_full (FP32 SIMT full-dimension GEMM + top-32)",
                    note="algorithmic 2D flops per (query, window) pair at the exact levels; peak = FP32 FMA "
                         "probe measured in this run")
    elif dom is not None:
        roof.update(note="dominant kernel without a roofline model in this script")
    if "search_tcf" in kern:
        # the exact_tc levels' full-dimension FP16 GEMM: 2 D flops per (query, window) pair
        fl = sum(2.0 * l["D"] * l["N"] * l["Q"] * it for l, m in zip(sizes, modes) if m == "exact_tc")
        ach = fl / (kern["search_tcf"]["ms_per_step"] / 1000.0) / 1e12
        roof["others"] = {"search_tcf": {
            "kernel": "k_search_tcf (FP16 tcgen05 full-dimension GEMM, scores to HBM)", "bound": "tensor",
            "achieved": ach, "peak": bf16_burst, "unit": "TFLOP/s", "frac": ach / bf16_burst,
            "note": f"algorithmic 2D flops per (query, window) pair at the exact_tc levels; peak = BF16 burst, "
                    f"{peak_src}"}}

    other_cfgs = {}
    if not args.no_precision_form:
        other_cfgs["precision_form"] = time_precision_form(pts, P, L, dev, stream, flush, args.steps, args.warmup,
                                                           bf16_burst, peak_src)

    if not args.no_robust:
        # section 2.1's own schedule: r = 0.8 with the stopping rule at every level, same search
        # modes and seeds; queries counted as the searches the schedule ran
        rob_ms, rob_q, rob_steps, rob_ratios = 0.0, 0, [], []
        for i in range(args.steps):
            x0 = init_dev(args.warmup + i)
            flush.zero_()
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            X, E, _ = synthesize_pyramid(pidx, x0, iters=0, mode=modes, schedule="robust")
            ev1.record(stream)
            ev1.synchronize()
            rob_ms += ev0.elapsed_time(ev1)
            rob_steps.append([len(e) - 1 for e in E])
            rob_q += sum(L_["Q"] * len(e) for L_, e in zip(sizes, E))
            rob_ratios.append(exact_energy(X) / ex_energies[i])
        other_cfgs["robust_schedule"] = {
            "schedule": "r = 0.8, IRLS weights max(d, 1e-3)^(r-2), EM at each level until the searched windows "
                        "repeat (at most 30 M-steps), search modes as level_modes",
            "value": rob_q / (rob_ms / 1000.0), "unit": "queries/s", "ms_per_step": rob_ms / args.steps,
            "m_steps_per_level": np.mean(rob_steps, axis=0).tolist(),
            "em_iterations_per_s": float(np.sum(rob_steps)) / (rob_ms / 1000.0),
            "final_energy_ratio_vs_exact_fixed_schedule": {"max": max(rob_ratios), "mean": float(np.mean(rob_ratios))}}

    if not args.no_batched:
        other_cfgs["batched"] = time_batched(dev, stream, flush, args.steps, args.warmup)

    if not args.no_proposal_large:
        other_cfgs["proposal_large_exemplar"] = time_proposal_large(pts, P, dev, stream, flush, args.steps,
                                                                    args.warmup)

    headline = None
    if also == "proposal" or args.mode == "proposal":
        pv = qps if args.mode == "proposal" else other["proposal"]["value"]
        pr = ratios if args.mode == "proposal" else None
        headline = {"proposal_vs_exact": pv / exact_qps,
                    "final_energy_within_1.01": bool(max(pr) <= 1.01) if pr else
                    other["proposal"]["final_energy_ratio_vs_exact"]["within_1.01"]}
    line = {
        "metric": METRIC, "value": qps, "headline_learned_proposal": headline, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"exact": "f32", "fp8c": "e4m3+f32", "proposal": "bf16+f16+f32"}.get(args.mode, "f16+f32"),
        "data": "synthetic",
        "config": dict(cfg, mode=args.mode, level_modes=modes, l2="flushed between steps (256 MB write)",
                       d_fast=[ix.info["d_fast"] for ix in pidx.indices],
                       queries_per_step=queries_per_step(cfg), index_build_s=index_build_s,
                       proposal_train_s=train_s, proposal_pairs=n_pairs, proposal_clusters=args.clusters,
                       proposal_train_loss=train_loss, parallelism=f"replicas x{world}"),
        "em_iterations_per_s": cfg["iters"] * cfg["levels"] * args.steps * world / (total_ms / 1000.0),
        "exact_fp32": {"value": exact_qps, "ms_per_step": ex_ms / args.steps,
                       "em_iterations_per_s": cfg["iters"] * cfg["levels"] * args.steps * world / (ex_ms / 1000.0),
                       "kernels_per_step": ex_kern, "roofline": ex_roof,
                       "full_pass_fraction_per_level": [r / max(1, a) for r, a in zip(route["range_queries"],
                                                                                       route["queries"])]},
        "fp32_fma_peak_tflops": fma_tf,
        "speedup_vs_exact": qps / exact_qps,
        "final_energy_ratio_vs_exact": {"max": max(ratios), "mean": float(np.mean(ratios)),
                                        "within_1.01": bool(max(ratios) <= 1.01)},
        "other_modes": other,
        "other_configs": other_cfgs,
        "roofline": roof,
        "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": int(inits[0].nbytes),
                "d2h_bytes_per_step": int(out_host.numel() * 4 + 8 * (cfg["iters"] + 1) * cfg["levels"])},
        "gpu_launches": int(launches),
        "kernels_per_step": kern,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        n = args.cpu_sample or 0
        # about 0.57 TFLOP of FP64 brute force (~10 s on the 16 host cores measured)
        per = [n] * 3 if n else [2048, 6144, 18432]
        rate, threads, timed, secs = oracle_sample_rate(per)
        line["cpu_baseline"] = {"value": rate, "unit": "queries/s", "cores": threads, "kind": "oracle",
                                "sample": f"{per} queries per level (coarse to fine) of one E-step each, "
                                          f"FP64 full-dimension brute force, {secs:.1f} s, rate weighted by the "
                                          "workload's query mix"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    pidx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
