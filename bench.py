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
                "windows 32/16/8, outputs 128/256/512, PCA 64, stride 2, 5 EM iterations/level",
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
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="exact", choices=["exact", "bf16", "fp8", "proposal"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=0, help="queries per level for the CPU baseline")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import ctypes

    import torch

    import paper_2006_11851_gb300 as pts
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
    L.pts_launch_count.restype = ctypes.c_longlong
    L.pts_profile_enable.argtypes = [ctypes.c_int]
    L.pts_profile_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_longlong)]

    cfg = WORKLOAD
    sizes = level_sizes(cfg)
    Z = P.synthetic_exemplar(0, cfg["exemplar"], cfg["shrink"])
    t_build0 = time.perf_counter()
    pidx = PyramidIndex(torch.from_numpy(Z).to(dev), cfg["windows"], d=cfg["d"])
    torch.cuda.synchronize()
    index_build_s = time.perf_counter() - t_build0
    z0 = pidx.exemplars[0].cpu().numpy()
    n_total = args.warmup + args.steps
    inits = [P.random_patch_init(z0, sizes[0]["Ho"], sizes[0]["Ho"], sizes[0]["w"], s) for s in range(n_total)]
    init_dev = [torch.from_numpy(x).to(dev) for x in inits]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(x0):
        X, E, _ = synthesize_pyramid(pidx, x0, iters=cfg["iters"], r=cfg["r"], mode=args.mode)
        return X, E

    # exact-mode reference energy for the energy-ratio check (seed 0)
    X_ex, E_ex = step(init_dev[0].clone())
    for i in range(args.warmup):
        step(init_dev[i].clone())
    torch.cuda.synchronize()

    # ---- device-timed region ----
    work = [init_dev[args.warmup + i].clone() for i in range(args.steps)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = L.pts_launch_count()
    L.pts_profile_enable(1)
    times = []
    energies = []
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            _, E = step(work[i])
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1))
            energies.append(E)
    torch.cuda.synchronize()
    launches = L.pts_launch_count() - launches0
    tk_ms, tk_n = ctypes.c_double(), ctypes.c_longlong()
    L.pts_profile_read(b"search_topk", ctypes.byref(tk_ms), ctypes.byref(tk_n))
    kern = {}
    for name in ("search_topk", "search_full", "rerank", "project", "m_step", "brute", "irls"):
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        L.pts_profile_read(name.encode(), ctypes.byref(ms), ctypes.byref(n))
        kern[name] = {"ms": ms.value / args.steps, "launches": n.value // args.steps}
    L.pts_profile_enable(0)
    total_ms = sum(times)
    if dist:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = t.item()
    qps = queries_per_step(cfg) * args.steps * world / (total_ms / 1000.0)

    # ---- end to end through the public API with host buffers ----
    pinned = [torch.from_numpy(inits[args.warmup + i]).pin_memory() for i in range(args.steps)]
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
        X, _ = step(x0)
        out_host.copy_(X, non_blocking=True)
        ev1.record(stream)
        ev1.synchronize()
        e2e_ms += ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = t.item()
    e2e_qps = queries_per_step(cfg) * args.steps * world / (e2e_ms / 1000.0)

    # ---- roofline of the dominant kernel (FP32 SIMT bound search) ----
    flops_per_step = sum(2.0 * (min(cfg["d"], 3 * l["w"] ** 2) + 1) * l["N"] * l["Q"] * (cfg["iters"] + 1)
                         for l in sizes)
    achieved_tflops = flops_per_step * args.steps / (tk_ms.value / 1000.0) / 1e12 if tk_ms.value > 0 else None
    peak_tflops = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    roof = {"kernel": "k_search (PCA-space lower-bound GEMM + top-32, FP32 SIMT)", "bound": "alu",
            "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved_tflops / peak_tflops if achieved_tflops else None, "traffic": None,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (derived)",
            "kernel_ms_per_step": tk_ms.value / args.steps, "launches_per_step": tk_n.value // args.steps}

    energy_ratio = float(np.mean([e[-1][-1] for e in energies]) / 1.0)
    line = {
        "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(cfg, mode=args.mode, l2="flushed between steps (256 MB write)",
                       queries_per_step=queries_per_step(cfg), index_build_s=index_build_s,
                       parallelism=f"replicas x{world}"),
        "roofline": roof,
        "e2e": {"value": e2e_qps, "unit": "queries/s",
                "h2d_bytes_per_step": int(inits[0].nbytes),
                "d2h_bytes_per_step": int(out_host.numel() * 4 + 8 * (cfg["iters"] + 1) * cfg["levels"])},
        "gpu_launches": int(launches),
        "kernels_per_step": kern,
        "final_energy": float(energies[0][-1][-1]),
        "final_energy_exact_seed0": float(E_ex[-1][-1]),
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        n = args.cpu_sample or 0
        per = [n] * 3 if n else [512, 1024, 3072]
        rate, threads, timed, secs = oracle_sample_rate(per)
        line["cpu_baseline"] = {"value": rate, "unit": "queries/s", "cores": threads, "kind": "oracle",
                                "sample": f"{per} queries per level (coarse to fine) of one E-step each, "
                                          f"FP64 full-dimension brute force, {secs:.1f} s, rate weighted by the "
                                          "workload's query mix"}
    del energy_ratio
    if rank == 0:
        print(json.dumps(line), flush=True)
    pidx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
