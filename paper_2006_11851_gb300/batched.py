"""Batched synthesis: many independent single-level jobs of uneven sizes replayed as one CUDA
graph (pts_batch_*), with the library's autotuner choosing each job's tensor-core split.

    python -m paper_2006_11851_gb300.batched --jobs 64 --runs 3

The job mix follows the batched workload: exemplar He = 128 + 2 floor(193 U) (even, 128..512),
output Ho even in 256..1024 with (Ho - w) even, w = 8 for even jobs and 16 for odd ones, d drawn
from {32, 48, 64}; seeded SplitMix64 draws, generator seed = job number.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import sys
import time

import numpy as np
import torch

from ._binding import ExemplarIndex, _check, _mode, _need, _ptr, _stream, downsample2, lib, synthesize_level

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import pts_inputs as P  # noqa: E402


class _Job(ctypes.Structure):
    _fields_ = [("index", ctypes.c_void_p), ("output", ctypes.c_void_p), ("Ho", ctypes.c_int),
                ("Wo", ctypes.c_int), ("stride", ctypes.c_int), ("mode", ctypes.c_int),
                ("energy", ctypes.c_void_p), ("parent", ctypes.c_int)]


def job_specs(n: int = 64, seed: int = 0, max_exemplar: int = 512, max_output: int = 1024,
              levels: int = 1) -> list[dict]:
    """The batched workload's jobs; levels > 1 makes each job a pyramid of that many levels
    (the output a multiple of 2^levels so that every level keeps (Ho - w) even)."""
    g = P.SplitMix64(seed)
    u = g.uniform(3 * n).reshape(n, 3)
    specs = []
    for j in range(n):
        w = 8 if j % 2 == 0 else 16
        he = min(max_exemplar, 128 + 2 * int(u[j, 0] * 193))
        ho = min(max_output, 256 + 2 * int(u[j, 1] * 385))
        ho -= (ho - w) % 2
        if levels > 1:
            ho -= ho % (1 << levels)
        d = (32, 48, 64)[min(2, int(u[j, 2] * 3))]
        specs.append({"job": j, "He": he, "Ho": ho, "w": w, "d": d, "seed": j, "levels": levels})
    return specs


def _declare(L):
    L.pts_batch_create.argtypes = [ctypes.POINTER(_Job), ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    L.pts_batch_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.pts_batch_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong), ctypes.c_void_p]
    L.pts_batch_destroy.argtypes = [ctypes.c_void_p]
    L.pts_batch_destroy.restype = None
    L.synthesize_batched.argtypes = [ctypes.POINTER(_Job), ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_void_p]


def synthesize_batched(indices: list, outputs: list, energies: list, mode="f16", iters: int = 5, r: float = 2.0,
                       delta: float = 1e-3, stride: int = 2) -> None:
    """One call of the library's synthesize_batched: job k runs `iters` EM iterations of
    outputs[k] (square Ho x Ho x 3, CUDA) against indices[k], then the final search; outputs and
    energies[k] (iters + 1 float64, CUDA) are written in place.  Synchronises the current stream."""
    L = lib()
    _declare(L)
    n = len(indices)
    if not (len(outputs) == len(energies) == n):
        raise ValueError("one output and one energy array per index")
    jobs = (_Job * n)()
    for k in range(n):
        _need(outputs[k], torch.float32, f"outputs[{k}]")
        _need(energies[k], torch.float64, f"energies[{k}]", (iters + 1,))
        Ho, Wo, C = outputs[k].shape
        if C != 3:
            raise ValueError(f"job {k}: output must be H x W x 3")
        jobs[k] = _Job(indices[k].handle.value, outputs[k].data_ptr(), Ho, Wo, stride, _mode(mode),
                       energies[k].data_ptr(), -1)
    _check(L.synthesize_batched(jobs, n, iters, r, delta, _stream()))


class Batch:
    """Indices, outputs and energies of a job list, and the captured graph over all of them.

    A spec is {"He", "Ho", "w", "d", "seed"} plus optionally "mode" (this job's search mode,
    default the batch's), "levels" (a pyramid of that many levels, coarse to fine, each level a
    job chained to the one before: its exemplar the finer one down-sampled, its output half the
    size); for mode "proposal" the proposal is trained first on the job's own exact runs
    (train_job_proposal), for mode "kmtree" the k-means tree is built.  self.levels[k] lists the
    batch jobs of spec k, coarsest first."""

    def __init__(self, specs: list[dict], mode="f16", iters: int = 5, r: float = 2.0, delta: float = 1e-3,
                 n_streams: int = 8, tune: bool = True, shrink: float = 4.0, device=None,
                 proposal_params: dict | None = None):
        L = lib()
        _declare(L)
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.specs, self.iters, self.r, self.delta, self.mode = specs, iters, r, delta, mode
        self.indices, self.inits, self.outputs, self.energies = [], [], [], []
        self.sizes, self.parents, self.modes, self.levels = [], [], [], []
        for s in specs:
            z = torch.from_numpy(P.synthetic_exemplar(s["seed"], s["He"], shrink)).to(self.device)
            nlev = int(s.get("levels", 1))
            pyr = [z]
            for _ in range(nlev - 1):
                pyr.append(downsample2(pyr[-1]))
            pyr = pyr[::-1]
            jm = s.get("mode", mode)
            ks = []
            for lev in range(nlev):
                ho = s["Ho"] >> (nlev - 1 - lev)
                ix = ExemplarIndex(pyr[lev], s["w"], d=s["d"])
                if jm == "kmtree":
                    from ._binding import build_kmeans_tree
                    build_kmeans_tree(ix, 10)
                if jm == "proposal":
                    from .proposal import train_job_proposal
                    train_job_proposal(ix, pyr[lev], ho, s["w"], [2000 + 10 * s["seed"] + t for t in range(2)],
                                       iters=iters, **(proposal_params or {}))
                x0 = torch.from_numpy(P.random_patch_init(pyr[lev].cpu().numpy(), ho, ho, s["w"],
                                                          1000 + s["seed"])).to(self.device)
                ks.append(len(self.indices))
                self.parents.append(ks[-2] if lev > 0 else -1)
                self.indices.append(ix)
                self.inits.append(x0)
                self.outputs.append(x0.clone())
                self.energies.append(torch.zeros(iters + 1, dtype=torch.float64, device=self.device))
                self.sizes.append((ho, s["w"]))
                self.modes.append(jm)
            self.levels.append(ks)
        jobs = (_Job * len(self.indices))()
        for k, ix in enumerate(self.indices):
            ho = self.sizes[k][0]
            jobs[k] = _Job(ix.handle.value, self.outputs[k].data_ptr(), ho, ho, 2, _mode(self.modes[k]),
                           self.energies[k].data_ptr(), self.parents[k])
        self._jobs = jobs
        self._h = ctypes.c_void_p()
        _check(L.pts_batch_create(jobs, len(self.indices), iters, r, delta, n_streams, 1 if tune else 0, _stream(),
                                  ctypes.byref(self._h)))
        n = ctypes.c_longlong()
        parts = np.zeros(len(self.indices), dtype=np.int32)
        _check(L.pts_batch_info(self._h, ctypes.byref(n), parts.ctypes.data_as(ctypes.c_void_p)))
        self.launches_per_run, self.parts = int(n.value), parts

    def reset(self):
        for x, x0 in zip(self.outputs, self.inits):
            x.copy_(x0)

    def run(self):
        _check(lib().pts_batch_run(self._h, _stream()))

    def queries(self) -> int:
        return sum(((ho - w) // 2 + 1) ** 2 * (self.iters + 1) for ho, w in self.sizes)

    def close(self):
        if getattr(self, "_h", None):
            lib().pts_batch_destroy(self._h)
            self._h = ctypes.c_void_p()
        for ix in self.indices:
            ix.close()


def run_eager(b: Batch) -> None:
    """The batch's jobs one by one through synthesize_level (chained levels up-sampled between)."""
    from ._binding import upsample2
    for k, (ix, x) in enumerate(zip(b.indices, b.outputs)):
        if b.parents[k] >= 0:
            x.copy_(upsample2(b.outputs[b.parents[k]]))
        synthesize_level(ix, x, b.iters, r=b.r, delta=b.delta, mode=b.modes[k])


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--runs", type=int, default=3)
    ap.add_argument("--mode", default="f16")
    ap.add_argument("--levels", type=int, default=1)
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--max-exemplar", type=int, default=512)
    ap.add_argument("--max-output", type=int, default=1024)
    args = ap.parse_args()
    specs = job_specs(args.jobs, max_exemplar=args.max_exemplar, max_output=args.max_output, levels=args.levels)
    t0 = time.perf_counter()
    b = Batch(specs, mode=args.mode, n_streams=args.streams)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    st = torch.cuda.current_stream()

    def timed(fn):
        b.reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1)

    graph_ms = min(timed(b.run) for _ in range(args.runs))
    eager_ms = min(timed(lambda: run_eager(b)) for _ in range(args.runs))
    q = b.queries()
    out = {"jobs": args.jobs, "levels": args.levels, "mode": args.mode, "queries_per_run": q, "graph_ms": graph_ms,
           "graph_queries_per_s": q / (graph_ms / 1e3), "eager_ms": eager_ms, "eager_queries_per_s": q / (eager_ms / 1e3),
           "em_iterations_per_s": len(b.indices) * b.iters / (graph_ms / 1e3), "launches_per_run": b.launches_per_run,
           "autotuned_parts": b.parts.tolist(), "index_build_and_tune_s": build_s}
    print(json.dumps(out))
    b.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
