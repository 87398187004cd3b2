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

from ._binding import ExemplarIndex, _check, _mode, _need, _ptr, _stream, lib, synthesize_level

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import pts_inputs as P  # noqa: E402


class _Job(ctypes.Structure):
    _fields_ = [("index", ctypes.c_void_p), ("output", ctypes.c_void_p), ("Ho", ctypes.c_int),
                ("Wo", ctypes.c_int), ("stride", ctypes.c_int), ("mode", ctypes.c_int),
                ("energy", ctypes.c_void_p)]


def job_specs(n: int = 64, seed: int = 0, max_exemplar: int = 512, max_output: int = 1024) -> list[dict]:
    g = P.SplitMix64(seed)
    u = g.uniform(3 * n).reshape(n, 3)
    specs = []
    for j in range(n):
        w = 8 if j % 2 == 0 else 16
        he = min(max_exemplar, 128 + 2 * int(u[j, 0] * 193))
        ho = min(max_output, 256 + 2 * int(u[j, 1] * 385))
        ho -= (ho - w) % 2
        d = (32, 48, 64)[min(2, int(u[j, 2] * 3))]
        specs.append({"job": j, "He": he, "Ho": ho, "w": w, "d": d, "seed": j})
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
                       energies[k].data_ptr())
    _check(L.synthesize_batched(jobs, n, iters, r, delta, _stream()))


class Batch:
    """Indices, outputs and energies of a job list, and the captured graph over all of them."""

    def __init__(self, specs: list[dict], mode="f16", iters: int = 5, r: float = 2.0, delta: float = 1e-3,
                 n_streams: int = 8, tune: bool = True, shrink: float = 4.0, device=None):
        L = lib()
        _declare(L)
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.specs, self.iters, self.r, self.delta, self.mode = specs, iters, r, delta, mode
        self.indices, self.inits, self.outputs, self.energies = [], [], [], []
        for s in specs:
            z = P.synthetic_exemplar(s["seed"], s["He"], shrink)
            zt = torch.from_numpy(z).to(self.device)
            self.indices.append(ExemplarIndex(zt, s["w"], d=s["d"]))
            x0 = torch.from_numpy(P.random_patch_init(z, s["Ho"], s["Ho"], s["w"], 1000 + s["seed"])).to(self.device)
            self.inits.append(x0)
            self.outputs.append(x0.clone())
            self.energies.append(torch.zeros(iters + 1, dtype=torch.float64, device=self.device))
        jobs = (_Job * len(specs))()
        for k, s in enumerate(specs):
            jobs[k] = _Job(self.indices[k].handle.value, self.outputs[k].data_ptr(), s["Ho"], s["Ho"], 2, _mode(mode),
                           self.energies[k].data_ptr())
        self._jobs = jobs
        self._h = ctypes.c_void_p()
        _check(L.pts_batch_create(jobs, len(specs), iters, r, delta, n_streams, 1 if tune else 0, _stream(),
                                  ctypes.byref(self._h)))
        n = ctypes.c_longlong()
        parts = np.zeros(len(specs), dtype=np.int32)
        _check(L.pts_batch_info(self._h, ctypes.byref(n), parts.ctypes.data_as(ctypes.c_void_p)))
        self.launches_per_run, self.parts = int(n.value), parts

    def reset(self):
        for x, x0 in zip(self.outputs, self.inits):
            x.copy_(x0)

    def run(self):
        _check(lib().pts_batch_run(self._h, _stream()))

    def queries(self) -> int:
        return sum(((s["Ho"] - s["w"]) // 2 + 1) ** 2 * (self.iters + 1) for s in self.specs)

    def close(self):
        if getattr(self, "_h", None):
            lib().pts_batch_destroy(self._h)
            self._h = ctypes.c_void_p()
        for ix in self.indices:
            ix.close()


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--runs", type=int, default=3)
    ap.add_argument("--mode", default="f16")
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--max-exemplar", type=int, default=512)
    ap.add_argument("--max-output", type=int, default=1024)
    args = ap.parse_args()
    specs = job_specs(args.jobs, max_exemplar=args.max_exemplar, max_output=args.max_output)
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

    def eager():
        for ix, x in zip(b.indices, b.outputs):
            synthesize_level(ix, x, b.iters, r=b.r, delta=b.delta, mode=args.mode)
    eager_ms = min(timed(eager) for _ in range(args.runs))
    q = b.queries()
    out = {"jobs": args.jobs, "mode": args.mode, "queries_per_run": q, "graph_ms": graph_ms,
           "graph_queries_per_s": q / (graph_ms / 1e3), "eager_ms": eager_ms, "eager_queries_per_s": q / (eager_ms / 1e3),
           "em_iterations_per_s": len(specs) * b.iters / (graph_ms / 1e3), "launches_per_run": b.launches_per_run,
           "autotuned_parts": b.parts.tolist(), "index_build_and_tune_s": build_s}
    print(json.dumps(out))
    b.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
