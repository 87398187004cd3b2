"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module holds no arithmetic of the synthesis method itself: it only draws
random numbers and paints images.  Everything it produces is an *input*:

* ``synthetic_exemplar``: a perspective-like exemplar standing in for the
  paper's photographs (Figs. 1, 8, 9): elliptic texels whose radius and
  spacing shrink linearly from the bottom row to the top row (the paper puts
  the largest texel at the bottom-left origin, Methodology section 1), hue
  uniform, plus Gaussian pixel noise, clipped to [0, 1].
* ``random_patch_init``: the initial output of the energy optimisation,
  non-overlapping w x w exemplar windows drawn uniformly at random.
* ``random_nn`` / ``random_weights`` / ``sample_indices``: seeded index and
  weight arrays for step-wise tests.
* ``uniform_field``: per-pixel uniforms for the scale-guided initialisation.
* ``batched_jobs``: the job list of the 64-job batched workload.

All randomness comes from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) written out below, so that the
streams do not depend on the numpy version.  Normal deviates use the
Box-Muller transform.
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass

import numpy as np

_GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64: output k (k = 1, 2, ...) is mix(seed + k*gamma)."""

    def __init__(self, seed: int):
        self._state = np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)
        self._counter = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self._counter + 1, self._counter + 1 + n, dtype=np.uint64)
        self._counter += n
        with np.errstate(over="ignore"):
            z = self._state + k * _GOLDEN_GAMMA
            z = (z ^ (z >> np.uint64(30))) * _MIX1
            z = (z ^ (z >> np.uint64(27))) * _MIX2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """n doubles uniform in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """n standard normal deviates (Box-Muller)."""
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        rad = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 is in (0, 1]
        z = np.concatenate([rad * np.cos(2.0 * math.pi * u2), rad * np.sin(2.0 * math.pi * u2)])
        return z[:n]

    def randint(self, n: int, high: int) -> np.ndarray:
        """n integers uniform in [0, high) (floor of a uniform; bias < 2^-40 for high < 2^13)."""
        return np.minimum((self.uniform(n) * high).astype(np.int64), high - 1)


def _hsv_to_rgb(h: float, s: float, v: float) -> tuple[float, float, float]:
    i = int(h * 6.0) % 6
    f = h * 6.0 - math.floor(h * 6.0)
    p, q, t = v * (1 - s), v * (1 - f * s), v * (1 - (1 - f) * s)
    return [(v, t, p), (q, v, p), (p, v, t), (p, q, v), (t, p, v), (v, p, q)][i]


def synthetic_exemplar(seed: int, size: int, shrink: float, noise_sigma: float = 0.02) -> np.ndarray:
    """Seeded size x size x 3 float32 exemplar in [0, 1], HWC row-major.

    Row 0 of the array is the TOP of the image; the texel radius is r0 = size/16
    at the bottom row and r0/shrink at the top row, varying linearly in
    between, and the spacing between texel centres is 2.5 x the local radius
    (jittered), so a shrink factor s mimics a plane whose scale ratio
    S_max/S_min = 1/cos^2(sigma) equals s (Methodology, Eq. 1).
    """
    H = W = int(size)
    rng = SplitMix64(seed * 1000003 + 17)
    img = np.full((H, W, 3), 0.5, dtype=np.float64)
    r0 = size / 16.0

    def radius(y_up: float) -> float:
        t = min(max(y_up / max(H - 1, 1), 0.0), 1.0)
        return r0 * (1.0 - (1.0 - 1.0 / shrink) * t)

    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    y_up_grid = (H - 1) - yy  # bottom-left origin
    y_up = radius(0.0) * 0.8
    while y_up - radius(y_up) < H:
        r = radius(y_up)
        spacing = 2.5 * r
        x = -spacing + float(rng.uniform(1)[0]) * spacing
        while x - r < W:
            jx, jy, ar, ang, hue = rng.uniform(5)
            cx = x + (jx - 0.5) * 0.4 * r
            cy = y_up + (jy - 0.5) * 0.4 * r
            a = r
            b = r * (0.6 + 0.4 * ar)
            th = ang * math.pi
            color = _hsv_to_rgb(hue, 0.8, 0.9)
            x0, x1 = max(int(cx - a) - 1, 0), min(int(cx + a) + 2, W)
            r_lo, r_hi = (H - 1) - (cy + a), (H - 1) - (cy - a)
            y0, y1 = max(int(r_lo) - 1, 0), min(int(r_hi) + 2, H)
            if x0 < x1 and y0 < y1:
                dx = xx[y0:y1, x0:x1] - cx
                dy = y_up_grid[y0:y1, x0:x1] - cy
                u = dx * math.cos(th) + dy * math.sin(th)
                v = -dx * math.sin(th) + dy * math.cos(th)
                inside = (u / a) ** 2 + (v / b) ** 2 <= 1.0
                patch = img[y0:y1, x0:x1]
                patch[inside] = color
            x += spacing
        y_up += spacing
    img += noise_sigma * rng.normal(H * W * 3).reshape(H, W, 3)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def num_windows(H: int, W: int, w: int, stride: int) -> tuple[int, int]:
    """(rows, cols) of window origins (y0, x0) with y0 in {0, stride, ..., H - w}."""
    if w > H or w > W or (H - w) % stride or (W - w) % stride:
        raise ValueError(f"bad window grid H={H} W={W} w={w} stride={stride}")
    return (H - w) // stride + 1, (W - w) // stride + 1


def random_patch_init(exemplar: np.ndarray, Ho: int, Wo: int, w: int, seed: int) -> np.ndarray:
    """Output initialised from non-overlapping w x w exemplar windows drawn uniformly.

    Blocks start at multiples of w; the last block row/column is cropped at the
    border.  Returns float32 Ho x Wo x 3.
    """
    He, We, _ = exemplar.shape
    ny, nx = He - w + 1, We - w + 1
    nby, nbx = -(-Ho // w), -(-Wo // w)
    rng = SplitMix64(seed * 7919 + 3)
    pick = rng.randint(nby * nbx, ny * nx)
    out = np.empty((Ho, Wo, 3), dtype=np.float32)
    for b in range(nby * nbx):
        by, bx = divmod(b, nbx)
        ey, ex = divmod(int(pick[b]), nx)
        h = min(w, Ho - by * w)
        ww = min(w, Wo - bx * w)
        out[by * w:by * w + h, bx * w:bx * w + ww] = exemplar[ey:ey + h, ex:ex + ww]
    return out


def uniform_field(seed: int, H: int, W: int) -> np.ndarray:
    """H x W float64 uniforms in [0, 1) (seeded): the per-pixel draws of an initialisation that
    picks one of several equally good exemplar pixels."""
    return SplitMix64(seed * 47 + 23).uniform(H * W).reshape(H, W)


def random_nn(seed: int, Q: int, N: int) -> np.ndarray:
    """Q exemplar-window indices uniform in [0, N), int32."""
    return SplitMix64(seed * 31 + 5).randint(Q, N).astype(np.int32)


def random_weights(seed: int, Q: int, lo: float = 0.05, hi: float = 2.0) -> np.ndarray:
    """Q positive weights uniform in [lo, hi), float32."""
    return (lo + (hi - lo) * SplitMix64(seed * 37 + 11).uniform(Q)).astype(np.float32)


def sample_indices(seed: int, count: int, k: int) -> np.ndarray:
    """k distinct sorted indices from range(count), int32 (seeded)."""
    k = min(k, count)
    keys = SplitMix64(seed * 41 + 13).u64(count)
    return np.sort(np.argsort(keys, kind="stable")[:k]).astype(np.int32)


def random_matrix(seed: int, rows: int, cols: int, scale: float = 1.0) -> np.ndarray:
    """rows x cols float64 with N(0, scale^2) entries (seeded)."""
    return scale * SplitMix64(seed * 43 + 19).normal(rows * cols).reshape(rows, cols)


@dataclass(frozen=True)
class Job:
    """One synthesis job of the batched workload."""

    seed: int
    He: int
    Ho: int
    w: int
    d: int


def batched_jobs(n_jobs: int = 64, seed: int = 0) -> list[Job]:
    """The 64-job batched workload: exemplars 128..512 px square (even),
    outputs 256..1024 px square (even), w = 8 for even job ids and 16 for odd,
    d drawn from {32, 48, 64}."""
    rng = SplitMix64(seed * 53 + 29)
    jobs = []
    for j in range(n_jobs):
        u = rng.uniform(3)
        He = 128 + 2 * int(u[0] * 193)
        Ho = 256 + 2 * int(u[1] * 385)
        w = 8 if j % 2 == 0 else 16
        d = (32, 48, 64)[min(int(u[2] * 3), 2)]
        jobs.append(Job(seed=j, He=He, Ho=Ho, w=w, d=d))
    return jobs


def array_digest(a: np.ndarray) -> str:
    """SHA-256 of an array's dtype, shape and bytes (C order)."""
    h = hashlib.sha256()
    h.update(str(a.dtype).encode())
    h.update(str(a.shape).encode())
    h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()
