"""Plain FP64 CPU oracle for perspective texture synthesis by energy optimisation.

TEST INFRASTRUCTURE ONLY: the slow, obviously correct reference the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product package never
does, and nothing here imports the product package.

The arithmetic lives in ``pts_oracle.c`` (plain C, FP64, OpenMP only across
independent queries/rows); this module builds it with gcc on first use and
marshals numpy arrays.  Images are H x W x C with C = 3 (RGB) or 4 (RGBS: the
scale map of section 1 as a fourth channel); the channel count comes from the
image's shape.  Histogram matching (section 3, Eq. 9) is plain numpy in
``histogram.py``, the scale map (Eqs. 1-3) and its use in synthesis in
``scale.py``, the k-means tree checks in ``kmtree.py``.  The EM driver below follows the paper's two phases
(section 2.1: search phase, then optimization phase, repeated).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, f) for f in ("pts_oracle.c", "pts_oracle_learn.c")]
_LOCK = threading.Lock()
_LIB = None


def _lib_path() -> str:
    return os.path.join(_HERE, "_build", f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp) into oracle/_build/."""
    out = _lib_path()
    srcs = [s for s in _SRC if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall", "-Wno-unknown-pragmas",
           "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def lib() -> ctypes.CDLL:
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = ctypes.CDLL(build())
            _declare(_LIB)
    return _LIB


_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_I = ctypes.c_int
_D = ctypes.c_double


def _declare(L: ctypes.CDLL) -> None:
    L.or_max_threads.argtypes = [_I]
    L.or_max_threads.restype = _I
    L.or_nn_bruteforce.argtypes = [_d, _I, _I, _d, _I, _I, _I, _I, _I, _i32, _I, _i32, _d, _I]
    L.or_pair_dist2.argtypes = [_d, _I, _I, _d, _I, _I, _I, _I, _I, _i32, _i32, _I, _d]
    L.or_window_mean.argtypes = [_d, _I, _I, _I, _I, _d]
    L.or_window_cov.argtypes = [_d, _I, _I, _I, _I, _d, _d, _I]
    L.or_jacobi_eigh.argtypes = [_d, _I, _d, _d, _I]
    L.or_jacobi_eigh.restype = _I
    L.or_pca_fit.argtypes = [_d, _I, _I, _I, _I, _I, _d, _d, _d, _I]
    L.or_pca_fit.restype = _I
    L.or_project.argtypes = [_d, _I, _I, _I, _I, _I, _d, _d, _I, _i32, _I, _d, _d, _d]
    L.or_irls.argtypes = [_d, _I, _D, _D, _d, _d, _d]
    L.or_m_step.argtypes = [_i32, _d, _d, _I, _I, _I, _I, _I, _I, _I, _d]
    L.or_downsample2.argtypes = [_d, _I, _I, _I, _d]
    L.or_upsample2.argtypes = [_d, _I, _I, _I, _d]
    if hasattr(L, "or_kmeans_assign"):
        _declare_learn(L)


def _declare_learn(L: ctypes.CDLL) -> None:
    L.or_kmeans_pp.argtypes = [_d, _I, _I, _I, _d, _d, _i32]
    L.or_kmeans_assign.argtypes = [_d, _I, _I, _d, _I, _i32, _d]
    L.or_kmeans_update.argtypes = [_d, _I, _I, _i32, _I, _d, _i32, _d]
    L.or_mlp_forward.argtypes = [_d, _I, _I, _I, _I, _I] + [_d] * 11
    L.or_ce_loss.argtypes = [_d, _I, _I, _i32, _d]
    L.or_ce_loss.restype = _D
    L.or_mlp_backward.argtypes = [_d, _I, _I, _I, _I, _I] + [_d] * 11 + [_i32] + [_d] * 6


def _p(a: np.ndarray, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32a(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _image(a) -> np.ndarray:
    """FP64 copy of an H x W x C image; C = 3 (RGB) or 4 (RGBS, section 3's scale channel)."""
    a = _f64(a)
    if a.ndim != 3 or a.shape[2] not in (3, 4):
        raise ValueError(f"expected an H x W x 3 or H x W x 4 image, got shape {a.shape}")
    return a


def _same_channels(*imgs) -> int:
    C = imgs[0].shape[2]
    if any(im.shape[2] != C for im in imgs):
        raise ValueError("images differ in their channel count")
    return C


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count the oracle uses."""
    return lib().or_max_threads(int(n))


# ---------------------------------------------------------------------------
# window grids (section 2.1 neighbourhoods; section 2.2 patch stride)
# ---------------------------------------------------------------------------
def grid(H: int, W: int, w: int, stride: int) -> tuple[int, int]:
    if w > H or w > W or (H - w) % stride or (W - w) % stride:
        raise ValueError(f"bad window grid H={H} W={W} w={w} stride={stride}")
    return (H - w) // stride + 1, (W - w) // stride + 1


def num_exemplar_windows(He: int, We: int, w: int) -> int:
    a, b = grid(He, We, w, 1)
    return a * b


def num_queries(Ho: int, Wo: int, w: int, stride: int = 2) -> int:
    a, b = grid(Ho, Wo, w, stride)
    return a * b


# ---------------------------------------------------------------------------
# E-step: exact brute-force full-dimension NN (Eq. 4)
# ---------------------------------------------------------------------------
def nn_bruteforce(X, Z, w: int, stride: int = 2, qlist=None, nthreads: int = 0):
    """(nn int32, d2 float64) of the listed queries (all if qlist is None)."""
    X, Z = _image(X), _image(Z)
    C = _same_channels(X, Z)
    Ho, Wo, _ = X.shape
    He, We, _ = Z.shape
    Q = num_queries(Ho, Wo, w, stride)
    num_exemplar_windows(He, We, w)
    if qlist is None:
        ql, nq = None, Q
    else:
        ql = _i32a(qlist)
        nq = len(ql)
        if nq and (ql.min() < 0 or ql.max() >= Q):
            raise ValueError("query index out of range")
    nn = np.empty(nq, np.int32)
    d2 = np.empty(nq, np.float64)
    lib().or_nn_bruteforce(_p(X), Ho, Wo, _p(Z), He, We, w, C, stride,
                           None if ql is None else _p(ql, ctypes.c_int32), nq,
                           _p(nn, ctypes.c_int32), _p(d2), int(nthreads))
    return nn, d2


def pair_dist2(X, Z, w: int, stride: int, q, n) -> np.ndarray:
    """Full-dimension squared distance for each (query q[i], exemplar window n[i])."""
    X, Z = _image(X), _image(Z)
    C = _same_channels(X, Z)
    q, n = _i32a(q), _i32a(n)
    Ho, Wo, _ = X.shape
    He, We, _ = Z.shape
    Q = num_queries(Ho, Wo, w, stride)
    N = num_exemplar_windows(He, We, w)
    if len(q) != len(n) or (len(q) and (q.min() < 0 or q.max() >= Q or n.min() < 0 or n.max() >= N)):
        raise ValueError("bad pair list")
    out = np.empty(len(q), np.float64)
    lib().or_pair_dist2(_p(X), Ho, Wo, _p(Z), He, We, w, C, stride, _p(q, ctypes.c_int32),
                        _p(n, ctypes.c_int32), len(q), _p(out))
    return out


# ---------------------------------------------------------------------------
# PCA (section 2.2)
# ---------------------------------------------------------------------------
def window_mean(Z, w: int) -> np.ndarray:
    Z = _image(Z)
    He, We, C = Z.shape
    num_exemplar_windows(He, We, w)
    mu = np.empty(C * w * w)
    lib().or_window_mean(_p(Z), He, We, w, C, _p(mu))
    return mu


def window_cov(Z, w: int, nthreads: int = 0) -> np.ndarray:
    Z = _image(Z)
    He, We, C = Z.shape
    mu = window_mean(Z, w)
    D = C * w * w
    cov = np.empty((D, D))
    lib().or_window_cov(_p(Z), He, We, w, C, _p(mu), _p(cov), int(nthreads))
    return cov


def jacobi_eigh(A, nthreads: int = 0):
    """(eigenvalues descending, eigenvectors as columns, sweeps) by Jacobi's method."""
    A = _f64(A).copy()
    n = A.shape[0]
    ev = np.empty(n)
    V = np.empty((n, n))
    sweeps = lib().or_jacobi_eigh(_p(A), n, _p(ev), _p(V), int(nthreads))
    return ev, V, sweeps


def pca_fit(Z, w: int, d: int, nthreads: int = 0):
    """(mu[D], basis[d, D], eigenvalues[min(N, D)] descending, sweeps)."""
    Z = _image(Z)
    He, We, C = Z.shape
    N = num_exemplar_windows(He, We, w)
    D = C * w * w
    if not 0 < d <= min(D, N):
        raise ValueError("bad d")
    mu = np.empty(D)
    basis = np.empty((d, D))
    ev = np.empty(min(N, D))
    sweeps = lib().or_pca_fit(_p(Z), He, We, w, C, d, _p(mu), _p(basis), _p(ev), int(nthreads))
    return mu, basis, ev, sweeps


def project(img, w: int, stride: int, mu, basis, lst=None):
    """(y [n, d], ||v - mu||^2 [n], residual norm [n]) of the listed windows."""
    img, mu, basis = _image(img), _f64(mu), _f64(basis)
    H, W, C = img.shape
    total = np.prod(grid(H, W, w, stride))
    d = basis.shape[0]
    if mu.shape != (C * w * w,) or basis.shape[1:] != (C * w * w,):
        raise ValueError("mu / basis do not match the image's window dimension")
    if lst is None:
        lp, cnt = None, int(total)
    else:
        lst = _i32a(lst)
        lp, cnt = _p(lst, ctypes.c_int32), len(lst)
    y = np.empty((cnt, d))
    un = np.empty(cnt)
    rs = np.empty(cnt)
    lib().or_project(_p(img), H, W, w, C, stride, _p(mu), _p(basis), d, lp, cnt, _p(y), _p(un), _p(rs))
    return y, un, rs


# ---------------------------------------------------------------------------
# IRLS weights and energy (Eqs. 5-8), M-step (Eq. 8)
# ---------------------------------------------------------------------------
def irls(d2, r: float = 2.0, delta: float = 1e-3):
    """(W [Q], E_r, E_delta); see or_irls in pts_oracle.c."""
    d2 = _f64(d2)
    W = np.empty(len(d2))
    er, ed = ctypes.c_double(), ctypes.c_double()
    lib().or_irls(_p(d2), len(d2), float(r), float(delta), _p(W), ctypes.byref(er), ctypes.byref(ed))
    return W, er.value, ed.value


def m_step(nn, Wt, Z, w: int, Ho: int, Wo: int, stride: int = 2, X_prev=None) -> np.ndarray:
    """New output image (Ho x Wo x C, float64, C the exemplar's channels) from matched windows and
    weights."""
    Z = _image(Z)
    He, We, C = Z.shape
    Q = num_queries(Ho, Wo, w, stride)
    N = num_exemplar_windows(He, We, w)
    nn = _i32a(nn)
    if nn.shape != (Q,) or (Q and (nn.min() < 0 or nn.max() >= N)):
        raise ValueError("bad nn")
    X = np.zeros((Ho, Wo, C)) if X_prev is None else _image(X_prev).copy()
    if X.shape != (Ho, Wo, C):
        raise ValueError("X_prev does not match the output size and the exemplar's channels")
    Wp = None if Wt is None else _f64(Wt)
    lib().or_m_step(_p(nn, ctypes.c_int32), None if Wp is None else _p(Wp), _p(Z), He, We, w, C, Ho, Wo,
                    stride, _p(X))
    return X


def downsample2(img) -> np.ndarray:
    img = _image(img)
    H, W, C = img.shape
    out = np.empty(((H + 1) // 2, (W + 1) // 2, C))
    lib().or_downsample2(_p(img), H, W, C, _p(out))
    return out


def upsample2(img) -> np.ndarray:
    img = _image(img)
    H, W, C = img.shape
    out = np.empty((2 * H, 2 * W, C))
    lib().or_upsample2(_p(img), H, W, C, _p(out))
    return out


def exemplar_pyramid(Z, levels: int) -> list[np.ndarray]:
    """[coarsest, ..., finest] Gaussian pyramid of the exemplar (section 2.1)."""
    pyr = [_f64(Z)]
    for _ in range(levels - 1):
        pyr.append(downsample2(pyr[-1]))
    return pyr[::-1]


# ---------------------------------------------------------------------------
# EM driver (section 2.1): search phase then optimization phase, repeated
# ---------------------------------------------------------------------------
def synthesize_level(Z, X0, w: int, iters: int, r: float = 2.0, delta: float = 1e-3, stride: int = 2,
                     nthreads: int = 0, keep_trajectory: bool = False, f32_io: bool = True):
    """Run `iters` EM iterations from X0, then one last search phase.

    Returns a dict with the final image X, the energies E (iters + 1 entries:
    E[t] is the energy of the iterate entering iteration t, E[iters] of the
    final image), the delta-form energies, and optionally the trajectory
    (X_t, nn_t, d2_t, W_t).  With f32_io the iterate is rounded to float32
    between iterations, as the GPU path stores images in float32; weights are
    rounded to float32 before the M-step for the same reason.
    """
    Z = _f64(Z)
    X = _f64(X0)
    Ho, Wo, _ = X.shape
    E, Ed, traj = [], [], []
    for _ in range(iters + 1):
        if f32_io:
            X = X.astype(np.float32).astype(np.float64)
        nn, d2 = nn_bruteforce(X, Z, w, stride, nthreads=nthreads)
        W, er, ed = irls(d2, r, delta)
        if f32_io:
            W = W.astype(np.float32).astype(np.float64)
        E.append(er)
        Ed.append(ed)
        if keep_trajectory:
            traj.append((X.copy(), nn, d2, W))
        if len(E) == iters + 1:
            break
        X = m_step(nn, W, Z, w, Ho, Wo, stride, X_prev=X)
    out = {"X": X, "E": np.array(E), "E_delta": np.array(Ed)}
    if keep_trajectory:
        out["trajectory"] = traj
    return out


def synthesize_level_converge(Z, X0, w: int, max_iters: int, r: float = 0.8, delta: float = 1e-3, stride: int = 2,
                              nthreads: int = 0, f32_io: bool = True):
    """EM iterations until the search phase returns, for every query, the window it returned the
    iteration before (the set {z_p} no longer changes: section 2.1's stopping rule), or until
    max_iters M-steps have run; the last search phase gives the final energy.  Returns a dict with
    X, E and E_delta (iters + 1 entries, as synthesize_level) and iters, the M-steps run."""
    Z = _f64(Z)
    X = _f64(X0)
    Ho, Wo, _ = X.shape
    E, Ed = [], []
    nn_prev = None
    it = 0
    while True:
        if f32_io:
            X = X.astype(np.float32).astype(np.float64)
        nn, d2 = nn_bruteforce(X, Z, w, stride, nthreads=nthreads)
        W, er, ed = irls(d2, r, delta)
        if f32_io:
            W = W.astype(np.float32).astype(np.float64)
        E.append(er)
        Ed.append(ed)
        if it == max_iters or (nn_prev is not None and np.array_equal(nn, nn_prev)):
            break
        X = m_step(nn, W, Z, w, Ho, Wo, stride, X_prev=X)
        nn_prev = nn
        it += 1
    return {"X": X, "E": np.array(E), "E_delta": np.array(Ed), "iters": it}


# ---------------------------------------------------------------------------
# learned cluster proposal (replaces the k-means tree of section 2.2)
# ---------------------------------------------------------------------------
def kmeans_pp(Y, k: int, u):
    """k-means++ seeding with the given uniforms u[k] in [0, 1)."""
    Y, u = _f64(Y), _f64(u)
    n, d = Y.shape
    C = np.empty((k, d))
    idx = np.empty(k, np.int32)
    lib().or_kmeans_pp(_p(Y), n, d, k, _p(u), _p(C), _p(idx, ctypes.c_int32))
    return C, idx


def kmeans_assign(Y, C):
    Y, C = _f64(Y), _f64(C)
    n, d = Y.shape
    a = np.empty(n, np.int32)
    cost = np.empty(n)
    lib().or_kmeans_assign(_p(Y), n, d, _p(C), C.shape[0], _p(a, ctypes.c_int32), _p(cost))
    return a, cost


def kmeans_update(Y, assign, k: int, cost=None):
    Y = _f64(Y)
    assign = _i32a(assign)
    n, d = Y.shape
    C = np.zeros((k, d))
    cnt = np.empty(k, np.int32)
    cst = None if cost is None else _f64(cost)
    lib().or_kmeans_update(_p(Y), n, d, _p(assign, ctypes.c_int32), k, _p(C), _p(cnt, ctypes.c_int32),
                           None if cst is None else _p(cst))
    return C, cnt


def kmeans(Y, k: int, u, iters: int = 25):
    """(centroids, assignment, inertia per iteration): k-means++ then Lloyd,
    stopping early when the assignment no longer changes."""
    C, _ = kmeans_pp(Y, k, u)
    a_prev, hist = None, []
    for _ in range(iters):
        a, cost = kmeans_assign(Y, C)
        hist.append(float(cost.sum()))
        if a_prev is not None and np.array_equal(a, a_prev):
            break
        C, _ = kmeans_update(Y, a, k, cost)
        a_prev = a
    a, cost = kmeans_assign(Y, C)
    return C, a, hist


MLP_SHAPES = (64, 256, 256, 1024)


def mlp_forward(X, params):
    """params: dict W1 b1 W2 b2 W3 b3 (rows = outputs).  Returns the cache."""
    X = _f64(X)
    B, din = X.shape
    W1, b1, W2, b2, W3, b3 = (_f64(params[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    h1, h2, out = W1.shape[0], W2.shape[0], W3.shape[0]
    c = {"A1": np.empty((B, h1)), "H1": np.empty((B, h1)), "A2": np.empty((B, h2)),
         "H2": np.empty((B, h2)), "Z": np.empty((B, out))}
    lib().or_mlp_forward(_p(X), B, din, h1, h2, out, _p(W1), _p(b1), _p(W2), _p(b2), _p(W3), _p(b3),
                         _p(c["A1"]), _p(c["H1"]), _p(c["A2"]), _p(c["H2"]), _p(c["Z"]))
    return c


def ce_loss(Z, labels):
    Z = _f64(Z)
    labels = _i32a(labels)
    P = np.empty_like(Z)
    loss = lib().or_ce_loss(_p(Z), Z.shape[0], Z.shape[1], _p(labels, ctypes.c_int32), _p(P))
    return loss, P


def mlp_backward(X, params, cache, P, labels):
    X = _f64(X)
    labels = _i32a(labels)
    B, din = X.shape
    W1, b1, W2, b2, W3, b3 = (_f64(params[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    h1, h2, out = W1.shape[0], W2.shape[0], W3.shape[0]
    g = {"W1": np.empty_like(W1), "b1": np.empty_like(b1), "W2": np.empty_like(W2), "b2": np.empty_like(b2),
         "W3": np.empty_like(W3), "b3": np.empty_like(b3)}
    lib().or_mlp_backward(_p(X), B, din, h1, h2, out, _p(W1), _p(b1), _p(W2), _p(b2), _p(W3), _p(b3),
                          _p(_f64(cache["A1"])), _p(_f64(cache["H1"])), _p(_f64(cache["A2"])),
                          _p(_f64(cache["H2"])), _p(_f64(P)), _p(labels, ctypes.c_int32),
                          _p(g["W1"]), _p(g["b1"]), _p(g["W2"]), _p(g["b2"]), _p(g["W3"]), _p(g["b3"]))
    return g
