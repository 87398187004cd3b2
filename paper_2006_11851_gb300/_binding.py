"""ctypes binding of libpts (include/pts.h): argument marshalling only.

Tensors must be contiguous CUDA tensors on the current device; every call
runs on torch's current CUDA stream.  Errors from the library raise PtsError
with the library's message.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

MODES = {"exact": 0, "f16": 1, "fp8": 2, "proposal": 3, "kmtree": 4, "exact_tc": 5}  # pts_mode

_LOCK = threading.Lock()
_LIB = None


class PtsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pts status {status}: {msg}")
        self.status = status


class _IndexParams(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("var_frac", ctypes.c_double), ("max_iters", ctypes.c_int),
                ("d_fast", ctypes.c_int), ("channels", ctypes.c_int)]


class _IndexInfo(ctypes.Structure):
    _fields_ = [("He", ctypes.c_int), ("We", ctypes.c_int), ("w", ctypes.c_int), ("D", ctypes.c_int),
                ("N", ctypes.c_int), ("d", ctypes.c_int), ("da", ctypes.c_int), ("d_fast", ctypes.c_int),
                ("var_retained", ctypes.c_double), ("eig_top", ctypes.c_double),
                ("eig_iters", ctypes.c_int), ("unorm2_max", ctypes.c_float), ("channels", ctypes.c_int),
                ("exact_dims", ctypes.c_int), ("exact_var", ctypes.c_double)]


class _SearchStats(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_longlong), ("certified", ctypes.c_longlong),
                ("range_queries", ctypes.c_longlong), ("range_pairs", ctypes.c_longlong),
                ("brute_queries", ctypes.c_longlong), ("fallback_queries", ctypes.c_longlong),
                ("full_splits", ctypes.c_longlong), ("second_certified", ctypes.c_longlong),
                ("full_queries", ctypes.c_longlong), ("second_queries", ctypes.c_longlong)]


class _ProposalParams(ctypes.Structure):
    _fields_ = [("n_clusters", ctypes.c_int), ("kmeans_iters", ctypes.c_int), ("epochs", ctypes.c_int),
                ("batch", ctypes.c_int), ("lr", ctypes.c_float), ("weight_decay", ctypes.c_float),
                ("fallback_factor", ctypes.c_float), ("seed", ctypes.c_ulonglong)]


_vp = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_Dd = ctypes.c_double


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libpts (building it with nvcc if needed)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.lib_path()
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libpts is not built ({path}); run python -m paper_2006_11851_gb300.build")
        L = ctypes.CDLL(path)
        L.pts_last_error.restype = ctypes.c_char_p
        L.pts_version.restype = ctypes.c_char_p
        L.pca_fit.argtypes = [_vp, _I, _I, _I, _I, _Dd, _vp, _vp, _vp, ctypes.POINTER(_I), _vp]
        L.pca_fit_channels.argtypes = [_vp, _I, _I, _I, _I, _I, _Dd, _vp, _vp, _vp, ctypes.POINTER(_I), _vp]
        L.pts_scale_map.argtypes = [_I, _I, _Dd, _Dd, _vp, _vp]
        L.pts_scale_resample.argtypes = [_vp, _I, _I, _I, _I, _vp, _vp]
        L.pts_scale_guided_init.argtypes = [_vp, _vp, _I, _I, _vp, _vp, _I, _I, _I, _vp, _vp, _vp]
        L.pts_rgbs.argtypes = [_vp, _vp, _Dd, _I, _I, _vp, _vp]
        L.pts_rgb_of.argtypes = [_vp, _I, _I, _vp, _vp]
        L.build_exemplar_index.argtypes = [_vp, _I, _I, _I, ctypes.POINTER(_IndexParams), _vp,
                                           ctypes.POINTER(_vp)]
        L.pts_index_destroy.argtypes = [_vp]
        L.pts_index_destroy.restype = None
        L.pts_index_get_info.argtypes = [_vp, ctypes.POINTER(_IndexInfo)]
        L.pts_index_device_status.argtypes = [_vp, _vp]
        L.pts_index_set_tc_parts.argtypes = [_vp, _I]
        L.pts_index_set_exact_bound.argtypes = [_vp, _I]
        L.nn_search.argtypes = [_vp, _vp, _I, _I, _I, _I, _vp, _vp, _vp]
        L.pts_index_search_stats.argtypes = [_vp, ctypes.POINTER(_SearchStats), _vp]
        L.irls_weights.argtypes = [_vp, _I, _F, _F, _vp, _vp, _vp]
        L.m_step.argtypes = [_vp, _vp, _vp, _I, _I, _I, _vp, _vp]
        L.synthesize_level.argtypes = [_vp, _vp, _I, _I, _I, _I, _F, _F, _I, _vp, _vp]
        L.synthesize_level_hist.argtypes = [_vp, _vp, _I, _I, _I, _I, _F, _F, _I, _I, _vp, _vp]
        L.synthesize_level_async.argtypes = [_vp, _vp, _I, _I, _I, _I, _F, _F, _I, _vp, _vp]
        L.m_step_hist.argtypes = [_vp, _vp, _vp, _I, _I, _I, _I, _vp, _vp, _vp]
        L.pts_histogram_match.argtypes = [_vp, _vp, _I, _I, _I, _vp]
        L.pts_build_kmeans_tree.argtypes = [_vp, _I, _vp]
        L.pts_kmtree_info.argtypes = [_vp, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]
        L.pts_kmtree_export.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.pts_kmtree_last_leaves.argtypes = [_vp, _vp, _I, _vp]
        L.synthesize_level_converge.argtypes = [_vp, _vp, _I, _I, _I, _I, _F, _F, _I, _I, _vp,
                                                ctypes.POINTER(_I), _vp]
        L.pts_downsample2.argtypes = [_vp, _I, _I, _vp, _vp]
        L.pts_upsample2.argtypes = [_vp, _I, _I, _vp, _vp]
        _declare_optional(L)
        _LIB = L
        return L


def _declare_optional(L: ctypes.CDLL) -> None:
    """Entry points of the learned proposal and the test-support self-tests."""
    L.pts_project_queries.argtypes = [_vp, _vp, _I, _I, _I, _vp, _vp]
    L.pts_index_pca.argtypes = [_vp, _vp, _vp, _vp]
    L.pts_query_rows_f16.argtypes = [_vp, _vp, _I, _I, _I, _I, _vp, _vp, _vp]
    L.pts_train_proposal.argtypes = [_vp, _vp, _vp, _vp, _I, ctypes.POINTER(_ProposalParams), _vp, _vp]
    L.pts_kmeans.argtypes = [_vp, _I, _I, _I, _vp, _I, _vp, _vp, ctypes.POINTER(_I), _vp]
    L.pts_mlp_grad.argtypes = [_I, _vp, _vp, _vp, _I, _vp, ctypes.POINTER(_Dd), _vp]
    L.pts_gemm_selftest.argtypes = [_I, _I, _I, ctypes.POINTER(_Dd)]
    L.pts_tc_selftest.argtypes = [_I, _I, _I, ctypes.POINTER(_Dd), ctypes.POINTER(_Dd)]
    L.pts_proposal_info.argtypes = [_vp, ctypes.POINTER(_I), _vp, _vp]
    L.pts_proposal_top4.argtypes = [_vp, _vp, _I, _I, _I, _I, _vp, _vp]
    L.pts_launch_count.restype = ctypes.c_longlong
    L.pts_profile_enable.argtypes = [_I]
    L.pts_profile_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(_Dd), ctypes.POINTER(ctypes.c_longlong)]
    L.pts_fp32_fma_peak.argtypes = [_I, _I, _vp, ctypes.POINTER(_Dd), ctypes.POINTER(_Dd)]
    L.pts_wait_selftest.argtypes = [_I, _I, ctypes.POINTER(_I)]
    L.pts_index_save.argtypes = [_vp, ctypes.c_char_p]
    L.pts_index_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(_vp)]
    L.pts_set_allocator.argtypes = [_vp, _vp, _vp]
    L.pts_live_allocations.restype = ctypes.c_longlong


def _check(status: int) -> None:
    if status != 0:
        raise PtsError(status, lib().pts_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, dtype: torch.dtype, name: str, shape=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _image_of(index: "ExemplarIndex", img: torch.Tensor, name: str = "output"):
    """(H, W) of a float32 CUDA image whose channel count is the index's (3 RGB, 4 RGBS)."""
    _need(img, torch.float32, name)
    if img.dim() != 3 or img.shape[2] != index.C:
        raise ValueError(f"{name} must be H x W x {index.C} for this index")
    return img.shape[0], img.shape[1]


def _mode(mode) -> int:
    if isinstance(mode, str):
        return MODES[mode]
    return int(mode)


def pca_fit(exemplar: torch.Tensor, w: int, d: int, var_frac: float = 0.95):
    """(mean[D] f32, basis[d, D] f32, eigenvalues[d] f64, d_used) on the GPU; the exemplar is
    H x W x 3 (RGB) or H x W x 4 (RGBS), D = C w^2."""
    _need(exemplar, torch.float32, "exemplar")
    He, We, C = exemplar.shape
    if C not in (3, 4):
        raise ValueError("exemplar must be H x W x 3 or H x W x 4")
    D = C * w * w
    cap = d if d > 0 else 64
    mean = torch.empty(D, device=exemplar.device, dtype=torch.float32)
    basis = torch.empty(cap, D, device=exemplar.device, dtype=torch.float32)
    eig = torch.empty(cap, device=exemplar.device, dtype=torch.float64)
    dout = ctypes.c_int(0)
    _check(lib().pca_fit_channels(_ptr(exemplar), He, We, C, w, d, var_frac, _ptr(mean), _ptr(basis), _ptr(eig),
                                  ctypes.byref(dout), _stream()))
    k = dout.value
    return mean, basis[:k].contiguous(), eig[:k].contiguous(), k


class ExemplarIndex:
    """Owns a pts_index (build_exemplar_index); freed by close() or on GC.  The exemplar is
    H x W x 3 (RGB) or H x W x 4 (RGBS: the scale map as a fourth channel); every image searched
    or updated with the index has the same channel count."""

    def __init__(self, exemplar: torch.Tensor, w: int, d: int = 0, var_frac: float = 0.95,
                 max_iters: int = 0, d_fast: int = 0):
        L = lib()
        _need(exemplar, torch.float32, "exemplar")
        He, We, C = exemplar.shape
        if C not in (3, 4):
            raise ValueError("exemplar must be H x W x 3 (RGB) or H x W x 4 (RGBS)")
        self._h = ctypes.c_void_p()
        p = _IndexParams(int(d), float(var_frac), int(max_iters), int(d_fast), int(C))
        _check(L.build_exemplar_index(_ptr(exemplar), He, We, w, ctypes.byref(p), _stream(),
                                      ctypes.byref(self._h)))
        self.device = exemplar.device
        self._read_info()

    def _read_info(self) -> None:
        info = _IndexInfo()
        _check(lib().pts_index_get_info(self._h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _IndexInfo._fields_}
        self.w, self.N, self.d, self.D = info.w, info.N, info.d, info.D
        self.He, self.We, self.C = info.He, info.We, info.channels

    def save(self, path: str) -> None:
        """Write the index (PCA, search tables, and any trained proposal or k-means tree) to a file
        (pts_index_save; synchronises the device)."""
        _check(lib().pts_index_save(self.handle, os.fsencode(path)))

    @classmethod
    def load(cls, path: str) -> "ExemplarIndex":
        """An index read from a file written by save(), on the current CUDA device
        (pts_index_load; synchronises the device)."""
        L = lib()
        self = cls.__new__(cls)
        self._h = ctypes.c_void_p()
        _check(L.pts_index_load(os.fsencode(path), ctypes.byref(self._h)))
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._read_info()
        return self

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("index is closed")
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().pts_index_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_queries(self, Ho: int, Wo: int, stride: int = 2) -> int:
        return ((Ho - self.w) // stride + 1) * ((Wo - self.w) // stride + 1)

    def search_stats(self) -> dict:
        s = _SearchStats()
        _check(lib().pts_index_search_stats(self.handle, ctypes.byref(s), _stream()))
        return {f: getattr(s, f) for f, _ in _SearchStats._fields_}

    def device_status(self) -> None:
        _check(lib().pts_index_device_status(self.handle, _stream()))

    def set_tc_parts(self, parts: int) -> None:
        """Exemplar split of the tensor-core searches (0 = automatic); results do not depend on it."""
        _check(lib().pts_index_set_tc_parts(self.handle, int(parts)))

    def set_exact_bound(self, fast) -> None:
        """Components of the exact search's PCA bound: 0 / False (the default) the first d, then
        d_fast for what that bound leaves uncertified; 1 / True d_fast only; 2 the first d only.
        The certified results do not depend on it."""
        _check(lib().pts_index_set_exact_bound(self.handle, int(fast)))
        self._read_info()


def index_save(index: ExemplarIndex, path: str) -> None:
    """pts_index_save: ExemplarIndex.save."""
    index.save(path)


def index_load(path: str) -> ExemplarIndex:
    """pts_index_load: ExemplarIndex.load."""
    return ExemplarIndex.load(path)


def live_allocations() -> int:
    """Device allocations the library holds (pts_live_allocations)."""
    return int(lib().pts_live_allocations())


_ALLOC_FNS = None


def set_allocator(alloc=None, free=None) -> None:
    """Route the library's device allocations through alloc(bytes) -> int pointer and free(ptr)
    (pts_set_allocator); with no arguments, back to cudaMalloc / cudaFree.  Allowed only while
    the library holds no device memory.  use_torch_allocator() installs torch's caching
    allocator."""
    global _ALLOC_FNS
    L = lib()
    if alloc is None and free is None:
        _check(L.pts_set_allocator(None, None, None))
        _ALLOC_FNS = None
        return
    if alloc is None or free is None:
        raise ValueError("give both alloc and free, or neither")
    alloc_t = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    free_t = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

    def _alloc(nbytes, stream, user):
        try:
            return alloc(int(nbytes)) or None
        except Exception:  # an exception must not cross into C: report failure instead
            return None

    def _free(ptr, stream, user):
        try:
            free(int(ptr))
        except Exception:
            pass

    fns = (alloc_t(_alloc), free_t(_free))  # kept alive while registered
    _check(L.pts_set_allocator(ctypes.cast(fns[0], _vp), ctypes.cast(fns[1], _vp), None))
    _ALLOC_FNS = fns


def use_torch_allocator() -> None:
    """Serve the library's device memory from torch's CUDA caching allocator (current device)."""
    set_allocator(lambda n: torch.cuda.caching_allocator_alloc(n), torch.cuda.caching_allocator_delete)


def build_exemplar_index(exemplar: torch.Tensor, w: int, d: int = 0, var_frac: float = 0.95,
                         max_iters: int = 0) -> ExemplarIndex:
    return ExemplarIndex(exemplar, w, d, var_frac, max_iters)


def nn_search(index: ExemplarIndex, output: torch.Tensor, stride: int = 2, mode="exact",
              nn_out: torch.Tensor | None = None, d2_out: torch.Tensor | None = None):
    """(nn int32[Q], dist2 float32[Q]) of every query window of `output`."""
    Ho, Wo = _image_of(index, output)
    Q = index.num_queries(Ho, Wo, stride) if (Ho - index.w) % stride == 0 and (Wo - index.w) % stride == 0 else 0
    if nn_out is None:
        nn_out = torch.empty(max(Q, 1), device=output.device, dtype=torch.int32)
    if d2_out is None:
        d2_out = torch.empty(max(Q, 1), device=output.device, dtype=torch.float32)
    _check(lib().nn_search(index.handle, _ptr(output), Ho, Wo, stride, _mode(mode), _ptr(nn_out),
                           _ptr(d2_out), _stream()))
    return nn_out[:Q], d2_out[:Q]


def irls_weights(dist2: torch.Tensor, r: float = 2.0, delta: float = 1e-3):
    """(weights float32[Q], energy float64 scalar tensor)."""
    _need(dist2, torch.float32, "dist2")
    W = torch.empty_like(dist2)
    E = torch.empty(1, device=dist2.device, dtype=torch.float64)
    _check(lib().irls_weights(_ptr(dist2), dist2.numel(), r, delta, _ptr(W), _ptr(E), _stream()))
    return W, E[0]


def m_step(index: ExemplarIndex, nn: torch.Tensor, weights: torch.Tensor | None, Ho: int, Wo: int,
           stride: int = 2, out: torch.Tensor | None = None) -> torch.Tensor:
    _need(nn, torch.int32, "nn")
    if weights is not None:
        _need(weights, torch.float32, "weights")
    if out is None:
        if index.C != 3:
            raise ValueError("an RGBS M-step updates R, G and B of an existing image: pass out")
        out = torch.empty(Ho, Wo, 3, device=nn.device, dtype=torch.float32)
    _need(out, torch.float32, "out", (Ho, Wo, index.C))
    Q = index.num_queries(Ho, Wo, stride)
    if nn.numel() != Q or (weights is not None and weights.numel() != Q):
        raise ValueError("nn/weights must have one entry per query")
    _check(lib().m_step(index.handle, _ptr(nn), _ptr(weights), Ho, Wo, stride, _ptr(out), _stream()))
    return out


def synthesize_level(index: ExemplarIndex, output: torch.Tensor, iters: int, r: float = 2.0,
                     delta: float = 1e-3, mode="exact", stride: int = 2, hist_bins: int = 0) -> np.ndarray:
    """Runs EM in place on `output`; returns the iters + 1 energies (host).  hist_bins > 0 uses
    the M-step with the histogram weights of Eq. 9 (synthesize_level_hist)."""
    Ho, Wo = _image_of(index, output)
    E = np.zeros(iters + 1, dtype=np.float64)
    if hist_bins:
        _check(lib().synthesize_level_hist(index.handle, _ptr(output), Ho, Wo, stride, iters, r, delta, _mode(mode),
                                           int(hist_bins), E.ctypes.data_as(ctypes.c_void_p), _stream()))
    else:
        _check(lib().synthesize_level(index.handle, _ptr(output), Ho, Wo, stride, iters, r, delta,
                                      _mode(mode), E.ctypes.data_as(ctypes.c_void_p), _stream()))
    return E


def synthesize_level_async(index: ExemplarIndex, output: torch.Tensor, iters: int, r: float = 2.0,
                           delta: float = 1e-3, mode="exact", stride: int = 2,
                           energy: torch.Tensor | None = None) -> torch.Tensor:
    """synthesize_level without the closing synchronisation: returns the iters + 1 energies as a
    device float64 tensor; kernel errors wait in the device status (index.device_status())."""
    Ho, Wo = _image_of(index, output)
    if energy is None:
        energy = torch.empty(iters + 1, device=output.device, dtype=torch.float64)
    _need(energy, torch.float64, "energy", (iters + 1,))
    _check(lib().synthesize_level_async(index.handle, _ptr(output), Ho, Wo, stride, iters, r, delta, _mode(mode),
                                        _ptr(energy), _stream()))
    return energy


def synthesize_level_converge(index: ExemplarIndex, output: torch.Tensor, max_iters: int, r: float = 0.8,
                              delta: float = 1e-3, mode="exact", stride: int = 2, hist_bins: int = 0):
    """EM in place on `output` until the searched windows repeat (or max_iters M-steps);
    returns (energies [iters + 1] on the host, iters)."""
    Ho, Wo = _image_of(index, output)
    E = np.zeros(max_iters + 1, dtype=np.float64)
    it = _I(0)
    _check(lib().synthesize_level_converge(index.handle, _ptr(output), Ho, Wo, stride, int(max_iters), r, delta,
                                           _mode(mode), int(hist_bins), E.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.byref(it), _stream()))
    return E[:it.value + 1], it.value


def m_step_hist(index: ExemplarIndex, nn: torch.Tensor, weights: torch.Tensor | None, current: torch.Tensor,
                nbins: int, stride: int = 2, out: torch.Tensor | None = None) -> torch.Tensor:
    """The M-step with the weights of Eq. 9, histograms of `current` against the exemplar's (RGB
    indices only)."""
    if index.C != 3:
        raise ValueError("histogram weights need an RGB index")
    _need(nn, torch.int32, "nn")
    _need(current, torch.float32, "current")
    if weights is not None:
        _need(weights, torch.float32, "weights")
    Ho, Wo, _ = current.shape
    if out is None:
        out = torch.empty_like(current)
    _need(out, torch.float32, "out", (Ho, Wo, 3))
    Q = index.num_queries(Ho, Wo, stride)
    if nn.numel() != Q or (weights is not None and weights.numel() != Q):
        raise ValueError("nn/weights must have one entry per query")
    _check(lib().m_step_hist(index.handle, _ptr(nn), _ptr(weights), Ho, Wo, stride, int(nbins), _ptr(current),
                             _ptr(out), _stream()))
    return out


def histogram_match(index: ExemplarIndex, image: torch.Tensor, nbins: int) -> torch.Tensor:
    """Maps each channel of `image` (in place) onto the exemplar's histogram; returns it."""
    _need(image, torch.float32, "image")
    H, W, _ = image.shape
    _check(lib().pts_histogram_match(index.handle, _ptr(image), H, W, int(nbins), _stream()))
    return image


def downsample2(img: torch.Tensor) -> torch.Tensor:
    _need(img, torch.float32, "img")
    H, W, _ = img.shape
    out = torch.empty((H + 1) // 2, (W + 1) // 2, 3, device=img.device, dtype=torch.float32)
    _check(lib().pts_downsample2(_ptr(img), H, W, _ptr(out), _stream()))
    return out


def upsample2(img: torch.Tensor) -> torch.Tensor:
    _need(img, torch.float32, "img")
    H, W, _ = img.shape
    out = torch.empty(2 * H, 2 * W, 3, device=img.device, dtype=torch.float32)
    _check(lib().pts_upsample2(_ptr(img), H, W, _ptr(out), _stream()))
    return out


# ---------------------------------------------------------------------------
# learned cluster proposal
# ---------------------------------------------------------------------------
def project_queries(index: ExemplarIndex, output: torch.Tensor, stride: int = 2) -> torch.Tensor:
    """PCA coordinates [Q, d] of every query window of `output`."""
    Ho, Wo = _image_of(index, output)
    y = torch.empty(index.num_queries(Ho, Wo, stride), index.d, device=output.device, dtype=torch.float32)
    _check(lib().pts_project_queries(index.handle, _ptr(output), Ho, Wo, stride, _ptr(y), _stream()))
    return y


def index_pca(index: ExemplarIndex) -> tuple[torch.Tensor, torch.Tensor]:
    """(mean [D], basis [d_fast, D]) of the index's PCA, float32 on its device."""
    mean = torch.empty(index.D, device=index.device, dtype=torch.float32)
    basis = torch.empty(index.info["d_fast"], index.D, device=index.device, dtype=torch.float32)
    _check(lib().pts_index_pca(index.handle, _ptr(mean), _ptr(basis), _stream()))
    return mean, basis


def query_rows_f16(index: ExemplarIndex, output: torch.Tensor, stride: int = 2,
                   tensor_cores: bool = True) -> tuple[torch.Tensor, torch.Tensor]:
    """(rows [Q, K] float16, ||u||^2 [Q] float32): the FP16 search's query rows (y, r, 1, 1, 1,
    0, ...), projected on the tensor cores (the search's own route) or by the FP32 SIMT kernel."""
    Ho, Wo = _image_of(index, output)
    Q = index.num_queries(Ho, Wo, stride)
    K = (index.info["d_fast"] + 4 + 15) // 16 * 16
    rows = torch.empty(Q, K, device=output.device, dtype=torch.float16)
    norm = torch.empty(Q, device=output.device, dtype=torch.float32)
    _check(lib().pts_query_rows_f16(index.handle, _ptr(output), Ho, Wo, stride, int(bool(tensor_cores)), _ptr(rows),
                                    _ptr(norm), _stream()))
    return rows, norm


def train_proposal(index: ExemplarIndex, y: torch.Tensor, nn: torch.Tensor, d2: torch.Tensor, n_clusters: int = 1024,
                   kmeans_iters: int = 25, epochs: int = 8, batch: int = 4096, lr: float = 1e-3,
                   weight_decay: float = 1e-4, fallback_factor: float = 1.2, seed: int = 0) -> np.ndarray:
    """Builds the proposal of mode "proposal" on `index`; returns the per-epoch loss."""
    _need(y, torch.float32, "y")
    _need(nn, torch.int32, "nn")
    _need(d2, torch.float32, "d2")
    n = y.shape[0]
    if y.shape[1] != index.d or nn.numel() != n or d2.numel() != n:
        raise ValueError("y must be [n, d] with one nn and d2 per row")
    p = _ProposalParams(n_clusters, kmeans_iters, epochs, batch, lr, weight_decay, fallback_factor, seed)
    loss = np.zeros(max(epochs, 1))
    _check(lib().pts_train_proposal(index.handle, _ptr(y), _ptr(nn), _ptr(d2), n, ctypes.byref(p),
                                    loss.ctypes.data_as(ctypes.c_void_p), _stream()))
    return loss


def proposal_top4(index: ExemplarIndex, output: torch.Tensor, stride: int = 2, fused: bool = True) -> torch.Tensor:
    """[Q, 4] int32: the network's 4 best-ranked clusters per query (fused kernel or GEMM path)."""
    Ho, Wo = _image_of(index, output)
    top = torch.empty(index.num_queries(Ho, Wo, stride), 4, dtype=torch.int32, device=output.device)
    _check(lib().pts_proposal_top4(index.handle, _ptr(output), Ho, Wo, stride, 1 if fused else 0, _ptr(top), _stream()))
    return top


def proposal_info(index: ExemplarIndex):
    """(cluster sizes [C], cluster of each exemplar window [N]) of the index's trained proposal."""
    L = lib()
    C = ctypes.c_int(0)
    _check(L.pts_proposal_info(index.handle, ctypes.byref(C), None, None))
    sizes = np.zeros(C.value, dtype=np.int32)
    assign = np.zeros(index.N, dtype=np.int32)
    _check(L.pts_proposal_info(index.handle, ctypes.byref(C), sizes.ctypes.data_as(ctypes.c_void_p),
                               assign.ctypes.data_as(ctypes.c_void_p)))
    return sizes, assign


def kmeans(points: torch.Tensor, k: int, u: np.ndarray, iters: int = 25):
    """(centroids [k, d], assignment [n], Lloyd iterations) on the GPU."""
    _need(points, torch.float32, "points")
    n, d = points.shape
    u = np.ascontiguousarray(u, dtype=np.float64)
    C = torch.empty(k, d, device=points.device, dtype=torch.float32)
    a = torch.empty(n, device=points.device, dtype=torch.int32)
    it = ctypes.c_int(0)
    _check(lib().pts_kmeans(_ptr(points), n, d, k, u.ctypes.data_as(ctypes.c_void_p), iters, _ptr(C), _ptr(a),
                            ctypes.byref(it), _stream()))
    return C, a, it.value


def mlp_grad(C: int, params: torch.Tensor, X: torch.Tensor, labels: torch.Tensor):
    """(gradients, loss) of one forward/backward pass of the proposal network."""
    _need(params, torch.float32, "params")
    _need(X, torch.float32, "X")
    _need(labels, torch.int32, "labels")
    g = torch.empty_like(params)
    loss = ctypes.c_double(0.0)
    _check(lib().pts_mlp_grad(C, _ptr(params), _ptr(X), _ptr(labels), X.shape[0], _ptr(g), ctypes.byref(loss),
                              _stream()))
    return g, loss.value


def gemm_selftest(M: int, N: int, K: int) -> float:
    e = ctypes.c_double(0.0)
    _check(lib().pts_gemm_selftest(M, N, K, ctypes.byref(e)))
    return e.value


def wait_selftest(arrive: bool, abortable: bool = False) -> tuple[int, bool]:
    """(status, completed) of pts_wait_selftest: status 0 when the phase completed, the library's
    PTS_ERR_TIMEOUT (-5) when the bounded wait gave up."""
    done = ctypes.c_int(0)
    st = lib().pts_wait_selftest(1 if arrive else 0, 1 if abortable else 0, ctypes.byref(done))
    return int(st), bool(done.value)


def fp32_fma_peak(iters: int = 20000, reps: int = 5) -> tuple[float, float]:
    """(TFLOP/s, ms) of the best of `reps` launches of the FP32 FMA probe on the current stream."""
    tf, ms = _Dd(), _Dd()
    _check(lib().pts_fp32_fma_peak(int(iters), int(reps), _stream(), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def build_kmeans_tree(index: ExemplarIndex, iters: int = 10) -> dict:
    """Builds the k = 4 hierarchical k-means tree of mode "kmtree"; returns its shape."""
    _check(lib().pts_build_kmeans_tree(index.handle, int(iters), _stream()))
    return kmtree_info(index)


def kmtree_info(index: ExemplarIndex) -> dict:
    a, b, c = _I(), _I(), _I()
    _check(lib().pts_kmtree_info(index.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"internal": a.value, "leaves": b.value, "depth": c.value}


def kmtree_export(index: ExemplarIndex) -> dict:
    """The tree as numpy arrays: child [internal, 4], leaf_begin, leaf_end, perm, cent [internal, 4, d]."""
    info = kmtree_info(index)
    ni, nl, d, N = info["internal"], info["leaves"], index.d, index.info["N"]
    child = np.zeros((ni, 4), dtype=np.int32)
    lb, le = np.zeros(nl, dtype=np.int32), np.zeros(nl, dtype=np.int32)
    perm = np.zeros(N, dtype=np.int32)
    cent = np.zeros((ni, 4, d), dtype=np.float32)
    _check(lib().pts_kmtree_export(index.handle, child.ctypes.data_as(ctypes.c_void_p), lb.ctypes.data_as(ctypes.c_void_p),
                                   le.ctypes.data_as(ctypes.c_void_p), perm.ctypes.data_as(ctypes.c_void_p),
                                   cent.ctypes.data_as(ctypes.c_void_p), _stream()))
    return {"child": child, "leaf_begin": lb, "leaf_end": le, "perm": perm, "cent": cent}


def kmtree_last_leaves(index: ExemplarIndex, Q: int) -> np.ndarray:
    out = np.zeros(Q, dtype=np.int32)
    _check(lib().pts_kmtree_last_leaves(index.handle, out.ctypes.data_as(ctypes.c_void_p), int(Q), _stream()))
    return out


# ---------------------------------------------------------------------------
# the scale map (section 1, Eqs. 1-3) and its use in synthesis (section 3)
# ---------------------------------------------------------------------------
def scale_map(h: int, w: int, slant_deg: float, tilt_deg: float, device=None) -> torch.Tensor:
    """Eq. 3's local scale of every pixel of an h x w image: float64 [h, w] on the GPU."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    S = torch.empty(h, w, device=dev, dtype=torch.float64)
    _check(lib().pts_scale_map(int(h), int(w), float(slant_deg), float(tilt_deg), _ptr(S), _stream()))
    return S


def scale_resample(S: torch.Tensor, Ho: int, Wo: int) -> torch.Tensor:
    """The map S resampled bilinearly (corner-aligned) to Ho x Wo: float64 [Ho, Wo]."""
    _need(S, torch.float64, "S")
    out = torch.empty(Ho, Wo, device=S.device, dtype=torch.float64)
    _check(lib().pts_scale_resample(_ptr(S), S.shape[0], S.shape[1], int(Ho), int(Wo), _ptr(out), _stream()))
    return out


def scale_guided_init(exemplar: torch.Tensor, S_z: torch.Tensor, S_x: torch.Tensor, u: torch.Tensor,
                      nbins: int = 64):
    """(initial output Ho x Wo x 3 float32, source pixel per output pixel int32 [Ho, Wo]): every
    output pixel copies an exemplar pixel of its scale bin."""
    _need(exemplar, torch.float32, "exemplar")
    _need(S_z, torch.float64, "S_z")
    _need(S_x, torch.float64, "S_x")
    _need(u, torch.float64, "u")
    He, We, C = exemplar.shape
    Ho, Wo = S_x.shape
    if C != 3 or tuple(S_z.shape) != (He, We) or tuple(u.shape) != (Ho, Wo):
        raise ValueError("exemplar H x W x 3, S_z H x W, u of S_x's shape")
    out = torch.empty(Ho, Wo, 3, device=exemplar.device, dtype=torch.float32)
    src = torch.empty(Ho, Wo, device=exemplar.device, dtype=torch.int32)
    _check(lib().pts_scale_guided_init(_ptr(exemplar), _ptr(S_z), He, We, _ptr(S_x), _ptr(u), Ho, Wo, int(nbins),
                                       _ptr(out), _ptr(src), _stream()))
    return out, src


def rgbs(rgb: torch.Tensor, S: torch.Tensor, lam: float = 1.0) -> torch.Tensor:
    """The H x W x 4 image (R, G, B, lam S)."""
    _need(rgb, torch.float32, "rgb")
    _need(S, torch.float64, "S")
    H, W, C = rgb.shape
    if C != 3 or tuple(S.shape) != (H, W):
        raise ValueError("rgb H x W x 3 and S H x W")
    out = torch.empty(H, W, 4, device=rgb.device, dtype=torch.float32)
    _check(lib().pts_rgbs(_ptr(rgb), _ptr(S), float(lam), H, W, _ptr(out), _stream()))
    return out


def rgb_of(img: torch.Tensor) -> torch.Tensor:
    """R, G and B of an H x W x 4 image."""
    _need(img, torch.float32, "img")
    H, W, C = img.shape
    if C != 4:
        raise ValueError("img must be H x W x 4")
    out = torch.empty(H, W, 3, device=img.device, dtype=torch.float32)
    _check(lib().pts_rgb_of(_ptr(img), H, W, _ptr(out), _stream()))
    return out
