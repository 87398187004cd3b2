"""irls_weights_noalloc: the IRLS entry point for callers that cannot allocate.

Callers that run inside a framework owning the whole device memory budget,
or that cannot afford the device-wide synchronisation of cudaFree, use this
variant; it keeps its reduction scratch in a fixed array inside the library.
This test calls it through the C ABI and checks it against irls_weights on
two calls in a row (the second with a different size, so stale scratch from
the first call would show up).  It lives in its own file so that pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest

import pts_inputs as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2006_11851_gb300 as pts  # noqa: E402

DEV = torch.device("cuda:0")


def _noalloc(L, d2, r, delta, W, E):
    L.irls_weights_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return L.irls_weights_noalloc(ctypes.c_void_p(d2.data_ptr()), d2.numel(), r, delta,
                                  ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_irls_weights_two_calls():
    L = pts.lib()
    for seed, n, r in [(21, 300_001, 0.8), (22, 4_099, 2.0)]:
        d2 = torch.from_numpy((P.SplitMix64(seed).uniform(n) * 3.0).astype(np.float32)).to(DEV)
        W_ref, E_ref = pts.irls_weights(d2, r, 1e-3)
        W = torch.full_like(d2, -1.0)
        E = torch.full((1,), -1.0, dtype=torch.float64, device=DEV)
        assert _noalloc(L, d2, r, 1e-3, W, E) == 0, L.pts_last_error()
        torch.cuda.synchronize()
        np.testing.assert_allclose(W.cpu().numpy(), W_ref.cpu().numpy(), rtol=2e-6)
        assert abs(E.item() / E_ref.item() - 1.0) < 1e-6


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = pts.lib()
    L.pts_last_error.restype = ctypes.c_char_p
    L.irls_weights_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    st = L.irls_weights_noalloc(ctypes.c_void_p(16), 8_388_609, 2.0, 1e-3, None, None, None)
    assert st == -1
    assert b"scratch limit" in L.pts_last_error()
