"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/pts.h declares, and rejects
bad arguments before launching anything."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, re.M):
            name = m.group(1)
            if name not in ("if", "while", "sizeof", "defined"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpts():
    from paper_2006_11851_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pca_fit", "build_exemplar_index", "nn_search", "m_step", "synthesize_level"):
        assert must in names


def test_every_declared_symbol_is_exported(libpts):
    missing = [n for n in _declared() if not hasattr(libpts, n)]
    assert not missing, missing


def test_bad_arguments_rejected_on_host(libpts):
    libpts.pts_last_error.restype = ctypes.c_char_p
    libpts.nn_search.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] * 4 + [ctypes.c_void_p] * 3
    assert libpts.nn_search(None, None, 16, 16, 2, 0, None, None, None) == -1
    assert b"null" in libpts.pts_last_error()
    libpts.pca_fit.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p]
    assert libpts.pca_fit(None, 8, 8, 4, 2, 0.9, None, None, None, None, None) == -1
    libpts.irls_weights.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert libpts.irls_weights(ctypes.c_void_p(16), 10, 3.0, 1e-3, None, None, None) == -1
    libpts.synthesize_level.argtypes = [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int] * 4 + \
        [ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    assert libpts.synthesize_level(None, None, 16, 16, 2, 1, 2.0, 1e-3, 0, None, None) == -1
    vp, i, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    libpts.synthesize_level_async.argtypes = [vp, vp, i, i, i, i, f, f, i, vp, vp]
    assert libpts.synthesize_level_async(None, None, 16, 16, 2, 1, 2.0, 1e-3, 0, None, None) == -1
    libpts.synthesize_level_hist.argtypes = [vp, vp, i, i, i, i, f, f, i, i, vp, vp]
    assert libpts.synthesize_level_hist(None, None, 16, 16, 2, 1, 2.0, 1e-3, 0, 32, None, None) == -1
    libpts.synthesize_level_converge.argtypes = [vp, vp, i, i, i, i, f, f, i, i, vp, vp, vp]
    assert libpts.synthesize_level_converge(None, None, 16, 16, 2, 5, 0.8, 1e-3, 0, 0, None, None, None) == -1
    libpts.m_step_hist.argtypes = [vp, vp, vp, i, i, i, i, vp, vp, vp]
    assert libpts.m_step_hist(None, None, None, 16, 16, 2, 32, None, None, None) == -1
    libpts.pts_histogram_match.argtypes = [vp, vp, i, i, i, vp]
    assert libpts.pts_histogram_match(None, None, 16, 16, 32, None) == -1
    libpts.pts_build_kmeans_tree.argtypes = [vp, i, vp]
    assert libpts.pts_build_kmeans_tree(None, 10, None) == -1
    libpts.pts_kmtree_info.argtypes = [vp, vp, vp, vp]
    assert libpts.pts_kmtree_info(None, None, None, None) == -1
    libpts.pts_index_set_tc_parts.argtypes = [vp, i]
    assert libpts.pts_index_set_tc_parts(None, 1) == -1
    libpts.pts_fp32_fma_peak.argtypes = [i, i, vp, vp, vp]
    assert libpts.pts_fp32_fma_peak(0, 1, None, None, None) == -1


def test_python_binding_fails_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2006_11851_gb300 as pts
    with pytest.raises(TypeError):
        pts.nn_search(None, torch.zeros(16, 16, 3), 2)
