"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/pts.h declares, and rejects
bad arguments before launching anything."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        # function declarations (typedefs of function-pointer types are not functions)
        for m in re.finditer(r"^(?!\s*typedef\b)\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                             src, re.M):
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
    libpts.pts_wait_selftest.argtypes = [i, i, vp]
    assert libpts.pts_wait_selftest(0, 1, None) == -1


def test_python_binding_fails_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2006_11851_gb300 as pts
    with pytest.raises(TypeError):
        pts.nn_search(None, torch.zeros(16, 16, 3), 2)


def test_allocator_registration_on_host(libpts):
    libpts.pts_set_allocator.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    libpts.pts_live_allocations.restype = ctypes.c_longlong
    alloc_t = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    free_t = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    calls = []
    a = alloc_t(lambda n, s, u: calls.append(n) or None)
    fr = free_t(lambda p, s, u: calls.append(p))
    cast = ctypes.cast
    assert libpts.pts_set_allocator(cast(a, ctypes.c_void_p), None, None) == -1       # one of the two
    assert libpts.pts_set_allocator(None, cast(fr, ctypes.c_void_p), None) == -1
    assert libpts.pts_live_allocations() == 0                                        # nothing allocated here
    assert libpts.pts_set_allocator(cast(a, ctypes.c_void_p), cast(fr, ctypes.c_void_p), None) == 0
    assert libpts.pts_set_allocator(None, None, None) == 0                           # back to cudaMalloc
    assert calls == []
    libpts.synthesize_batched.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_void_p]
    assert libpts.synthesize_batched(None, 0, 1, 2.0, 1e-3, None) == -1


# index files: the header layout of persist.cu, written field by field in host byte order
_HEADER = "<8sII16ifddiifiiiii"


def _index_file(tables=None, **over):
    """Bytes of a consistent index file for a 12 x 12 exemplar, w = 4, d = 8, d_fast = 16 (every
    table zero), with header fields replaced by `over`.  `tables` adds a trained proposal
    ("prop": C = 4 clusters) and/or a k-means tree ("tree": a root with four leaves), given as
    {tag: int32 array} for their integer tables; tables left out are valid ones."""
    import struct
    tables = tables or {}
    N, C = 81, 4
    f = dict(He=12, We=12, w=4, D=48, N=N, d=8, da=12, d_fast=16, da_fast=20, ny=9, nx=9, ntiles=1,
             ktc=32, kf8=32, eig_iters=5, tc_parts=0, unorm2_max=1.0, var=0.9, eig_top=1.0)
    f.update(over)
    prop, tree = "prop" in tables, "tree" in tables
    head = struct.pack(_HEADER, over.get("magic", b"PTSINDEX"), over.get("version", 2),
                       over.get("order", 0x01020304), f["He"], f["We"], f["w"], f["D"], f["N"], f["d"], f["da"],
                       f["d_fast"], f["da_fast"], f["ny"], f["nx"], f["ntiles"], f["ktc"], f["kf8"],
                       f["eig_iters"], f["tc_parts"], f["unorm2_max"], f["var"], f["eig_top"],
                       int(prop), C if prop else 0, 1.2 if prop else 0.0, int(tree), 1 if tree else 0,
                       4 if tree else 0, 1 if tree else 0, over.get("C", 3))
    tcr = 256  # one tensor-core tile of 256 windows
    secs = [(b"EXEM", 4, 12 * 12 * 3), (b"EXE4", 16, 144), (b"MEAN", 4, 48), (b"BASI", 4, 128 * 48),
            (b"BAST", 4, 48 * 128), (b"EIGV", 8, 128), (b"ETIL", 4, 12 * 128), (b"EROW", 4, 81 * 12),
            (b"ENRM", 4, 128), (b"EFUL", 4, 64 * 128), (b"EFST", 4, 20 * 128), (b"ETCH", 2, tcr * 32),
            (b"ETC8", 1, tcr * 32), (b"F8SC", 4, 17), (b"UMAX", 4, 1)]
    ints = {}
    bounds = np.array([0, 20, 40, 60, N], np.int32)          # four ranges of windows
    if prop:
        assign = np.repeat(np.arange(C, dtype=np.int32), np.diff(bounds))
        ints.update({b"PASG": assign, b"PCNT": np.diff(bounds).astype(np.int32), b"POFF": bounds,
                     b"PMEM": np.arange(N, dtype=np.int32)})
        ints.update(tables["prop"])
        secs += [(b"PCEN", 4, C * 8), (b"PASG", 4, N), (b"PCNT", 4, C), (b"POFF", 4, C + 1), (b"PMEM", 4, N),
                 (b"PMED", 4, C), (b"PETC", 2, tcr * 32), (b"PMLP", 4, 256 * 64 + 256 + 256 * 256 + 256 + C * 256 + C)]
    if tree:
        ints.update({b"TCHI": np.array([-2, -3, -4, -5], np.int32), b"TLBG": bounds[:4], b"TLEN": bounds[1:],
                     b"TPRM": np.arange(N, dtype=np.int32)})
        ints.update(tables["tree"])
        secs += [(b"TCEN", 4, 4 * 8), (b"TCHI", 4, 4), (b"TLBG", 4, 4), (b"TLEN", 4, 4), (b"TPRM", 4, N)]

    def payload(t, e, c):
        if t in ints:
            a = np.ascontiguousarray(ints[t], dtype=np.int32)
            assert a.size == c
            return a.tobytes()
        return bytes(e * c)
    body = b"".join(t + struct.pack("<IQ", e, c) + payload(t, e, c) for t, e, c in secs)
    return head + body


def test_index_files_checked_on_host(libpts, tmp_path):
    libpts.pts_last_error.restype = ctypes.c_char_p
    libpts.pts_index_load.argtypes = [ctypes.c_char_p, ctypes.c_void_p]
    libpts.pts_index_save.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
    libpts.pts_index_destroy.argtypes = [ctypes.c_void_p]
    out = ctypes.c_void_p()

    def load(data):
        p = tmp_path / "idx.bin"
        p.write_bytes(data)
        rc = libpts.pts_index_load(str(p).encode(), ctypes.byref(out))
        return rc, libpts.pts_last_error().decode()

    assert libpts.pts_index_save(None, str(tmp_path / "x").encode()) == -1
    assert libpts.pts_index_load(str(tmp_path / "missing.bin").encode(), ctypes.byref(out)) == -1
    assert libpts.pts_index_load(None, ctypes.byref(out)) == -1
    good = _index_file()
    for data, msg in [(b"", "ends early"),
                      (_index_file(magic=b"NOTINDEX"), "not an index file"),
                      (_index_file(order=0x04030201), "byte order"),
                      (_index_file(version=1), "version"),
                      (_index_file(C=5), "channels"),
                      (_index_file(C=4), "window grid"),
                      (_index_file(D=49), "window grid"),
                      (_index_file(N=80), "window count"),
                      (_index_file(da=16), "PCA dimensions"),
                      (_index_file(ktc=48), "tile sizes"),
                      (good[:-1], "length"),
                      (good + b"\0", "length")]:
        rc, err = load(data)
        assert rc == -1 and msg in err, (msg, rc, err)
        assert not out.value
    # a consistent file passes every check and reaches the device: without a GPU that step fails
    rc, err = load(good)
    if rc == 0:  # pragma: no cover - only where a GPU is present
        libpts.pts_index_destroy(out)
    else:
        assert rc == -2 and "CUDA" in err, (rc, err)


def test_allocator_returning_null_fails_the_build_cleanly(libpts):
    """Host-side fault injection: a registered allocator that always fails.  The index build
    returns PTS_ERR_OOM at its first allocation, before any device work, and holds nothing."""
    class Params(ctypes.Structure):
        _fields_ = [("d", ctypes.c_int), ("var_frac", ctypes.c_double), ("max_iters", ctypes.c_int),
                    ("d_fast", ctypes.c_int), ("channels", ctypes.c_int)]
    libpts.pts_last_error.restype = ctypes.c_char_p
    libpts.pts_set_allocator.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    libpts.pts_live_allocations.restype = ctypes.c_longlong
    libpts.build_exemplar_index.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(Params), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    alloc_t = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    free_t = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    asked, freed = [], []
    a = alloc_t(lambda n, s, u: asked.append(n) or None)
    fr = free_t(lambda p, s, u: freed.append(p))
    assert libpts.pts_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(fr, ctypes.c_void_p), None) == 0
    try:
        out = ctypes.c_void_p()
        p = Params(16, 0.95, 0, 0, 0)
        rc = libpts.build_exemplar_index(ctypes.c_void_p(16), 32, 32, 8, ctypes.byref(p), None, ctypes.byref(out))
        assert rc == -3 and b"registered allocator failed" in libpts.pts_last_error()
        assert asked == [32 * 32 * 3 * 4] and freed == [] and not out.value
        assert libpts.pts_live_allocations() == 0
    finally:
        assert libpts.pts_set_allocator(None, None, None) == 0


def test_index_file_integer_tables_checked_on_host(libpts, tmp_path):
    """Cluster lists and tree links are indices the search kernels follow: one damaged value in
    a saved file must be refused on the host (PTS_ERR_INVALID_ARG) before any device work; the
    same file undamaged passes every check and reaches the device (which fails without a GPU)."""
    libpts.pts_last_error.restype = ctypes.c_char_p
    libpts.pts_index_load.argtypes = [ctypes.c_char_p, ctypes.c_void_p]
    libpts.pts_index_destroy.argtypes = [ctypes.c_void_p]
    out = ctypes.c_void_p()

    def load(data):
        p = tmp_path / "idx.bin"
        p.write_bytes(data)
        rc = libpts.pts_index_load(str(p).encode(), ctypes.byref(out))
        return rc, libpts.pts_last_error().decode()

    perm_dup = np.arange(81, dtype=np.int32)
    perm_dup[5] = 6
    perm_big = np.arange(81, dtype=np.int32)
    perm_big[80] = 81
    bad_assign = np.repeat(np.arange(4, dtype=np.int32), [20, 20, 20, 21])
    bad_assign[3] = 4
    moved = np.repeat(np.arange(4, dtype=np.int32), [20, 20, 20, 21])
    moved[3] = 1
    cases = [
        ({"tree": {b"TCHI": np.array([-2, -3, 7, -5], np.int32)}}, "child reference"),       # no node 7
        ({"tree": {b"TCHI": np.array([-2, 0, -4, -5], np.int32)}}, "child reference"),       # a cycle
        ({"tree": {b"TCHI": np.array([-2, -3, -4, -6], np.int32)}}, "child reference"),      # leaf 4 of 4
        ({"tree": {b"TLEN": np.array([20, 40, 60, 82], np.int32)}}, "leaf range"),
        ({"tree": {b"TLBG": np.array([0, 41, 40, 60], np.int32)}}, "leaf range"),
        ({"tree": {b"TPRM": perm_dup}}, "permutation"),
        ({"tree": {b"TPRM": perm_big}}, "permutation"),
        ({"prop": {b"POFF": np.array([0, 20, 40, 60, 80], np.int32)}}, "0 to N"),
        ({"prop": {b"POFF": np.array([0, 40, 20, 60, 81], np.int32)}}, "offsets or sizes"),
        ({"prop": {b"PCNT": np.array([20, 20, 20, 20], np.int32)}}, "offsets or sizes"),
        ({"prop": {b"PASG": bad_assign}}, "out of range"),
        ({"prop": {b"PMEM": perm_dup}}, "permutation"),
        ({"prop": {b"PASG": moved}}, "another cluster"),
    ]
    for tables, msg in cases:
        rc, err = load(_index_file(tables))
        assert rc == -1 and msg in err, (tables, msg, rc, err)
        assert not out.value
    for tables in ({"tree": {}}, {"prop": {}}, {"tree": {}, "prop": {}}):
        rc, err = load(_index_file(tables))
        if rc == 0:  # pragma: no cover - only where a GPU is present
            libpts.pts_index_destroy(out)
        else:
            assert rc == -2 and "CUDA" in err, (tables, rc, err)
