"""Index files, the allocator hook, the one-call batched form and device-memory bookkeeping on
the GPU, through the C ABI:

  - an index saved and loaded back (with a trained proposal and the k-means tree) searches
    exactly like the original in every mode, and a whole EM level on it gives the same image and
    energies; saving the loaded index writes the same bytes;
  - a file whose section does not match its header is refused;
  - with torch's caching allocator registered, the library allocates through it and returns
    everything on destroy, and results do not change (in a child process, so the registration
    meets a library that holds no memory);
  - synthesize_batched equals the captured batch it wraps;
  - building, training and destroying an index leaves no library allocation behind.

These exercise host-side bookkeeping over kernels the other GPU tests check against the oracle,
so the file is collected after them.
"""
import filecmp
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import pts_inputs as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2006_11851_gb300 as pts  # noqa: E402
from paper_2006_11851_gb300 import batched  # noqa: E402
from paper_2006_11851_gb300.proposal import collect_pairs, subsample  # noqa: E402
from paper_2006_11851_gb300.pyramid import PyramidIndex  # noqa: E402

DEV = torch.device("cuda:0")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODES = ["exact", "f16", "fp8", "proposal", "kmtree"]


def _t(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(DEV)


@pytest.fixture(scope="module")
def level():
    """Two-level pyramid (128² exemplar, windows 16/8, outputs 128/256); the fine index gets a
    proposal of 64 clusters and the k-means tree; X is a mid-synthesis image of the fine level."""
    Z = P.synthetic_exemplar(5, 128, 4.0)
    pidx = PyramidIndex(_t(Z), [16, 8], d=64)
    z0 = pidx.exemplars[0].cpu().numpy()
    init = lambda s: _t(P.random_patch_init(z0, 128, 128, 16, s))  # noqa: E731
    y, nn, d2 = collect_pairs(pidx, 1, init, range(2), iters=3)
    y, nn, d2 = subsample(y, nn, d2, 100_000)
    pts.train_proposal(pidx.indices[1], y, nn, d2, n_clusters=64, epochs=2, batch=4096, seed=2)
    pts.build_kmeans_tree(pidx.indices[1], 10)
    X = init(40)
    pts.synthesize_level(pidx.indices[0], X, 3, mode="exact")
    X = pts.upsample2(X)
    pts.synthesize_level(pidx.indices[1], X, 2, mode="exact")
    yield pidx, X
    pidx.close()


def test_loaded_index_searches_identically(level, tmp_path):
    pidx, X = level
    ix = pidx.indices[1]
    path = str(tmp_path / "fine.ptsidx")
    ix.save(path)
    iy = pts.ExemplarIndex.load(path)
    try:
        assert iy.info == ix.info
        for mode in MODES:
            nn_a, d2_a = pts.nn_search(ix, X, 2, mode)
            nn_b, d2_b = pts.nn_search(iy, X, 2, mode)
            assert torch.equal(nn_a, nn_b) and torch.equal(d2_a, d2_b), mode
        Xa, Xb = X.clone(), X.clone()
        Ea = pts.synthesize_level(ix, Xa, 3, mode="f16")
        Eb = pts.synthesize_level(iy, Xb, 3, mode="f16")
        assert torch.equal(Xa, Xb) and list(Ea) == list(Eb)
        sa, aa = pts.proposal_info(ix)
        sb, ab = pts.proposal_info(iy)
        assert np.array_equal(sa, sb) and np.array_equal(aa, ab)
        ta, tb = pts.kmtree_export(ix), pts.kmtree_export(iy)
        assert ta.keys() == tb.keys() and all(np.array_equal(ta[k], tb[k]) for k in ta)
        path2 = str(tmp_path / "again.ptsidx")
        iy.save(path2)
        assert filecmp.cmp(path, path2, shallow=False)
    finally:
        iy.close()


def test_file_with_a_foreign_section_is_refused(level, tmp_path):
    pidx, _ = level
    path = str(tmp_path / "coarse.ptsidx")
    pidx.indices[0].save(path)
    data = bytearray(open(path, "rb").read())
    k = data.find(b"MEAN")
    assert k > 0
    data[k:k + 4] = b"MEAM"
    bad = tmp_path / "bad.ptsidx"
    bad.write_bytes(bytes(data))
    with pytest.raises(pts.PtsError, match="section"):
        pts.ExemplarIndex.load(str(bad))
    with pytest.raises(pts.PtsError, match="length"):
        (tmp_path / "short.ptsidx").write_bytes(bytes(data[:-3]))
        pts.ExemplarIndex.load(str(tmp_path / "short.ptsidx"))


def test_destroy_returns_every_allocation():
    before = pts.live_allocations()
    Z = P.synthetic_exemplar(7, 96, 4.0)
    pidx = PyramidIndex(_t(Z), [16, 8], d=64)
    z0 = pidx.exemplars[0].cpu().numpy()
    init = lambda s: _t(P.random_patch_init(z0, 96, 96, 16, s))  # noqa: E731
    y, nn, d2 = collect_pairs(pidx, 1, init, range(1), iters=2)
    pts.train_proposal(pidx.indices[1], y, nn, d2, n_clusters=64, epochs=1, batch=4096, seed=3)
    pts.build_kmeans_tree(pidx.indices[1], 5)
    assert pts.live_allocations() > before
    pidx.close()
    assert pts.live_allocations() == before


_CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np, torch
    import pts_inputs as P
    import paper_2006_11851_gb300 as pts
    dev = torch.device("cuda:0")
    Z = torch.from_numpy(P.synthetic_exemplar(9, 64, 3.0)).to(dev)
    X0 = torch.from_numpy(P.random_patch_init(Z.cpu().numpy(), 128, 128, 8, 1)).to(dev)

    def run():
        ix = pts.ExemplarIndex(Z, 8, d=24)
        X = X0.clone()
        E = pts.synthesize_level(ix, X, 2, mode="f16")
        nn, d2 = pts.nn_search(ix, X, 2, "exact")
        live = pts.live_allocations()
        ix.close()
        return X.cpu(), list(E), nn.cpu(), d2.cpu(), live

    assert pts.live_allocations() == 0
    ref = run()
    assert pts.live_allocations() == 0
    calls = {{"alloc": 0, "free": 0}}

    def alloc(n):
        calls["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(n)

    def free(p):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(p)

    pts.set_allocator(alloc, free)
    held0 = torch.cuda.memory_allocated()
    got = run()
    assert calls["alloc"] > 0 and calls["alloc"] == calls["free"], calls
    assert torch.cuda.memory_allocated() == held0
    pts.set_allocator()
    assert torch.equal(ref[0], got[0]) and ref[1] == got[1]
    assert torch.equal(ref[2], got[2]) and torch.equal(ref[3], got[3]) and ref[4] == got[4] > 0
    print("allocator ok", calls)
""")


def test_torch_allocator_serves_the_library():
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "allocator ok" in r.stdout


def test_synthesize_batched_equals_the_batch():
    specs = batched.job_specs(6, seed=3, max_exemplar=160, max_output=288)
    b = batched.Batch(specs, mode="f16", iters=2, n_streams=3)
    try:
        b.reset()
        b.run()
        torch.cuda.synchronize()
        want = [x.clone() for x in b.outputs]
        want_e = [e.clone() for e in b.energies]
        outs = [x.clone() for x in b.inits]
        energies = [torch.zeros_like(e) for e in b.energies]
        batched.synthesize_batched(b.indices, outs, energies, mode="f16", iters=2)
        for k in range(len(specs)):
            assert torch.equal(outs[k], want[k]), k
            assert torch.equal(energies[k], want_e[k]), k
    finally:
        b.close()
