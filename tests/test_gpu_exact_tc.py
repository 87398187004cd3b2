"""The exact search through the full-dimension FP16 tensor-core GEMM (mode "exact_tc"), against
the FP64 oracle and against the FP32 exact mode.

The mode certifies the FP32 re-rank of its 32 best FP16 scores with a worst-case slack for the
FP16 operands and the FP32 accumulation (include/pts.h), and sends what it cannot certify to the
FP32 full-dimension pass of exact mode.  So its results must be exact mode's: the same window
and the same FP32 distance bit for bit, wherever the nearest window is unique.  The tests cover
ragged query blocks and window tiles, K padding (D not a multiple of 64), fewer windows than
candidates, four channels, the benchmark's coarsest level (w = 32, D = 3,072), near-ties far
below the FP16 resolution (which the slack must leave uncertified), and values past the FP16
range (whose queries must not be certified from the GEMM)."""
import numpy as np
import pytest

import oracle
import pts_inputs as P
from _util import check_nn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2006_11851_gb300 as pts  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def _same_as_exact(idx, X, stride):
    """Runs both exact routes; asserts equal distances everywhere and equal windows wherever the
    distance has no tie; returns the tensor-core route's results and statistics."""
    nn_e, d2_e = pts.nn_search(idx, X, stride, "exact")
    nn_t, d2_t = pts.nn_search(idx, X, stride, "exact_tc")
    st = idx.search_stats()
    assert torch.equal(d2_t, d2_e)
    diff = (nn_t != nn_e).nonzero().flatten()
    assert diff.numel() <= max(1, nn_t.numel() // 1000), diff.numel()
    return nn_t.cpu().numpy(), d2_t.cpu().numpy(), st, diff.cpu().numpy()


@pytest.mark.parametrize("He,Ho,w,d,stride", [
    (64, 128, 8, 24, 2),   # D = 192 (K = 192), N = 3,249: 13 tiles, the last ragged; Q = 3,721
    (24, 29, 5, 10, 1),    # D = 75 padded to K = 128, stride 1
    (10, 20, 8, 8, 2),     # N = 9 windows: fewer than 32 candidates
    (33, 36, 16, 40, 2),   # D = 768, Q = 121: one ragged query block
    (30, 40, 8, 20, 4),    # stride 4
])
def test_exact_tc_against_oracle_and_exact(He, Ho, w, d, stride):
    Z = P.synthetic_exemplar(4, He, 3.0)
    X = P.random_patch_init(Z, Ho, Ho, w, 2)
    idx = pts.ExemplarIndex(_t(Z), w, d=d)
    nn, d2, st, diff = _same_as_exact(idx, _t(X), stride)
    nn_o, d2_o = oracle.nn_bruteforce(X, Z, w, stride)
    check_nn(X, Z, w, stride, nn, d2, nn_o, d2_o)
    assert st["queries"] == len(nn_o)
    assert st["certified"] + st["range_queries"] == st["queries"]
    idx.close()


def test_exact_tc_four_channels():
    """RGBS windows (section 3): the scale channel is a fourth component of every pixel."""
    Z3 = P.synthetic_exemplar(6, 40, 3.0)
    s = np.linspace(0.2, 1.0, 40, dtype=np.float32)[:, None, None] * np.ones((40, 40, 1), np.float32)
    Z = np.ascontiguousarray(np.concatenate([Z3, s], axis=2))
    # the generator copies 3-channel blocks: the same seed picks the same blocks of the scale map
    X = np.ascontiguousarray(np.concatenate([P.random_patch_init(Z3, 52, 52, 8, 3),
                                             P.random_patch_init(np.repeat(s, 3, axis=2), 52, 52, 8, 3)[..., :1]],
                                            axis=2))
    idx = pts.ExemplarIndex(_t(Z), 8, d=24)
    nn, d2, st, _ = _same_as_exact(idx, _t(X), 2)
    nn_o, d2_o = oracle.nn_bruteforce(X, Z, 8, 2)
    check_nn(X, Z, 8, 2, nn, d2, nn_o, d2_o)
    idx.close()


def test_exact_tc_benchmark_coarsest_level():
    """The benchmark's coarsest level (64x64 exemplar, w = 32, D = 3,072, 2,401 queries), where
    the PCA keeps under 85% of the variance: the random-patch initialisation and the oracle's next
    two iterates, all queries against the FP64 brute force.  Nearly every query is certified from
    the FP16 scores."""
    Z = oracle.exemplar_pyramid(P.synthetic_exemplar(0, 256, 4.0), 3)[0].astype(np.float32)
    idx = pts.ExemplarIndex(_t(Z), 32, d=64)
    X0 = P.random_patch_init(Z, 128, 128, 32, 100)
    ref = oracle.synthesize_level(Z, X0, 32, 2, keep_trajectory=True)
    for Xt, nn_o, d2_o, _ in ref["trajectory"]:
        nn, d2, st, _ = _same_as_exact(idx, _t(Xt), 2)
        check_nn(Xt, Z, 32, 2, nn, d2, nn_o, d2_o, max_mismatch_frac=0.01)
        print(f"\ncoarsest level: {st['certified']} of {st['queries']} certified from the FP16 scores")
        assert st["queries"] == 2401 and st["certified"] >= 0.9 * 2401, st
    idx.close()


def test_exact_tc_near_ties_stay_uncertified():
    """An exemplar that is a horizontal ramp plus noise of amplitude 1e-3: the windows of one
    column differ by about 1e-4 in squared distance, far inside the FP16 slack (about 2^-9 of
    the norms, which the ramp makes large), so more than 32 windows tie with each query's best
    within the slack and the certificate must fail, sending the query to the FP32 pass.  The
    results must be the oracle's nearest windows (tie rule of tests/_util.py) on every query.
    (Exact mode's PCA bound, whose FP32 slack is a model rather than a worst-case bound, returns
    on this input a window up to 1.1e-4 relative farther than the nearest for a few queries; the
    tensor-core route never returns a farther window than it.)"""
    He, w = 48, 8
    rng = P.SplitMix64(11)
    ramp = np.linspace(0.0, 1.0, He, dtype=np.float32)[None, :, None] * np.ones((He, He, 3), np.float32)
    Z = np.ascontiguousarray(ramp + 1e-3 * rng.uniform(He * He * 3).reshape(He, He, 3).astype(np.float32))
    X = P.random_patch_init(Z, 64, 64, w, 5)
    idx = pts.ExemplarIndex(_t(Z), w, d=24)
    _, d2_e = pts.nn_search(idx, _t(X), 2, "exact")
    nn, d2 = pts.nn_search(idx, _t(X), 2, "exact_tc")
    st = idx.search_stats()
    nn_o, d2_o = oracle.nn_bruteforce(X, Z, w, 2)
    check_nn(X, Z, w, 2, nn.cpu().numpy(), d2.cpu().numpy(), nn_o, d2_o)
    assert torch.all(d2 <= d2_e)
    print(f"\nramp exemplar: {st['range_queries']} of {st['queries']} queries left to the FP32 pass")
    assert st["range_queries"] > st["queries"] // 2, st
    idx.close()


def test_exact_tc_values_past_the_fp16_range():
    """A query window holding a value 40 above the exemplar mean (past 2^12 x 40 > 65504 after
    scaling) saturates in FP16; its slack becomes infinite, so it is never certified from the
    GEMM, and its result is exact mode's."""
    Z = P.synthetic_exemplar(9, 40, 3.0)
    X = P.random_patch_init(Z, 48, 48, 8, 1)
    X[10, 10, 1] = 40.0
    idx = pts.ExemplarIndex(_t(Z), 8, d=24)
    nn, d2, st, _ = _same_as_exact(idx, _t(X), 2)
    nn_o, d2_o = oracle.nn_bruteforce(X, Z, 8, 2)
    check_nn(X, Z, 8, 2, nn, d2, nn_o, d2_o)
    assert st["range_queries"] >= 1
    idx.close()


def test_exact_tc_on_an_exemplar_past_the_fp16_range():
    """An exemplar value 40 above the mean cannot be held by the FP16 tiles: the mode runs the
    FP32 exact search instead, with the same results."""
    Z = P.synthetic_exemplar(10, 32, 3.0)
    Z[5, 5, 0] = 40.0
    X = P.random_patch_init(Z, 40, 40, 8, 1)
    idx = pts.ExemplarIndex(_t(Z), 8, d=24)
    nn, d2, _, _ = _same_as_exact(idx, _t(X), 2)
    nn_o, d2_o = oracle.nn_bruteforce(X, Z, 8, 2)
    check_nn(X, Z, 8, 2, nn, d2, nn_o, d2_o)
    idx.close()


def test_exact_tc_synthesis_matches_exact_mode():
    """Two EM iterations (search, IRLS weights, M-step) in each exact route from the same
    initialisation give the same image."""
    Z = P.synthetic_exemplar(0, 64, 3.0)
    idx = pts.ExemplarIndex(_t(Z), 8, d=24)
    X0 = P.random_patch_init(Z, 96, 96, 8, 7)
    xa, xb = _t(X0), _t(X0)
    ea = pts.synthesize_level(idx, xa, 2, r=2.0, mode="exact")
    eb = pts.synthesize_level(idx, xb, 2, r=2.0, mode="exact_tc")
    assert torch.equal(xa, xb)
    np.testing.assert_array_equal(np.asarray(ea), np.asarray(eb))
    idx.close()
