"""Batched synthesis (one CUDA graph over jobs of uneven sizes): against the FP64 oracle run job
by job, and against the same jobs run one by one through synthesize_level (identical outputs and
energies, and identical on a second replay)."""
import numpy as np
import pytest

import oracle
import pts_inputs as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2006_11851_gb300 as pts  # noqa: E402
from paper_2006_11851_gb300.batched import Batch, job_specs  # noqa: E402


@pytest.mark.parametrize("mode", ["f16", "exact"])
def test_batch_matches_sequential(mode):
    specs = job_specs(6, seed=3, max_exemplar=160, max_output=288)
    b = Batch(specs, mode=mode, iters=3, n_streams=3)
    b.reset()
    b.run()
    torch.cuda.synchronize()
    outs = [x.clone() for x in b.outputs]
    ens = [e.cpu().numpy().copy() for e in b.energies]
    # replay: same results from the same inputs
    b.reset()
    b.run()
    torch.cuda.synchronize()
    for x, o in zip(b.outputs, outs):
        assert torch.equal(x, o)
    # each job alone through the public API
    for k, (ix, x0) in enumerate(zip(b.indices, b.inits)):
        x = x0.clone()
        E = pts.synthesize_level(ix, x, 3, mode=mode)
        assert torch.equal(x, outs[k]), k
        np.testing.assert_array_equal(E, ens[k])
    assert b.launches_per_run > 0
    if mode == "f16":
        assert all(p in (0, 1, 2, 4) for p in b.parts)  # 0: the automatic split
    b.close()


# Uneven jobs small enough for the oracle: 8x8 and 16x16 windows, exemplars 36..64, outputs 48..96.
SMALL_JOBS = [
    {"job": 0, "He": 48, "Ho": 80, "w": 8, "d": 24, "seed": 0},
    {"job": 1, "He": 40, "Ho": 64, "w": 16, "d": 32, "seed": 1},
    {"job": 2, "He": 64, "Ho": 96, "w": 8, "d": 32, "seed": 2},
    {"job": 3, "He": 36, "Ho": 48, "w": 16, "d": 48, "seed": 3},
]


@pytest.mark.parametrize("mode", ["exact", "f16"])
def test_batch_against_oracle(mode):
    """Each job of one graph replay against the oracle's EM run of that job (section 2.1, Eq. 4),
    from the same seeded exemplar and initialisation.  Exact mode: every energy within 1e-3
    relative (the first, an E-step on the initialisation, within 1e-5) and 99% of the pixels
    within 1e-4 (a near-tie may flip a match).  FP16 mode: the final image's energy, measured by
    the oracle's exact search, within 1.01x of the oracle's exact run."""
    iters = 3
    b = Batch(SMALL_JOBS, mode=mode, iters=iters, n_streams=2)
    b.reset()
    b.run()
    torch.cuda.synchronize()
    for k, s in enumerate(SMALL_JOBS):
        Z = P.synthetic_exemplar(s["seed"], s["He"], 4.0)
        X0 = P.random_patch_init(Z, s["Ho"], s["Ho"], s["w"], 1000 + s["seed"])
        np.testing.assert_array_equal(b.inits[k].cpu().numpy(), X0)
        ref = oracle.synthesize_level(Z, X0, s["w"], iters, r=2.0)
        E = b.energies[k].cpu().numpy()
        X = b.outputs[k].cpu().numpy()
        if mode == "exact":
            assert abs(E[0] / ref["E"][0] - 1) < 1e-5, (k, E[0], ref["E"][0])
            np.testing.assert_allclose(E, ref["E"], rtol=1e-3)
            assert np.mean(np.abs(X - ref["X"]) < 1e-4) > 0.99, k
        else:
            _, d2 = oracle.nn_bruteforce(X, Z, s["w"], 2)
            assert d2.sum() <= 1.01 * ref["E"][-1], (k, d2.sum(), ref["E"][-1])
    b.close()


def test_batch_refuses_to_run_after_its_indices_change():
    """The captured graph holds raw pointers into each job's index.  A search that makes the index
    reallocate its workspace (a larger output), or destroying a job's index, must make the next
    pts_batch_run refuse with PTS_ERR_INVALID_ARG before launching anything."""
    specs = SMALL_JOBS[:2]
    b = Batch(specs, mode="f16", iters=1, n_streams=2)
    b.run()
    torch.cuda.synchronize()
    x = torch.zeros(specs[0]["Ho"], specs[0]["Ho"], 3, device="cuda")
    pts.nn_search(b.indices[0], x, 2, "f16")          # same size and mode: nothing moves
    b.run()
    torch.cuda.synchronize()
    big = torch.zeros(specs[0]["Ho"] + 96, specs[0]["Ho"] + 96, 3, device="cuda")
    pts.nn_search(b.indices[0], big, 2, "f16")        # more queries: the workspace grows
    with pytest.raises(pts.PtsError, match="create the batch again"):
        b.run()
    b.close()
    b = Batch(specs, mode="exact", iters=1, n_streams=1)
    b.indices[1].close()
    with pytest.raises(pts.PtsError, match="destroyed"):
        b.run()
    b.close()


def test_batch_pyramid_levels_against_oracle():
    """Pyramid levels inside one batch (section 2.1's coarse to fine): two 3-level jobs whose
    finer levels start from the coarser results up-sampled by 2 within the graph.  Every level's
    final energy against the oracle's run of the same pyramid (its FP64 exemplar pyramid, its
    up-sampling) within 1e-3, and the batch equal to the same levels run one by one."""
    from paper_2006_11851_gb300.batched import run_eager
    specs = [{"job": 0, "He": 48, "Ho": 96, "w": 8, "d": 16, "seed": 4, "levels": 3},
             {"job": 1, "He": 64, "Ho": 128, "w": 8, "d": 16, "seed": 5, "levels": 3}]
    iters = 3
    b = Batch(specs, mode="exact", iters=iters, n_streams=2)
    assert b.parents == [-1, 0, 1, -1, 3, 4]
    b.reset()
    b.run()
    torch.cuda.synchronize()
    outs = [x.clone() for x in b.outputs]
    ens = [e.cpu().numpy().copy() for e in b.energies]
    for s, ks in zip(specs, b.levels):
        pyr_o = oracle.exemplar_pyramid(P.synthetic_exemplar(s["seed"], s["He"], 4.0), 3)
        Xo = b.inits[ks[0]].cpu().numpy()
        for lev, k in enumerate(ks):
            ref = oracle.synthesize_level(pyr_o[lev].astype(np.float32), Xo, s["w"], iters)
            assert abs(ens[k][-1] / ref["E"][-1] - 1) < 1e-3, (s["job"], lev, ens[k], ref["E"])
            Xo = oracle.upsample2(ref["X"]) if lev < 2 else ref["X"]
    b.reset()
    run_eager(b)
    torch.cuda.synchronize()
    for k, x in enumerate(b.outputs):
        assert torch.equal(x, outs[k]), k
    b.close()


def test_batch_with_proposal_and_tree_jobs():
    """The learned proposal (trained on the job's own exact runs) and the paper's k-means tree as
    job modes of a batch, beside an FP16 job: the graph replay equals each job run alone through
    synthesize_level, bit for bit."""
    from paper_2006_11851_gb300.batched import run_eager
    specs = [{"job": 0, "He": 96, "Ho": 160, "w": 8, "d": 32, "seed": 6, "mode": "f16"},
             {"job": 1, "He": 96, "Ho": 160, "w": 8, "d": 32, "seed": 7, "mode": "proposal"},
             {"job": 2, "He": 80, "Ho": 128, "w": 16, "d": 48, "seed": 8, "mode": "kmtree"}]
    b = Batch(specs, iters=2, n_streams=3, proposal_params={"n_clusters": 64, "epochs": 2, "batch": 1024})
    assert b.modes == ["f16", "proposal", "kmtree"]
    b.reset()
    b.run()
    torch.cuda.synchronize()
    outs = [x.clone() for x in b.outputs]
    ens = [e.clone() for e in b.energies]
    b.reset()
    run_eager(b)
    torch.cuda.synchronize()
    for k in range(3):
        assert torch.equal(b.outputs[k], outs[k]), k
    # the eager path returns host energies; the graph's device energies are those of the same run
    for k, (ix, x0) in enumerate(zip(b.indices, b.inits)):
        x = x0.clone()
        E = pts.synthesize_level(ix, x, 2, mode=b.modes[k])
        np.testing.assert_array_equal(E, ens[k].cpu().numpy())
    b.close()
