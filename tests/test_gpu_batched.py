"""Batched synthesis (one CUDA graph over jobs of uneven sizes) against the same jobs run one by
one through synthesize_level: identical outputs and energies, and identical on a second replay."""
import numpy as np
import pytest

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
        assert all(p >= 1 for p in b.parts)
    b.close()
