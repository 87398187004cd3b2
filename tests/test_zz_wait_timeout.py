"""Failure detection of the device waits, without a fault: the library's bounded mbarrier waits
(both variants) complete when their phase completes, and when nothing completes it they give up
after about a second, report PTS_ERR_TIMEOUT through the status word, and leave the context
usable for the next call.  The wait is made to run out by a barrier no thread arrives at."""
import time

import numpy as np
import pytest

import pts_inputs as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2006_11851_gb300 as pts  # noqa: E402

PTS_ERR_TIMEOUT = -5


@pytest.mark.parametrize("abortable", [False, True])
def test_wait_completes_when_its_phase_does(abortable):
    assert pts.wait_selftest(True, abortable) == (0, True)


@pytest.mark.parametrize("abortable", [False, True])
def test_wait_gives_up_and_reports_timeout(abortable):
    t0 = time.perf_counter()
    status, completed = pts.wait_selftest(False, abortable)
    elapsed = time.perf_counter() - t0
    assert status == PTS_ERR_TIMEOUT and not completed
    assert 0.5 < elapsed < 30.0
    assert "gave up" in pts.lib().pts_last_error().decode()
    # the context is still usable: a small search afterwards runs and is sane
    z = torch.from_numpy(P.synthetic_exemplar(1, 48, 3.0)).cuda()
    ix = pts.ExemplarIndex(z, 8, d=16)
    try:
        x = z[:40, :40].contiguous()
        nn, d2 = pts.nn_search(ix, x, 2, "exact")
        assert float(d2.max()) == 0.0          # a crop of the exemplar matches itself
        assert np.all(nn.cpu().numpy() >= 0)
    finally:
        ix.close()
