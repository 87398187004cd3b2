"""Comparison helpers shared by the GPU parity tests."""
import numpy as np

import oracle

# NN parity (exact mode): indices must agree where the true minimum is unique
# by a margin above 1e-5 relative; elsewhere the GPU's window must be within
# 1e-5 relative of the oracle minimum.
NN_REL = 1e-5
NN_ABS = 1e-9


def check_nn(X, Z, w, stride, nn_g, d2_g, nn_o, d2_o, qlist=None, max_mismatch_frac=1.0):
    """Asserts the NN parity rule; returns the number of index mismatches."""
    nn_g = np.asarray(nn_g)
    d2_g = np.asarray(d2_g, dtype=np.float64)
    qs = np.arange(len(nn_o)) if qlist is None else np.asarray(qlist)
    mism = np.nonzero(nn_g != nn_o)[0]
    if len(mism):
        dt = oracle.pair_dist2(X, Z, w, stride, qs[mism], nn_g[mism])
        bad = dt > d2_o[mism] * (1 + NN_REL) + NN_ABS
        assert not bad.any(), (
            f"{bad.sum()} queries matched a window farther than the tie tolerance: "
            f"q={qs[mism][bad][:5]} gpu_d2={dt[bad][:5]} oracle_d2={d2_o[mism][bad][:5]}")
    # the reported distance is the FP32 full-dimension distance of that window
    dsel = d2_o.copy()
    if len(mism):
        dsel[mism] = oracle.pair_dist2(X, Z, w, stride, qs[mism], nn_g[mism])
    np.testing.assert_allclose(d2_g, dsel, rtol=NN_REL, atol=1e-6)
    assert len(mism) <= max_mismatch_frac * len(nn_o)
    return len(mism)
