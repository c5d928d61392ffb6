"""Slices with undephased sites (eta_i = 0) on the GPU against the oracle.

The block inversions skip the pivot search only on slices where every site dephases; a slice
with an undephased site takes partial pivoting: the warp's register routine (complex64,
W <= 16) and the CTA routine with row interchanges and a final column unscramble (complex64
above W = 16, complex128 at every width).  These wires mix dephased and undephased sites so
that both kinds of slice occur in one sweep.

Bars: weights elementwise within 1e-5 (FP32) / 1e-10 (FP64) of the oracle's row sum, row sums
within the same relative bar, Monte Carlo T against the direct probe solve with every
|z| <= z_bar(m) and sum z^2 <= chi2_bar(m) (mc_bars: the 3-SE bar as a 0.27 % family-wise
false-alarm rate).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from mc_bars import chi2_bar, z_bar  # noqa: E402
from oracle import pipeline  # noqa: E402
from paper_1805_10164_gb300 import inputs, negf  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_10164_gb300 import build
    build.build()
    c = negf.negf_create(0)
    yield c
    negf.negf_destroy(c)


def _partly_undephased(seed, W, L, n_energy=2):
    w = inputs.small_wire(seed, W=W, L=L, n_energy=n_energy, eta=0.08, disorder=0.8,
                          e_lo=-1.7, e_hi=1.3)
    eta = w.eta.copy()
    eta[::2, ::3] = 0.0            # every other slice has undephased sites
    eta[1, :] = 0.0                # and one slice has none dephased
    return inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=w.onsite, eta=eta, energy=w.energy,
                       energy_weight=w.energy_weight)


def _wires():
    return [_partly_undephased(401, W=8, L=7), _partly_undephased(402, W=20, L=5),
            _partly_undephased(403, W=3, L=9)]


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp64", 1e-10)])
def test_pivoted_slices_match_oracle(ctx, precision, tol):
    wires = _wires()
    refs = [pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False)
            for w in wires for E in w.energy]
    tables = negf.negf_build_tables(ctx, wires, precision=precision, keep_weights=True)
    try:
        for task, ref in enumerate(refs):
            w_ref = ref["tab"]["w"]
            rs_ref = w_ref.sum(1)
            w = negf.negf_export_tables(ctx, tables, task, "weights").reshape(w_ref.shape)
            bad = np.abs(w - w_ref) > tol * rs_ref[:, None] + 1e-30
            assert not bad.any(), (precision, task, np.argwhere(bad)[:5])
            rs = negf.negf_export_tables(ctx, tables, task, "rowsum")
            assert np.allclose(rs, rs_ref, rtol=tol, atol=1e-300), (precision, task)
        N = 300_000
        tally = negf.negf_walk(ctx, tables, 0, 2024, N)
        res = negf.negf_current(ctx, tables, tally, 3.5, -3.5, 0.025)
        negf.negf_tally_free(tally)
        z = []
        for task, ref in enumerate(refs):
            T_ref = ref["T_direct"][1, 0]
            if res["T_se"][task] > 0:
                z.append((res["T"][task] - T_ref) / (res["T_se"][task] + 1e-6 * T_ref))
            else:
                assert abs(res["T"][task] - T_ref) <= 1e-6 * T_ref + 1e-12, task
        z = np.asarray(z)
        assert np.max(np.abs(z)) <= z_bar(z.size) and np.sum(z ** 2) <= chi2_bar(z.size), z
    finally:
        negf.negf_tables_free(tables)
