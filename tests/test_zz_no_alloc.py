"""The allocation-free table build (negf_build_tables_noalloc) against the allocating one.

Callers that cannot allocate device memory (a host framework owning every device byte through
its own pool, a process whose device footprint is fixed after start-up) use this entry point;
it must give the same tables as negf_build_tables.  Calls in a row (wide wires first, then
smaller ones, so later calls run on scratch earlier ones left behind) are each compared with
negf_build_tables: alias entries bit for bit (same kernels, deterministic), c_p to the FP64
table bar of the parity tests (1e-10 relative).  The FP32 cases of W = 24 and W = 64 take the
CTA-wide block-column chains; they are also compared with the FP64 oracle: every alias row's
exact implied distribution within the quantisation bound (K + 2) 2^-32 plus the FP32 table bar
(1e-5 of the row) of the oracle's weights over their row sum, c_p within 1e-5.  Kept in a file
collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import alias as oalias, pipeline  # noqa: E402
from paper_1805_10164_gb300 import inputs, negf  # noqa: E402


def _reference(ctx, wire, precision):
    tables = negf.negf_build_tables(ctx, [wire], precision=precision)
    try:
        out = []
        for task in range(len(wire.energy)):
            info = negf.negf_get_task_info(ctx, tables, task)
            out.append((negf.negf_export_tables(ctx, tables, task, "alias"),
                        negf.negf_export_tables(ctx, tables, task, "mode_alias"), info["c"]))
        return out
    finally:
        negf.negf_tables_free(tables)


def _check_against_oracle(wire, alias_rows, c):
    n, W = wire.W * wire.L, wire.W
    rows, K = n + 2 * W, n + 2
    rng = np.random.default_rng(wire.W)
    for k, E in enumerate(wire.energy):
        ref = pipeline.task_reference(wire.onsite, wire.eta, wire.t, E, with_alias=False,
                                      with_direct=False)
        w = ref["tab"]["w"]
        assert np.allclose(c[k], ref["tab"]["c"], rtol=1e-5, atol=0.0), k
        ent = alias_rows[k].reshape(rows, K)
        for r in np.concatenate([rng.choice(rows, size=24, replace=False), [0, n - 1, n, rows - 1]]):
            A = w[r].sum()
            if A <= 0:
                continue
            p = oalias.implied_distribution(ent[r])
            assert np.max(np.abs(p - w[r] / A)) <= (K + 2) * 2.0**-32 + 1e-5, (k, r)


def test_noalloc_build_matches_allocating_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_10164_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = negf.negf_create(0, stream)
    try:
        cases = [(inputs.small_wire(65, W=24, L=5, n_energy=3, eta=0.06), "fp32"),
                 (inputs.small_wire(66, W=64, L=3, n_energy=2, eta=0.05, disorder=0.5), "fp32"),
                 (inputs.small_wire(61, W=6, L=12, n_energy=5, eta=0.08), "fp32"),
                 (inputs.small_wire(62, W=3, L=5, n_energy=2, eta=0.2), "fp64"),
                 # a multi-orbital slice block (its modes from the device eigensolver)
                 (inputs.sp3_wire(67, 3, 4, n_energy=2, eta=0.1), "fp32")]
        for wire, prec in cases:
            n_e, W, L = len(wire.energy), wire.W, wire.L
            n = W * L
            rows, K = n + 2 * W, n + 2
            d_alias = torch.zeros(n_e * rows * K, dtype=torch.int64, device="cuda")
            d_mode = torch.zeros(n_e * 2 * W, dtype=torch.int64, device="cuda")
            d_c = torch.zeros(n_e * 2, dtype=torch.float64, device="cuda")
            st = negf.negf_build_tables_noalloc(wire, prec, stream, d_alias, d_mode, d_c)
            assert st == negf.NEGF_OK, st
            alias = d_alias.cpu().numpy().view(np.uint64).reshape(n_e, rows * K)
            mode = d_mode.cpu().numpy().view(np.uint64).reshape(n_e, 2 * W)
            c = d_c.cpu().numpy().reshape(n_e, 2)
            ref = _reference(ctx, wire, prec)
            for k, (a_ref, m_ref, c_ref) in enumerate(ref):
                assert np.array_equal(alias[k], a_ref), (W, prec, k)
                assert np.array_equal(mode[k], m_ref), (W, prec, k)
                assert np.allclose(c[k], c_ref, rtol=1e-10, atol=0.0), (W, prec, k)
            if W > 16:
                _check_against_oracle(wire, alias, c)
    finally:
        negf.negf_destroy(ctx)


def test_noalloc_rejects_oversized_problems():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stream = torch.cuda.current_stream()
    big = inputs.small_wire(63, W=40, L=170, n_energy=1)          # W*L > 6400 sites limit
    buf = torch.zeros(8, dtype=torch.int64, device="cuda")
    c = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert negf.negf_build_tables_noalloc(big, "fp32", stream, buf, buf, c) == negf.NEGF_E_INVALID
    many = inputs.small_wire(64, W=10, L=50, n_energy=40)         # scratch beyond 64 MiB
    assert negf.negf_build_tables_noalloc(many, "fp64", stream, buf, buf, c) == negf.NEGF_E_NOMEM
