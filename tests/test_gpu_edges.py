"""Edge cases of the GPU path through the C ABI: empty batches, wires without energies, zero
walkers, single-site wires, no dephasing (every walk ends on its first draw), and the largest
one-level (W*L = 6400) and two-level (W*L = 65536) wires, with sizes beyond those rejected."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from mc_bars import z_bar  # noqa: E402
from oracle import alias, columns, pipeline  # noqa: E402
from paper_1805_10164_gb300 import inputs, negf  # noqa: E402

MU = (3.5, -3.5, 0.025)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_10164_gb300 import build
    build.build()
    c = negf.negf_create(0)
    yield c
    negf.negf_destroy(c)


def test_empty_batch_and_empty_wire(ctx):
    t = negf.negf_build_tables(ctx, [])
    try:
        assert negf.negf_tables_num_tasks(t) == 0
        tl = negf.negf_walk(ctx, t, 0, 1, 100)
        res = negf.negf_current(ctx, t, tl, *MU)
        assert res["I"].size == 0 and res["T"].size == 0 and not res["stepcap"]
        negf.negf_tally_free(tl)
    finally:
        negf.negf_tables_free(t)
    # a wire without energies between two wires with energies: no tasks, zero current
    w1 = inputs.small_wire(301, W=3, L=4, n_energy=2)
    w0 = inputs.Wire(W=2, L=3, t=1.0, onsite=np.zeros((3, 2)), eta=np.full((3, 2), 0.1),
                     energy=np.zeros(0), energy_weight=np.zeros(0))
    w2 = inputs.small_wire(302, W=2, L=5, n_energy=1)
    t = negf.negf_build_tables(ctx, [w1, w0, w2])
    try:
        assert negf.negf_tables_num_tasks(t) == 3
        assert [negf.negf_get_task_info(ctx, t, k)["wire"] for k in range(3)] == [0, 0, 2]
        tl = negf.negf_walk(ctx, t, 0, 7, 20000)
        res = negf.negf_current(ctx, t, tl, *MU)
        negf.negf_tally_free(tl)
        assert res["I"][1] == 0.0 and res["se"][1] == 0.0 and res["I"][0] != 0.0
    finally:
        negf.negf_tables_free(t)


def test_zero_walkers_and_single_site(ctx):
    w = inputs.small_wire(303, W=1, L=1, n_energy=2, eta=0.2, e_lo=-1.0, e_hi=1.0)
    t = negf.negf_build_tables(ctx, [w], precision="fp64", keep_weights=True)
    try:
        tl = negf.negf_walk(ctx, t, 0, 3, 0)
        counts = negf.negf_tally_counts(ctx, tl, 2)
        res = negf.negf_current(ctx, t, tl, *MU)
        negf.negf_tally_free(tl)
        assert not counts.any() and np.all(res["T"] == 0.0) and np.all(res["I"] == 0.0)
        # one site: rows are the site and one mode per lead; sum rule and MC transmission
        for k, E in enumerate(w.energy):
            ref = pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False)
            wts = negf.negf_export_tables(ctx, t, k, "weights").reshape(ref["tab"]["w"].shape)
            assert np.allclose(wts, ref["tab"]["w"], rtol=1e-10, atol=1e-14)
        tl = negf.negf_walk(ctx, t, 1, 4, 200_000)
        res = negf.negf_current(ctx, t, tl, *MU)
        negf.negf_tally_free(tl)
        for k, E in enumerate(w.energy):
            ref = pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False)
            assert abs(res["T"][k] - ref["T_direct"][0, 1]) <= z_bar(2) * res["T_se"][k] + 1e-12
    finally:
        negf.negf_tables_free(t)


def test_no_dephasing_ends_every_walk_on_its_first_draw(ctx):
    """eta = 0: no Buttiker site can be drawn, so every walk is absorbed on its first transition
    and the estimator is the coherent transmission (Landauer), within its binomial SE."""
    w = inputs.small_wire(304, W=4, L=6, n_energy=2, eta=0.0, e_lo=-0.7, e_hi=0.9)
    t = negf.negf_build_tables(ctx, [w], precision="fp32")
    try:
        N = 300_000
        tl = negf.negf_walk(ctx, t, 0, 5, N)
        counts = negf.negf_tally_counts(ctx, tl, 2)
        res = negf.negf_current(ctx, t, tl, *MU)
        negf.negf_tally_free(tl)
        assert np.all(counts[:, 4] == counts[:, 1] + counts[:, 2])      # one step per walk
        for k, E in enumerate(w.energy):
            ref = pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False)
            assert abs(res["T"][k] - ref["T_direct"][1, 0]) <= z_bar(2) * res["T_se"][k] + 1e-6
    finally:
        negf.negf_tables_free(t)


def test_largest_one_level_wire(ctx):
    """W = 64, L = 100 (6400 sites) with one-level tables forced: sampled rows realise the
    oracle's weights (1e-5 of the row plus quantisation), T_LR = T_RL within 3 SE."""
    w = inputs.small_wire(305, W=64, L=100, n_energy=1, eta=0.05, disorder=0.5, e_lo=0.21,
                          e_hi=0.21)
    n = 6400
    rows = np.array([0, 3333, n - 1, n, n + 64 + 5])
    ref_rows = columns.sampled_rows(w.energy[0], w.onsite, w.eta, w.t, rows)
    t = negf.negf_build_tables(ctx, [w], precision="fp32", layout="one_level")
    try:
        info = negf.negf_get_task_info(ctx, t, 0)
        assert info["layout"] == "one_level" and info["K"] == n + 2
        for j, r in enumerate(rows):
            ent = negf.negf_export_table_rows(ctx, t, 0, "alias", r, 1)
            p = alias.implied_distribution(ent)
            A = ref_rows["w"][j].sum()
            assert np.max(np.abs(p - ref_rows["w"][j] / A)) <= (n + 4) * 2.0**-32 + 1e-5
        tl = negf.negf_walk(ctx, t, 0, 6, 400_000)
        res = negf.negf_current(ctx, t, tl, *MU)
        negf.negf_tally_free(tl)
        tl = negf.negf_walk(ctx, t, 1, 7, 400_000)
        res1 = negf.negf_current(ctx, t, tl, *MU)
        negf.negf_tally_free(tl)
        # reciprocity at this size (the dense direct solve is left to the smaller cases)
        assert abs(res["T"][0] - res1["T"][0]) <= 3.0 * np.hypot(res["T_se"][0], res1["T_se"][0])
    finally:
        negf.negf_tables_free(t)


def test_size_limits(ctx):
    # largest two-level wire: W = 64, L = 1024 (65536 sites, 34 GB of tables)
    w = inputs.small_wire(306, W=64, L=1024, n_energy=1, eta=0.01, disorder=0.5, e_lo=-0.45,
                          e_hi=-0.45)
    n = 65536
    t = negf.negf_build_tables(ctx, [w], precision="fp32")
    try:
        info = negf.negf_get_task_info(ctx, t, 0)
        assert info["layout"] == "two_level" and info["n"] == n
        rows = np.array([17, n - 2, n + 3])
        ref_rows = columns.sampled_rows(w.energy[0], w.onsite, w.eta, w.t, rows)
        for j, r in enumerate(rows):
            rs = negf.negf_export_table_rows(ctx, t, 0, "rowsum", r, 1)[0]
            A = ref_rows["w"][j].sum()
            assert abs(rs - A) <= 1e-5 * A
    finally:
        negf.negf_tables_free(t)
    too_long = inputs.small_wire(307, W=64, L=1025, n_energy=1)
    with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
        negf.negf_build_tables(ctx, [too_long])
    too_wide = inputs.small_wire(308, W=65, L=2, n_energy=1)
    with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
        negf.negf_build_tables(ctx, [too_wide])
    one_level_too_long = inputs.small_wire(309, W=64, L=101, n_energy=1)
    with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
        negf.negf_build_tables(ctx, [one_level_too_long], layout="one_level")
