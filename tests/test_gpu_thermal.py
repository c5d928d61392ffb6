"""Continuous-energy sampling of the linear conductance (negf_walk_thermal) against the oracle.

Bars: walks bit-exact against the oracle's replay walker on the exported tables, given the
device's energy interval and alpha; those energy draws equal to the oracle's from the same
Philox words (interval exactly, alpha within 2^-20); G against the exact expectation of the
interpolated chain (quadrature of the oracle's FP64 chain) with every |z| <= z_bar(m) and
sum z^2 <= chi2_bar(m) over the m wires (mc_bars: the 3-SE bar as a 0.27 % family-wise
false-alarm rate); with a fine grid, G within 3 SE plus the linear-interpolation error bound of
the direct conductance.  Two-level tables: the same replay and expectation bars.  The adaptive
grid: interval distances against the oracle's (FP64 tables 1e-9, FP32 tables 1e-4 absolute:
the FP32 table bar of 1e-5 per entry summed over a row's few dominant entries) and the refined
grid equal to the oracle's (same midpoints in the same rounds).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from mc_bars import chi2_bar, z_bar  # noqa: E402
from oracle import pipeline, thermal  # noqa: E402
from oracle.philox import philox4x32_10  # noqa: E402
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


def _on_grid(w, grid):
    g = np.asarray(grid, dtype=np.float64)
    return inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=w.onsite, eta=w.eta, energy=g,
                       energy_weight=np.ones_like(g))


def _cases():
    w = inputs.small_wire(601, W=3, L=5, n_energy=1, eta=0.12, disorder=0.8)
    chain = inputs.small_wire(602, W=1, L=9, n_energy=1, eta=0.1, disorder=0.5)
    return [(_on_grid(w, [-0.3, -0.05, 0.2, 0.45]), 0.1, 0.09),
            # the last energy lies outside the chain's band: no open channel there
            (_on_grid(chain, [1.55, 1.8, 2.25]), 1.9, 0.12)]


def _export(ctx, tables, task0, M, two_level=False):
    ent, ment, c, l2 = [], [], [], []
    for e in range(M):
        info = negf.negf_get_task_info(ctx, tables, task0 + e)
        if two_level:
            W, L = info["W"], info["L"]
            ent.append(negf.negf_export_tables(ctx, tables, task0 + e, "alias_level1")
                       .reshape(info["rows"], L + 2))
            l2.append(negf.negf_export_tables(ctx, tables, task0 + e, "alias").view(np.uint32)
                      .reshape(info["rows"], L, negf.level2_words(W)))
        else:
            ent.append(negf.negf_export_tables(ctx, tables, task0 + e, "alias")
                       .reshape(info["rows"], info["K"]))
        ment.append(negf.negf_export_tables(ctx, tables, task0 + e, "mode_alias")
                    .reshape(2, info["W"]))
        c.append(np.asarray(info["c"], dtype=np.float64))
    level2 = (l2, info["L"]) if two_level else None
    return ent, ment, c, info["n"], info["W"], level2


@pytest.mark.parametrize("layout", ["one_level", "two_level"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_thermal_walks_replay_bit_exact(ctx, precision, layout):
    cases = _cases()
    wires = [cw[0] for cw in cases]
    two = layout == "two_level"
    tables = negf.negf_build_tables(ctx, wires, precision=precision, layout=layout)
    try:
        task0 = 0
        for wi, (w, mu, kT) in enumerate(cases):
            M = w.energy.size
            ent, ment, c, n, W, level2 = _export(ctx, tables, task0, M, two)
            info = negf.negf_get_task_info(ctx, tables, task0)
            assert info["layout"] == layout
            for lead0, off in ((0, 0), (1, 2 ** 35 + 3)):
                N = 1500
                tr = {k: torch.empty(N, dtype=torch.int32, device="cuda")
                      for k in ("lead", "steps", "interval", "a")}
                res = negf.negf_walk_thermal(ctx, tables, wi, lead0, 0xFEED + wi, N, mu, kT,
                                             walker_id_offset=off, trace=tr)
                dl = tr["lead"].cpu().numpy()
                ds = tr["steps"].cpu().numpy().astype(np.uint32)
                di = tr["interval"].cpu().numpy().astype(np.int64)
                da = tr["a"].cpu().numpy().view(np.uint32).astype(np.uint64)
                wids = off + np.arange(N, dtype=np.uint64)
                # the energy draws from the same Philox words
                x = philox4x32_10(np.zeros(N, np.uint64), wids & np.uint64(0xFFFFFFFF),
                                  wids >> np.uint64(32),
                                  np.full(N, 0x80000000 | wi, np.uint64), (0xFEED + wi),
                                  0)
                _, oi, oa = thermal.energy_draw(x[0], x[1], w.energy, mu, kT)
                assert np.array_equal(oi, di), (wi, lead0)
                assert np.max(np.abs(oa.astype(np.int64) - da.astype(np.int64))) <= 4096
                lead, steps, _, _ = thermal.walk(ent, ment, c, n, W, wi, lead0, 0xFEED + wi,
                                                 wids, w.energy, mu, kT, 1 << 20,
                                                 energy=(di, da), level2=level2)
                assert np.array_equal(lead, dl), (wi, lead0, np.argwhere(lead != dl)[:5])
                assert np.array_equal(steps, ds), (wi, lead0)
                assert res["walkers"] == N
                assert res["absorbed"][0] + res["absorbed"][1] + res["closed"] == N
            task0 += M
    finally:
        negf.negf_tables_free(tables)


@pytest.mark.parametrize("precision,layout", [("fp32", "one_level"), ("fp64", "one_level"),
                                              ("fp32", "two_level")])
def test_thermal_conductance_matches_interpolated_chain(ctx, precision, layout):
    cases = _cases()
    wires = [cw[0] for cw in cases]
    tables = negf.negf_build_tables(ctx, wires, precision=precision, layout=layout)
    try:
        z = []
        for wi, (w, mu, kT) in enumerate(cases):
            tabs = [pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False)["tab"]
                    for E in w.energy]
            G_ref = thermal.conductance_interpolated(tabs, w.energy, mu, kT, n_quad=24)
            res = negf.negf_walk_thermal(ctx, tables, wi, 0, 77 + wi, 2_000_000, mu, kT)
            assert not res["stepcap"]
            z.append((res["G"] - G_ref) / (res["se"] + 1e-6 * G_ref))
            assert abs(z[-1]) <= z_bar(len(cases)), (wi, res, G_ref)
            window = thermal.th_cdf(w.energy[-1], mu, kT) - thermal.th_cdf(w.energy[0], mu, kT)
            assert abs(res["window"] - window) < 1e-12
        assert np.sum(np.square(z)) <= chi2_bar(len(z)), z
    finally:
        negf.negf_tables_free(tables)


def test_thermal_fine_grid_approaches_direct_conductance(ctx):
    w0 = inputs.small_wire(603, W=4, L=6, n_energy=1, eta=0.1, disorder=0.6)
    mu, kT = 0.15, 0.06
    grid = np.linspace(mu - 5 * kT, mu + 5 * kT, 21)
    w = _on_grid(w0, grid)
    G_dir = thermal.conductance_direct(w.onsite, w.eta, w.t, grid, mu, kT, n_quad=8)
    coarse = grid[::4]
    tabs = [pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False)["tab"]
            for E in coarse]
    G_coarse = thermal.conductance_interpolated(tabs, coarse, mu, kT)
    # the interpolation error falls like h^2: a quarter of the coarse error bounds the fine one
    bound = abs(G_coarse - G_dir) / 16.0 * 4.0 + 1e-4 * G_dir
    tables = negf.negf_build_tables(ctx, [w], precision="fp32")
    try:
        res = negf.negf_walk_thermal(ctx, tables, 0, 0, 99, 4_000_000, mu, kT)
        assert abs(res["G"] - G_dir) <= 3.0 * res["se"] + bound, (res, G_dir, bound)
    finally:
        negf.negf_tables_free(tables)


def test_thermal_refusals(ctx):
    w = inputs.small_wire(604, W=3, L=4, n_energy=1)
    one = _on_grid(w, [0.3])
    desc = _on_grid(w, [0.5, 0.2, 0.7])
    ok = _on_grid(w, [0.1, 0.4])
    t = negf.negf_build_tables(ctx, [one, desc, ok])
    try:
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_walk_thermal(ctx, t, 0, 0, 1, 100, 0.3, 0.05)       # one energy
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_walk_thermal(ctx, t, 1, 0, 1, 100, 0.3, 0.05)       # not ascending
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_walk_thermal(ctx, t, 3, 0, 1, 100, 0.3, 0.05)       # no such wire
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_walk_thermal(ctx, t, 2, 0, 1, 100, 0.3, 0.0)        # kT = 0
        assert negf.negf_walk_thermal(ctx, t, 2, 0, 1, 0, 0.3, 0.05)["walkers"] == 0
    finally:
        negf.negf_tables_free(t)
    t = negf.negf_build_tables(ctx, [ok, one])                     # no keep_weights
    try:
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_interval_distance(ctx, t, 0, 2)
    finally:
        negf.negf_tables_free(t)
    t = negf.negf_build_tables(ctx, [ok, one], keep_weights=True)
    try:
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_interval_distance(ctx, t, 1, 1)                 # one energy
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_interval_distance(ctx, t, 2, 2)                 # no such wire
    finally:
        negf.negf_tables_free(t)
    for args in ((0.4, 0.1, 5), (0.1, 0.4, 1), (0.1, 0.4, 9, 0.05, 8), (0.1, 0.4, 5, 0.0)):
        with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
            negf.negf_thermal_grid(ctx, w, *args)


def _tabs(w, grid):
    return [pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False,
                                    with_direct=False)["tab"] for E in grid]


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_interval_distance_matches_oracle(ctx, precision, bar):
    w0 = inputs.small_wire(605, W=4, L=7, n_energy=1, eta=0.09, disorder=0.7)
    grid = np.array([-0.9, -0.6, -0.5, -0.45, 0.1, 0.12, 0.8])
    tabs = _tabs(w0, grid)
    chain = inputs.small_wire(606, W=1, L=8, n_energy=1, eta=0.1, disorder=0.4)
    cgrid = np.array([1.5, 1.7, 1.95, 2.3])                      # the last one has no channel
    ctabs = _tabs(chain, cgrid)
    t = negf.negf_build_tables(ctx, [_on_grid(w0, grid), _on_grid(chain, cgrid)],
                               precision=precision, keep_weights=True)
    try:
        for wi, (g, tb) in enumerate(((grid, tabs), (cgrid, ctabs))):
            for p in (0, 1):
                d = negf.negf_interval_distance(ctx, t, wi, g.size, start_lead=p)
                ref = np.array([thermal.interval_distance(tb[i], tb[i + 1], p)
                                for i in range(g.size - 1)])
                assert np.max(np.abs(d - ref)) <= bar, (wi, p, d, ref)
    finally:
        negf.negf_tables_free(t)


def test_thermal_grid_matches_oracle_refinement(ctx):
    w0 = inputs.small_wire(607, W=3, L=6, n_energy=1, eta=0.1, disorder=0.9)
    for (lo, hi, n0, tol, cap) in ((-0.6, 0.6, 5, 0.05, 65), (-0.6, 0.6, 3, 0.02, 12)):
        ref, dref = thermal.refine_grid(w0.onsite, w0.eta, w0.t, lo, hi, n0, tol, cap)
        got = negf.negf_thermal_grid(ctx, w0, lo, hi, n0, tol, cap, precision="fp64")
        assert got.size == ref.size, (got.size, ref.size)
        assert np.max(np.abs(got - ref)) <= 1e-14, (got, ref)
        if ref.size < cap:
            assert np.all(dref <= tol)
