"""Multi-orbital slices (sp3-like slice blocks, the exact lead of the slice block) and k-point
batching on the GPU against the oracle.

Bars (those of the parity tests):
  * weights: FP64 1e-10 |w_ref| + 1e-13 rowsum_ref per element, FP32 1e-5 rowsum_ref; row sums,
    mode weights and c_p relative 1e-10 / 1e-5; the slice block's eigenvectors enter only
    through weights, which do not see their signs.
  * alias rows (one- and two-level) realise their weights within the quantisation bound.
  * walks bit-exact against the oracle's walker on the exported tables.
  * Monte Carlo T against the direct probe solve: every |z| <= z_bar(m), sum z^2 <= chi2_bar(m).
  * clean strip (no dephasing, no reflection): c_p = Tr[Gamma_p G Gamma_p G^dag] + T = twice the
    number N of open channels of the slice block (1e-10 FP64), every walker leaves on its first
    draw, half of them at each lead (within z_bar of the binomial SE), so T = c_p n_q / N_w
    estimates N.
  * k-points: a film's k-point wires (slice block shifted by -2 t_z cos k) in one batch equal
    the oracle per k (tables as above, T at the z bars); the current of the batch is the
    k-average.
  * gradient (block-column adjoint, exact-expectation tallies): per component
    1e-6 abs(ref) + 1e-9 max (FP64).
  * an asymmetric or non-finite slice block is NEGF_E_INVALID (host and device inputs).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from mc_bars import chi2_bar, z_bar  # noqa: E402
from oracle import adjoint, alias, buttiker, current as ocur, pipeline, walker, wire  # noqa: E402
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


def _wires():
    return [inputs.sp3_wire(801, 2, 6, n_energy=2, eta=0.12),            # W = 8 (registers)
            inputs.sp3_wire(802, 4, 5, n_energy=2, eta=0.08),            # W = 16
            inputs.sp3_wire(803, 6, 4, n_energy=1, eta=0.06),            # W = 24 (CTA chain)
            inputs.sp3_wire(804, 16, 3, n_energy=1, eta=0.05, disorder=0.3),   # W = 64
            inputs.sp3_wire(805, 3, 4, n_energy=2, eta=0.1, lead_model=1, gamma_lead=0.7)]


def _refs(wires):
    out = []
    for w in wires:
        for E in w.energy:
            out.append(pipeline.task_reference(w.onsite, w.eta, w.t, E, w.lead_model,
                                               w.gamma_lead, with_alias=False,
                                               slice_h=w.slice_h))
    return out


@pytest.fixture(scope="module")
def batch(ctx):
    wires = _wires()
    return wires, _refs(wires)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multiorbital_tables_match_oracle(ctx, batch, precision):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision=precision, keep_weights=True)
    try:
        rt = 1e-10 if precision == "fp64" else 1e-5
        rng = np.random.default_rng(3)
        for task, ref in enumerate(refs):
            tab = ref["tab"]
            w_ref = tab["w"]
            rs_ref = w_ref.sum(1)
            w = negf.negf_export_tables(ctx, tables, task, "weights").reshape(w_ref.shape)
            if precision == "fp64":
                tol = 1e-10 * np.abs(w_ref) + 1e-13 * rs_ref[:, None] + 1e-300
            else:
                tol = 1e-5 * rs_ref[:, None] + 1e-30
            bad = np.abs(w - w_ref) > tol
            assert not bad.any(), (task, np.argwhere(bad)[:5])
            rs = negf.negf_export_tables(ctx, tables, task, "rowsum")
            assert np.allclose(rs, rs_ref, rtol=rt, atol=1e-300)
            mw = negf.negf_export_tables(ctx, tables, task, "mode_weights").reshape(2, -1)
            assert np.allclose(mw, tab["mode_w"], rtol=rt, atol=rt * tab["c"].max() + 1e-300)
            info = negf.negf_get_task_info(ctx, tables, task)
            assert np.allclose(info["c"], tab["c"], rtol=rt, atol=1e-300)
            ent = negf.negf_export_tables(ctx, tables, task, "alias").reshape(w_ref.shape)
            K = w_ref.shape[1]
            for r in rng.choice(w_ref.shape[0], size=min(10, w_ref.shape[0]), replace=False):
                if rs[r] > 0:
                    p = alias.implied_distribution(ent[r])
                    assert np.max(np.abs(p - w[r] / rs[r])) <= (K + 2) / 2**32 + 1e-12, (task, r)
    finally:
        negf.negf_tables_free(tables)


def test_multiorbital_two_level_tables(ctx, batch):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="fp32", layout="two_level")
    try:
        rng = np.random.default_rng(4)
        for task, ref in enumerate(refs):
            info = negf.negf_get_task_info(ctx, tables, task)
            rows, L, W = info["rows"], info["L"], info["W"]
            l2 = negf.negf_export_tables(ctx, tables, task, "alias").view(np.uint32).reshape(
                rows, L, negf.level2_words(W))
            l1 = negf.negf_export_tables(ctx, tables, task, "alias_level1").reshape(rows, L + 2)
            w_ref = ref["tab"]["w"]
            rs_ref = w_ref.sum(1)
            for r in rng.choice(rows, size=min(8, rows), replace=False):
                p = alias.implied_two_level(l1[r], l2[r], W)
                assert np.max(np.abs(p - w_ref[r] / rs_ref[r])) <= (L + W + 4) * 2.0**-32 + 1e-5
    finally:
        negf.negf_tables_free(tables)


def test_multiorbital_walks_bit_exact(ctx, batch):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="fp32")
    try:
        n_w = 2000
        for task in range(len(refs)):
            info = negf.negf_get_task_info(ctx, tables, task)
            ent = negf.negf_export_tables(ctx, tables, task, "alias").reshape(info["rows"], info["K"])
            ment = negf.negf_export_tables(ctx, tables, task, "mode_alias").reshape(2, info["W"])
            for lead0, off in ((0, 0), (1, 2**33 + 5)):
                d_lead = torch.empty(n_w, dtype=torch.int32, device="cuda")
                d_steps = torch.empty(n_w, dtype=torch.int32, device="cuda")
                negf.negf_walk_trace(ctx, tables, task, lead0, 0xD00D + task, off, d_lead,
                                     d_steps)
                lead, steps = walker.walk(ent, ment, info["n"], info["W"], info["c"] > 0, task,
                                          lead0, 0xD00D + task, off + np.arange(n_w), 1 << 20)
                assert np.array_equal(d_lead.cpu().numpy(), lead), (task, lead0)
                assert np.array_equal(d_steps.cpu().numpy().astype(np.uint32), steps)
    finally:
        negf.negf_tables_free(tables)


def test_multiorbital_monte_carlo_transmission(ctx, batch):
    wires, refs = batch
    tables = negf.negf_build_tables(ctx, wires, precision="fp32")
    try:
        N = 400_000
        z = []
        for lead0 in (0, 1):
            tally = negf.negf_walk(ctx, tables, lead0, 31 + lead0, N)
            res = negf.negf_current(ctx, tables, tally, 3.5, -3.5, 0.025)
            negf.negf_tally_free(tally)
            for task, ref in enumerate(refs):
                if ref["tab"]["c"][lead0] > 0:
                    T_ref = ref["T_direct"][1 - lead0, lead0]
                    z.append((res["T"][task] - T_ref) / (res["T_se"][task] + 1e-6 * T_ref))
        z = np.asarray(z)
        assert np.max(np.abs(z)) <= z_bar(z.size) and np.sum(z ** 2) <= chi2_bar(z.size), z
    finally:
        negf.negf_tables_free(tables)


def test_clean_multiorbital_strip_staircase(ctx):
    h = inputs.sp3_slice(3)
    W, L, t = h.shape[0], 4, 1.0
    eps = np.linalg.eigvalsh(h)
    edges = np.sort(np.concatenate([eps - 2 * t, eps + 2 * t]))
    mids = 0.5 * (edges[1:] + edges[:-1])
    mids = mids[np.min(np.abs(mids[:, None] - edges[None, :]), axis=1) > 0.02]
    zeros = np.zeros((L, W))
    w = inputs.Wire(W=W, L=L, t=t, onsite=zeros, eta=zeros, energy=mids,
                    energy_weight=np.ones_like(mids), slice_h=h)
    tables = negf.negf_build_tables(ctx, [w], precision="fp64")
    try:
        N = 200_000
        tally = negf.negf_walk(ctx, tables, 0, 5, N)
        counts = negf.negf_tally_counts(ctx, tally, mids.size)
        res = negf.negf_current(ctx, tables, tally, 1.0, 0.0, 0.1)
        negf.negf_tally_free(tally)
        z = []
        for k, E in enumerate(mids):
            n_open = int(np.sum(np.abs(E - eps) < 2 * t))
            c = negf.negf_get_task_info(ctx, tables, k)["c"][0]
            assert abs(c - 2 * n_open) <= 1e-10 * max(1, n_open), (E, c, n_open)
            if n_open:
                assert counts[k, 1] + counts[k, 2] == N and counts[k, 4] == N   # one draw each
                z.append((counts[k, 2] / N - 0.5) / np.sqrt(0.25 / N))
                assert abs(res["T"][k] - c * counts[k, 2] / N) <= 1e-12 * c
        z = np.asarray(z)
        assert np.max(np.abs(z)) <= z_bar(z.size) and np.sum(z ** 2) <= chi2_bar(z.size), z
    finally:
        negf.negf_tables_free(tables)


def test_film_kpoints_batch(ctx):
    base = inputs.sp3_wire(806, 2, 5, n_energy=3, eta=0.1, e_lo=-1.5, e_hi=2.5)
    n_k, t_z = 4, 0.3
    kw = inputs.film_kpoints(base, t_z, n_k)
    tables = negf.negf_build_tables(ctx, kw, precision="fp64", keep_weights=True)
    try:
        N = 300_000
        tally = negf.negf_walk(ctx, tables, 0, 77, N)
        res = negf.negf_current(ctx, tables, tally, 0.8, 0.2, 0.3)
        negf.negf_tally_free(tally)
        z, task = [], 0
        I_ref = 0.0
        for wk in kw:
            T_ref = []
            for E in wk.energy:
                ref = pipeline.task_reference(wk.onsite, wk.eta, wk.t, E, with_alias=False,
                                              slice_h=wk.slice_h)
                info = negf.negf_get_task_info(ctx, tables, task)
                assert np.allclose(info["c"], ref["tab"]["c"], rtol=1e-10)
                w_gpu = negf.negf_export_tables(ctx, tables, task, "weights").reshape(
                    ref["tab"]["w"].shape)
                rs = ref["tab"]["w"].sum(1)
                assert np.all(np.abs(w_gpu - ref["tab"]["w"]) <=
                              1e-10 * np.abs(ref["tab"]["w"]) + 1e-13 * rs[:, None] + 1e-300)
                T_ref.append(ref["T_direct"][1, 0])
                z.append((res["T"][task] - T_ref[-1]) / (res["T_se"][task] + 1e-9))
                task += 1
            I_k, _ = ocur.current(wk.energy, wk.energy_weight, np.array(T_ref), np.zeros(3),
                                  0.8, 0.2, 0.3)
            I_ref += I_k
        z = np.asarray(z)
        assert np.max(np.abs(z)) <= z_bar(z.size) and np.sum(z ** 2) <= chi2_bar(z.size), z
        # the film's current: the k-average (energy weights already carry 1 / n_k)
        I = float(np.sum(res["I"]))
        se = float(np.sqrt(np.sum(np.square(res["se"]))))
        assert abs(I - I_ref) <= z_bar(1) * se + 1e-12, (I, I_ref, se)
    finally:
        negf.negf_tables_free(tables)


def test_multiorbital_gradient_exact_tallies(ctx):
    w = inputs.sp3_wire(807, 2, 4, n_energy=1, eta=0.15, e_lo=0.1, e_hi=0.3)   # E = 0.2
    p, N = 0, float(2 ** 52)
    tables = negf.negf_build_tables(ctx, [w], precision="fp64", keep_weights=True)
    tally = negf.negf_walk_score(ctx, tables, p, 1, 0)
    try:
        E = float(w.energy[0])
        g = wire.green_retarded(E, w.onsite, w.eta, w.t, slice_h=w.slice_h)
        from oracle import markov
        phi, _, gam = wire.lead_modes(E, w.W, w.t, slice_h=w.slice_h)
        tab = markov.transition_weights(g, (phi, gam))
        n, W = w.W * w.L, w.W
        P = tab["w"] / tab["w"].sum(1, keepdims=True)
        rows, K = P.shape
        IQ = np.eye(n) - P[:n, :n]
        hq = np.linalg.solve(IQ, P[:n, n:])
        u = tab["mode_w"][p] / tab["mode_w"][p].sum()
        inj = slice(n + p * W, n + (p + 1) * W)
        nu = np.zeros(rows)
        nu[inj] = u
        nu[:n] = np.linalg.solve(IQ.T, P[inj, :n].T @ u)
        sc = np.zeros((2, negf.load().negf_tally_score_size(tally)), dtype=np.uint64)
        md = np.zeros((2, negf.load().negf_tally_mode_size(tally)), dtype=np.uint64)
        for rr in range(2):
            hb = np.concatenate([hq[:, rr], [1.0 if rr == 0 else 0.0, 1.0 if rr == 1 else 0.0]])
            sc[rr, :rows * K] = np.rint(N * (nu[:, None] * P * hb[None, :])).reshape(-1)
        v = P[inj, n:] + P[inj, :n] @ hq
        for rr in range(2):
            md[rr, p * W:(p + 1) * W] = np.rint(N * u * v[:, rr])
        Pr = u @ v
        negf.negf_tally_accumulate(ctx, tally, np.rint(np.array([[N, N * Pr[0], N * Pr[1], 0, 0]]))
                                   .astype(np.uint64))
        negf.negf_tally_score_accumulate(ctx, tally, sc, md)
        mu_p, mu_q, kT = 0.6, -0.4, 0.3
        dV, dE, cap = negf.negf_current_backward_rgf(ctx, tables, tally, mu_p, mu_q, kT, [1.0], n)
        assert not cap
        f = w.energy_weight[0] * (ocur.fermi(E, mu_p, kT) - ocur.fermi(E, mu_q, kT))
        _, gV, gE = adjoint.transmission_gradient(w.onsite, w.eta, w.t, E, p, 1 - p,
                                                  slice_h=w.slice_h)
        gV, gE = f * gV.reshape(-1), f * gE.reshape(-1)
        scale = max(np.abs(gV).max(), np.abs(gE).max())
        for got, ref in ((dV, gV), (dE, gE)):
            assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref) + 1e-9 * scale), \
                np.abs(got - ref).max() / scale
    finally:
        negf.negf_tally_free(tally)
        negf.negf_tables_free(tables)


def test_slice_block_device_inputs_and_refusals(ctx):
    w = inputs.sp3_wire(808, 2, 4, n_energy=2, eta=0.1)
    host = negf.negf_build_tables(ctx, [w], precision="fp32")
    dev = inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=torch.from_numpy(w.onsite).cuda(),
                      eta=torch.from_numpy(w.eta).cuda(), energy=torch.from_numpy(w.energy).cuda(),
                      energy_weight=torch.from_numpy(w.energy_weight).cuda(),
                      slice_h=torch.from_numpy(w.slice_h).cuda())
    t_dev = negf.negf_build_tables(ctx, [dev], precision="fp32", memspace="device")
    try:
        for k in range(2):
            a = negf.negf_export_tables(ctx, host, k, "alias")
            b = negf.negf_export_tables(ctx, t_dev, k, "alias")
            assert np.array_equal(a, b), k
    finally:
        negf.negf_tables_free(host)
        negf.negf_tables_free(t_dev)
    bad = inputs.sp3_wire(808, 2, 4, n_energy=1, eta=0.1)
    bad.slice_h = bad.slice_h.copy()
    bad.slice_h[0, 1] += 1e-3                                   # not symmetric
    with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
        negf.negf_build_tables(ctx, [bad])
    bad_dev = inputs.Wire(W=bad.W, L=bad.L, t=bad.t, onsite=torch.from_numpy(bad.onsite).cuda(),
                          eta=torch.from_numpy(bad.eta).cuda(),
                          energy=torch.from_numpy(bad.energy).cuda(),
                          energy_weight=torch.from_numpy(bad.energy_weight).cuda(),
                          slice_h=torch.from_numpy(bad.slice_h).cuda())
    with pytest.raises(negf.NegfError, match="NEGF_E_INVALID"):
        t = negf.negf_build_tables(ctx, [bad_dev], memspace="device")
        try:
            negf.negf_get_task_info(ctx, t, 0)      # device values are checked on the device
            negf.negf_export_tables(ctx, t, 0, "alias")
        finally:
            negf.negf_tables_free(t)
