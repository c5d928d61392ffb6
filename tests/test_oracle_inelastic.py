"""Pins of the inelastic oracle (Step 7', oracle/inelastic.py), all on the CPU.

* sigma = 0 (lambda~ ~ delta(E - E')) is the elastic limit: every injection energy's absorption
  probabilities and mean steps equal those of its own elastic chain (markov.absorption).
* A grid of one repeated energy: the tables of every grid point are the same, so any energy
  hop leaves the walk's law unchanged and any sigma gives the elastic chain.
* Probability conservation, P(L | p, E_0) + P(R | p, E_0) = 1 at every open energy.
* The energy draw is the one of Eq. draw_E_last under the model's lambda~: the hop weights are
  w_e' K A_ii(E_e'), and their alias rows realise them exactly (integer implied distribution).
* The CPU walker's samples (Philox streams, alias rows of both draws) against the exact chain:
  absorption probabilities and mean steps within the family-wise z bars.
* A planted mistake (the hop weighted by the spectral weight at the current energy instead of
  the drawn one) moves the absorption probabilities beyond the rounding bar, so the pins above
  would see it.
"""
import numpy as np
import pytest

from mc_bars import z_bar
from oracle import alias, inelastic, markov, pipeline
from paper_1805_10164_gb300 import inputs


def _wire_tabs(seed, W, L, E, eta):
    rng = np.random.default_rng(seed)
    on = rng.uniform(-1, 1, (L, W))
    et = np.full((L, W), eta)
    refs = [pipeline.task_reference(on, et, 1.0, e, with_direct=False) for e in E]
    return refs


def test_elastic_limit_is_the_elastic_chain():
    E, wE = inputs.midpoint_grid(-2.5, 2.5, 5)
    refs = _wire_tabs(3, 3, 5, E, 0.3)
    ch = inelastic.chain([r["tab"] for r in refs], E, wE, 0.0)
    for e, r in enumerate(refs):
        ex = markov.absorption(r["tab"])
        for p in range(2):
            if r["tab"]["c"][p] <= 0:
                continue
            assert np.allclose(ch["P_inj"][e, p], ex["P_inj"][p], rtol=0, atol=1e-12)
            assert abs(ch["steps_inj"][e, p] - ex["steps_inj"][p]) <= 1e-10 * ex["steps_inj"][p]
        assert np.allclose(ch["T"][e], ex["T_eff"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("sigma", [0.1, 1.0, 10.0])
def test_repeated_energy_grid_is_elastic_for_any_sigma(sigma):
    E = np.full(3, 0.35)
    wE = np.full(3, 0.2)
    refs = _wire_tabs(5, 2, 6, E, 0.5)
    ch = inelastic.chain([r["tab"] for r in refs], E, wE, sigma)
    ex = markov.absorption(refs[0]["tab"])
    for e in range(3):
        assert np.allclose(ch["P_inj"][e], ex["P_inj"], rtol=0, atol=1e-12)
        assert np.allclose(ch["steps_inj"][e], ex["steps_inj"], rtol=1e-10, atol=0)


def test_probability_is_conserved_and_hops_follow_the_model():
    E, wE = inputs.midpoint_grid(-3.0, 3.0, 6)
    refs = _wire_tabs(7, 3, 4, E, 0.4)
    sigma = 0.7
    ch = inelastic.chain([r["tab"] for r in refs], E, wE, sigma)
    for e, r in enumerate(refs):
        for p in range(2):
            if r["tab"]["c"][p] > 0:
                assert abs(ch["P_inj"][e, p].sum() - 1.0) < 1e-12
    # Eq. draw_E_last with the model's lambda~: p(e'|i, e) ~ w_e' K(E_e' - E_e) A_ii(E_e')
    n = refs[0]["n"]
    i, e = 5, 2
    A = np.array([r["tab"]["w"][i].sum() for r in refs])
    want = wE * np.exp(-(E - E[e]) ** 2 / (2 * sigma ** 2)) * A
    assert np.allclose(ch["H"][i, e], want / want.sum(), rtol=1e-14, atol=0)
    # the alias rows of the hops realise them within the quantisation bound
    ent = inelastic.energy_tables(ch["weights"])
    for ii in range(0, n, 3):
        for ee in range(E.size):
            got = alias.implied_distribution(ent[ii, ee])
            assert np.max(np.abs(got - ch["H"][ii, ee])) <= (E.size + 2) / 2**32


def test_walker_samples_match_the_exact_chain():
    E, wE = inputs.midpoint_grid(-2.0, 2.0, 4)
    refs = _wire_tabs(11, 2, 4, E, 0.6)
    sigma = 0.8
    ch = inelastic.chain([r["tab"] for r in refs], E, wE, sigma)
    ent = np.stack([r["entries"] for r in refs])
    ment = np.stack([r["mode_entries"] for r in refs])
    c_open = np.stack([r["c_open"] for r in refs])
    eent = inelastic.energy_tables(ch["weights"])
    n, W = refs[0]["n"], refs[0]["W"]
    N = 20000
    zs = []
    for e0 in range(E.size):
        for p in range(2):
            if not c_open[e0, p]:
                continue
            lead, steps = inelastic.walk(ent, ment, eent, n, W, c_open, e0, 9 + e0, p, 4242,
                                         np.arange(N), 10**6)
            assert np.all(lead >= 0)
            P = ch["P_inj"][e0, p, 1]
            zs.append((np.mean(lead == 1) - P) / np.sqrt(max(P * (1 - P), 1e-300) / N))
            m = ch["steps_inj"][e0, p]
            zs.append((steps.mean() - m) / (steps.std() / np.sqrt(N)))
    zs = np.array(zs)
    assert np.all(np.abs(zs) <= z_bar(zs.size)), zs


def test_planted_hop_mistake_is_caught():
    E, wE = inputs.midpoint_grid(-2.5, 2.5, 5)
    refs = _wire_tabs(13, 3, 4, E, 0.5)
    tabs = [r["tab"] for r in refs]
    sigma = 0.6
    good = inelastic.chain(tabs, E, wE, sigma)
    real = inelastic.energy_weights

    def wrong(A, E_, wE_, s):            # A_ii at the current energy, not at the drawn one
        K = inelastic.energy_kernel(E_, s)
        return K[None, :, :] * (np.asarray(wE_)[None, None, :] * np.asarray(A).T[:, :, None])

    inelastic.energy_weights = wrong
    try:
        bad = inelastic.chain(tabs, E, wE, sigma)
    finally:
        inelastic.energy_weights = real
    assert np.max(np.abs(bad["P_inj"] - good["P_inj"])) > 1e-4
