"""Pins of the continuous-energy (thermal) sampler's oracle, no GPU.

What fixes each part:
  * Th(E) = -df/dE: the central difference of the Fermi function of oracle.current, its
    integral against the closed-form CDF, the inverse CDF round trip;
  * the direct conductance: a clean chain (T = 1 inside the band) and a clean W = 3 wire
    (T = number of open channels) give G = sums of CDF differences in closed form;
  * the interpolated chain: at alpha = 0 and 1 it is the exact absorbing chain of the grid
    energies (markov.absorption); refining the grid drives its conductance to the direct one at
    the rate of linear interpolation (error ratio near 4 per halving);
  * the replay walker and the estimator: the sampled G within 4 SE of the interpolated chain's
    exact expectation, the energy draws against the restricted logistic CDF (Kolmogorov-Smirnov).
"""
import numpy as np
import pytest

from oracle import alias, current, markov, pipeline, thermal
from paper_1805_10164_gb300 import inputs


def test_th_is_minus_fermi_derivative():
    mu, kT, h = 0.2, 0.04, 1e-6
    E = np.linspace(-0.5, 0.9, 57)
    fd = (current.fermi(E - h, mu, kT) - current.fermi(E + h, mu, kT)) / (2 * h)
    assert np.allclose(thermal.th_density(E, mu, kT), fd, rtol=1e-6, atol=1e-9)
    x = np.linspace(-1.0, 1.5, 200001)
    integral = np.trapezoid(thermal.th_density(x, mu, kT), x)
    assert abs(integral - (thermal.th_cdf(1.5, mu, kT) - thermal.th_cdf(-1.0, mu, kT))) < 1e-8
    assert np.allclose(thermal.th_cdf(E, mu, kT), 1.0 - current.fermi(E, mu, kT), atol=1e-15)
    p = np.array([1e-6, 0.2, 0.5, 0.93])
    assert np.allclose(thermal.th_cdf(thermal.th_inverse(p, mu, kT), mu, kT), p, rtol=1e-12)


def test_direct_conductance_closed_forms():
    mu, kT = 0.05, 0.1
    grid = np.linspace(-0.6, 0.7, 5)
    L = 12
    G = thermal.conductance_direct(np.zeros((L, 1)), np.zeros((L, 1)), 1.0, grid, mu, kT,
                                   n_quad=8)
    assert abs(G - (thermal.th_cdf(0.7, mu, kT) - thermal.th_cdf(-0.6, mu, kT))) < 1e-9
    # clean W = 3 wire: channel m open for |E - eps_m| < 2t
    W, t = 3, 1.0
    grid = np.linspace(-3.4, -2.2, 7)          # crosses the lowest channel's band edges only
    mu, kT = -2.8, 0.15
    eps = -2.0 * t * np.cos(np.arange(1, W + 1) * np.pi / (W + 1))
    ref = 0.0
    for e in eps:
        lo, hi = max(grid[0], e - 2 * t), min(grid[-1], e + 2 * t)
        if hi > lo:
            ref += thermal.th_cdf(hi, mu, kT) - thermal.th_cdf(lo, mu, kT)
    # the staircase is discontinuous inside the span: split the quadrature at the edges
    edges = np.sort(np.concatenate([grid, [e - 2 * t for e in eps if grid[0] < e - 2 * t
                                            < grid[-1]]]))
    G = thermal.conductance_direct(np.zeros((6, W)), np.zeros((6, W)), t, edges, mu, kT,
                                   n_quad=12)
    assert abs(G - ref) < 1e-7, (G, ref)


def _wire():
    return inputs.small_wire(501, W=3, L=6, n_energy=1, eta=0.15, disorder=0.8)


def _tabs(w, grid):
    return [pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False)["tab"]
            for E in grid]


def test_interpolated_chain_endpoints_and_convergence():
    w = _wire()
    grid = np.array([0.1, 0.35])
    ti, tj = _tabs(w, grid)
    for alpha, tab in ((0.0, ti), (1.0, tj)):
        P = thermal.interpolated_absorption(ti, tj, alpha, p=0)
        assert np.allclose(P, markov.absorption(tab)["P_inj"][0], atol=1e-12)
    # grid refinement: error of the interpolated conductance falls like h^2
    mu, kT = 0.2, 0.08
    lo, hi = -0.2, 0.6
    G_ref = thermal.conductance_direct(w.onsite, w.eta, w.t, np.linspace(lo, hi, 9), mu, kT)
    errs = []
    for m in (3, 5, 9):
        g = np.linspace(lo, hi, m)
        errs.append(abs(thermal.conductance_interpolated(_tabs(w, g), g, mu, kT) - G_ref))
    assert errs[2] < errs[1] < errs[0]
    assert 2.0 < errs[1] / errs[2] < 8.0, errs
    assert errs[2] < 2e-3 * G_ref


def test_replay_walker_matches_interpolated_expectation():
    w = _wire()
    grid = np.linspace(-0.2, 0.6, 4)
    mu, kT = 0.2, 0.08
    tabs = _tabs(w, grid)
    entries = [alias.build_tables(t["w"]) for t in tabs]
    mode_entries = [np.stack([alias.build_tables(t["mode_w"][p][None, :])[0] for p in (0, 1)])
                    for t in tabs]
    c = [t["c"] for t in tabs]
    n, W = tabs[0]["n"], tabs[0]["W"]
    N = 3000
    lead, steps, iv, a = thermal.walk(entries, mode_entries, c, n, W, 7, 0, 0xC0FFEE,
                                      np.arange(N, dtype=np.uint64), grid, mu, kT, 1 << 16)
    window = thermal.th_cdf(grid[-1], mu, kT) - thermal.th_cdf(grid[0], mu, kT)
    G, se = thermal.estimate(lead, a, iv, c, window, 0)
    G_exact = thermal.conductance_interpolated(tabs, grid, mu, kT)
    assert abs(G - G_exact) <= 3.0 * se, (G, G_exact, se)
    # the energy draws follow Th restricted to the span (Kolmogorov-Smirnov, 1 % level)
    E = grid[iv] + (a.astype(np.float64) / 2.0 ** 32) * (grid[iv + 1] - grid[iv])
    F = (thermal.th_cdf(np.sort(E), mu, kT) - thermal.th_cdf(grid[0], mu, kT)) / window
    D = np.max(np.maximum(np.arange(1, N + 1) / N - F, F - np.arange(N) / N))
    assert D < 1.63 / np.sqrt(N), D


@pytest.mark.parametrize("bad", ["drop_c_interp", "uniform_energy"])
def test_planted_mistakes_are_caught(bad):
    """A sampler that ignores the interpolation of c, or draws E uniformly, misses the exact
    expectation (each would pass a test too weak to pin the estimator)."""
    w = _wire()
    grid = np.linspace(-0.2, 0.6, 3)
    mu, kT = 0.1, 0.06
    tabs = _tabs(w, grid)
    G_exact = thermal.conductance_interpolated(tabs, grid, mu, kT)
    xg, wg = np.polynomial.legendre.leggauss(16)
    total = 0.0
    for i in range(grid.size - 1):
        lo, hi = grid[i], grid[i + 1]
        for x, wq in zip(xg, wg):
            alpha = 0.5 * (x + 1.0)
            E = lo + alpha * (hi - lo)
            P = thermal.interpolated_absorption(tabs[i], tabs[i + 1], alpha, 0)
            c = tabs[i]["c"][0] if bad == "drop_c_interp" else \
                (1 - alpha) * tabs[i]["c"][0] + alpha * tabs[i + 1]["c"][0]
            dens = thermal.th_density(E, mu, kT) if bad == "drop_c_interp" else \
                (thermal.th_cdf(grid[-1], mu, kT) - thermal.th_cdf(grid[0], mu, kT)) / \
                (grid[-1] - grid[0])
            total += 0.5 * (hi - lo) * wq * dens * c * P[1]
    assert abs(total - G_exact) > 1e-3 * G_exact


def test_interval_distance_properties():
    w = inputs.small_wire(611, W=3, L=5, n_energy=1, eta=0.12)
    ta, tb = _tabs(w, [0.31, 0.37])
    assert thermal.interval_distance(ta, ta) == 0.0
    d = thermal.interval_distance(ta, tb)
    assert d == thermal.interval_distance(tb, ta)
    assert 0.0 < d <= 1.0
    # a closed start lead at one end only: the relative change of c is 1
    closed = dict(ta, c=np.array([0.0, ta["c"][1]]), mode_w=np.zeros_like(ta["mode_w"]))
    assert thermal.interval_distance(closed, tb) == 1.0


def test_refined_grid_meets_tolerance_and_converges():
    """The paper's rule (interpolate where the ends differ by less than 5 %): every interval of
    the refined grid passes, and the interpolated conductance approaches the direct one as the
    tolerance shrinks, about as its square (interval widths scale with the tolerance)."""
    w = inputs.small_wire(603, W=4, L=6, n_energy=1, eta=0.1, disorder=0.6)
    mu, kT = 0.15, 0.06
    errs = []
    for tol in (0.2, 0.05):
        grid, d = thermal.refine_grid(w.onsite, w.eta, w.t, mu - 5 * kT, mu + 5 * kT, 3, tol=tol)
        assert np.all(d <= tol) and np.all(np.diff(grid) > 0)
        tabs = _tabs(w, grid)
        G_int = thermal.conductance_interpolated(tabs, grid, mu, kT, n_quad=24)
        G_dir = thermal.conductance_direct(w.onsite, w.eta, w.t, grid, mu, kT, n_quad=8)
        errs.append(abs(G_int - G_dir) / G_dir)
    assert errs[1] < errs[0] / 8.0 and errs[1] < 1e-3, errs
    # the cap on the number of points is honoured
    grid, d = thermal.refine_grid(w.onsite, w.eta, w.t, mu - 5 * kT, mu + 5 * kT, 3, tol=1e-4,
                                  max_points=9)
    assert grid.size == 9 and np.any(d > 1e-4)
