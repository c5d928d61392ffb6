"""Pins of the oracle's multi-orbital slices and k-point batching (CPU).

* A slice block equal to the square-lattice cross-section (-t between neighbours) reproduces
  the default model: H, G and every Step 6' weight (the slice's eigenvectors are the sine
  modes up to sign, which no weight sees).
* Channel staircase of a clean multi-orbital strip (no dephasing, exact leads): the direct
  transmission Tr[Gamma_L G Gamma_R G^dag] equals the number of slice levels eps_m with
  |E - eps_m| < 2t, counted from the eigenvalues of the slice block alone.
* The modal lead self-energy solves the surface Dyson equation of the semi-infinite lead,
  Sigma = t^2 (E - h - Sigma)^{-1}, with Im Sigma <= 0 (retarded), in and out of the bands.
* k-points: without dephasing, the transmission of a film slab periodic over n_z cells in z
  (real space, its slice block n_z copies of the wire's coupled by -t_z) equals the sum over
  the n_z Bloch wavevectors of the wire with onsite energies shifted by -2 t_z cos k (Bloch's
  theorem; the disorder is the same in every z cell).
"""
import numpy as np

from oracle import buttiker, markov, wire
from paper_1805_10164_gb300 import inputs


def _square_slice(W, t):
    h = np.zeros((W, W))
    for a in range(W - 1):
        h[a, a + 1] = h[a + 1, a] = -t
    return h


def test_square_lattice_slice_reproduces_default_model():
    w = inputs.small_wire(701, W=4, L=5, n_energy=1, eta=0.12)
    E = 0.37
    h = _square_slice(w.W, w.t)
    g0 = wire.green_retarded(E, w.onsite, w.eta, w.t)
    g1 = wire.green_retarded(E, w.onsite, w.eta, w.t, slice_h=h)
    assert np.array_equal(g0["H"], g1["H"])
    assert np.max(np.abs(g0["G"] - g1["G"])) <= 1e-12 * np.abs(g0["G"]).max()
    t0 = markov.transition_weights(g0, wire.lead_modes(E, w.W, w.t)[0::2])
    t1 = markov.transition_weights(g1, wire.lead_modes(E, w.W, w.t, slice_h=h)[0::2])
    assert np.max(np.abs(t0["w"] - t1["w"])) <= 1e-11 * t0["w"].max()
    assert np.allclose(t0["mode_w"], t1["mode_w"], rtol=1e-10, atol=1e-14)
    assert np.allclose(t0["c"], t1["c"], rtol=1e-10)


def test_clean_multiorbital_strip_staircase():
    n_atoms, L, t = 3, 4, 1.0
    h = inputs.sp3_slice(n_atoms)
    W = h.shape[0]
    eps = np.linalg.eigvalsh(h)
    edges = np.sort(np.concatenate([eps - 2 * t, eps + 2 * t]))
    # energies halfway between consecutive band edges, plus one below and one above all bands
    probes = np.concatenate([[edges[0] - 0.3], 0.5 * (edges[1:] + edges[:-1]), [edges[-1] + 0.3]])
    probes = probes[np.min(np.abs(probes[:, None] - edges[None, :]), axis=1) > 1e-3]
    zeros = np.zeros((L, W))
    seen = set()
    for E in probes:
        g = wire.green_retarded(E, zeros, zeros, t, slice_h=h)
        T = buttiker.effective_transmission(g)[1, 0]
        n_open = int(np.sum(np.abs(E - eps) < 2 * t))
        seen.add(n_open)
        assert abs(T - n_open) <= 1e-9, (E, T, n_open)
    assert len(seen) >= 5


def test_modal_lead_self_energy_solves_surface_dyson():
    h = inputs.sp3_slice(2)
    W = h.shape[0]
    t = 1.0
    for E in (-2.7, -0.4, 0.9, 2.2, 4.6):
        phi, sig, gam = wire.lead_modes(E, W, t, slice_h=h)
        S = phi @ np.diag(sig) @ phi.T
        rhs = t * t * np.linalg.inv(E * np.eye(W) - h - S)
        assert np.max(np.abs(S - rhs)) <= 1e-11, E
        assert np.all(np.linalg.eigvalsh(-S.imag) >= -1e-12)
        assert np.allclose(phi @ phi.T, np.eye(W), atol=1e-12)
        assert np.allclose(gam, -2.0 * sig.imag)


def test_film_kpoints_equal_periodic_slab():
    n_atoms, L, n_z, t_z = 2, 4, 3, 0.35
    w = inputs.sp3_wire(702, n_atoms, L, n_energy=1, eta=0.0, disorder=0.6)
    w.eta = np.zeros_like(w.eta)
    slab_h = inputs.film_slab_slice(w.slice_h, n_z, t_z)
    slab_on = np.tile(w.onsite, (1, n_z))           # the same disorder in every z cell
    zeros = np.zeros_like(slab_on)
    # energies at least 0.05 from every channel edge of every k (the surface Green's functions
    # lose digits next to an edge)
    edges = np.concatenate([np.linalg.eigvalsh(wk.slice_h) + s * 2 * w.t
                            for wk in inputs.film_kpoints(w, t_z, n_z) for s in (-1, 1)])
    grid = np.linspace(-3.0, 4.0, 701)
    ok = grid[np.min(np.abs(grid[:, None] - edges[None, :]), axis=1) > 0.05]
    for E in ok[:: max(1, ok.size // 4)][:4]:
        g = wire.green_retarded(E, slab_on, zeros, w.t, slice_h=slab_h)
        T_slab = buttiker.effective_transmission(g)[1, 0]
        T_k = 0.0
        for wk in inputs.film_kpoints(w, t_z, n_z):
            gk = wire.green_retarded(E, wk.onsite, wk.eta, wk.t, slice_h=wk.slice_h)
            T_k += buttiker.effective_transmission(gk)[1, 0]
            assert np.isclose(wk.energy_weight[0] * n_z, w.energy_weight[0])
        assert abs(T_slab - T_k) <= 1e-9 * max(1.0, T_slab), (E, T_slab, T_k)
