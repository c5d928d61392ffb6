"""Seeded synthetic wires shaped like the paper's nanowires (Sec. IV: narrow, long,
dephasing-dominated).  The paper's CdTe tight-binding parameters are not available, so square
lattices with uniform onsite disorder stand in for them.

This module only draws inputs (numpy PCG64 from a seed); it holds none of the method's
arithmetic, and both the GPU path and the CPU oracle take their inputs from it.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Wire:
    W: int
    L: int
    t: float
    onsite: np.ndarray          # [L, W] float64
    eta: np.ndarray             # [L, W] float64, Buttiker gamma_i (Sigma_s = -i eta / 2)
    energy: np.ndarray          # [n_energy] float64
    energy_weight: np.ndarray   # [n_energy] float64 quadrature weights
    lead_model: int = 0
    gamma_lead: float = 0.0
    slice_h: np.ndarray = None  # [W, W] multi-orbital slice block (None: square lattice)


@dataclass
class Workload:
    name: str
    wires: list
    walkers_per_task: int
    mu_p: float
    mu_q: float
    kT: float
    precision: str              # "fp64" | "fp32" | "split_tf32"
    seed: int
    meta: dict = field(default_factory=dict)


def midpoint_grid(e_min, e_max, n):
    de = (e_max - e_min) / n
    return e_min + de * (np.arange(n) + 0.5), np.full(n, de)


def random_wire(rng, W, L, t, disorder, eta, energy, energy_weight, lead_model=0,
                gamma_lead=0.0):
    onsite = rng.uniform(-disorder, disorder, size=(L, W))
    eta_arr = np.full((L, W), float(eta))
    return Wire(W=W, L=L, t=t, onsite=onsite, eta=eta_arr, energy=np.asarray(energy, float),
                energy_weight=np.asarray(energy_weight, float), lead_model=lead_model,
                gamma_lead=gamma_lead)


def chain_l20(seed=0, walkers=100_000):
    """1D chain, L = 20, t = 1, onsite U[-0.5, 0.5], eta = 0.1 on every site, one energy
    E = 0.5, bias window mu = 0.5 +- 0.025 at kT = 0.025, FP64."""
    rng = np.random.default_rng(seed)
    w = random_wire(rng, 1, 20, 1.0, 0.5, 0.1, [0.5], [1.0])
    return Workload("chain_L20_eta0.1_E0.5", [w], walkers, 0.525, 0.475, 0.025, "fp64", seed)


def wire_10x50(seed=1, walkers=1_000_000, n_energy=64, precision="fp32"):
    """2D wire W = 10 x L = 50, t = 1, onsite U[-1, 1], eta = 0.05, 64 midpoint energies on
    [-3.5, 3.5]; the grid is the bias window (mu_L = 3.5, mu_R = -3.5, kT = 0.025)."""
    rng = np.random.default_rng(seed)
    E, wE = midpoint_grid(-3.5, 3.5, n_energy)
    w = random_wire(rng, 10, 50, 1.0, 1.0, 0.05, E, wE)
    return Workload("wire_W10_L50_eta0.05_64E", [w], walkers, 3.5, -3.5, 0.025, precision, seed)


def batched_uneven(seed=2, n_wires=256, walkers=1_000_000, n_energy=32, precision="fp32"):
    """256 wires, W uniform in {4..32}, L uniform in {20..200}, eta log-uniform in
    [0.01, 0.2], onsite U[-1, 1], 32 midpoint energies on [-3.5, 3.5] each."""
    rng = np.random.default_rng(seed)
    E, wE = midpoint_grid(-3.5, 3.5, n_energy)
    wires = []
    for _ in range(n_wires):
        W = int(rng.integers(4, 33))
        L = int(rng.integers(20, 201))
        eta = float(np.exp(rng.uniform(np.log(0.01), np.log(0.2))))
        wires.append(random_wire(rng, W, L, 1.0, 1.0, eta, E, wE))
    return Workload("batched_256_wires_W4-32_L20-200_32E", wires, walkers, 3.5, -3.5, 0.025,
                    precision, seed)


def wire_16x100(seed=3, walkers=1_000_000, n_energy=16, precision="fp64"):
    """Differentiation case: W = 16 x L = 100, onsite U[-1, 1], eta = 0.05, 16 energies."""
    rng = np.random.default_rng(seed)
    E, wE = midpoint_grid(-3.5, 3.5, n_energy)
    w = random_wire(rng, 16, 100, 1.0, 1.0, 0.05, E, wE)
    return Workload("wire_W16_L100_eta0.05_16E", [w], walkers, 3.5, -3.5, 0.025, precision,
                    seed)


def wire_64x1000(seed=4, n_energy=256, precision="fp32", walkers=32_000_000):
    """Weak scattering: W = 64 x L = 1000, onsite U[-0.5, 0.5], eta = 0.005, 256 energies.
    About 3.1 transitions per walk, so 3.2e7 walkers per energy give ~1e8 walker steps.
    FP32 tables (CUDA-core block products); precision="split_tf32" selects the tensor-core
    block products."""
    rng = np.random.default_rng(seed)
    E, wE = midpoint_grid(-3.5, 3.5, n_energy)
    w = random_wire(rng, 64, 1000, 1.0, 0.5, 0.005, E, wE)
    return Workload("wire_W64_L1000_eta0.005_256E", [w], walkers, 3.5, -3.5, 0.025, precision,
                    seed, meta=dict(steps_per_task=100_000_000))


def wire_32x100(seed=6, n_energy=8, precision="fp32", walkers=1_000_000):
    """W = 32 x L = 100, onsite U[-1, 1], eta = 0.05, 8 energies: slices as wide as the widest
    of the batched wires, on a case small enough for full ncu captures (tables ~0.7 GB)."""
    rng = np.random.default_rng(seed)
    E, wE = midpoint_grid(-3.5, 3.5, n_energy)
    w = random_wire(rng, 32, 100, 1.0, 1.0, 0.05, E, wE)
    return Workload("wire_W32_L100_eta0.05_8E", [w], walkers, 3.5, -3.5, 0.025, precision,
                    seed)


def wire_64x100(seed=5, n_energy=8, precision="fp32", walkers=1_000_000):
    """W = 64 x L = 100, onsite U[-0.5, 0.5], eta = 0.005, 8 energies: the wide-slice kernels
    on a case small enough for full ncu captures (tables ~0.7 GB)."""
    rng = np.random.default_rng(seed)
    E, wE = midpoint_grid(-3.5, 3.5, n_energy)
    w = random_wire(rng, 64, 100, 1.0, 0.5, 0.005, E, wE)
    return Workload("wire_W64_L100_eta0.005_8E", [w], walkers, 3.5, -3.5, 0.025, precision,
                    seed)


def small_wire(seed, W, L, n_energy=3, eta=0.1, disorder=1.0, t=1.0, e_lo=-2.9, e_hi=2.9,
               lead_model=0, gamma_lead=0.0):
    """Small seeded wire for parity tests (sizes the oracle finishes in seconds)."""
    rng = np.random.default_rng(seed)
    E, wE = midpoint_grid(e_lo, e_hi, n_energy)
    return random_wire(rng, W, L, t, disorder, eta, E, wE, lead_model, gamma_lead)


# ---------------------------------------------------------------- multi-orbital slices, k-points

# Synthetic sp3-like parameters (units of the slice-to-slice hopping t): onsite energies of the
# s, px, py, pz orbitals (the p levels split so that no two slice modes are degenerate) and the
# two-centre couplings of neighbouring atoms along the slice (ss sigma, sp sigma, pp sigma,
# pp pi).  The paper's CdTe parameters are not available.
SP3 = dict(Es=-1.0, Epx=1.2, Epy=1.5, Epz=1.8, ss=-0.6, sp=0.5, pps=0.7, ppp=-0.25)


def sp3_slice(n_atoms, params=None):
    """[4 n_atoms, 4 n_atoms] block of a slice: n_atoms atoms in a row along y, orbitals
    (s, px, py, pz) per atom (index 4 a + orbital); neighbouring atoms coupled by the
    two-centre blocks of the bond direction y (direction cosines (0, 1, 0))."""
    p = dict(SP3, **(params or {}))
    W = 4 * n_atoms
    h = np.zeros((W, W))
    for a in range(n_atoms):
        o = 4 * a
        h[o, o], h[o + 1, o + 1], h[o + 2, o + 2], h[o + 3, o + 3] = (
            p["Es"], p["Epx"], p["Epy"], p["Epz"])
        if a + 1 < n_atoms:
            q = o + 4
            blk = np.zeros((4, 4))
            blk[0, 0] = p["ss"]
            blk[0, 2] = p["sp"]          # s on a, py on a + 1
            blk[2, 0] = -p["sp"]         # py on a, s on a + 1
            blk[1, 1] = p["ppp"]
            blk[2, 2] = p["pps"]
            blk[3, 3] = p["ppp"]
            h[o:o + 4, q:q + 4] = blk
            h[q:q + 4, o:o + 4] = blk.T
    return h


def sp3_wire(seed, n_atoms, L, n_energy=3, eta=0.1, disorder=0.5, t=1.0, e_lo=-2.5, e_hi=3.5,
             lead_model=0, gamma_lead=0.0, params=None):
    """Multi-orbital wire: the sp3-like slice block on every slice (W = 4 n_atoms orbitals),
    onsite disorder U[-disorder, disorder] per orbital, Buttiker rate eta per orbital,
    orbital-diagonal hopping -t between slices."""
    rng = np.random.default_rng(seed)
    E, wE = midpoint_grid(e_lo, e_hi, n_energy)
    w = random_wire(rng, 4 * n_atoms, L, t, disorder, eta, E, wE, lead_model, gamma_lead)
    w.slice_h = sp3_slice(n_atoms, params)
    return w


def film_kpoints(w, t_z, n_k):
    """A film periodic along z (period one slice cross-section; hopping -t_z between the same
    orbital of z-neighbours, t_z a scalar or one value per orbital): its Bloch Hamiltonian at
    k_j = 2 pi j / n_k, leads included, is the wire's with the slice block shifted by
    diag(-2 t_z cos k_j).  Returns one wire per k-point, energy weights divided by n_k (the
    k-average), for the batch."""
    h0 = w.slice_h
    if h0 is None:                      # the square-lattice cross-section as a slice block
        h0 = np.zeros((w.W, w.W))
        for a in range(w.W - 1):
            h0[a, a + 1] = h0[a + 1, a] = -w.t
    tz = np.broadcast_to(np.asarray(t_z, dtype=np.float64), (w.W,))
    out = []
    for j in range(n_k):
        hk = h0 + np.diag(-2.0 * tz * np.cos(2.0 * np.pi * j / n_k))
        out.append(Wire(W=w.W, L=w.L, t=w.t, onsite=w.onsite, eta=w.eta, energy=w.energy,
                        energy_weight=w.energy_weight / n_k, lead_model=w.lead_model,
                        gamma_lead=w.gamma_lead, slice_h=hk))
    return out


def film_slab_slice(slice_h, n_z, t_z):
    """The slice block of the same film in real space over n_z periods along z (periodic):
    n_z copies of slice_h (index z W + a) with -t_z between the same orbital of z-neighbours."""
    W = slice_h.shape[0]
    h = np.kron(np.eye(n_z), slice_h)
    for z in range(n_z):
        z2 = (z + 1) % n_z
        if z2 == z:
            continue
        for a in range(W):
            h[z * W + a, z2 * W + a] += -t_z
            h[z2 * W + a, z * W + a] += -t_z
    return h
