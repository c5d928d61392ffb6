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
