"""torch.autograd.Function over the Monte Carlo current of one wire.

Forward: negf_build_tables (keeping the weights when a gradient is wanted, or the dense G for
the dense adjoint), negf_walk_score (negf_walk when not), negf_current.  Backward:
negf_current_backward_rgf (block-column adjoint, left- and right-connected blocks checkpointed
every ckpt_stride slices) or negf_current_backward (dense G), the score-function gradient of
the Monte Carlo current w.r.t. the onsite energies and the Buttiker dephasing of every site.
All arithmetic runs in libnegf's CUDA kernels; this module only marshals arguments.

The current follows Eq. iqof_t_el_db with the estimator of Eq. elast_lin_xpq:
I = sum_E w_E (f(E; mu_p) - f(E; mu_q)) T_qp(E).
"""
from dataclasses import dataclass

import torch

from . import negf

PRECISIONS = ("fp64", "fp32")
ADJOINTS = ("rgf", "dense")


@dataclass
class CurrentSpec:
    """Everything about the current except the differentiable parameters."""
    W: int
    L: int
    t: float
    energy: object                 # 1-D float64 array or tensor
    energy_weight: object = None   # 1-D float64 array or tensor, or None for all 1
    mu_p: float = 0.0
    mu_q: float = 0.0
    kT: float = 0.025
    start_lead: int = 0            # p: walkers are injected from lead p and counted at q = 1 - p
    walkers_per_task: int = 100_000
    seed: int = 0
    walker_id_offset: int = 0
    max_steps: int = 1 << 20
    precision: str = "fp32"
    lead_model: int = 0
    gamma_lead: float = 0.0
    adjoint: str = "rgf"           # "rgf": block-column adjoint; "dense": keeps the n x n G
    ckpt_stride: int = 0           # rgf: keep g^L, g^R every this many slices (0: default 10)
    layout: str = "auto"           # table layout (the dense adjoint needs one-level tables)


@dataclass
class _Wire:
    W: int
    L: int
    t: float
    onsite: object
    eta: object
    energy: object
    energy_weight: object
    lead_model: int
    gamma_lead: float


class _Handles:
    """Owns the tables and tally handles kept from forward for backward."""

    def __init__(self, tables, tally):
        self.tables, self.tally = tables, tally

    def release(self):
        if self.tally is not None:
            negf.negf_tally_free(self.tally)
            self.tally = None
        if self.tables is not None:
            negf.negf_tables_free(self.tables)
            self.tables = None

    def __del__(self):
        self.release()


def _as_device(x, device):
    if x is None:
        return None
    return torch.as_tensor(x, dtype=torch.float64, device=device).contiguous()


class NegfCurrent(torch.autograd.Function):
    """I, SE(I) = NegfCurrent.apply(onsite [L, W], eta [L, W], ctx, spec).

    onsite and eta are float64 CUDA tensors; I and its binomial standard error come back as
    0-d float64 tensors on the same device.  The gradient flows to onsite and eta only; it is
    an unbiased Monte Carlo estimate drawn from the same walks as I.
    """

    @staticmethod
    def forward(fctx, onsite, eta, ctx, spec):
        if spec.precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {PRECISIONS}")
        if spec.adjoint not in ADJOINTS:
            raise ValueError(f"adjoint must be one of {ADJOINTS}")
        if not (onsite.is_cuda and eta.is_cuda):
            raise ValueError("onsite and eta must be CUDA tensors")
        if tuple(onsite.shape) != (spec.L, spec.W) or tuple(eta.shape) != (spec.L, spec.W):
            raise ValueError(f"onsite and eta must have shape ({spec.L}, {spec.W})")
        dev = onsite.device
        wire = _Wire(spec.W, spec.L, spec.t, onsite.detach().to(torch.float64).contiguous(),
                     eta.detach().to(torch.float64).contiguous(),
                     _as_device(spec.energy, dev), _as_device(spec.energy_weight, dev),
                     spec.lead_model, spec.gamma_lead)
        grad = any(fctx.needs_input_grad[:2])
        dense = spec.adjoint == "dense"
        tables = negf.negf_build_tables(ctx, [wire], precision=spec.precision, memspace="device",
                                        keep_weights=grad and not dense,
                                        keep_green=grad and dense, layout=spec.layout)
        walk = negf.negf_walk_score if grad else negf.negf_walk
        try:
            tally = walk(ctx, tables, spec.start_lead, spec.seed, spec.walkers_per_task,
                         walker_id_offset=spec.walker_id_offset, max_steps=spec.max_steps)
        except Exception:
            negf.negf_tables_free(tables)
            raise
        handles = _Handles(tables, tally)
        res = negf.negf_current(ctx, tables, tally, spec.mu_p, spec.mu_q, spec.kT)
        if res["stepcap"]:
            handles.release()
            raise negf.NegfError(negf.NEGF_E_STEPCAP, "walks hit max_steps; raise max_steps")
        if grad:
            fctx.handles = handles
        else:
            handles.release()
        fctx.ctx, fctx.spec = ctx, spec
        I = torch.tensor(float(res["I"][0]), dtype=torch.float64, device=dev)
        se = torch.tensor(float(res["se"][0]), dtype=torch.float64, device=dev)
        fctx.mark_non_differentiable(se)
        return I, se

    @staticmethod
    def backward(fctx, gI, gse):
        spec = fctx.spec
        h = fctx.handles
        if h.tables is None:
            raise RuntimeError("NegfCurrent.backward called twice (retain_graph is not supported)")
        dI = [float(gI.item())]
        try:
            if spec.adjoint == "dense":
                dV, dE, cap = negf.negf_current_backward(fctx.ctx, h.tables, h.tally, spec.mu_p,
                                                         spec.mu_q, spec.kT, dI, spec.W * spec.L)
            else:
                dV, dE, cap = negf.negf_current_backward_rgf(fctx.ctx, h.tables, h.tally,
                                                             spec.mu_p, spec.mu_q, spec.kT, dI,
                                                             spec.W * spec.L, spec.ckpt_stride)
        finally:
            h.release()
        if cap:
            raise negf.NegfError(negf.NEGF_E_STEPCAP, "walks hit max_steps; raise max_steps")
        dev = gI.device
        gV = torch.from_numpy(dV).to(dev).reshape(spec.L, spec.W)
        gEta = torch.from_numpy(dE).to(dev).reshape(spec.L, spec.W)
        return (gV if fctx.needs_input_grad[0] else None,
                gEta if fctx.needs_input_grad[1] else None, None, None)


def current(onsite, eta, ctx, spec):
    """(I, SE) of one wire with autograd support; see NegfCurrent."""
    return NegfCurrent.apply(onsite, eta, ctx, spec)
