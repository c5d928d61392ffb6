"""One task (wire, energy) through the oracle end to end (oracle; test infrastructure only).

Composes the pieces in the paper's order: G^r (Eq. eq_for_gr) -> Step 6' weights and Step 4
injection distribution -> Vose alias tables -> exact walk expectation and the direct probe
solve (Eq. buteq).  Nothing here adds arithmetic of its own.

Pinned by: the pins of the functions it composes (wire, markov, buttiker, alias).
"""
import numpy as np

from . import alias, buttiker, markov, wire


def task_reference(onsite, eta, t, E, lead_model=0, gamma_lead=0.0, with_alias=True,
                   with_direct=True, slice_h=None):
    onsite = np.asarray(onsite, dtype=np.float64)
    L, W = onsite.shape
    g = wire.green_retarded(E, onsite, eta, t, lead_model, gamma_lead, slice_h)
    phi, sig, gam = wire.lead_modes(E, W, t, lead_model, gamma_lead, slice_h)
    tab = markov.transition_weights(g, (phi, gam))
    out = dict(g=g, tab=tab, sigma_modes=sig, gamma_modes=gam, W=W, L=L, n=L * W, K=L * W + 2)
    out["exact"] = markov.absorption(tab)
    if with_direct:
        out["T_direct"] = buttiker.effective_transmission(g)
    if with_alias:
        out["entries"] = alias.build_tables(tab["w"])
        out["mode_entries"] = np.stack([alias.vose(tab["mode_w"][p]) for p in range(2)])
        out["c_open"] = tab["c"] > 0
    return out
