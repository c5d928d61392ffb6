"""Writes oracle_small_wires.json: reference values of the CPU FP64 oracle (and of nothing
else) for three seeded small workloads, so that any later change of the oracle's arithmetic
shows up as a failing regression test and has to be justified.

Quantities per (workload, energy), all from oracle/:
  T_direct  effective transmission T^eff_RL of the floating-probe solve (Eq. buteq);
  T_chain   c_L P(R | L) of the exact absorbing Step 6' chain (Eq. elast_lin_xpq, Appendix B);
  c         c_p = Tr Gamma_p A for p = L, R (Eq. lead_out_probability);
  steps     mean transitions of a walk injected from L (Sec. IV.B);
  I         the current of the workload's energy grid and bias (Eq. iqof_t_el_db).

Run from the repository root: python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import current, pipeline  # noqa: E402
from paper_1805_10164_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small_wires.json")


def cases():
    ch = inputs.chain_l20()
    return [
        ("chain_L20_E0.5", ch.wires[0], ch.mu_p, ch.mu_q, ch.kT),
        ("wire_W3_L5_3E", inputs.small_wire(901, W=3, L=5, n_energy=3, eta=0.1), 0.6, -0.4, 0.3),
        ("wire_W4_L4_wideband_2E", inputs.small_wire(902, W=4, L=4, n_energy=2, eta=0.2,
                                                     lead_model=1, gamma_lead=0.7), 0.5, -0.5, 0.2),
    ]


def compute():
    out = {}
    for name, w, mu_p, mu_q, kT in cases():
        rows = []
        T = []
        for E in w.energy:
            r = pipeline.task_reference(w.onsite, w.eta, w.t, E, w.lead_model, w.gamma_lead,
                                        with_alias=False)
            ex = r["exact"]
            rows.append(dict(E=float(E), T_direct=float(r["T_direct"][1, 0]),
                             T_chain=float(ex["T_eff"][1, 0]),
                             c=[float(v) for v in r["tab"]["c"]],
                             steps=float(ex["steps_inj"][0])))
            T.append(float(ex["T_eff"][1, 0]))
        I, _ = current.current(w.energy, w.energy_weight, np.array(T), np.zeros(len(T)), mu_p,
                               mu_q, kT)
        out[name] = dict(energies=rows, mu_p=mu_p, mu_q=mu_q, kT=kT, I=float(I))
    return out


if __name__ == "__main__":
    with open(OUT, "w") as fh:
        json.dump(compute(), fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(OUT)
