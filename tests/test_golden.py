"""The oracle against its stored reference values (tests/golden/oracle_small_wires.json,
written by tests/golden/make_oracle_golden.py, which calls only oracle/): any change of the
oracle's arithmetic shows up here.  The paper prints no worked example whose inputs can be
rebuilt (its CdTe parameters are missing), so these values come from the oracle itself; they
are pinned independently by tests/test_oracle_pins.py (the probe solve and the absorbing chain
agree, T_direct == T_chain below to 1e-10, as Appendix B states)."""
import importlib.util
import json
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _generator():
    spec = importlib.util.spec_from_file_location(
        "make_oracle_golden", os.path.join(HERE, "golden", "make_oracle_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _close(a, b, rtol=1e-10, atol=1e-13):
    return abs(a - b) <= atol + rtol * abs(b)


def test_oracle_reproduces_its_golden_values():
    with open(os.path.join(HERE, "golden", "oracle_small_wires.json")) as fh:
        stored = json.load(fh)
    now = _generator().compute()
    assert sorted(now) == sorted(stored)
    for name, ref in stored.items():
        got = now[name]
        assert _close(got["I"], ref["I"]), name
        for g, r in zip(got["energies"], ref["energies"], strict=True):
            for key in ("E", "T_direct", "T_chain", "steps"):
                assert _close(g[key], r[key]), (name, key, g[key], r[key])
            for gc, rc in zip(g["c"], r["c"], strict=True):
                assert _close(gc, rc), (name, "c")


@pytest.mark.parametrize("name", ["chain_L20_E0.5", "wire_W3_L5_3E", "wire_W4_L4_wideband_2E"])
def test_golden_routes_agree(name):
    """Within the stored values: the direct probe solve and the exact chain agree (the central
    identity, Appendix B), and the walks are injected with c_p > 0 where T > 0."""
    with open(os.path.join(HERE, "golden", "oracle_small_wires.json")) as fh:
        ref = json.load(fh)[name]
    for e in ref["energies"]:
        assert abs(e["T_direct"] - e["T_chain"]) <= 1e-10 * max(1.0, e["T_direct"])
        if e["T_direct"] > 0:
            assert e["c"][0] > 0 and e["steps"] >= 1.0
