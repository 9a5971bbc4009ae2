"""The oracle reproduces its stored values on the chain workload (regression pin)."""
import json
import os

import ccsd_synth as cs
from oracle import ccsd_k, driver

GOLD = os.path.join(os.path.dirname(__file__), "golden", "chain_k4_o4_v8.json")


def test_chain_golden():
    g = json.load(open(GOLD))
    spec = cs.spec_for(g["workload"])
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, cs.generate(spec))
    r = driver.solve(P, n_iter=3)
    N = spec.nk
    assert abs(r["energies"][0].real / N - g["e_mp2_per_cell"]) < 1e-12
    assert abs(r["energies"][2].real / N - g["e_iter3_per_cell"]) < 1e-12
