"""Writes the stored oracle values under tests/golden/ (run from the repo root).

The paper prints no numerical example, so every stored value here comes from
the CPU oracle on the seeded synthetic chain workload: N_k = 4 (1D, k = 2 pi n / 4),
4 occupied and 8 virtual spin orbitals per k, seed 1001.  Energies are per unit cell
(total supercell energy / N_k)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ccsd_synth as cs  # noqa: E402
from oracle import ccsd_k, driver  # noqa: E402


def main():
    name = "chain_k4_o4_v8"
    spec = cs.spec_for(name)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, cs.generate(spec))
    jac = driver.solve(P, tol=1e-10, max_iter=100)
    dii = driver.solve(P, tol=1e-10, max_iter=100, diis_depth=6)
    N = spec.nk
    out = {
        "workload": name,
        "source": "oracle (tests/golden/make_golden.py); the paper prints no worked example",
        "e_mp2_per_cell": jac["energies"][0].real / N,
        "e_iter3_per_cell": jac["energies"][2].real / N,
        "e_ccsd_per_cell": jac["energies"][-1].real / N,
        "e_ccsd_per_cell_diis6": dii["energies"][-1].real / N,
        "jacobi_iterations_to_1e-10": jac["iters"],
        "diis6_iterations_to_1e-10": dii["iters"],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name + ".json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
