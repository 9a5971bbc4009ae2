"""Writes the stored oracle values under tests/golden/ (run from the repo root).

  python tests/golden/make_golden.py [chain_k4_o4_v8] [grid222_o8_v32]

The paper prints no numerical example, so every stored value here comes from
the CPU oracle (form A and its driver) on seeded synthetic workloads:
  chain_k4_o4_v8  N_k = 4 (1D, k = 2 pi n / 4), 4 occupied and 8 virtual spin
                  orbitals per k, seed 1001: converged energies;
  grid222_o8_v32  2x2x2 k grid (N_k = 8), 8 occupied and 32 virtual spin orbitals
                  per k, seed 1002 (vvvv 8.6 GB): the first two updates from t = 0
                  with DIIS(6), the second one extrapolated (about 10 minutes and
                  40 GB on 8 cores).
Energies are per unit cell (total supercell energy / N_k)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ccsd_synth as cs  # noqa: E402
from oracle import ccsd_k, driver  # noqa: E402


def chain():
    name = "chain_k4_o4_v8"
    spec = cs.spec_for(name)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, cs.generate(spec))
    jac = driver.solve(P, tol=1e-10, max_iter=100)
    dii = driver.solve(P, tol=1e-10, max_iter=100, diis_depth=6)
    N = spec.nk
    return name, {
        "workload": name,
        "source": "oracle (tests/golden/make_golden.py); the paper prints no worked example",
        "e_mp2_per_cell": jac["energies"][0].real / N,
        "e_iter3_per_cell": jac["energies"][2].real / N,
        "e_ccsd_per_cell": jac["energies"][-1].real / N,
        "e_ccsd_per_cell_diis6": dii["energies"][-1].real / N,
        "jacobi_iterations_to_1e-10": jac["iters"],
        "diis6_iterations_to_1e-10": dii["iters"],
    }


def grid222():
    name = "grid222_o8_v32"
    spec = cs.spec_for(name)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, cs.generate(spec))
    r = driver.solve(P, n_iter=2, diis_depth=6)
    N = spec.nk
    return name, {
        "workload": name,
        "source": "oracle (tests/golden/make_golden.py): form-A residuals, Jacobi update, DIIS(6); "
                  "the paper prints no worked example",
        "diis_depth": 6,
        "e_per_cell_after_update": [e.real / N for e in r["energies"]],
        "e_imag_per_cell_after_update": [e.imag / N for e in r["energies"]],
        "max_resid_after_update": [float(x) for x in r["max_r"]],
    }


def main(names):
    makers = {"chain_k4_o4_v8": chain, "grid222_o8_v32": grid222}
    for n in names or ["chain_k4_o4_v8"]:
        name, out = makers[n]()
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name + ".json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main(sys.argv[1:])
