"""Writes the stored expected values under tests/golden/ by calling only the
oracle (never the CUDA path).  Re-run after a justified oracle change:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import etdm_synth as synth  # noqa: E402
from oracle.etdm_kpoints import BlochOracle  # noqa: E402
from oracle.etdm_oracle import Oracle, minimize  # noqa: E402


def tiny_crystal():
    d = synth.tiny_crystal()
    o = BlochOracle(d)
    E, g = o.energy_grad(d["a0"])
    ref = o.reference_k()
    return {
        "_source": "oracle/etdm_kpoints.py on etdm_synth.tiny_crystal() (2 atoms, M=4, "
                   "2x2x2 Monkhorst-Pack, kT = 0.5 eV, 24x12x12 grid, variables ~ N(0, 0.05) "
                   "seed 6)",
        "E_a0": E,
        "g_a0": g.tolist(),
        "mu": ref["mu"],
        "f": [f.tolist() for f in ref["f"]],
        "eps_core": [e.tolist() for e in ref["eps_core"]],
    }


def main():
    d = synth.config_small_molecule()
    o = Oracle(d)
    E, g = o.energy_grad(d["a0"])
    hist, _ = minimize(o, d["a0"], n_steps=20)
    out = {
        "_source": "oracle/etdm_oracle.py on etdm_synth.config_small_molecule() "
                   "(8 atoms, M=16, N=4, 32^3 grid, A_ov ~ N(0, 0.05) seed 0)",
        "E_a0": E,
        "g_a0": g.tolist(),
        "order": o.reference()["order"].tolist(),
        "trajectory": [{"E": h[0], "alpha": h[1], "trials": h[2]} for h in hist],
    }
    with open(os.path.join(HERE, "small_molecule_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    with open(os.path.join(HERE, "tiny_crystal_oracle.json"), "w") as f:
        json.dump(tiny_crystal(), f, indent=1)


if __name__ == "__main__":
    main()
