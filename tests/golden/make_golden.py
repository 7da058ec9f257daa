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
from oracle.etdm_oracle import Oracle, minimize  # noqa: E402


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


if __name__ == "__main__":
    main()
