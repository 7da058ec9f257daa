"""Writes the stored expected values under tests/golden/ by calling only the
oracle (never the CUDA path).  Re-run after a justified oracle change:

    python tests/golden/make_golden.py            (small molecule, tiny crystal)
    python tests/golden/make_golden.py crystal64  (the 64-atom crystal, ~10 min)
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


def crystal64():
    """The 64-atom crystal (M = 512, 8 k-points): what is free of eigenvector
    phases with the oracle's own reference (eigenvalues of h_core(k),
    occupations, E and the gradient norm per k-point at A = 0), and E and
    seeded gradient entries at the seeded A with the Loewdin reference
    S(k)^(-1/2) and the same occupations.  About ten minutes on eight cores."""
    import numpy as np
    d = synth.config_crystal64()
    o = BlochOracle(d, cache_x=False)
    ref = o.reference_k()
    z = np.zeros(o.nk * o.nvar)
    E0, g0 = o.energy_grad(z)
    o.set_reference(o.lowdin_reference())
    E1, g1 = o.energy_grad(d["a0"])
    idx = np.sort(np.random.default_rng(64).choice(len(g1), size=256, replace=False))
    return {
        "_source": "oracle/etdm_kpoints.py on etdm_synth.config_crystal64() (64 atoms, M=512, "
                   "8 k-points, kT = 0.1 eV, 56^3 grid); E_a0 and g_a0 with the Loewdin "
                   "reference S(k)^(-1/2) and the oracle's occupations, variables a0 ~ N(0, 0.01) "
                   "seed 4; sampled entries at the sorted indices drawn by default_rng(64)",
        "mu": ref["mu"],
        "f": [f.tolist() for f in ref["f"]],
        "eps_core": [e.tolist() for e in ref["eps_core"]],
        "E_0": E0,
        "gnorm_0": [float(np.linalg.norm(g0[k * o.nvar:(k + 1) * o.nvar])) for k in range(o.nk)],
        "E_a0_lowdin": E1,
        "gnorm_a0_lowdin": [float(np.linalg.norm(g1[k * o.nvar:(k + 1) * o.nvar]))
                            for k in range(o.nk)],
        "g_idx": idx.tolist(),
        "g_a0_lowdin": g1[idx].tolist(),
    }


def main():
    if sys.argv[1:] == ["crystal64"]:
        with open(os.path.join(HERE, "crystal64_oracle.json"), "w") as f:
            json.dump(crystal64(), f, indent=1)
        return
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
