"""GPU parity of the Perdew-Zunger self-interaction correction on the full-A
path at the Gamma point (Sec. 2, Eq. 16-18 as read: one self-interaction per
electron, unit orbital densities, spin-polarized exchange; the L of the
orbital-dependent Hamiltonians with each orbital potential weighted by its own
occupation) against the oracle, element by element.  The functional is not
unitary invariant, so the occupied-occupied rotations are variables too."""
import numpy as np
import pytest

import etdm_synth as synth
from oracle.etdm_kpoints import BlochOracle
from oracle.etdm_oracle import minimize

pytestmark = pytest.mark.gpu


def _gamma_full(d):
    g = dict(d)
    g.update(kpts=np.zeros((1, 3)), kw=np.ones(1), kT=0.0)
    return g


CASES = {"small": lambda: _gamma_full(synth.config_small_molecule()),
         "tiny": lambda: _gamma_full(synth.tiny())}


@pytest.fixture(scope="module")
def cases():
    from paper_2101_12597_gb300.etdm import ETDM
    out = {}
    for name, make in CASES.items():
        d = make()
        bo = BlochOracle(d, sic=True)
        s = ETDM(d, functional="pzsic")
        ref = bo.reference_k()
        s.set_reference(np.array(ref["C0"]), np.array(ref["f"]))
        out[name] = (d, bo, s)
    yield out
    for _, _, s in out.values():
        s.close()


@pytest.mark.parametrize("which", list(CASES))
@pytest.mark.parametrize("scale", [0.0, 0.05])
def test_pzsic_energy_gradient_parity(which, scale, cases):
    import torch
    d, bo, s = cases[which]
    a = np.random.default_rng(11).normal(0.0, scale, bo.nvar) if scale else np.zeros(bo.nvar)
    E, g = s.energy_grad(torch.tensor(a, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    s.check()
    E_ref, g_ref, ex = bo.energy_grad(a, want=True)
    g = g.cpu().numpy()
    dE = abs(float(E.item()) - E_ref)
    dg = np.abs(g - g_ref).max() / np.abs(g_ref).max()
    print(f"{which} a~N(0,{scale}): E_SIC={ex['terms']['sic']:.6f} |dE|={dE:.3e} Ha grad err={dg:.3e}")
    assert dE < 1e-9
    assert dg <= 1e-9


def test_pzsic_minimization_trajectory(cases):
    """Ten L-BFGS steps of the small molecule with PZ-SIC from A = 0 (the SIC
    gradient is nonzero there in the occupied-occupied block): energies,
    steps and trials equal the oracle's."""
    import torch
    d, _, s = cases["small"]
    bo = BlochOracle(d, sic=True)
    a = torch.zeros(s.var_shape, dtype=torch.float64, device="cuda")
    s.lbfgs_reset()
    E, al, tr = s.minimize(a, 10)
    hist, a_ref = minimize(bo, np.zeros(bo.nvar), 10)
    E_ref = np.array([h[0] for h in hist])
    print("PZ-SIC trajectory:", np.abs(E - E_ref).max(), E_ref[0] - E_ref[-1])
    assert np.abs(E - E_ref).max() < 1e-9
    assert list(tr) == [h[2] for h in hist]
    assert np.abs(a.cpu().numpy() - a_ref).max() < 1e-6
