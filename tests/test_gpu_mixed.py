"""Mixed-precision path (tensor-core grid passes) against the FP64 oracle.

Bars: truncation lists of the 4x4x8 tiles bit-exact; energy within 1e-6 Ha;
gradient within 1e-5 of max|g| (max-abs); the minimization trajectory of the
8-atom system identical in accepted steps and within 1e-6 Ha per step.
"""
import numpy as np
import pytest

import etdm_synth as synth
from oracle.etdm_oracle import Oracle, minimize

pytestmark = pytest.mark.gpu

E_TOL = 1e-6
G_TOL = 1e-5


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def _solver(d):
    _torch()
    from paper_2101_12597_gb300.etdm import ETDM
    return ETDM(d, precision="mixed")


@pytest.fixture(scope="module")
def cases():
    out = {}
    # "odd": every grid extent odd (an unpaired real z line, odd half spectrum,
    # ragged tiles in all three directions)
    for name, fn in [("tiny", synth.tiny), ("small", synth.config_small_molecule),
                     ("ragged", synth.ragged_water),
                     ("odd", lambda: synth.ragged_water(grid=(27, 25, 45), seed=12))]:
        d = fn()
        out[name] = (d, Oracle(d), _solver(d))
    return out


def _grad_err(g, gref):
    return float(np.abs(g - gref).max() / max(np.abs(gref).max(), 1e-300))


@pytest.mark.parametrize("which", ["tiny", "small", "ragged", "odd"])
def test_tc_truncation_lists_bit_exact(which, cases):
    d, o, s = cases[which]
    ptr = s.get_array("tile_ptr_tc")
    keys = s.get_array("tile_keys_tc")
    nu = s.get_array("tile_nu_tc")
    tile = (4, 4, 8)
    nt = o.n_tiles(tile)
    assert len(ptr) == nt + 1 and len(nu) == nt
    funcs = []
    for t in range(nt):
        ref = o.tile_list(tile, t)
        np.testing.assert_array_equal(keys[ptr[t]:ptr[t + 1]], ref)
        # functions per tile: periodic images of one function merged
        funcs.append(np.unique(np.asarray(ref, dtype=np.int64) // 512))
        assert nu[t] == len(funcs[t])
    # V groups: greedy runs of at most two consecutive tiles whose union has at
    # most 128 functions; a tile starts a new group only when joining it to the
    # previous one-tile group would exceed 128
    t0 = s.get_array("vgroup_t0")
    gnu = s.get_array("vgroup_nu")
    assert t0[0] == 0 and t0[-1] == nt and len(gnu) == len(t0) - 1
    assert np.all(np.diff(t0) >= 1) and np.all(np.diff(t0) <= 2)
    for g in range(len(gnu)):
        un = np.unique(np.concatenate(funcs[t0[g]:t0[g + 1]]))
        assert gnu[g] == len(un) <= 128
        if t0[g + 1] - t0[g] == 1 and t0[g + 1] < nt:
            assert len(np.union1d(funcs[t0[g]], funcs[t0[g + 1]])) > 128


@pytest.mark.parametrize("which", ["tiny", "small", "ragged"])
def test_mixed_tensor_core_chains_on_small_systems(which, cases):
    """Every product of the float-pair chains on the tensor cores for systems
    whose matrices are far smaller than one 128 x 64 tile (padding, one K
    step): energy and gradient against the oracle."""
    torch = _torch()
    from paper_2101_12597_gb300.etdm import ETDM
    d, o, _ = cases[which]
    s = ETDM(d, precision="mixed", dense_tc=1)
    E_ref, g_ref = o.energy_grad(d["a0"])
    E, g = s.energy_grad(torch.tensor(d["a0"], device="cuda"))
    torch.cuda.synchronize()
    print(f"{which} status words: {s.get_array('status').tolist()}")
    s.check()
    dE = abs(float(E.item()) - E_ref)
    dg = _grad_err(g.cpu().numpy(), g_ref)
    print(f"{which} tensor-core chains: |dE|={dE:.3e} Ha  grad err={dg:.3e}")
    assert dE < E_TOL
    assert dg <= G_TOL
    s.close()


@pytest.mark.parametrize("which", ["tiny", "small", "ragged", "odd"])
def test_mixed_energy_gradient_parity(which, cases):
    torch = _torch()
    d, o, s = cases[which]
    for a in (d["a0"], synth.direction(d["a0"].shape, seed=31, scale=0.3)):
        E_ref, g_ref, ex = o.energy_grad(a, want=True)
        E, g = s.energy_grad(torch.tensor(a, device="cuda"))
        torch.cuda.synchronize()
        s.check()
        dE = abs(float(E.item()) - E_ref)
        dg = _grad_err(g.cpu().numpy(), g_ref)
        print(f"{which}: |dE|={dE:.3e} Ha  grad err={dg:.3e}")
        assert dE < E_TOL
        assert dg <= G_TOL
        rho = s.get_array("rho").reshape(tuple(o.n))
        assert np.abs(rho - ex["rho"]).max() < 1e-5 * ex["rho"].max()
        # accessors of the float-pair dense chain: H is the grid part V (rebuilt
        # symmetric from its upper triangle), U_occ has orthonormal columns
        M, N = o.M, o.N
        H = s.get_array("H").reshape(M, M)
        Vref = ex["H"] - s.get_array("T").reshape(M, M)
        assert np.array_equal(H, H.T)
        assert np.abs(H - Vref).max() < 1e-5 * np.abs(Vref).max()
        U = s.get_array("Uocc").reshape(M, N)
        assert np.abs(U.T @ U - np.eye(N)).max() < 1e-11


def test_mixed_energy_only_call(cases):
    torch = _torch()
    d, o, s = cases["small"]
    E_ref, _ = o.energy_grad(d["a0"])
    E, g = s.energy_grad(torch.tensor(d["a0"], device="cuda"), want_grad=False)
    s.check()
    assert g is None and abs(float(E.item()) - E_ref) < E_TOL


def test_mixed_minimization_trajectory(cases):
    torch = _torch()
    d, o, s = cases["small"]
    s.lbfgs_reset()
    hist, a_ref = minimize(o, d["a0"], n_steps=20)
    a = torch.tensor(d["a0"], device="cuda")
    E, al, tr = s.minimize(a, 20)
    for k in range(21):
        assert abs(E[k] - hist[k][0]) < E_TOL, (k, E[k], hist[k][0])
        assert tr[k] == hist[k][2]
        assert al[k] == pytest.approx(hist[k][1], abs=1e-9)
    s.lbfgs_reset()


def test_mixed_minimization_converges_to_the_oracle_minimum(cases):
    """300 L-BFGS steps of the 8-atom system: the mixed path lands on the
    oracle's minimum (energy within the bar) and is stationary there (Eq. 15:
    the occupied-virtual block of C^T H C vanishes; the GPU side checked
    through its own gradient)."""
    torch = _torch()
    d, o, s = cases["small"]
    s.lbfgs_reset()
    hist, a_ref = minimize(o, d["a0"], n_steps=300)
    E_ref, g_ref = o.energy_grad(a_ref)
    a = torch.tensor(d["a0"], device="cuda")
    E, al, tr = s.minimize(a, 300)
    E_gpu, g = s.energy_grad(a)
    torch.cuda.synchronize()
    s.check()
    print(f"converged: |E_gpu - E_ref|={abs(float(E_gpu.item()) - E_ref):.3e} Ha  "
          f"max|g_gpu|={float(g.abs().max()):.3e}  max|g_ref|={np.abs(g_ref).max():.3e}")
    assert abs(float(E_gpu.item()) - E_ref) < E_TOL
    assert abs(E[-1] - E_ref) < E_TOL
    assert float(g.abs().max()) < 2e-6  # from max|g| ~ 4 at the start; 3e-7 measured
    s.lbfgs_reset()


def test_water32_mixed_full_size(cases):
    torch = _torch()
    d = synth.config_water32()
    o = Oracle(d)
    s = _solver(d)
    E_ref, g_ref = o.energy_grad(d["a0"])
    E, g = s.energy_grad(torch.tensor(d["a0"], device="cuda"))
    torch.cuda.synchronize()
    s.check()
    dE = abs(float(E.item()) - E_ref)
    dg = _grad_err(g.cpu().numpy(), g_ref)
    print(f"water32 mixed: |dE|={dE:.3e} Ha  grad err={dg:.3e}")
    assert dE < E_TOL
    assert dg <= G_TOL
    ptr = s.get_array("tile_ptr_tc")
    keys = s.get_array("tile_keys_tc")
    nt = o.n_tiles((4, 4, 8))
    for t in list(range(0, nt, nt // 9)) + [nt - 1]:
        np.testing.assert_array_equal(keys[ptr[t]:ptr[t + 1]], o.tile_list((4, 4, 8), t))
    s.close()


def test_water576_mixed_vs_fp64_path():
    """The largest workload (1728 atoms, M=4608, N=2304, 192^3 grid): too big for
    the CPU oracle's energy, so the mixed path is held to the FP64 GPU path (itself
    pinned to the oracle on every smaller case) at the same bars, plus the
    properties that hold at any size: unitary U, and sampled 4x4x8 truncation
    lists bit-exact against the oracle's."""
    torch = _torch()
    from paper_2101_12597_gb300.etdm import ETDM
    d = synth.config_water576()
    a = torch.tensor(d["a0"], device="cuda")
    s = _solver(d)  # the large products of the chains on the tensor cores
    E, g = s.energy_grad(a)
    torch.cuda.synchronize()
    s.check()
    E, g = float(E.item()), g.cpu().numpy()
    s2 = ETDM(d, precision="mixed", dense_tc=-1)  # every product on float pairs
    E2, g2 = s2.energy_grad(a)
    torch.cuda.synchronize()
    s2.check()
    print(f"water576 tensor-core vs float-pair chains: |dE|={abs(E - float(E2.item())):.3e} Ha "
          f"grad err={_grad_err(g, g2.cpu().numpy()):.3e}")
    s2.close()
    U = s.get_array("Uocc").reshape(s.M, s.N)
    assert np.abs(U.T @ U - np.eye(s.N)).max() < 1e-11
    o = Oracle(d)
    ptr = s.get_array("tile_ptr_tc")
    keys = s.get_array("tile_keys_tc")
    nt = o.n_tiles((4, 4, 8))
    assert len(ptr) == nt + 1
    for t in (0, nt // 3, nt - 1):
        np.testing.assert_array_equal(keys[ptr[t]:ptr[t + 1]], o.tile_list((4, 4, 8), t))
    s.close()
    from paper_2101_12597_gb300.etdm import ETDM
    f = ETDM(d, precision="fp64")
    E64, g64 = f.energy_grad(a)
    torch.cuda.synchronize()
    f.check()
    dE = abs(E - float(E64.item()))
    dg = _grad_err(g, g64.cpu().numpy())
    print(f"water576 mixed vs FP64 path: |dE|={dE:.3e} Ha  grad err={dg:.3e}")
    assert dE < E_TOL
    assert dg <= G_TOL
    f.close()


@pytest.mark.parametrize("which", ["small", "odd"])
def test_mixed_potential_at_float_pair_accuracy(which, cases):
    """The potential of the mixed path (float-pair half-spectrum transforms,
    Slater exchange, v_ext) against the oracle's potential of the same density:
    the GPU's own rho is read back exactly, so the difference is the potential
    arithmetic alone.  Float-pair accuracy leaves about 1e-13 of max|v|;
    butterflies at FP32 accuracy would leave about 1e-8 (the helpers use
    explicit-rounding intrinsics, so the compiler cannot fuse them into that)."""
    torch = _torch()
    d, o, s = cases[which]
    s.energy_grad(torch.tensor(d["a0"], device="cuda"))
    torch.cuda.synchronize()
    s.check()
    rho = s.get_array("rho").reshape(tuple(o.n))
    v = s.get_array("vtot").reshape(tuple(o.n))
    _, vx = o.lda_x(rho)
    vref = o.reference()["vext"] + o.hartree_potential(rho) + vx
    err = float(np.abs(v - vref).max() / np.abs(vref).max())
    print(f"{which}: potential error {err:.2e} of max|v|")
    assert err < 1e-11, f"potential error {err:.2e} of max|v|"


@pytest.fixture(scope="module")
def water75():
    """The oracle's evaluation of the 75-unit water box (M = 600, N = 300,
    64^3 grid), shared by the cases below."""
    d = synth.config_water75()
    o = Oracle(d)
    E, g, ex = o.energy_grad(d["a0"], want=True)
    return d, o, E, g, ex


@pytest.mark.parametrize("precision,dense_blocks,dense_tc", [
    ("fp64", 0, 0), ("fp64", 4, 0), ("mixed", 0, -1), ("mixed", 4, -1), ("mixed", 0, 1)])
def test_water75_against_oracle(water75, precision, dense_blocks, dense_tc):
    """Both GPU paths at a size that runs the density pass over three orbital
    chunks (N = 300 > 128) and, with the dense grid fixed at 4 blocks, puts
    every product of the dense chains on the 64 x 64 output tiles (the
    automatic grid keeps them on 8 x 16 tiles): energy, gradient, density and
    the Hamiltonian (its grid part V on the mixed path) element by element
    against the oracle.  dense_tc = 1 runs every product of the float-pair
    chains on the tensor cores (exact BF16 slices)."""
    torch = _torch()
    from paper_2101_12597_gb300.etdm import ETDM
    d, o, E_ref, g_ref, ex = water75
    s = ETDM(d, precision=precision, dense_blocks=dense_blocks, dense_tc=dense_tc)
    E, g = s.energy_grad(torch.tensor(d["a0"], device="cuda"))
    torch.cuda.synchronize()
    print(f"water75 status words: {s.get_array('status').tolist()}")
    s.check()
    dE = abs(float(E.item()) - E_ref)
    dg = _grad_err(g.cpu().numpy(), g_ref)
    rho = s.get_array("rho").reshape(tuple(o.n))
    drho = float(np.abs(rho - ex["rho"]).max() / ex["rho"].max())
    M = o.M
    H = s.get_array("H").reshape(M, M)
    Href = ex["H"] - (s.get_array("T").reshape(M, M) if precision == "mixed" else 0.0)
    dH = float(np.abs(H - Href).max() / np.abs(Href).max())
    print(f"water75 {precision} dense_blocks={dense_blocks} dense_tc={dense_tc}: |dE|={dE:.3e} Ha "
          f"grad err={dg:.3e} rho err={drho:.2e} H err={dH:.2e}")
    assert dE < E_TOL
    assert dg <= G_TOL
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert drho < tol and dH < tol
    U = s.get_array("Uocc").reshape(M, o.N)
    assert np.abs(U.T @ U - np.eye(o.N)).max() < 1e-11
    s.close()


def test_autograd_backward_water32_against_oracle_differences():
    """The autograd Function on the mixed path (water32: M = 256, N = 128):
    its backward against central differences (h = 1e-5) of the oracle's
    energy on 32 seeded entries of A_ov, within the gradient bar."""
    torch = _torch()
    from paper_2101_12597_gb300.etdm import energy_function
    d = synth.config_water32()
    o = Oracle(d)
    s = _solver(d)
    a = torch.tensor(d["a0"], device="cuda", requires_grad=True)
    E = energy_function().apply(a, s)
    E.backward()
    g = a.grad.cpu().numpy()
    rng = np.random.default_rng(32)
    N, V = d["a0"].shape
    idx = rng.choice(N * V, size=32, replace=False)
    h = 1e-5
    fd = []
    for k in idx:
        ap, am = d["a0"].copy(), d["a0"].copy()
        ap.flat[k] += h
        am.flat[k] -= h
        fd.append((o.energy(ap) - o.energy(am)) / (2 * h))
    fd = np.array(fd)
    err = float(np.abs(g.flat[idx] - fd).max() / np.abs(g).max())
    print(f"water32 autograd vs oracle central differences: {err:.2e} of max|g|")
    assert err <= G_TOL
    s.close()
