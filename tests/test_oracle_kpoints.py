"""Pins of the k-point / full-A oracle (Bloch basis, fractional occupation)
against what the paper and the mathematics fix: quadrature of the Bloch
functions, time reversal, the Gamma-point oracle as a special case, finite
differences of E in the real and imaginary variables, the Eq. 31 diagonal
Hessian, invariances of the functional and stationarity (Eq. 15)."""
import math

import numpy as np
import pytest

import etdm_synth as synth
from oracle.etdm_kpoints import BlochOracle, fermi_dirac, fermi_level
from oracle.etdm_oracle import Oracle, minimize


@pytest.fixture(scope="module")
def tiny():
    d = synth.tiny_crystal()
    return d, BlochOracle(d)


def _with(d, **over):
    e = dict(d)
    e.update(over)
    return e


# ---- Bloch basis, S(k), T(k) (Eq. 4-5, Eq. 11) -----------------------------------

def test_bloch_basis_at_gamma_is_the_gamma_basis(tiny):
    d, _ = tiny
    g = _with(d, kpts=np.zeros((1, 3)), kw=np.ones(1))
    bo, o = BlochOracle(g), Oracle(g)
    X = o.X()
    assert np.abs(bo.Xk(0) - X).max() <= 1e-15 * np.abs(X).max()
    S, T = o.overlap_kinetic()
    Sk, Tk = bo.overlap_kinetic_k(0)
    assert np.abs(Sk - S).max() < 1e-15 and np.abs(Tk - T).max() < 1e-14


def test_overlap_and_kinetic_match_grid_quadrature(tiny):
    """S(k) = dV X_k^dag X_k; T(k) from the spectral Laplacian of the periodic
    part u = exp(-i k.r) chi_k, whose plane waves carry G + k."""
    d, bo = tiny
    g = [2 * math.pi * np.fft.fftfreq(int(bo.n[a]), d=bo.h[a]) for a in range(3)]
    r = [bo.coords(a) for a in range(3)]
    for k in (0, 3, 6):
        X = bo.Xk(k)
        S, T = bo.overlap_kinetic_k(k)
        assert np.abs(S - bo.dV * X.conj().T @ X).max() < 1e-9
        kc = 2 * math.pi * bo.kfrac[k] / bo.L
        ph = np.exp(-1j * (kc[0] * r[0][:, None, None] + kc[1] * r[1][None, :, None]
                           + kc[2] * r[2][None, None, :]))
        U = np.fft.fftn(X.reshape(*tuple(bo.n), bo.M) * ph[..., None], axes=(0, 1, 2))
        Gk2 = ((g[0] + kc[0]) ** 2)[:, None, None] + ((g[1] + kc[1]) ** 2)[None, :, None] \
            + ((g[2] + kc[2]) ** 2)[None, None, :]
        U = U.reshape(-1, bo.M)
        Tq = 0.5 * bo.dV / bo.G * (U.conj().T @ (Gk2.reshape(-1, 1) * U))
        assert np.abs(T - Tq).max() < 1e-7


def test_time_reversal_pairs(tiny):
    """Real eta: chi_{-k} = conj(chi_k), so S(-k) = conj S(k), h_core(-k) =
    conj h_core(k), and both k-points get the same bands and occupations."""
    d, bo = tiny
    ref = bo.reference_k()
    kf = bo.kfrac
    for k in range(bo.nk):
        m = int(np.argmin(np.abs(kf + kf[k]).sum(1)))
        assert np.allclose(kf[m], -kf[k])
        assert np.abs(ref["S"][m] - ref["S"][k].conj()).max() < 1e-14
        assert np.abs(ref["hcore"][m] - ref["hcore"][k].conj()).max() < 1e-13
        assert np.abs(ref["eps_core"][m] - ref["eps_core"][k]).max() < 1e-12
        assert np.abs(ref["f"][m] - ref["f"][k]).max() < 1e-12


# ---- reference and occupations ---------------------------------------------------------

def test_fermi_dirac_and_level():
    x = np.array([-1e4, -30.0, -1.0, 0.0, 1.0, 30.0, 1e4])
    f = fermi_dirac(x)
    assert np.all(np.isfinite(f)) and f[3] == 0.5
    assert np.allclose(f + fermi_dirac(-x), 1.0, atol=1e-16, rtol=0)
    assert abs(f[2] - 1 / (1 + math.e ** -1)) < 1e-16 and f[0] == 1.0 and f[-1] == 0.0
    rng = np.random.default_rng(2)
    eps = [np.sort(rng.normal(size=6)) for _ in range(4)]
    w = np.full(4, 0.25)
    for n_e, kT in ((2, 0.05), (5, 0.3), (11, 1e-3)):
        mu = fermi_level(eps, w, n_e, kT)
        cnt = sum(2 * w[k] * fermi_dirac((eps[k] - mu) / kT).sum() for k in range(4))
        assert abs(cnt - n_e) < 1e-12
        lo = sum(2 * w[k] * fermi_dirac((eps[k] - mu + 1e-3) / kT).sum() for k in range(4))
        assert lo < cnt  # the count increases with mu


def test_reference_orthonormal_sorted_and_occupations(tiny):
    d, bo = tiny
    ref = bo.reference_k()
    tot = 0.0
    for k in range(bo.nk):
        C = ref["C0"][k]
        assert np.abs(C.conj().T @ ref["S"][k] @ C - np.eye(bo.M)).max() < 1e-12
        # C0 diagonalizes h_core(k) with the eigenvalues in ascending order
        Hc = C.conj().T @ ref["hcore"][k] @ C
        assert np.abs(Hc - np.diag(ref["eps_core"][k])).max() < 1e-12
        assert np.all(np.diff(ref["eps_core"][k]) >= 0)
        f = ref["f"][k]
        assert np.all((f >= 0) & (f <= 2 * bo.kw[k])) and np.all(np.diff(f) <= 0)
        tot += f.sum()
    assert abs(tot - d["n_electrons"]) < 1e-12
    # genuinely fractional: the full-A parametrization is needed
    assert any(np.any((ref["f"][k] > 1e-3 * bo.kw[k]) & (ref["f"][k] < 1.999 * bo.kw[k]))
               for k in range(bo.nk))


def test_density_integrates_to_electron_count(tiny):
    d, bo = tiny
    orbs = bo.orbitals_k(d["a0"])
    Ds = bo.density_matrices(orbs)
    ref = bo.reference_k()
    assert abs(sum(np.sum(Ds[k] * ref["S"][k].T).real for k in range(bo.nk))
               - d["n_electrons"]) < 1e-12
    _, _, rho, _ = bo.energy_terms_k(Ds)
    assert abs(bo.dV * rho.sum() - d["n_electrons"]) < 1e-8
    assert rho.min() > -1e-14
    for k, (A, O) in enumerate(orbs):  # unitary exp(A(k)): O^dag S O = I
        assert np.abs(O.conj().T @ ref["S"][k] @ O - np.eye(bo.M)).max() < 1e-12
        assert np.abs(A + A.conj().T).max() == 0.0


# ---- the Gamma point as a special case ------------------------------------------------------

def test_gamma_only_integer_occupation_reduces_to_gamma_oracle(tiny):
    """One k-point at Gamma, weight 1, kT far below the gap: integer occupations,
    and E, g over the occupied-virtual real variables equal the Gamma-point
    oracle's with the same (phase-fixed, real) reference orbitals."""
    d, _ = tiny
    g = _with(d, kpts=np.zeros((1, 3)), kw=np.ones(1), kT=1e-5)
    bo, o = BlochOracle(g), Oracle(g)
    ref = bo.reference_k()
    assert np.abs(ref["f"][0] - np.array([2.0] + [0.0] * (bo.M - 1))).max() < 1e-15
    C = ref["C0"][0]
    piv = C[np.argmax(np.abs(C), axis=0), np.arange(bo.M)]
    C = C * (np.abs(piv) / piv)[None, :]
    assert np.abs(C.imag).max() < 1e-14
    ref["C0"][0] = C.real.astype(np.complex128)
    Aov = synth.direction((o.N, o.V), seed=8, scale=0.2)
    v = np.zeros(bo.nvar)
    nre = bo.M * (bo.M - 1) // 2
    pos = {(i, j): p for p, (i, j) in enumerate(zip(*bo._iu))}
    for i in range(o.N):
        for j in range(o.V):
            v[pos[(i, o.N + j)]] = Aov[i, j]
    Eb, gb = bo.energy_grad(v)
    Eg, gg = o.energy_grad(Aov, C0=C.real)
    assert abs(Eb - Eg) < 1e-12
    for i in range(o.N):
        for j in range(o.V):
            assert abs(gb[pos[(i, o.N + j)]] - gg[i, j]) < 1e-11
    assert np.abs(gb[nre:]).max() < 1e-12  # real A: no force on the imaginary parts


# ---- energy and gradient (Eq. 1, Eq. 14, Eq. 20) ---------------------------------------------

def test_gradient_central_differences_real_and_imaginary(tiny):
    d, bo = tiny
    a = d["a0"]
    E, g = bo.energy_grad(a)
    rng = np.random.default_rng(11)
    nre = bo.M * (bo.M - 1) // 2
    idx = list(rng.choice(len(a), 24, replace=False))
    idx += [3 * bo.nvar + nre, 5 * bo.nvar + nre + 4]  # two Im a_ii
    h = 1e-5
    for i in idx:
        e = np.zeros_like(a); e[i] = h
        fd = (bo.energy(a + e) - bo.energy(a - e)) / (2 * h)
        assert abs(fd - g[i]) < max(1e-9, 1e-6 * abs(fd)), (i, fd, g[i])


def test_gradient_at_zero_is_eq42(tiny):
    """At A = 0, dE/da_ij = (2 - d_ij)/2 L_ji (Eq. 42 with fractional f): the
    imaginary diagonal has no force (L_ii = 0)."""
    d, bo = tiny
    E, g, ex = bo.energy_grad(np.zeros(bo.nk * bo.nvar), want=True)
    for k in range(bo.nk):
        L = ex["k"][k]["L"]
        fac = np.where(np.eye(bo.M, dtype=bool), 0.5, 1.0)
        assert np.abs(ex["k"][k]["dEda"] - fac * L.T).max() < 1e-14
        assert np.abs(np.diag(L)).max() < 1e-15


def test_energy_invariances(tiny):
    """Rephasing the reference orbitals, C0' = C0 P with P diagonal and unitary,
    together with A' = P^dag A P gives O' = O P and the same D, hence the same
    E at any A (this exercises the variable <-> A(k) mapping); with integer
    occupations a unitary mixing of the occupied orbitals of each k-point
    leaves E unchanged."""
    d, bo = tiny
    a = d["a0"]
    rng = np.random.default_rng(5)
    b2 = BlochOracle(d)
    r1, r2 = bo.reference_k(), b2.reference_k()
    nre = bo.M * (bo.M - 1) // 2
    ap = np.empty_like(a)
    for k in range(bo.nk):
        p = np.exp(1j * rng.uniform(0, 2 * np.pi, bo.M))
        r2["C0"][k] = r1["C0"][k] * p[None, :]
        A = bo.A_of(a[k * bo.nvar:(k + 1) * bo.nvar])
        Ap = p.conj()[:, None] * A * p[None, :]
        ap[k * bo.nvar:k * bo.nvar + nre] = Ap[bo._iu].real
        ap[k * bo.nvar + nre:(k + 1) * bo.nvar] = Ap[bo._iud].imag
        assert np.abs(b2.A_of(ap[k * bo.nvar:(k + 1) * bo.nvar]) - Ap).max() < 1e-16
    assert abs(b2.energy(ap) - bo.energy(a)) < 1e-12

    gi = _with(d, kT=1e-5)
    b3, b4 = BlochOracle(gi), BlochOracle(gi)
    r4 = b4.reference_k()
    z = np.zeros(b3.nk * b3.nvar)
    E3 = b3.energy(z)
    for k in range(b4.nk):
        n = int(np.sum(r4["f"][k] > 0))
        assert np.abs(r4["f"][k][:n] - 2 * b4.kw[k]).max() < 1e-15  # integer to rounding
        Q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
        C = r4["C0"][k].copy()
        C[:, :n] = C[:, :n] @ Q
        r4["C0"][k] = C
    assert abs(b4.energy(z) - E3) < 1e-12


# ---- preconditioner (Eq. 31-34 with k-point weights) ---------------------------------------

def test_preconditioner_gamma0_is_inverse_fd_hessian_real_and_imaginary():
    """Fixed potential, reference = eigenvectors of h_core(k): with gamma = 0,
    1 / P equals the second difference of E along Re a_ij and along Im a_ij
    (i < j) at every sampled k-point; f carries the k-point weight."""
    d = synth.tiny_crystal()
    bo = BlochOracle(d, hartree=False, exchange=False)
    ref = bo.reference_k()
    with np.errstate(divide="ignore"):
        P0 = bo.precond(ref["eps_core"], beta=3.0, gamma=0.0)
    nre = bo.M * (bo.M - 1) // 2
    pos_re = {(i, j): p for p, (i, j) in enumerate(zip(*bo._iu))}
    pos_im = {(i, j): nre + p for p, (i, j) in enumerate(zip(*bo._iud))}
    z = np.zeros(bo.nk * bo.nvar)
    E0 = bo.energy(z)
    h = 1e-4
    for k in (0, 5):
        for ij in [(0, 1), (0, 3), (1, 2)]:
            for pos in (pos_re[ij], pos_im[ij]):
                e = np.zeros_like(z); e[k * bo.nvar + pos] = h
                fd2 = (bo.energy(e) - 2 * E0 + bo.energy(-e)) / h ** 2
                assert abs(1.0 / P0[k * bo.nvar + pos] - fd2) < 1e-5 * fd2, (k, ij, pos)
    Pg = bo.precond(ref["eps_core"], beta=3.0, gamma=0.25)
    k, p = 2, pos_im[(1, 1)]  # equal occupations: only the beta term remains
    assert abs(1.0 / Pg[k * bo.nvar + p] - 0.25 * 3.0 * bo.kw[k]) < 1e-15


# ---- minimization over all k-points (Sec. 3, Eq. 15) ----------------------------------------

def test_minimization_reaches_stationarity(tiny):
    d, _ = tiny
    bo = BlochOracle(d)
    hist, a = minimize(bo, np.zeros(bo.nk * bo.nvar), n_steps=40)
    Es = [h[0] for h in hist]
    assert all(Es[i + 1] <= Es[i] + 1e-12 for i in range(len(Es) - 1))
    assert Es[-1] < Es[0]
    E, g, ex = bo.energy_grad(a, want=True)
    assert np.abs(g).max() < 1e-8
    # Eq. 15 with fractional occupation: [F, H_mo] = 0 at the minimum
    assert max(np.abs(x["L"]).max() for x in ex["k"]) < 1e-8


def test_streamed_planes_equal_the_cached_basis(tiny):
    """Large systems build the Bloch basis one x-plane at a time; the sums are
    the same, in a different association order."""
    d, bo = tiny
    bs = BlochOracle(d, cache_x=False)
    E1, g1 = bo.energy_grad(d["a0"])
    E2, g2 = bs.energy_grad(d["a0"])
    assert not bs._Xk and abs(E1 - E2) < 1e-13 and np.abs(g1 - g2).max() < 1e-13


def test_oracle_matches_stored_tiny_crystal_values(tiny):
    # stored values come from tests/golden/make_golden.py (oracle only); this
    # guards the k-point oracle against unreviewed arithmetic changes
    import json
    import os
    d, bo = tiny
    with open(os.path.join(os.path.dirname(__file__), "golden", "tiny_crystal_oracle.json")) as f:
        gold = json.load(f)
    E, g = bo.energy_grad(d["a0"])
    ref = bo.reference_k()
    assert abs(E - gold["E_a0"]) < 1e-11
    assert np.abs(g - np.array(gold["g_a0"])).max() < 1e-10
    assert abs(ref["mu"] - gold["mu"]) < 1e-11
    assert np.abs(np.array(ref["f"]) - np.array(gold["f"])).max() < 1e-11
    assert np.abs(np.array(ref["eps_core"]) - np.array(gold["eps_core"])).max() < 1e-11


def test_imaginary_diagonal_force_vanishes_only_at_zero(tiny):
    """Im a_ii: zero gradient at A = 0 (L_ii = 0), generally non-zero elsewhere
    (a diagonal step commutes with A only in special cases), so these variables
    stay in the parametrization."""
    d, bo = tiny
    nre = bo.M * (bo.M - 1) // 2
    diag = [nre + p for p, (i, j) in enumerate(zip(*bo._iud)) if i == j]
    idx = [k * bo.nvar + p for k in range(bo.nk) for p in diag]
    _, g0 = bo.energy_grad(np.zeros_like(d["a0"]))
    _, g = bo.energy_grad(d["a0"])
    assert np.abs(g0[idx]).max() == 0.0
    assert np.abs(g[idx]).max() > 1e-5


def test_orbital_energies_sum_is_trace_per_k(tiny):
    """Eq. 33 at k-points: sum_m eps_m(k) = Tr(C0^dag H C0) = Tr(S(k)^-1 H(k)) at
    A = 0, for any reference with C0 C0^dag = S^-1."""
    d, bo = tiny
    eps = bo.orbital_energies()
    _, _, ex = bo.energy_grad(np.zeros(bo.nk * bo.nvar), want=True)
    ref = bo.reference_k()
    for k in range(bo.nk):
        tr = np.trace(np.linalg.solve(ref["S"][k], ex["k"][k]["H"]))
        assert abs(tr.imag) < 1e-12 and abs(eps[k].sum() - tr.real) < 1e-11


def test_lowdin_reference_is_s_orthonormal(tiny):
    """S(k)^(-1/2): Hermitian and C0^dagger S C0 = I for every k-point."""
    d, bo = tiny
    for k, C in enumerate(bo.lowdin_reference()):
        S, _ = bo.overlap_kinetic_k(k)
        assert np.abs(C - C.conj().T).max() < 1e-13
        assert np.abs(C.conj().T @ S @ C - np.eye(bo.M)).max() < 1e-12


def test_reference_update_identity(tiny):
    """E with reference C0 at A equals E with reference C0 exp(A) at A = 0:
    the identity behind the reference update C <- C exp(A) of Sec. 3.5."""
    d, _ = tiny
    bo = BlochOracle(d)
    a = d["a0"]
    E_a = bo.energy(a)
    ref = bo.reference_k()
    moved = [ref["C0"][k] @ bo.expm_eig(bo.A_of(a[k * bo.nvar:(k + 1) * bo.nvar]))
             for k in range(bo.nk)]
    bo2 = BlochOracle(d)
    bo2.set_reference(moved)
    assert abs(bo2.energy(np.zeros_like(a)) - E_a) < 1e-12
    # and the energy does not depend on which S-orthonormal basis of the same
    # occupied space is the reference when A = 0 and occupations are equal
    # within it: here a phase on every column
    ph = [np.exp(1j * np.arange(bo.M)) for _ in range(bo.nk)]
    bo3 = BlochOracle(d)
    bo3.set_reference([ref["C0"][k] * ph[k][None, :] for k in range(bo.nk)])
    assert abs(bo3.energy(np.zeros_like(a)) - bo.energy(np.zeros_like(a))) < 1e-12


def test_scaling_and_squaring_equals_the_eigendecomposition_route(tiny):
    """Eq. 38 (Pade scaling and squaring) and Eq. 35 give the same exp(A),
    also for a rotation large enough to need several squarings."""
    d, bo = tiny
    for k in (0, 5):
        A = bo.A_of(d["a0"][k * bo.nvar:(k + 1) * bo.nvar])
        for t in (1.0, 40.0):
            U = bo.expm_ss(t * A)
            assert np.abs(U - bo.expm_eig(t * A)).max() < 1e-13
            assert np.abs(U.conj().T @ U - np.eye(bo.M)).max() < 1e-13


def test_approximate_gradient_is_the_first_term_of_eq19(tiny):
    """Eq. 42 is the first term of the Eq. 19 series: with the L of the
    approximate evaluation, L + [A, L]/2! + [A, [A, L]]/3! + ... summed to
    convergence gives the exact Eq. 39 gradient; at A = 0 the two are equal."""
    d, bo = tiny
    z = np.zeros_like(d["a0"])
    E0, g0 = bo.energy_grad(z)
    E1, g1 = bo.energy_grad_approx(z)
    assert E0 == E1 and np.array_equal(g0, g1)
    a = d["a0"]
    Ee, ge = bo.energy_grad(a)
    Ea, ga, ex = bo.energy_grad_approx(a, want=True)
    assert abs(Ee - Ea) < 1e-14
    fac = np.where(np.eye(bo.M, dtype=bool), 0.5, 1.0)
    gs = np.empty_like(ge)
    for k, (A, L, _) in enumerate(ex["L"]):
        term, S = L.copy(), L.copy()
        for n in range(1, 40):
            term = (A @ term - term @ A) / (n + 1)
            S = S + term
        gs[k * bo.nvar:(k + 1) * bo.nvar] = bo.vars_of_grad(fac * S.T)
    assert np.abs(gs - ge).max() <= 1e-12 * np.abs(ge).max()
    assert np.abs(ga - ge).max() > 1e-6 * np.abs(ge).max()  # the approximation is visible


def test_ss_minimization_with_reference_updates(tiny):
    """The "ss" route with reference updates (every 5 steps, and by the
    Sec. 3.5 test) lowers E monotonically and ends where the exact-gradient
    minimization ends; after an update the new reference at A = 0 reproduces
    the energy of the point it was taken at (C <- C exp(A))."""
    d, _ = tiny
    z = np.zeros_like(d["a0"])
    h_ex, _ = minimize(BlochOracle(d), z, 20)
    for ru in (5, -1):
        bo = BlochOracle(d)
        h, a, nu = bo.minimize_ss(d["a0"], 20, ru)
        E = np.array([x[0] for x in h])
        assert np.all(np.diff(E) <= 1e-12)
        assert abs(E[-1] - h_ex[-1][0]) < 1e-9
        if ru == 5:
            assert nu == 3
        assert abs(bo.energy_grad_approx(a)[0] - E[-1]) < 1e-12


def _gamma_full(d):
    g = dict(d)
    g.update(kpts=np.zeros((1, 3)), kw=np.ones(1), kT=0.0)
    return g


def test_pzsic_gradient_central_differences():
    """PZ-SIC (Eq. 16-18 as read): the Eq. 39 gradient with the SIC L matches
    central differences of E in real and imaginary variables."""
    d = _gamma_full(synth.config_small_molecule())
    bo = BlochOracle(d, sic=True)
    rng = np.random.default_rng(3)
    a = rng.normal(0.0, 0.05, bo.nvar)
    _, g = bo.energy_grad(a)
    h = 1e-5
    for i in rng.choice(bo.nvar, 16, replace=False):
        ap, am = a.copy(), a.copy()
        ap[i] += h
        am[i] -= h
        fd = (bo.energy(ap) - bo.energy(am)) / (2 * h)
        assert abs(g[i] - fd) < 2e-9, (i, g[i], fd)


def test_pzsic_two_electrons_in_one_orbital():
    """One doubly occupied orbital: the self-interaction correction removes the
    exchange exactly (E_x[2n] = 2 E_x^pol[n]) and leaves the Hartree energy of
    the two electrons in each other's field, 2 E_H[n] = E_H[2n] / 2."""
    d = _gamma_full(synth.tiny())
    bo = BlochOracle(d, sic=True)
    assert bo.n_e == 2
    a = 0.1 * np.random.default_rng(5).normal(size=bo.nvar)
    E, _, ex = bo.energy_grad(a, want=True)
    t = ex["terms"]
    assert abs(E - (t["kinetic"] + t["external"] + 0.5 * t["hartree"])) < 1e-12 * abs(E) + 1e-14
    assert abs(t["exchange"] + t["sic"] + 0.5 * t["hartree"]) < 1e-12 * abs(t["hartree"])


def test_pzsic_is_not_unitary_invariant():
    """Rotations among the occupied orbitals leave the Kohn-Sham energy alone
    but change the SIC energy; at A = 0 the occupied-occupied gradient is zero
    for Kohn-Sham (Eq. 42) and not for PZ-SIC."""
    d = _gamma_full(synth.config_small_molecule())
    ks, pz = BlochOracle(d), BlochOracle(d, sic=True)
    N, M = ks.n_e // 2, ks.M
    A = np.zeros((M, M))
    A[0, 1], A[1, 0] = 0.3, -0.3   # a real rotation of occupied orbitals 0 and 1
    a = np.zeros(ks.nvar)
    a[:M * (M - 1) // 2] = A[ks._iu]
    z = np.zeros(ks.nvar)
    assert abs(ks.energy(a) - ks.energy(z)) < 1e-12
    assert abs(pz.energy(a) - pz.energy(z)) > 1e-6
    iu = list(zip(*ks._iu))
    occ = [p for p, (i, j) in enumerate(iu) if j < N]
    g_ks, g_pz = ks.energy_grad(z)[1], pz.energy_grad(z)[1]
    assert np.abs(g_ks[occ]).max() < 1e-12
    assert np.abs(g_pz[occ]).max() > 1e-6
