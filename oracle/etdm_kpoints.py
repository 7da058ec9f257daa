"""Plain FP64 / complex128 CPU oracle of the ETDM evaluation with k-point
sampling and the full skew-Hermitian A(k) of each k-point (fractional
occupation).

TEST INFRASTRUCTURE ONLY, under the same rule as ``etdm_oracle``: only tests/,
``__graft_entry__.smoke()`` and the baseline legs of ``bench.py`` may import it;
it shares no code with the CUDA path.

It extends the Gamma-point oracle (whose grid, potentials, exponential and
Eq. 39 adjoint it reuses) to:

* Bloch basis functions (Eq. 5) chi_mu,k(r) = sum_R exp(i k.R) eta_mu(r - R - d_mu)
  over the images within the truncation radius, without the 1/sqrt(N) factor
  (per-cell normalization, so that S(k) is the overlap over one cell);
* S(k), T(k) (Eq. 4, Eq. 11) summed over lattice images with the phase
  exp(i k.R);
* one unitary exp(A(k)) per k-point (Eq. 7, Eq. 35) and O(k) = C0(k) exp(A(k));
* the density of Eq. 2 summed over k-points, rho_mu,nu(k) = sum_m f_m(k)
  O_mu,m(k) conj(O_nu,m(k)) (Eq. 12), and E of Eq. 1;
* H(k) (Eq. 11), L(k) = [F(k), O^dag H O] (Eq. 13) and the gradient of Eq. 14
  with respect to the real and imaginary parts of the upper-triangular
  elements a_ij(k), i <= j (Eq. 20-24), Re a_ii being zero;
* the Eq. 33 preconditioner with beta multiplied by the k-point weight
  (Sec. 3.3), for the real and the imaginary parts alike.

Readings of what the paper leaves open (parity of the first two is pinned only
through the properties the tests check):

* f_m(k) carries the k-point weight and the spin factor,
  f_m(k) = 2 w_k / (1 + exp((eps_m(k) - mu) / kT)), so sum_k,m f_m(k) = n_e
  with mu found by bisection; the occupations are set once, at the reference,
  and then stay fixed (variational occupations with thermal smearing are the
  paper's future work, Sec. 5).
* The reference orbitals C0(k) are the generalized eigenvectors of
  h_core(k) = T(k) + V_ext(k) with S(k) (ascending eigenvalues eps_m(k)); the
  orbital energies of Eq. 33 are the diagonal of C0^dag H[rho(A = 0)] C0, and
  the orbital-energy term enters with its absolute value as at the Gamma point.
* Variables of one k-point, in this order: Re a_ij for i < j (row-major), then
  Im a_ij for i <= j (row-major), M^2 real numbers; the k-points follow one
  another.  With dE/da_ij the complex derivative of Eq. 20,
  dE/dRe a_ij = 2 Re dE/da_ij and dE/dIm a_ij = -2 Im dE/da_ij.
"""
from __future__ import annotations

import math

import numpy as np

from .etdm_oracle import GAMMA, LBFGS, Oracle, _fsum, line_search


def fermi_dirac(x):
    """1 / (1 + exp(x)) without overflow."""
    x = np.asarray(x, dtype=np.float64)
    e = np.exp(-np.abs(x))
    return np.where(x > 0, e / (1.0 + e), 1.0 / (1.0 + e))


def fermi_level(eps, w, n_e, kT, tol=1e-13, max_iter=400):
    """mu with sum_k w_k sum_m 2 f((eps_mk - mu) / kT) = n_e, by bisection (the
    count is increasing in mu).  eps: list of per-k eigenvalue arrays."""
    def count(mu):
        return _fsum([2.0 * w[k] * fermi_dirac((eps[k] - mu) / kT).sum()
                      for k in range(len(w))])
    lo = min(float(e.min()) for e in eps) - 50.0 * kT - 1.0
    hi = max(float(e.max()) for e in eps) + 50.0 * kT + 1.0
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        if count(mid) < n_e:
            lo = mid
        else:
            hi = mid
        if hi - lo <= tol * max(1.0, abs(mid)):
            break
    return 0.5 * (lo + hi)


class BlochOracle(Oracle):
    """One periodic system with k-point sampling and a full skew-Hermitian A(k)
    per k-point."""

    def __init__(self, sysd, sic=False, **kw):
        super().__init__(sysd, **kw)
        self.sic = bool(sic)
        self.kfrac = np.atleast_2d(np.asarray(sysd["kpts"], dtype=np.float64))
        self.kw = np.asarray(sysd["kw"], dtype=np.float64)
        self.kT = float(sysd["kT"])
        self.nk = len(self.kw)
        self.nvar = self.M * self.M
        self._iu = np.triu_indices(self.M, 1)
        self._iud = np.triu_indices(self.M)
        self._Xk = {}
        self._kref = None

    # ---- lattice images ---------------------------------------------------
    def image_range(self, reach):
        """All n with |n_a| L_a < reach + L_a per axis: every image of a point of
        the cell within `reach` of another point of the cell."""
        nm = [int(math.floor(reach / self.L[a])) + 1 for a in range(3)]
        return [(i, j, k) for i in range(-nm[0], nm[0] + 1)
                for j in range(-nm[1], nm[1] + 1) for k in range(-nm[2], nm[2] + 1)]

    def bloch_phase(self, k, n):
        """exp(i k.R) for R = n L, k in fractional reciprocal coordinates."""
        return np.exp(2j * math.pi * float(np.dot(self.kfrac[k], n)))

    # ---- Bloch basis on the grid (Eq. 5) ------------------------------------
    def basis_plane_k(self, i, k):
        """chi_mu,k at all points of the x-plane i, shape (ny*nz, M), complex."""
        ny, nz = int(self.n[1]), int(self.n[2])
        x = self.coords(0)[i]
        y, z = self.coords(1), self.coords(2)
        out = np.zeros((ny, nz, self.M), dtype=np.complex128)
        for mu in range(self.M):
            rc2 = self.rcut[mu] * self.rcut[mu]
            for n in self.image_range(self.rcut[mu]):
                c = self.image_center(mu, n)
                dx = x - c[0]
                dx2 = dx * dx
                if not dx2 < rc2:
                    continue
                dy = y - c[1]
                dz = z - c[2]
                r2 = (dx2 + (dy * dy)[:, None]) + (dz * dz)[None, :]
                m = r2 < rc2
                if not m.any():
                    continue
                out[:, :, mu] += self.bloch_phase(k, n) * np.where(
                    m, self.norm[mu] * np.exp(-self.alpha[mu] * r2), 0.0)
        return out.reshape(ny * nz, self.M)

    def Xk(self, k):
        """Dense Bloch basis matrix X_k[r, mu] = chi_mu,k(r), grid in C order."""
        if k in self._Xk:
            return self._Xk[k]
        X = np.concatenate([self.basis_plane_k(i, k) for i in range(int(self.n[0]))])
        if self._cache_x:
            self._Xk[k] = X
        return X

    def _planes_k(self, k):
        """(x-plane index, basis rows of that plane): from the cached X_k, or
        built one plane at a time when caching is off (large systems)."""
        per = int(self.n[1] * self.n[2])
        if self._cache_x or k in self._Xk:
            X = self.Xk(k)
            for i in range(int(self.n[0])):
                yield i, X[i * per:(i + 1) * per]
        else:
            for i in range(int(self.n[0])):
                yield i, self.basis_plane_k(i, k)

    # ---- S(k), T(k) ------------------------------------------------------------
    def overlap_kinetic_k(self, k):
        """S(k), T(k) of normalized s-Gaussians summed over images R with
        |d_mu - d_nu - R| < r_c,mu + r_c,nu, each with the phase exp(i k.R)."""
        M = self.M
        S = np.zeros((M, M), dtype=np.complex128)
        T = np.zeros((M, M), dtype=np.complex128)
        a = self.alpha[:, None]
        b = self.alpha[None, :]
        xi = a * b / (a + b)
        pre = (2.0 * np.sqrt(a * b) / (a + b)) ** 1.5
        cut = self.rcut[:, None] + self.rcut[None, :]
        d = self.centers[:, None, :] - self.centers[None, :, :]
        for n in self.image_range(2.0 * float(self.rcut.max())):
            R = d - np.array(n) * self.L
            R2 = (R * R).sum(-1)
            m = R2 < cut * cut
            if not m.any():
                continue
            s = np.where(m, pre * np.exp(-xi * R2), 0.0)
            ph = self.bloch_phase(k, n)
            S += ph * s
            T += ph * (xi * (3.0 - 2.0 * xi * R2) * s)
        return S, T

    # ---- density and Hamiltonian per k-point (Eq. 2, Eq. 11-12) ---------------
    def density_k(self, D, k):
        """sum_mu,nu chi_mu,k(r) D_mu,nu conj(chi_nu,k(r)) (real up to rounding)."""
        out = np.empty(self.G)
        per = int(self.n[1] * self.n[2])
        for i, Xp in self._planes_k(k):
            out[i * per:(i + 1) * per] = np.einsum("pa,pa->p", Xp @ D, Xp.conj()).real
        return out.reshape(tuple(self.n))

    def potential_matrix_k(self, v, k):
        """V_mu,nu(k) = dV sum_r conj(chi_mu,k(r)) v(r) chi_nu,k(r)."""
        Vm = np.zeros((self.M, self.M), dtype=np.complex128)
        per = int(self.n[1] * self.n[2])
        vf = v.reshape(-1)
        for i, Xp in self._planes_k(k):
            Vm += Xp.conj().T @ (vf[i * per:(i + 1) * per, None] * Xp)
        return self.dV * Vm

    # ---- reference orbitals and occupations ---------------------------------------
    def reference_k(self):
        """Per k-point: S, T, h_core = T + V_ext, the generalized eigenvectors C0
        (C0^dag S C0 = I, ascending eps); the Fermi level and the fixed
        occupations f_m(k) = 2 w_k FD((eps - mu) / kT)."""
        if self._kref is not None:
            return self._kref
        vext = self.vext()
        S, T, H0, C0, eps = [], [], [], [], []
        for k in range(self.nk):
            Sk, Tk = self.overlap_kinetic_k(k)
            hk = Tk + self.potential_matrix_k(vext, k)
            hk = 0.5 * (hk + hk.conj().T)
            Sk = 0.5 * (Sk + Sk.conj().T)
            # generalized Hermitian eigenproblem through S^(-1/2)
            w, Q = np.linalg.eigh(Sk)
            Sih = (Q / np.sqrt(w)) @ Q.conj().T
            e, Y = np.linalg.eigh(Sih @ hk @ Sih)
            S.append(Sk); T.append(Tk); H0.append(hk)
            C0.append(Sih @ Y); eps.append(e)
        if self.kT == 0.0:  # integer occupation (one k-point): the n_e / 2 lowest doubly
            assert self.nk == 1
            mu = 0.0
            f = [np.where(np.arange(self.M) < self.n_e // 2, 2.0 * self.kw[0], 0.0)]
        else:
            mu = fermi_level(eps, self.kw, self.n_e, self.kT)
            f = [2.0 * self.kw[k] * fermi_dirac((eps[k] - mu) / self.kT) for k in range(self.nk)]
        self._kref = dict(S=S, T=T, hcore=H0, C0=C0, eps_core=eps, mu=mu, f=f, vext=vext)
        return self._kref

    def set_reference(self, C0, f=None):
        """Replace the reference orbitals C0(k) that O(k) = C0(k) exp(A(k))
        rotates (Eq. 6-7) and, optionally, the occupations; the rest of the
        reference (S, T, v_ext) stays."""
        ref = dict(self.reference_k())
        ref["C0"] = [np.asarray(c, dtype=np.complex128) for c in C0]
        if f is not None:
            ref["f"] = [np.asarray(x, dtype=np.float64) for x in f]
        self._kref = ref

    def lowdin_reference(self):
        """S(k)^(-1/2) per k-point (a matrix function, free of the eigenvector
        phases): the Loewdin orthonormal orbitals of the Bloch basis."""
        out = []
        for k in range(self.nk):
            S, _ = self.overlap_kinetic_k(k)
            S = 0.5 * (S + S.conj().T)
            w, Q = np.linalg.eigh(S)
            out.append((Q / np.sqrt(w)) @ Q.conj().T)
        return out

    # ---- variables <-> A(k) (Eq. 22-24) ----------------------------------------
    def A_of(self, v):
        """Skew-Hermitian A from the M^2 real variables of one k-point."""
        M = self.M
        nre = M * (M - 1) // 2
        A = np.zeros((M, M), dtype=np.complex128)
        A[self._iu] = v[:nre]
        A[self._iud] += 1j * v[nre:]
        diag = 1j * np.diag(A).imag
        A = A - A.conj().T
        A[np.diag_indices(M)] = diag
        return A

    def vars_of_grad(self, dEda):
        """Real-variable gradient from the complex derivatives dE/da_ij (Eq. 20)."""
        return np.concatenate([2.0 * dEda[self._iu].real, -2.0 * dEda[self._iud].imag])

    # ---- energy and gradient -----------------------------------------------------
    def orbitals_k(self, a):
        ref = self.reference_k()
        out = []
        for k in range(self.nk):
            A = self.A_of(a[k * self.nvar:(k + 1) * self.nvar])
            out.append((A, ref["C0"][k] @ self.expm_eig(A)))
        return out

    def energy_terms_k(self, Ds):
        ref = self.reference_k()
        rho = np.zeros(tuple(self.n))
        for k in range(self.nk):
            rho += self.density_k(Ds[k], k)
        vH = self.hartree_potential(rho)
        ex, vx = self.lda_x(rho)
        vext = ref["vext"]
        kin = [float(np.sum(Ds[k] * ref["T"][k].T).real) for k in range(self.nk)]
        terms = dict(kinetic=_fsum(kin), external=self.dV * _fsum(rho * vext),
                     hartree=0.5 * self.dV * _fsum(rho * vH), exchange=self.dV * _fsum(ex))
        return _fsum(list(terms.values())), terms, rho, vext + vH + vx

    def density_matrices(self, orbs):
        ref = self.reference_k()
        return [(O * ref["f"][k][None, :]) @ O.conj().T for k, (_, O) in enumerate(orbs)]

    def energy(self, a):
        orbs = self.orbitals_k(a)
        E = self.energy_terms_k(self.density_matrices(orbs))[0]
        if self.sic:
            E += self.sic_terms(orbs[0][1], self.reference_k()["f"][0])[0]
        return E

    # ---- Perdew-Zunger self-interaction correction (Eq. 16-18 as read) -------------
    def lda_x_polarized(self, n):
        """Exchange of a fully spin-polarized density n (one spin channel):
        e_x = -(3/4)(6/pi)^(1/3) n^(4/3), v_x = -(6/pi)^(1/3) n^(1/3) (the
        unpolarized formula at 2n, halved: E_x^unpol[2n] = 2 E_x^pol[n])."""
        if not self.exchange:
            return np.zeros_like(n), np.zeros_like(n)
        r = np.maximum(n, 0.0)
        cx = (6.0 / math.pi) ** (1.0 / 3.0)
        r13 = np.cbrt(r)
        return -0.75 * cx * r * r13, -cx * r13

    def sic_terms(self, O, f):
        """PZ-SIC at one k-point (the Gamma point) for orbitals O (columns) with
        occupations f (spin included): E_SIC = -sum_k f_k (E_H[n_k] + E_x^pol[n_k])
        with the unit orbital densities n_k = |phi_k|^2, one self-interaction per
        electron; the orbital potentials V^k = v_H[n_k] + v_x^pol[n_k] and the
        matrix S with S_mk = <phi_m|V^k|phi_k>."""
        X = self.Xk(0) if self._cache_x else None
        E = 0.0
        S = np.zeros((self.M, self.M), dtype=np.complex128)
        for k in range(self.M):
            if f[k] == 0.0:
                continue
            if X is not None:
                phi = X @ O[:, k]
            else:
                phi = np.concatenate([Xp @ O[:, k] for _, Xp in self._planes_k(0)])
            n = (phi.conj() * phi).real.reshape(tuple(self.n))
            vH = self.hartree_potential(n)
            ex, vx = self.lda_x_polarized(n)
            E -= f[k] * (0.5 * self.dV * _fsum(n * vH) + self.dV * _fsum(ex))
            Vk = self.potential_matrix_k(vH + vx, 0)
            S[:, k] = O.conj().T @ (Vk @ O[:, k])
        return E, S

    def energy_grad(self, a, want=False):
        """E and the real-variable gradient (nk * M^2) at the variables a."""
        ref = self.reference_k()
        orbs = self.orbitals_k(a)
        Ds = self.density_matrices(orbs)
        E, terms, rho, v = self.energy_terms_k(Ds)
        if self.sic:
            assert self.nk == 1 and not np.any(self.kfrac), "PZ-SIC at the Gamma point only"
            E_sic, S = self.sic_terms(orbs[0][1], ref["f"][0])
            terms = dict(terms, sic=E_sic)
            E = E + E_sic
        g = np.empty(self.nk * self.nvar)
        extra = []
        for k, (A, O) in enumerate(orbs):
            H = ref["T"][k] + self.potential_matrix_k(v, k)
            Hmo = O.conj().T @ H @ O
            f = ref["f"][k]
            L = f[:, None] * Hmo - Hmo * f[None, :]
            if self.sic:
                # the orbital-dependent Hamiltonians H - V^k (E_SIC enters with a
                # minus sign): L_mk += f_k <m|V^k|k> - f_m <m|V^m|k>, the second
                # term the Hermitian conjugate of the first with m, k swapped
                L = L + S * f[None, :] - (S * f[None, :]).conj().T
            dEda = self.grad_eq39(A, L)
            g[k * self.nvar:(k + 1) * self.nvar] = self.vars_of_grad(dEda)
            extra.append(dict(H=H, Hmo=Hmo, L=L, dEda=dEda, O=O, D=Ds[k]))
        if want:
            return E, g, dict(terms=terms, rho=rho, v=v, k=extra)
        return E, g

    # ---- scaling and squaring with the approximate gradient (Eq. 38, 42-44) -----
    @staticmethod
    def expm_ss(A):
        """Eq. 38: exp(A) = exp(A / 2^m)^(2^m) with a [q, q] Pade approximant of
        exp(A / 2^m), m and q chosen by the algorithm of Al-Mohy and Higham
        (SciPy's expm, the implementation the paper names)."""
        from scipy.linalg import expm
        return expm(A)

    def energy_grad_approx(self, a, want=False):
        """E with exp(A(k)) by Eq. 38 and the approximate gradient of Eq. 42,
        G ~ L^T (the first term of the Eq. 19 expansion; exact at A = 0), in
        the real variables of Eq. 20-24."""
        ref = self.reference_k()
        orbs = []
        for k in range(self.nk):
            A = self.A_of(a[k * self.nvar:(k + 1) * self.nvar])
            orbs.append((A, ref["C0"][k] @ self.expm_ss(A)))
        Ds = self.density_matrices(orbs)
        E, terms, rho, v = self.energy_terms_k(Ds)
        g = np.empty(self.nk * self.nvar)
        Ls = []
        for k, (A, O) in enumerate(orbs):
            H = ref["T"][k] + self.potential_matrix_k(v, k)
            Hmo = O.conj().T @ H @ O
            f = ref["f"][k]
            L = f[:, None] * Hmo - Hmo * f[None, :]
            fac = np.where(np.eye(self.M, dtype=bool), 0.5, 1.0)
            g[k * self.nvar:(k + 1) * self.nvar] = self.vars_of_grad(fac * L.T)
            Ls.append((A, L, H))
        if want:
            return E, g, dict(terms=terms, rho=rho, v=v, L=Ls)
        return E, g

    @staticmethod
    def commutator_test(Ls, eps=3.0):
        """The reference-update test of Sec. 3.5 as read here: update when
        |L| < eps |[A, L]| (Frobenius norms over all k-points), eps = 3."""
        nL = math.sqrt(sum(float(np.vdot(L, L).real) for _, L, _ in Ls))
        nC = math.sqrt(sum(float(np.vdot(A @ L - L @ A, A @ L - L @ A).real)
                           for A, L, _ in Ls))
        return nL < eps * nC, nL, nC

    def minimize_ss(self, a0, n_steps, ref_update=-1):
        """ETDM with exp by Eq. 38 and the approximate gradient of Eq. 42 (the
        paper's "ss" route), with reference updates C <- C exp(A), A <- 0:
        ref_update = n > 0 after every n steps, -1 by the Sec. 3.5 test, 0
        never.  After an update the L-BFGS memory is erased (Sec. 3.5) and the
        Eq. 33 orbital energies are taken afresh at the new reference.
        Returns the (E, alpha, trials) history, the final variables and the
        number of updates."""
        eps = self.orbital_energies()
        lb = LBFGS(lambda beta: self.precond(eps, beta))
        a = np.array(a0, dtype=np.float64)
        E, g, ex = self.energy_grad_approx(a, want=True)
        hist = [(E, 0.0, 1)]
        since, updates = 0, 0
        for _ in range(n_steps):
            if ref_update > 0:
                upd = since >= ref_update
            elif ref_update < 0:
                upd = self.commutator_test(ex["L"])[0]
            else:
                upd = False
            if upd:
                ref = self.reference_k()
                self.set_reference([ref["C0"][k] @ self.expm_ss(
                    self.A_of(a[k * self.nvar:(k + 1) * self.nvar])) for k in range(self.nk)])
                a = np.zeros_like(a)
                lb.reset()
                eps = self.orbital_energies()
                lb.pfn = lambda beta, eps=eps: self.precond(eps, beta)
                E, g, ex = self.energy_grad_approx(a, want=True)
                since, updates = 0, updates + 1
            p = lb.step(a, g)
            d0 = float(np.vdot(g, p))
            if not d0 < 0.0:
                lb.reset()
                p = -self.precond(eps, lb.beta) * g
                lb.a_prev, lb.g_prev = a.copy(), g.copy()
                d0 = float(np.vdot(g, p))

            def phi(alpha, a=a, p=p):
                Et, gt, ext = self.energy_grad_approx(a + alpha * p, want=True)
                return Et, float(np.vdot(gt, p)), (gt, ext)

            alpha, Et, _, pay, trials = line_search(phi, E, d0)
            if pay is not None:
                E, (g, ex) = Et, pay
                a = a + alpha * p
            hist.append((E, alpha, trials))
            since += 1
        return hist, a, updates

    # ---- preconditioner (Eq. 33-34, k-point weight on beta) -----------------------
    def orbital_energies(self):
        """eps_m(k) = (C0^dag H[rho(A = 0)] C0)_mm per k-point."""
        ref = self.reference_k()
        _, _, ex = self.energy_grad(np.zeros(self.nk * self.nvar), want=True)
        return [np.einsum("mj,mn,nj->j", ref["C0"][k].conj(), ex["k"][k]["H"],
                          ref["C0"][k]).real for k in range(self.nk)]

    def precond(self, eps, beta, gamma=GAMMA):
        """P for every real variable: 1 / (2 (1-gamma) |(e_i - e_j)(f_i - f_j)|
        + gamma beta w_k), the same for Re a_ij and Im a_ij."""
        ref = self.reference_k()
        out = []
        for k in range(self.nk):
            e, f = eps[k], ref["f"][k]
            full = 1.0 / (2.0 * (1.0 - gamma) * np.abs((e[:, None] - e[None, :])
                                                       * (f[:, None] - f[None, :]))
                          + gamma * beta * self.kw[k])
            out.append(np.concatenate([full[self._iu], full[self._iud]]))
        return np.concatenate(out)
