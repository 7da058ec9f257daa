"""Plain FP64 CPU oracle of the ETDM energy + gradient evaluation.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product path (the CUDA library and its Python binding) never
calls it, and it shares no code with that path.

It follows the paper (Ivanov, Jonsson, Vegge, Jonsson, "Direct energy
minimization based on exponential transformation in density functional
calculations of finite and extended systems", arXiv:2101.12597) step by step,
in FP64 / complex128, with numpy's matmul, eigh and FFT as library steps:

* Sec. 2, Eq. 1-4 and Eq. 11-12: energy functional, density, LCAO orbitals,
  density matrix, Hamiltonian matrix.
* Eq. 7: O = C exp(A); Eq. 35: exp(A) from the eigendecomposition of iA.
* Eq. 13-14 with Eq. 39-41: the exact gradient through the commutator
  L = [F, H] (the divided-difference matrix written with the sign that makes
  A -> 0 reduce to Eq. 42; see ``grad_eq39``).
* Eq. 36-37: the occupied-virtual parametrization and its closed-form
  exponential (used here only as a cross-check of Eq. 35).
* Eq. 33-34: the diagonal preconditioner; Sec. 3.1: L-BFGS (m = 3);
  Eq. 25-29: line search conditions and parameter values.
* Eq. 45: the convergence criterion (residual of the Kohn-Sham equations of
  the occupied orbitals), with H psi represented in the span of the basis.

The model Hamiltonian (s-type normalized Gaussians, Gaussian ion charges,
spectral Poisson solve, Slater exchange) stands in for the paper's PAW/PBE
setting.  Readings of passages that are garbled or silent:

* Eq. 37 prints cos(P) and a garbled lower-right block; the closed form used
  is exp(A) = [[cos sqrt(P), s(P) A_ov], [-A_ov^T s(P), I + A_ov^T c(P) A_ov]]
  with s(p) = sin(sqrt p)/sqrt p and c(p) = (cos sqrt p - 1)/p.
* Eq. 40 as printed gives D_ii -> -1 at A = 0, contradicting Eq. 42; the
  divided difference used is (1 - exp(-i d))/(i d) = int_0^1 exp(-i t d) dt.
* Occupation numbers are closed-shell: f = 2 for the N occupied orbitals.
* The orbital energies in Eq. 33 are the diagonal of C0^T H C0 at A = 0 and
  the orbital-energy term enters with its absolute value so that the
  preconditioner stays positive for a non-aufbau reference.

Conventions the paper does not fix, whose parity is unpinned (both sides
implement the same choice; tests pin only the properties they must keep):

* beta^(0) = 1 Ha, and the curvature threshold s.y > 1e-30 below which a pair
  is not stored (the skip itself is pinned: the direction equals dense BFGS
  over the stored pairs and stays a descent direction).
* The line search's bracketing, interpolation safeguards and trial limit
  beyond the Eq. 25-29 conditions (pinned: the accepted point satisfies them).
"""
from __future__ import annotations

import math

import numpy as np

# Eq. 29 parameter values
C1, C2, DELTA, SIGMA, EPS_E = 1e-4, 0.9, 0.1, 0.9, 1e-6
GAMMA = 0.25          # Eq. 33
LBFGS_M = 3           # Sec. 3.1
BETA0 = 1.0           # beta^(0): no previous step exists yet
MAX_TRIALS = 20
IMG_MAX = 3           # |n| <= 3 lattice images per axis


def _fsum(x):
    return math.fsum(np.asarray(x, dtype=np.float64).ravel().tolist())


class Oracle:
    """One periodic system at the Gamma point, occupied-virtual rotations."""

    def __init__(self, sysd, hartree=True, exchange=True, vext=True,
                 cache_x=True):
        self.sys = sysd
        self.pos = np.asarray(sysd["pos"], dtype=np.float64)
        self.Z = np.asarray(sysd["Z"], dtype=np.float64)
        self.bf_atom = np.asarray(sysd["bf_atom"], dtype=np.int64)
        self.alpha = np.asarray(sysd["bf_exp"], dtype=np.float64)
        self.rcut = np.asarray(sysd["bf_rcut"], dtype=np.float64)
        self.L = np.asarray(sysd["box"], dtype=np.float64)
        self.n = np.asarray(sysd["grid"], dtype=np.int64)
        self.sigma = float(sysd["ion_sigma"])
        self.n_e = int(sysd["n_electrons"])
        self.M = len(self.alpha)
        self.N = self.n_e // 2
        self.V = self.M - self.N
        self.h = self.L / self.n                      # grid spacing per axis
        self.dV = float(self.h[0] * self.h[1] * self.h[2])
        self.G = int(np.prod(self.n))
        self.omega = float(self.L[0] * self.L[1] * self.L[2])
        self.centers = self.pos[self.bf_atom]          # d_mu
        self.norm = (2.0 * self.alpha / math.pi) ** 0.75
        self.hartree, self.exchange, self.use_vext = hartree, exchange, vext
        self.f = np.zeros(self.M)
        self.f[: self.N] = 2.0
        self._X = None
        self._cache_x = cache_x
        self._ref = None

    # ---- geometry ---------------------------------------------------------
    def coords(self, ax):
        """Grid coordinates x_i = i * (L / N) along one axis."""
        return np.arange(self.n[ax], dtype=np.float64) * self.h[ax]

    def images(self, mu):
        """Lattice images R = n L that can bring function mu within r_c."""
        out = []
        rng = [range(-IMG_MAX, IMG_MAX + 1)] * 3
        for nx in rng[0]:
            for ny in rng[1]:
                for nz in rng[2]:
                    n = (nx, ny, nz)
                    ok = all(abs(n[a]) <= math.floor(self.rcut[mu] / self.L[a]) + 1
                             for a in range(3))
                    if ok:
                        out.append(n)
        return out

    def image_center(self, mu, n):
        return np.array([self.centers[mu, a] + n[a] * self.L[a] for a in range(3)])

    # ---- basis on the grid (Eq. 3, Eq. 5 at the Gamma point) ---------------
    def basis_plane(self, i):
        """chi_mu at all points of the x-plane i, shape (ny*nz, M).

        chi_mu(r) = sum_R eta(r - d_mu - R) over images with |r - d_mu - R| < r_c,
        eta(r) = (2a/pi)^(3/4) exp(-a r^2).  r^2 = (dx^2 + dy^2) + dz^2.
        """
        ny, nz = int(self.n[1]), int(self.n[2])
        x = self.coords(0)[i]
        y, z = self.coords(1), self.coords(2)
        out = np.zeros((ny, nz, self.M))
        for mu in range(self.M):
            rc2 = self.rcut[mu] * self.rcut[mu]
            for n in self.images(mu):
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
                out[:, :, mu] += np.where(
                    m, self.norm[mu] * np.exp(-self.alpha[mu] * r2), 0.0)
        return out.reshape(ny * nz, self.M)

    def X(self):
        """Dense basis matrix X[r, mu] = chi_mu(r), grid in C order (x, y, z)."""
        if self._X is not None:
            return self._X
        X = np.concatenate([self.basis_plane(i) for i in range(int(self.n[0]))])
        if self._cache_x:
            self._X = X
        return X

    def _planes(self):
        if self._X is not None or self._cache_x:
            X = self.X()
            per = int(self.n[1] * self.n[2])
            for i in range(int(self.n[0])):
                yield i, X[i * per:(i + 1) * per]
        else:
            for i in range(int(self.n[0])):
                yield i, self.basis_plane(i)

    # ---- truncation lists (bit-exact index work) ---------------------------
    @staticmethod
    def pack_key(mu, n):
        return mu * 512 + (n[0] + 4) * 64 + (n[1] + 4) * 8 + (n[2] + 4)

    def tile_list(self, tile_dims, t):
        """Sorted keys of (mu, image) pairs with at least one point of tile t
        strictly inside the truncation sphere (brute force over the points)."""
        tx, ty, tz = tile_dims
        nbx = -(-int(self.n[0]) // tx)
        nby = -(-int(self.n[1]) // ty)
        nbz = -(-int(self.n[2]) // tz)
        bx, rem = divmod(t, nby * nbz)
        by, bz = divmod(rem, nbz)
        I = np.arange(bx * tx, min((bx + 1) * tx, int(self.n[0])))
        J = np.arange(by * ty, min((by + 1) * ty, int(self.n[1])))
        K = np.arange(bz * tz, min((bz + 1) * tz, int(self.n[2])))
        x, y, z = self.coords(0)[I], self.coords(1)[J], self.coords(2)[K]
        keys = []
        for mu in range(self.M):
            rc2 = self.rcut[mu] * self.rcut[mu]
            for n in self.images(mu):
                c = self.image_center(mu, n)
                dx, dy, dz = x - c[0], y - c[1], z - c[2]
                r2 = ((dx * dx)[:, None, None] + (dy * dy)[None, :, None]) \
                    + (dz * dz)[None, None, :]
                if (r2 < rc2).any():
                    keys.append(self.pack_key(mu, n))
        return np.array(sorted(keys), dtype=np.int32)

    def n_tiles(self, tile_dims):
        return int(np.prod([-(-int(self.n[a]) // tile_dims[a]) for a in range(3)]))

    # ---- analytic overlap and kinetic matrices (Eq. 4, Eq. 11) --------------
    def overlap_kinetic(self):
        """S and T of normalized s-Gaussians summed over lattice images with
        |d_mu - d_nu - R| < r_c,mu + r_c,nu."""
        M = self.M
        S = np.zeros((M, M))
        T = np.zeros((M, M))
        a = self.alpha[:, None]
        b = self.alpha[None, :]
        xi = a * b / (a + b)
        pre = (2.0 * np.sqrt(a * b) / (a + b)) ** 1.5
        cut = self.rcut[:, None] + self.rcut[None, :]
        d = self.centers[:, None, :] - self.centers[None, :, :]
        for nx in range(-IMG_MAX, IMG_MAX + 1):
            for ny in range(-IMG_MAX, IMG_MAX + 1):
                for nz in range(-IMG_MAX, IMG_MAX + 1):
                    R = d - np.array([nx, ny, nz]) * self.L
                    R2 = (R * R).sum(-1)
                    m = R2 < cut * cut
                    if not m.any():
                        continue
                    s = np.where(m, pre * np.exp(-xi * R2), 0.0)
                    S += s
                    T += xi * (3.0 - 2.0 * xi * R2) * s
        return S, T

    # ---- reciprocal space ---------------------------------------------------
    def gvectors(self):
        """|G|^2 on the FFT grid, fftfreq ordering (Nyquist at n = -N/2)."""
        g = [2.0 * math.pi * np.fft.fftfreq(int(self.n[a]), d=self.h[a])
             for a in range(3)]
        G2 = (g[0] ** 2)[:, None, None] + (g[1] ** 2)[None, :, None] \
            + (g[2] ** 2)[None, None, :]
        return g, G2

    def vext(self):
        """Potential of Gaussian ion charges (width sigma) on the grid:
        v(G) = -(4 pi / (Omega G^2)) sum_I Z_I exp(-G^2 s^2/2) exp(-i G.R_I),
        v(G=0) = 0, v(r) = Re sum_G v(G) exp(i G.r)."""
        if not self.use_vext:
            return np.zeros(tuple(self.n))
        g, G2 = self.gvectors()
        Sg = np.zeros(tuple(self.n), dtype=np.complex128)
        for I in range(len(self.Z)):
            ph = [np.exp(-1j * g[a] * self.pos[I, a]) for a in range(3)]
            Sg += self.Z[I] * ph[0][:, None, None] * ph[1][None, :, None] \
                * ph[2][None, None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            vg = -4.0 * math.pi / (self.omega * G2) * np.exp(-G2 * self.sigma ** 2 / 2.0) * Sg
        vg[0, 0, 0] = 0.0
        return (np.fft.ifftn(vg) * self.G).real

    def hartree_potential(self, rho):
        """Spectral Poisson solve: v_H(G) = 4 pi rho(G) / G^2, v_H(0) = 0."""
        if not self.hartree:
            return np.zeros_like(rho)
        _, G2 = self.gvectors()
        rg = np.fft.fftn(rho)
        with np.errstate(divide="ignore", invalid="ignore"):
            vg = 4.0 * math.pi * rg / G2
        vg[0, 0, 0] = 0.0
        return np.fft.ifftn(vg).real

    def lda_x(self, rho):
        """Slater (Dirac) exchange, spin-unpolarized: energy density and potential."""
        if not self.exchange:
            return np.zeros_like(rho), np.zeros_like(rho)
        r = np.maximum(rho, 0.0)
        cx = (3.0 / math.pi) ** (1.0 / 3.0)
        r13 = np.cbrt(r)
        return -0.75 * cx * r * r13, -cx * r13

    # ---- density and Hamiltonian matrix (Eq. 2, Eq. 11-12) ------------------
    @staticmethod
    def density_plane(Xp, D):
        """rho at the points of one x-plane: sum_{mu,nu} chi_mu D_mu,nu chi_nu."""
        return np.einsum("pa,pa->p", Xp @ D, Xp)

    @staticmethod
    def potential_plane(Xp, vp):
        """One x-plane's part of sum_r chi_mu(r) v(r) chi_nu(r) (without dV)."""
        return Xp.T @ (vp[:, None] * Xp)

    def density(self, D):
        """rho(r) = sum_{mu,nu} chi_mu(r) D_mu,nu chi_nu(r)."""
        out = np.empty(self.G)
        per = int(self.n[1] * self.n[2])
        for i, Xp in self._planes():
            out[i * per:(i + 1) * per] = self.density_plane(Xp, D)
        return out.reshape(tuple(self.n))

    def potential_matrix(self, v):
        """V_mu,nu = dV sum_r chi_mu(r) v(r) chi_nu(r)."""
        Vm = np.zeros((self.M, self.M))
        per = int(self.n[1] * self.n[2])
        vf = v.reshape(-1)
        for i, Xp in self._planes():
            Vm += self.potential_plane(Xp, vf[i * per:(i + 1) * per])
        return Vm * self.dV

    # ---- reference orbitals -------------------------------------------------
    def reference(self):
        """C0 = S^(-1/2) (Loewdin from the identity); its columns are ordered by
        ascending (C0^T h_core C0)_jj (ties: lower index first) and the first N
        are occupied.  Also returns S, T and v_ext."""
        if self._ref is not None:
            return self._ref
        S, T = self.overlap_kinetic()
        w, Q = np.linalg.eigh(S)
        Sih = (Q / np.sqrt(w)) @ Q.T
        vext = self.vext()
        hcore = T + self.potential_matrix(vext)
        diag = np.einsum("mj,mn,nj->j", Sih, hcore, Sih)
        order = np.argsort(diag, kind="stable")
        C0 = Sih[:, order]
        self._ref = dict(S=S, T=T, C0=C0, order=order, vext=vext, hcore=hcore)
        return self._ref

    # ---- matrix exponential ---------------------------------------------------
    def full_A(self, Aov):
        """Eq. 36: A = [[0, A_ov], [-A_ov^T, 0]]."""
        A = np.zeros((self.M, self.M))
        A[: self.N, self.N:] = Aov
        A[self.N:, : self.N] = -Aov.T
        return A

    @staticmethod
    def expm_eig(A):
        """Eq. 35: exp(A) = W exp(-i Omega) W^dagger with iA = W Omega W^dagger."""
        Om, W = np.linalg.eigh(1j * A)
        return (W * np.exp(-1j * Om)) @ W.conj().T

    def expm_occvirt(self, Aov):
        """Eq. 37 (as read above) via the eigendecomposition of P = A_ov A_ov^T."""
        P = Aov @ Aov.T
        p, W = np.linalg.eigh(P)
        p = np.maximum(p, 0.0)
        sq = np.sqrt(p)
        small = p < 1e-2
        s = np.where(small, 1 - p / 6 + p**2 / 120 - p**3 / 5040 + p**4 / 362880,
                     np.sin(sq) / np.where(small, 1.0, sq))
        c = np.where(small, -0.5 + p / 24 - p**2 / 720 + p**3 / 40320 - p**4 / 3628800,
                     (np.cos(sq) - 1) / np.where(small, 1.0, p))
        cosP = (W * np.cos(sq)) @ W.T
        sP = (W * s) @ W.T
        cP = (W * c) @ W.T
        N, M = self.N, self.M
        U = np.zeros((M, M))
        U[:N, :N] = cosP
        U[:N, N:] = sP @ Aov
        U[N:, :N] = -Aov.T @ sP
        U[N:, N:] = np.eye(M - N) + Aov.T @ cP @ Aov
        return U

    @staticmethod
    def expm_taylor(A, terms=30):
        """exp(A) by a truncated Taylor series with scaling and squaring, in
        numpy longdouble."""
        A = np.asarray(A, dtype=np.longdouble)
        nrm = float(np.abs(A).sum(axis=0).max())
        s = max(0, int(math.ceil(math.log2(nrm / 0.5))) if nrm > 0.5 else 0)
        B = A / np.longdouble(2 ** s)
        E = np.eye(len(A), dtype=np.longdouble)
        term = np.eye(len(A), dtype=np.longdouble)
        for k in range(1, terms + 1):
            term = term @ B / np.longdouble(k)
            E = E + term
        for _ in range(s):
            E = E @ E
        return E

    # ---- energy (Eq. 1) -------------------------------------------------------
    def orbitals(self, Aov, C0=None):
        ref = self.reference()
        C0 = ref["C0"] if C0 is None else C0
        U = self.expm_eig(self.full_A(Aov))
        assert np.abs(U.imag).max() < 1e-10
        return C0 @ U.real

    def density_matrix(self, O):
        """Eq. 12: D = O F O^T with f = 2 on the occupied columns."""
        Oc = O[:, : self.N]
        return 2.0 * Oc @ Oc.T

    def energy_terms(self, D):
        ref = self.reference()
        rho = self.density(D)
        vH = self.hartree_potential(rho)
        ex, vx = self.lda_x(rho)
        vext = ref["vext"]
        terms = dict(
            kinetic=_fsum(D * ref["T"]),
            external=self.dV * _fsum(rho * vext),
            hartree=0.5 * self.dV * _fsum(rho * vH),
            exchange=self.dV * _fsum(ex),
        )
        E = _fsum(list(terms.values()))
        return E, terms, rho, vext + vH + vx

    def energy(self, Aov, C0=None):
        D = self.density_matrix(self.orbitals(Aov, C0))
        return self.energy_terms(D)[0]

    # ---- gradient (Eq. 13-14, Eq. 39-41) ---------------------------------------
    def commutator_L(self, O, H):
        """Eq. 13: L = [F, O^T H O]."""
        Hmo = O.T @ H @ O
        return self.f[:, None] * Hmo - Hmo * self.f[None, :], Hmo

    @staticmethod
    def grad_eq39(A, L):
        """dE/da_ij for all i, j (complex Wirtinger form, Eq. 14):
        G^T = W ((W^dag L W) o Dt) W^dag with iA = W Omega W^dag and
        Dt_ab = int_0^1 exp(-i t (Omega_a - Omega_b)) dt; dE/da_ij = (2-d_ij)/2 G_ij."""
        Om, W = np.linalg.eigh(1j * A)
        Lt = W.conj().T @ L @ W
        d = Om[:, None] - Om[None, :]
        small = np.abs(d) < 1e-3
        dsafe = np.where(small, 1.0, d)
        Dt = np.where(small, 1 - 0.5j * d - d * d / 6 + 1j * d**3 / 24,
                      (1 - np.exp(-1j * dsafe)) / (1j * dsafe))
        G = (W @ (Lt * Dt) @ W.conj().T).T
        fac = np.where(np.eye(len(A), dtype=bool), 0.5, 1.0)
        return fac * G

    def energy_grad(self, Aov, C0=None, want=False):
        """E and g = dE/dA_ov (real occupied-virtual variables, Eq. 20)."""
        ref = self.reference()
        C0 = ref["C0"] if C0 is None else C0
        A = self.full_A(Aov)
        O = self.orbitals(Aov, C0)
        D = self.density_matrix(O)
        E, terms, rho, v = self.energy_terms(D)
        H = ref["T"] + self.potential_matrix(v)
        L, Hmo = self.commutator_L(O, H)
        dEda = self.grad_eq39(A, L)
        g = 2.0 * dEda[: self.N, self.N:].real
        if want:
            return E, g, dict(terms=terms, rho=rho, v=v, H=H, D=D, O=O, L=L,
                              Hmo=Hmo, dEda=dEda)
        return E, g

    # ---- convergence criterion (Eq. 45) ----------------------------------------
    def residual_eq45(self, Aov, C0=None):
        """Eq. 45: (1/N_e) sum_i f_i int |H psi_i - sum_j lambda_ij psi_j|^2 dr,
        lambda = O^T H O over the occupied orbitals, with H psi_i represented in
        the span of the basis (what an LCAO calculation holds of it): its
        coefficients are S^-1 (H O)_i, so the residual of orbital i has the
        coefficients r_i = S^-1 (H O)_i - sum_j O_j lambda_ji and the integral
        is r_i^T S r_i.  Hartree^2."""
        ref = self.reference()
        _, _, ex = self.energy_grad(Aov, C0, want=True)
        N = self.N
        O = ex["O"][:, :N]
        HO = ex["H"] @ O
        lam = O.T @ HO
        R = np.linalg.solve(ref["S"], HO) - O @ lam
        per = np.einsum("mi,mn,ni->i", R, ref["S"], R)
        return float(np.sum(self.f[:N] * per) / self.n_e)

    # ---- preconditioner (Eq. 33-34) ------------------------------------------
    def orbital_energies(self):
        """eps_j = (C0^T H[rho(A=0)] C0)_jj, computed once at the start."""
        ref = self.reference()
        C0 = ref["C0"]
        D = self.density_matrix(C0)
        _, _, _, v = self.energy_terms(D)
        H = ref["T"] + self.potential_matrix(v)
        return np.einsum("mj,mn,nj->j", C0, H, C0)

    def precond(self, eps, beta, gamma=GAMMA):
        """P_ij = 1 / (2 (1-gamma) |(e_i - e_j)(f_i - f_j)| + gamma beta) for
        i occupied, j virtual, as an N x V array."""
        ei = eps[: self.N][:, None]
        ej = eps[self.N:][None, :]
        fi = self.f[: self.N][:, None]
        fj = self.f[self.N:][None, :]
        return 1.0 / (2.0 * (1.0 - gamma) * np.abs((ei - ej) * (fi - fj)) + gamma * beta)


# ---- L-BFGS (Sec. 3.1, two-loop recursion) -------------------------------------
class LBFGS:
    """Limited-memory BFGS with m pairs and the Eq. 33 preconditioner as the
    initial inverse Hessian.  beta^(k) from Eq. 34 uses the latest pair."""

    def __init__(self, precond_fn, m=LBFGS_M, beta0=BETA0):
        self.pfn = precond_fn
        self.m = m
        self.beta = beta0
        self.s, self.y = [], []
        self.a_prev = self.g_prev = None

    def reset(self):
        self.s, self.y = [], []
        self.a_prev = self.g_prev = None

    def step(self, a, g):
        if self.a_prev is not None:
            s = a - self.a_prev
            y = g - self.g_prev
            sy = float(np.vdot(s, y))
            if sy > 1e-30:
                self.beta = float(np.vdot(y, y)) / sy
                self.s.append(s)
                self.y.append(y)
                if len(self.s) > self.m:
                    self.s.pop(0)
                    self.y.pop(0)
        self.a_prev, self.g_prev = a.copy(), g.copy()
        H0 = self.pfn(self.beta)
        q = g.copy()
        alphas = []
        for s, y in zip(reversed(self.s), reversed(self.y)):
            rho = 1.0 / float(np.vdot(y, s))
            al = rho * float(np.vdot(s, q))
            q = q - al * y
            alphas.append(al)
        r = H0 * q
        for (s, y), al in zip(zip(self.s, self.y), reversed(alphas)):
            rho = 1.0 / float(np.vdot(y, s))
            be = rho * float(np.vdot(y, r))
            r = r + s * (al - be)
        return -r


# ---- line search (Eq. 25-29) ------------------------------------------------------
def cubic_min(a, fa, da, b, fb, db):
    """Minimizer of the cubic through (a, fa, fa') and (b, fb, fb'), or None."""
    if a == b:
        return None
    d1 = da + db - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - da * db
    if disc < 0.0:
        return None
    d2 = math.copysign(math.sqrt(disc), b - a)
    den = db - da + 2.0 * d2
    if den == 0.0:
        return None
    return b - (b - a) * (db + d2 - d1) / den


def wolfe_ok(alpha, E, d, E0, d0):
    """Strong Wolfe (Eq. 25-26) or approximate Wolfe (Eq. 27) with Eq. 28."""
    strong = (E <= E0 + C1 * alpha * d0) and (abs(d) <= C2 * abs(d0))
    approx = ((2.0 * DELTA - 1.0) * d0 >= d >= SIGMA * d0) and \
        (E <= E0 + EPS_E * abs(E0))
    return strong or approx


def line_search(phi, E0, d0, max_trials=MAX_TRIALS):
    """Bracketing + zoom with cubic interpolation; alpha = 1 tried first.

    phi(alpha) -> (E, d, payload) with d = grad E(a + alpha p) . p.
    Returns (alpha, E, d, payload, trials)."""
    trials = 0
    prev = (0.0, E0, d0, None)
    alpha = 1.0
    lo = hi = None
    while trials < max_trials:
        E, d, pay = phi(alpha)
        trials += 1
        cur = (alpha, E, d, pay)
        if wolfe_ok(alpha, E, d, E0, d0):
            return alpha, E, d, pay, trials
        if E > E0 + C1 * alpha * d0 or (trials > 1 and E >= prev[1]):
            lo, hi = prev, cur
            break
        if d >= 0.0:
            lo, hi = cur, prev
            break
        nxt = cubic_min(prev[0], prev[1], prev[2], alpha, E, d)
        if nxt is None or not (1.1 * alpha <= nxt <= 4.0 * alpha):
            nxt = 2.0 * alpha
        prev, alpha = cur, nxt
    while lo is not None and trials < max_trials:
        a0, a1 = lo[0], hi[0]
        width = abs(a1 - a0)
        left, right = min(a0, a1), max(a0, a1)
        aj = cubic_min(lo[0], lo[1], lo[2], hi[0], hi[1], hi[2])
        if aj is None or not (left + 0.1 * width <= aj <= right - 0.1 * width):
            aj = 0.5 * (a0 + a1)
        E, d, pay = phi(aj)
        trials += 1
        cur = (aj, E, d, pay)
        if wolfe_ok(aj, E, d, E0, d0):
            return aj, E, d, pay, trials
        if E > E0 + C1 * aj * d0 or E >= lo[1]:
            hi = cur
        else:
            if d * (hi[0] - lo[0]) >= 0.0:
                hi = lo
            lo = cur
    # no acceptable point: take the best point seen
    best = lo if lo is not None else prev
    return best[0], best[1], best[2], best[3], trials


def minimize(oracle, a0, n_steps, eps=None):
    """ETDM minimization: L-BFGS direction, line search with alpha = 1 first.
    Returns the list of (E, alpha, trials) per step and the final a."""
    if eps is None:
        eps = oracle.orbital_energies()
    lb = LBFGS(lambda beta: oracle.precond(eps, beta))
    a = np.array(a0, dtype=np.float64)
    E, g = oracle.energy_grad(a)
    hist = [(E, 0.0, 1)]
    for _ in range(n_steps):
        p = lb.step(a, g)
        d0 = float(np.vdot(g, p))
        if not d0 < 0.0:
            lb.reset()
            p = -oracle.precond(eps, lb.beta) * g
            lb.a_prev, lb.g_prev = a.copy(), g.copy()
            d0 = float(np.vdot(g, p))

        def phi(alpha, a=a, p=p):
            Et, gt = oracle.energy_grad(a + alpha * p)
            return Et, float(np.vdot(gt, p)), gt

        alpha, Et, _, gt, trials = line_search(phi, E, d0)
        if gt is not None:
            E, g = Et, gt
            a = a + alpha * p
        hist.append((E, alpha, trials))
    return hist, a
