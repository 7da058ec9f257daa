"""Seeded synthetic inputs for the ETDM energy+gradient path.

This module is the single source of inputs for both the CUDA path and the
oracle.  It draws random numbers and lays out geometry; it holds none of the
method's arithmetic (no basis values, overlaps, exponentials or energies).

Every system is a plain dict of numpy arrays in atomic units:

    pos        (n_atoms, 3) float64   atom positions, bohr, wrapped into [0, L)
    Z          (n_atoms,)   float64   ion charge of each site
    bf_atom    (M,)         int32     atom carrying each basis function
    bf_exp     (M,)         float64   Gaussian exponent alpha, bohr^-2
    bf_rcut    (M,)         float64   hard truncation radius, bohr
    box        (3,)         float64   orthorhombic cell edges, bohr
    grid       (3,)         int32     real-space grid points per axis
    ion_sigma  float                  width of the Gaussian ion charge, bohr
    n_electrons int                   even; N = n_electrons / 2 doubly occupied
    a0         (N, M-N)     float64   starting occupied-virtual block A_ov

Crystals (k-point sampling, full A(k)) add:

    kpts       (n_k, 3)     float64   k-points, fractional reciprocal coordinates
    kw         (n_k,)       float64   k-point weights (sum 1)
    kT         float                  Fermi-Dirac temperature of the reference
                                      occupations, hartree
    a0         (n_k*M*M,)   float64   real variables of every A(k) (gradient checks)

The recipes (positions, exponents, grid, truncation, A_ov distribution) follow
the workloads the paper studies (small molecules, liquid-water boxes, insulating
crystals with k-point sampling), shrunk
to a model Hamiltonian of s-type Gaussians; the water-like boxes stand in for
the paper's liquid-water snapshots, which are not reproduced here.
"""
from __future__ import annotations

import math

import numpy as np

ANGSTROM = 1.8897261246  # bohr per angstrom (CODATA 2018)

HEAVY_EXPS = [0.3 * 10.0 ** (k / 3.0) for k in range(4)]  # 0.3 .. 3.0 bohr^-2
LIGHT_EXPS = [0.5, 1.5]


def _min_image_dist(d, box):
    d = d - box * np.round(d / box)
    return np.sqrt((d * d).sum(-1))


def _uniform_positions(rng, n, box, min_sep):
    pos = []
    while len(pos) < n:
        p = rng.uniform(0.0, 1.0, 3) * box
        if all(_min_image_dist(p - q, box) >= min_sep for q in pos):
            pos.append(p)
    return np.array(pos)


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _finish(pos, Z, exps_per_atom, box, grid, rcut, sigma, a_sigma, a_seed):
    bf_atom, bf_exp = [], []
    for ia, exps in enumerate(exps_per_atom):
        for e in exps:
            bf_atom.append(ia)
            bf_exp.append(e)
    bf_exp = np.array(bf_exp, dtype=np.float64)
    if rcut is None:
        # no radius given: cut where the Gaussian has fallen to 1e-16
        bf_rcut = np.sqrt(math.log(1e16) / bf_exp)
    else:
        bf_rcut = np.full(len(bf_exp), float(rcut))
    Zarr = np.asarray(Z, dtype=np.float64)
    n_e = int(round(Zarr.sum()))
    assert n_e % 2 == 0, "closed-shell systems only"
    M = len(bf_exp)
    N = n_e // 2
    box = np.asarray(box, dtype=np.float64)
    pos = np.mod(np.asarray(pos, dtype=np.float64), box)
    a0 = np.random.default_rng(a_seed).normal(0.0, a_sigma, size=(N, M - N))
    return dict(
        pos=pos,
        Z=Zarr,
        bf_atom=np.array(bf_atom, dtype=np.int32),
        bf_exp=bf_exp,
        bf_rcut=bf_rcut,
        box=box,
        grid=np.asarray(grid, dtype=np.int32),
        ion_sigma=float(sigma),
        n_electrons=n_e,
        a0=a0,
    )


def random_atoms(n_atoms=8, box_ang=6.4, grid=(32, 32, 32), min_sep_ang=1.0,
                 exps=(0.5, 1.5), Z=1.0, rcut_ang=None, sigma=0.5,
                 a_sigma=0.05, seed=0):
    """Atoms at seeded uniform positions in a cubic box (min-image separation)."""
    box = np.full(3, box_ang * ANGSTROM)
    rng = np.random.default_rng(seed + 1000)
    pos = _uniform_positions(rng, n_atoms, box, min_sep_ang * ANGSTROM)
    rcut = None if rcut_ang is None else rcut_ang * ANGSTROM
    return _finish(pos, [Z] * n_atoms, [list(exps)] * n_atoms, box, grid,
                   rcut, sigma, a_sigma, seed)


def water_box(lattice=(4, 4, 2), box_ang=9.9, grid=(96, 96, 96), rcut_ang=4.0,
              sigma=0.5, a_sigma=0.02, seed=1, jitter_ang=0.2):
    """Triatomic water-like units: heavy site Z=6 (4 Gaussians 0.3..3.0) and
    two light sites Z=1 (exponents 0.5, 1.5) at 0.96 A, 104.5 deg, heavy sites
    on a jittered lattice, each unit randomly oriented."""
    box = np.full(3, box_ang * ANGSTROM)
    rng = np.random.default_rng(seed + 1000)
    nx, ny, nz = lattice
    half = math.radians(104.5) / 2.0
    bond = 0.96 * ANGSTROM
    local = np.array([[0.0, 0.0, 0.0],
                      [bond * math.sin(half), 0.0, bond * math.cos(half)],
                      [-bond * math.sin(half), 0.0, bond * math.cos(half)]])
    pos, Z, exps = [], [], []
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                c = (np.array([i, j, k]) + 0.5) / np.array(lattice) * box
                c = c + rng.uniform(-jitter_ang, jitter_ang, 3) * ANGSTROM
                R = _random_rotation(rng)
                for s in range(3):
                    pos.append(c + R @ local[s])
                    Z.append(6.0 if s == 0 else 1.0)
                    exps.append(HEAVY_EXPS if s == 0 else LIGHT_EXPS)
    return _finish(np.array(pos), Z, exps, box, grid, rcut_ang * ANGSTROM,
                   sigma, a_sigma, seed)


# --- named workloads -------------------------------------------------------

def config_small_molecule():
    """8 atoms, M=16, N=4, 32^3 grid, A_ov ~ N(0, 0.05) (seed 0)."""
    return random_atoms()


def config_water32():
    """32 water-like units (96 atoms), M=256, N=128, 96^3 grid, r_c = 4 A,
    A_ov ~ N(0, 0.02) (seed 1)."""
    return water_box()


def config_water576():
    """576 water-like units (1728 atoms), M=4608, N=2304, 192^3 grid,
    r_c = 3.5 A, 25 A box, A_ov ~ N(0, 0.01) (seed 2)."""
    return water_box(lattice=(9, 8, 8), box_ang=25.0, grid=(192, 192, 192),
                     rcut_ang=3.5, a_sigma=0.01, seed=2)


def config_water216():
    """216 water-like units (648 atoms), M=1728, N=864, 128^3 grid over an
    18.03 A box (the water576 density), r_c = 3.5 A, A_ov ~ N(0, 0.01) (seed
    2): a mid-size box for profiler captures (a few GB on the device)."""
    return water_box(lattice=(6, 6, 6), box_ang=18.03, grid=(128, 128, 128),
                     rcut_ang=3.5, a_sigma=0.01, seed=2)


def config_water75():
    """75 water-like units (225 atoms), M=600, N=300, 64^3 grid over a 13.13 A
    box (the water32 density), r_c = 3.5 A, A_ov ~ N(0, 0.02) (seed 5): the
    largest case the CPU oracle evaluates in seconds that still spans several
    orbital chunks of 128 and large dense products."""
    return water_box(lattice=(5, 5, 3), box_ang=13.13, grid=(64, 64, 64),
                     rcut_ang=3.5, a_sigma=0.02, seed=5)


def tiny(grid=(16, 16, 16), seed=7):
    """2 atoms with 2 functions each in a 4 A box: brute-force sized."""
    return random_atoms(n_atoms=2, box_ang=4.0, grid=grid, a_sigma=0.1,
                        seed=seed)


def ragged_water(grid=(36, 28, 44), seed=11):
    """2 water-like units on a grid whose sizes are not tile multiples."""
    return water_box(lattice=(2, 1, 1), box_ang=6.0, grid=grid, rcut_ang=3.0,
                     a_sigma=0.05, seed=seed)


HA_PER_EV = 1.0 / 27.211386245988  # CODATA 2018


def monkhorst_pack(q):
    """q x q x q Monkhorst-Pack k-points in fractional reciprocal coordinates,
    k_a = (2 r - q - 1) / (2 q) for r = 1 .. q, and their equal weights."""
    ks = [(2.0 * r - q - 1.0) / (2.0 * q) for r in range(1, q + 1)]
    kpts = np.array([[a, b, c] for a in ks for b in ks for c in ks], dtype=np.float64)
    return kpts, np.full(len(kpts), 1.0 / len(kpts))


def crystal(cells=(4, 4, 4), spacing_ang=2.8, jitter_ang=0.05, n_exp=8, Z=4.0,
            grid=(56, 56, 56), rcut_ang=4.0, kmesh=2, kT_ev=0.1, sigma=0.5,
            a_sigma=0.01, seed=4, exps=None):
    """Simple-cubic crystal, one atom per lattice site with a seeded jitter, n_exp
    s-Gaussians per atom (exponents geometric in 0.3 .. 3.0 bohr^-2), a
    Monkhorst-Pack k-mesh and a Fermi-Dirac temperature for the reference
    occupations.  a0 holds the seeded real variables of the full A(k) of every
    k-point (M*M per k-point) for gradient checks; minimizations start at A = 0."""
    cells = np.asarray(cells)
    box = cells * spacing_ang * ANGSTROM
    rng = np.random.default_rng(seed + 1000)
    pos = []
    for i in range(cells[0]):
        for j in range(cells[1]):
            for k in range(cells[2]):
                site = (np.array([i, j, k]) + 0.5) * spacing_ang * ANGSTROM
                pos.append(site + rng.uniform(-jitter_ang, jitter_ang, 3) * ANGSTROM)
    if exps is None:
        exps = [0.3 * 10.0 ** (e / (n_exp - 1)) for e in range(n_exp)]
    n_at = len(pos)
    rcut = None if rcut_ang is None else rcut_ang * ANGSTROM
    d = _finish(np.array(pos), [Z] * n_at, [list(exps)] * n_at, box, grid,
                rcut, sigma, a_sigma, seed)
    kpts, kw = monkhorst_pack(kmesh)
    M = len(d["bf_exp"])
    d.update(kpts=kpts, kw=kw, kT=kT_ev * HA_PER_EV,
             a0=np.random.default_rng(seed).normal(0.0, a_sigma, size=len(kw) * M * M))
    return d


def config_crystal64():
    """64 atoms on a 4x4x4 simple-cubic lattice (2.8 A, 0.05 A jitter, seed 4),
    8 Gaussians per atom (M = 512), Z = 4 (256 electrons), 56^3 grid over the
    11.2 A cell, r_c = 4 A, 2x2x2 Monkhorst-Pack k-points, kT = 0.1 eV;
    gradient-check variables ~ N(0, 0.01)."""
    return crystal()


def tiny_crystal(kT_ev=0.5, kmesh=2, grid=(24, 12, 12), seed=6, rcut_ang=None):
    """Two atoms per cell (a 2x1x1 supercell of a 2.2 A simple-cubic lattice),
    2 Gaussians each (exponents 0.4 and 1.2, M = 4), Z = 1, with a k-mesh and a
    temperature at which the occupations are fractional; the 1e-16 truncation
    rule and an isotropic grid keep the analytic S and T within quadrature
    error of the grid.  Brute-force sized.  rcut_ang (a hard radius, below
    twice the shortest cell edge) makes it a system the GPU path accepts."""
    return crystal(cells=(2, 1, 1), spacing_ang=2.2, jitter_ang=0.1, Z=1.0,
                   exps=(0.4, 1.2), grid=grid, rcut_ang=rcut_ang, kmesh=kmesh,
                   kT_ev=kT_ev, a_sigma=0.05, seed=seed)


def small_crystal(seed=8):
    """Eight atoms (a 2x2x2 simple-cubic cell of 2.6 A, 0.1 A jitter), 3
    Gaussians each (M = 24), Z = 1.5 (12 electrons, the Fermi level inside a
    band: occupations from 1 to 0.02 of full), 2x2x2 k-points, kT = 0.5 eV,
    r_c = 3 A, a ragged 26 x 24 x 22 grid (tiles of 4^3 with partial tiles on
    every axis): the full-A path at a size that spans several tiles."""
    return crystal(cells=(2, 2, 2), spacing_ang=2.6, jitter_ang=0.1, n_exp=3, Z=1.5,
                   grid=(26, 24, 22), rcut_ang=3.0, kmesh=2, kT_ev=0.5, a_sigma=0.05,
                   seed=seed)


def molecule_batch(n_mol=148, atoms=(2, 20), p_heavy=1.0 / 3.0, cube_ang=4.8,
                   box_ang=9.6, grid=(48, 48, 48), rcut_ang=4.0, min_sep_ang=1.0,
                   sigma=0.5, a_sigma=0.05, seed=3):
    """Molecules of uneven size, each in its own cell: n_atoms uniform in
    [atoms[0], atoms[1]], each site heavy (Z = 6, 4 Gaussians 0.3 .. 3.0) with
    probability p_heavy, else light (Z = 1, exponents 0.5 and 1.5); when the
    electron count is odd the last light site becomes heavy.  Positions are
    uniform in a cube of edge cube_ang centred in the box, at least min_sep_ang
    apart.  Molecule i draws its A_ov from seed 1000 * seed + i."""
    rng = np.random.default_rng(seed + 1000)
    box = np.full(3, box_ang * ANGSTROM)
    half = 0.5 * cube_ang * ANGSTROM
    out = []
    for i in range(n_mol):
        n_at = int(rng.integers(atoms[0], atoms[1] + 1))
        heavy = rng.random(n_at) < p_heavy
        light = np.flatnonzero(~heavy)
        if len(light) % 2 == 1:
            heavy[light[-1]] = True
        pos = []
        while len(pos) < n_at:
            p = 0.5 * box + rng.uniform(-half, half, 3)
            if all(np.linalg.norm(p - q) >= min_sep_ang * ANGSTROM for q in pos):
                pos.append(p)
        Z = [6.0 if h else 1.0 for h in heavy]
        exps = [HEAVY_EXPS if h else LIGHT_EXPS for h in heavy]
        out.append(_finish(np.array(pos), Z, exps, box, grid, rcut_ang * ANGSTROM,
                           sigma, a_sigma, 1000 * seed + i))
    return out


def config_molecules148():
    """148 molecules of 2 to 20 atoms (M from 4 to 80), each on a 48^3 grid over
    a 9.6 A box (0.2 A spacing), r_c = 4 A, A_ov ~ N(0, 0.05) (seed 3)."""
    return molecule_batch()


def direction(shape, seed, scale=1.0):
    """A seeded random array (search directions, FD probes, test vectors)."""
    return np.random.default_rng(seed).normal(0.0, scale, size=shape)
