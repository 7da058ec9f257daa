"""The seeded synthetic workloads match the recipes they state (sizes, geometry,
distributions) and are reproducible: the parity tests and the benchmark rely
on both sides receiving the same, well-formed inputs."""
import numpy as np
import pytest

import etdm_synth as synth

A = synth.ANGSTROM


def _min_image(d, box):
    d = d - box * np.round(d / box)
    return np.sqrt((d * d).sum(-1))


@pytest.mark.parametrize("make,units,M,N,grid,box_ang,rc_ang,a_sigma", [
    (synth.config_water32, 32, 256, 128, 96, 9.9, 4.0, 0.02),
    (synth.config_water576, 576, 4608, 2304, 192, 25.0, 3.5, 0.01),
    (synth.config_water216, 216, 1728, 864, 128, 18.03, 3.5, 0.01),
    (synth.config_water75, 75, 600, 300, 64, 13.13, 3.5, 0.02),
])
def test_water_boxes(make, units, M, N, grid, box_ang, rc_ang, a_sigma):
    d = make()
    assert d["pos"].shape == (3 * units, 3)
    assert len(d["bf_exp"]) == M and d["n_electrons"] == 2 * N
    assert d["a0"].shape == (N, M - N)
    assert tuple(d["grid"]) == (grid,) * 3
    assert np.allclose(d["box"], box_ang * A)
    assert np.allclose(d["bf_rcut"], rc_ang * A)
    assert np.all((d["pos"] >= 0) & (d["pos"] < d["box"]))
    assert abs(d["a0"].std() - a_sigma) < 0.05 * a_sigma and abs(d["a0"].mean()) < 0.05 * a_sigma
    Z = d["Z"].reshape(units, 3)
    assert np.all(Z[:, 0] == 6.0) and np.all(Z[:, 1:] == 1.0)
    # heavy site with 4 exponents 0.3 .. 3.0, light sites with 0.5 and 1.5
    per_atom = np.bincount(d["bf_atom"], minlength=3 * units).reshape(units, 3)
    assert np.all(per_atom == [4, 2, 2])
    assert np.allclose(d["bf_exp"][:8], synth.HEAVY_EXPS + synth.LIGHT_EXPS * 2)
    # bonds of 0.96 A at 104.5 degrees (minimum image: units may wrap)
    p = d["pos"].reshape(units, 3, 3)
    box = d["box"]
    for s in (1, 2):
        assert np.allclose(_min_image(p[:, s] - p[:, 0], box), 0.96 * A, atol=1e-12)
    u = p[:, 1] - p[:, 0]; u -= box * np.round(u / box)
    v = p[:, 2] - p[:, 0]; v -= box * np.round(v / box)
    cosang = (u * v).sum(1) / (np.linalg.norm(u, axis=1) * np.linalg.norm(v, axis=1))
    assert np.allclose(np.degrees(np.arccos(cosang)), 104.5, atol=1e-9)


def test_small_molecule_recipe():
    d = synth.config_small_molecule()
    assert d["pos"].shape == (8, 3) and len(d["bf_exp"]) == 16 and d["n_electrons"] == 8
    assert tuple(d["grid"]) == (32, 32, 32) and np.allclose(d["box"], 6.4 * A)
    n = len(d["pos"])
    dist = [_min_image(d["pos"][i] - d["pos"][j], d["box"]) for i in range(n) for j in range(i)]
    assert min(dist) >= 1.0 * A
    # no radius given: the cut sits where the Gaussian has fallen to 1e-16
    assert np.allclose(np.exp(-d["bf_exp"] * d["bf_rcut"] ** 2), 1e-16)


def test_edge_case_grids_are_ragged():
    # against 4 x 4 x 8 point tiles: the ragged water grid is ragged along z
    # only, the all-odd grid along every axis (and has an unpaired z line)
    tile = np.array([4, 4, 8])
    g = synth.ragged_water()["grid"]
    assert tuple(g) == (36, 28, 44) and list(g % tile != 0) == [False, False, True]
    g = synth.ragged_water(grid=(27, 25, 45))["grid"]
    assert np.all(g % tile != 0) and np.all(g % 2 == 1)
    assert tuple(synth.tiny()["grid"]) == (16, 16, 16)


@pytest.mark.parametrize("make", [synth.config_small_molecule, synth.config_water32,
                                  synth.tiny, synth.ragged_water])
def test_reproducible(make):
    a, b = make(), make()
    for k in a:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


def test_distinct_seeds_differ():
    assert not np.array_equal(synth.water_box(seed=1)["pos"], synth.water_box(seed=2)["pos"])
    x = synth.direction((3, 4), seed=5, scale=0.1)
    assert x.shape == (3, 4) and np.array_equal(x, synth.direction((3, 4), seed=5, scale=0.1))
    y = synth.direction((400, 50), seed=1, scale=2.0)
    assert abs(y.std() - 2.0) < 0.05 and abs(y.mean()) < 0.05


def test_crystal64_recipe():
    d = synth.config_crystal64()
    assert d["pos"].shape == (64, 3) and len(d["bf_exp"]) == 512 and d["n_electrons"] == 256
    assert tuple(d["grid"]) == (56, 56, 56) and np.allclose(d["box"], 11.2 * A)
    assert np.allclose(d["bf_rcut"], 4.0 * A) and np.all(d["Z"] == 4.0)
    exps = d["bf_exp"][:8]
    assert np.allclose(exps[[0, -1]], [0.3, 3.0]) and np.allclose(exps[1:] / exps[:-1], 10 ** (1 / 7))
    # simple-cubic sites at (n + 1/2) 2.8 A with a jitter of at most 0.05 A per axis
    site = (np.floor(d["pos"] / (2.8 * A)) + 0.5) * 2.8 * A
    assert np.abs(d["pos"] - site).max() <= 0.05 * A + 1e-12
    kp, kw = d["kpts"], d["kw"]
    assert kp.shape == (8, 3) and np.all(np.abs(kp) == 0.25) and np.allclose(kw, 1 / 8)
    assert len({tuple(k) for k in kp}) == 8
    assert abs(d["kT"] - 0.1 / 27.211386245988) < 1e-18
    assert d["a0"].shape == (8 * 512 * 512,) and abs(d["a0"].std() - 0.01) < 1e-4


def test_monkhorst_pack():
    for q in (1, 2, 3, 4):
        kp, kw = synth.monkhorst_pack(q)
        assert kp.shape == (q ** 3, 3) and abs(kw.sum() - 1) < 1e-15
        # symmetric under k -> -k, inside the first zone, Gamma only for odd q
        s = {tuple(np.round(k, 12)) for k in kp}
        assert s == {tuple(np.round(-k, 12)) for k in kp}
        assert np.all(np.abs(kp) < 0.5)
        assert ((0.0, 0.0, 0.0) in s) == (q % 2 == 1)


def test_molecules148_recipe():
    ms = synth.config_molecules148()
    assert len(ms) == 148
    box = 9.6 * A
    for m in ms:
        n = len(m["Z"])
        assert 2 <= n <= 20 and m["n_electrons"] % 2 == 0
        assert tuple(m["grid"]) == (48, 48, 48) and np.allclose(m["box"], box)
        assert np.allclose(m["bf_rcut"], 4.0 * A)
        heavy = m["Z"] == 6.0
        assert np.all(heavy | (m["Z"] == 1.0))
        assert len(m["bf_exp"]) == 4 * heavy.sum() + 2 * (~heavy).sum()
        assert m["a0"].shape == (m["n_electrons"] // 2, len(m["bf_exp"]) - m["n_electrons"] // 2)
        # inside the centred 4.8 A cube, at least 1 A apart
        assert np.all(np.abs(m["pos"] - 0.5 * box) <= 2.4 * A)
        dd = np.linalg.norm(m["pos"][:, None] - m["pos"][None, :], axis=-1)
        assert dd[np.triu_indices(n, 1)].min() >= 1.0 * A
    M = [len(m["bf_exp"]) for m in ms]
    assert min(M) == 4 and max(M) <= 80
    na = [len(m["Z"]) for m in ms]
    assert set(na) == set(range(2, 21))  # every size occurs


def test_batch_molecule_through_the_oracle():
    from oracle.etdm_oracle import Oracle
    m = min(synth.config_molecules148(), key=lambda x: len(x["bf_exp"]))
    o = Oracle(m)
    D = o.density_matrix(o.orbitals(m["a0"]))
    assert abs(float(np.sum(D * o.reference()["S"])) - m["n_electrons"]) < 1e-12
    assert abs(o.dV * o.density(D).sum() - m["n_electrons"]) < 1e-8 * m["n_electrons"]


def test_gpu_sized_crystals():
    """The two crystals of the GPU k-point tests: the two-atom cell with a
    hard radius below twice its shortest edge, and the 8-atom cell with a
    ragged grid and the Fermi level inside a band."""
    t = synth.tiny_crystal(rcut_ang=3.0)
    assert len(t["bf_exp"]) == 4 and np.allclose(t["bf_rcut"], 3.0 * A)
    assert np.all(t["bf_rcut"] < 2.0 * t["box"].min())
    s = synth.small_crystal()
    assert len(s["bf_exp"]) == 24 and s["n_electrons"] == 12
    assert tuple(s["grid"]) == (26, 24, 22)
    assert np.all(s["bf_rcut"] < 2.0 * s["box"].min())
    assert len(s["kw"]) == 8 and abs(s["kw"].sum() - 1.0) < 1e-15
    assert s["a0"].shape == (8 * 24 * 24,)
