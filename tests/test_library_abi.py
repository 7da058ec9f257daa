"""Host-side checks of the C ABI: the library builds, loads and exports every
entry point that include/etdm.h declares; argument validation runs before any
device work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import etdm_synth as synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2101_12597_gb300 import build
    build.build()
    from paper_2101_12597_gb300.etdm import load_library
    return load_library()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "etdm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(etdm_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    from paper_2101_12597_gb300.etdm import EXPORTS
    assert sorted(EXPORTS) == names


def test_default_options(lib):
    from paper_2101_12597_gb300.etdm import EtdmOptions
    o = EtdmOptions()
    lib.etdm_default_options(ctypes.byref(o))
    assert (o.precision, o.lbfgs_m, o.gamma, o.beta0, o.device, o.dense_blocks,
            o.dense_tc, o.param, o.expm, o.ref_update, o.vgroup,
            o.functional) == (0, 3, 0.25, 1.0, 0, 0, 0, 0, 0, 0, 0, 0)


def _system(lib, d, **over):
    from paper_2101_12597_gb300.etdm import EtdmSystem
    keep = dict(pos=np.ascontiguousarray(d["pos"]), Z=np.ascontiguousarray(d["Z"]),
                bf_atom=np.ascontiguousarray(d["bf_atom"], dtype=np.int32),
                bf_exp=np.ascontiguousarray(d["bf_exp"]),
                bf_rcut=np.ascontiguousarray(d["bf_rcut"]))
    keep.update({k: v for k, v in over.items() if k in keep})
    s = EtdmSystem()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    s.n_atoms = len(keep["Z"]); s.pos = dp(keep["pos"]); s.Z = dp(keep["Z"])
    s.n_basis = len(keep["bf_exp"])
    s.bf_atom = keep["bf_atom"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    s.bf_exp = dp(keep["bf_exp"]); s.bf_rcut = dp(keep["bf_rcut"])
    for a in range(3):
        s.box[a] = float(d["box"][a]); s.grid[a] = int(over.get("grid", d["grid"])[a])
    s.ion_sigma = float(d["ion_sigma"])
    s.n_electrons = int(over.get("n_electrons", d["n_electrons"]))
    return s, keep


@pytest.mark.parametrize("over,frag", [
    (dict(grid=(34, 32, 32)), "prime factors"),
    (dict(n_electrons=7), "even"),
    (dict(n_electrons=40), "n_electrons"),
    (dict(n_electrons=32), "virtual orbital"),
    (dict(bf_rcut=np.full(16, 100.0)), "bf_rcut"),
    (dict(bf_exp=-np.ones(16)), "bf_exp"),
])
def test_invalid_arguments_rejected_before_device_work(lib, over, frag):
    d = synth.config_small_molecule()
    s, keep = _system(lib, d, **over)
    h = ctypes.c_void_p()
    rc = lib.etdm_init_basis(ctypes.byref(s), None, ctypes.byref(h))
    assert rc == -1
    assert frag in lib.etdm_last_error(None).decode()
    assert not h.value


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.etdm_energy_grad(None, None, None, None, None) == -6
    assert lib.etdm_lbfgs_reset(None) == -6
    assert lib.etdm_check(None, None) == -6
    lib.etdm_free(None)


def _kpoint_system(lib, d, nk=None, kfrac=None, kw=None, kT=None):
    s, keep = _system(lib, d)
    kf = np.ascontiguousarray(d["kpts"] if kfrac is None else kfrac, dtype=np.float64)
    w = np.ascontiguousarray(d["kw"] if kw is None else kw, dtype=np.float64)
    keep.update(kf=kf, w=w)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    s.n_k = len(w) if nk is None else nk
    s.k_frac, s.k_w = dp(kf), dp(w)
    s.kT = float(d["kT"] if kT is None else kT)
    return s, keep


@pytest.mark.parametrize("over,frag", [
    (dict(nk=-1), "n_k"),
    (dict(kw=np.full(8, 0.2)), "sum to 1"),
    (dict(kw=np.r_[-0.125, np.full(7, 1.125 / 7)]), "positive"),
    (dict(kfrac=np.full((8, 3), np.nan)), "finite"),
    (dict(kT=-1.0), "kT"),
    (dict(kT=0.0), "integer occupation"),
])
def test_kpoint_arguments_rejected_before_device_work(lib, over, frag):
    """The full-A path's k-point arrays and temperature are checked on the host."""
    d = synth.tiny_crystal(rcut_ang=3.0)
    s, keep = _kpoint_system(lib, d, **over)
    h = ctypes.c_void_p()
    rc = lib.etdm_init_basis(ctypes.byref(s), None, ctypes.byref(h))
    assert rc == -1
    assert frag in lib.etdm_last_error(None).decode()


@pytest.mark.parametrize("param,precision,nk,frag", [
    (1, 1, 8, "FP64 only"),   # full A in mixed precision
    (3, 0, 8, "unknown param"),
    (2, 0, 0, "unknown param"),
])
def test_full_a_options_checked(lib, param, precision, nk, frag):
    from paper_2101_12597_gb300.etdm import EtdmOptions
    d = synth.tiny_crystal(rcut_ang=3.0)
    if nk:
        s, keep = _kpoint_system(lib, d)
    else:
        s, keep = _system(lib, d)
    o = EtdmOptions()
    lib.etdm_default_options(ctypes.byref(o))
    o.param, o.precision = param, precision
    h = ctypes.c_void_p()
    rc = lib.etdm_init_basis(ctypes.byref(s), ctypes.byref(o), ctypes.byref(h))
    assert rc == -1
    assert frag in lib.etdm_last_error(None).decode()


@pytest.mark.parametrize("expm,ref,full,frag", [
    (1, 0, False, "needs the full-A path"),
    (2, 0, True, "unknown expm"),
    (1, -2, True, "ref_update"),
    (0, 5, True, "needs expm"),
])
def test_ss_options_checked(lib, expm, ref, full, frag):
    from paper_2101_12597_gb300.etdm import EtdmOptions
    d = synth.tiny_crystal(rcut_ang=3.0)
    s, keep = _kpoint_system(lib, d) if full else _system(lib, d)
    o = EtdmOptions()
    lib.etdm_default_options(ctypes.byref(o))
    o.expm, o.ref_update = expm, ref
    h = ctypes.c_void_p()
    rc = lib.etdm_init_basis(ctypes.byref(s), ctypes.byref(o), ctypes.byref(h))
    assert rc == -1
    assert frag in lib.etdm_last_error(None).decode()


@pytest.mark.parametrize("kT,kfrac,param,frag", [
    (0.0, None, 0, "full-A path"),
    (0.01, (0.0, 0.0, 0.0), 1, "kT = 0"),
    (0.0, (0.25, 0.0, 0.0), 1, "Gamma point"),
])
def test_pzsic_options_checked(lib, kT, kfrac, param, frag):
    from paper_2101_12597_gb300.etdm import EtdmOptions
    d = synth.config_small_molecule()
    s, keep = _system(lib, d)
    if kfrac is not None:
        kf = np.array(kfrac, dtype=np.float64)
        w = np.ones(1)
        keep.update(kf=kf, w=w)
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        s.n_k, s.k_frac, s.k_w = 1, dp(kf), dp(w)
    s.kT = kT
    o = EtdmOptions()
    lib.etdm_default_options(ctypes.byref(o))
    o.functional, o.param = 1, param
    h = ctypes.c_void_p()
    rc = lib.etdm_init_basis(ctypes.byref(s), ctypes.byref(o), ctypes.byref(h))
    assert rc == -1
    assert frag in lib.etdm_last_error(None).decode()


def test_set_reference_rejects_null_handle(lib):
    rc = lib.etdm_set_reference(None, 0, None, None)
    assert rc == -6


def test_single_system_binding_passes_vgroup(lib):
    """The single-system handle's V-group size reaches the options struct (the
    batch's tuned size can be reproduced on one system)."""
    import inspect
    from paper_2101_12597_gb300.etdm import ETDM, _options
    assert "vgroup" in inspect.signature(ETDM.__init__).parameters
    for vg in (0, 2, 4, 8):
        assert _options(lib, "mixed", 3, 0.25, 1.0, 0, 0, vgroup=vg).vgroup == vg


def test_init_batch_needs_systems(lib):
    """An empty batch is rejected before any system is read or device work done."""
    from paper_2101_12597_gb300.etdm import EtdmOptions
    d = synth.config_small_molecule()
    s, keep = _system(lib, d)
    o = EtdmOptions()
    lib.etdm_default_options(ctypes.byref(o))
    for sys_ptr, n in ((ctypes.byref(s), 0), (None, 3), (ctypes.byref(s), -2)):
        h = ctypes.c_void_p()
        assert lib.etdm_init_batch(sys_ptr, n, ctypes.byref(o), ctypes.byref(h)) == -1
        assert "n_sys" in lib.etdm_last_error(None).decode()
        assert not h.value


@pytest.mark.parametrize("field,value,frag", [
    ("precision", 2, "unknown precision"),
    ("lbfgs_m", 0, "lbfgs_m"),
    ("lbfgs_m", 17, "lbfgs_m"),
    ("gamma", 1.5, "gamma"),
    ("beta0", 0.0, "beta0"),
    ("dense_blocks", -1, "dense_blocks"),
    ("dense_tc", 2, "dense_tc"),
    ("vgroup", 9, "vgroup"),
    ("functional", 2, "unknown functional"),
])
def test_general_options_checked(lib, field, value, frag):
    """Every option outside its documented range is refused at set-up, before
    any device work, with a message naming it."""
    from paper_2101_12597_gb300.etdm import EtdmOptions
    s, keep = _system(lib, synth.config_small_molecule())
    o = EtdmOptions()
    lib.etdm_default_options(ctypes.byref(o))
    setattr(o, field, value)
    h = ctypes.c_void_p()
    assert lib.etdm_init_basis(ctypes.byref(s), ctypes.byref(o), ctypes.byref(h)) == -1
    assert frag in lib.etdm_last_error(None).decode()
    assert not h.value


def test_geometry_checked(lib):
    """Positions outside the cell, a function on a missing atom, a non-positive
    ion width or cell edge are refused at set-up with a message."""
    for mutate, frag in [
        (lambda s, k: k["pos"].__setitem__((0, 0), -0.1), "positions"),
        (lambda s, k: k["bf_atom"].__setitem__(0, 99), "bf_atom"),
        (lambda s, k: setattr(s, "ion_sigma", 0.0), "ion_sigma"),
        (lambda s, k: s.box.__setitem__(1, -1.0), "box"),
        (lambda s, k: setattr(s, "n_atoms", 0), "n_atoms"),
    ]:
        s, keep = _system(lib, synth.config_small_molecule())  # fresh arrays each time
        mutate(s, keep)
        h = ctypes.c_void_p()
        assert lib.etdm_init_basis(ctypes.byref(s), None, ctypes.byref(h)) == -1
        assert frag in lib.etdm_last_error(None).decode(), frag
        assert not h.value
