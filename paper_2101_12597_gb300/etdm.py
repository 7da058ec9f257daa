"""Thin ctypes binding of libetdm (include/etdm.h).

Argument marshalling only: every step of the ETDM evaluation runs in the CUDA
library.  Tensors are torch CUDA tensors (FP64, contiguous); torch supplies
device memory and streams.  There is no CPU fallback: if libetdm.so is missing
or no GPU is present, construction fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libetdm.so")

ETDM_OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "NOT_CONVERGED",
          -5: "TIMEOUT", -6: "STATE", -7: "NUMERIC"}
PRECISION = {"fp64": 0, "mixed": 1}
PARAM = {"occvirt": 0, "full": 1}
EXPM = {"eig": 0, "ss": 1}
FUNCTIONAL = {"ks": 0, "pzsic": 1}
ARRAYS = {"S": (0, np.float64), "T": (1, np.float64), "C0": (2, np.float64),
          "order": (3, np.int32), "vext": (4, np.float64), "rho": (5, np.float64),
          "vtot": (6, np.float64), "H": (7, np.float64), "D": (8, np.float64),
          "Uocc": (9, np.float64), "tile_ptr": (10, np.int32),
          "tile_keys": (11, np.int32), "eps": (12, np.float64),
          "eterms": (13, np.float64), "beta": (14, np.float64),
          "tile_ptr_tc": (15, np.int32), "tile_keys_tc": (16, np.int32),
          "tile_nu_tc": (17, np.int32), "vgroup_t0": (18, np.int32),
          "vgroup_nu": (19, np.int32), "doublings": (20, np.int32),
          "status": (21, np.int32),
          # full-A path: complex [n_k][M][M] matrices and [n_k][M] vectors
          "S_k": (0, np.complex128), "T_k": (1, np.complex128), "C0_k": (2, np.complex128),
          "H_k": (7, np.complex128), "D_k": (8, np.complex128), "occ": (22, np.float64),
          "eps_ref": (23, np.float64), "omega": (24, np.float64),
          # tiles per V group in use, then (tiles, ms per evaluation) pairs timed at set-up
          "tune": (25, np.float64)}
DIM_NAMES = ["M", "N", "V", "G", "n_tiles", "entries", "max_list", "tx", "ty",
             "tz", "sum_npt2", "precision"]

EXPORTS = ["etdm_default_options", "etdm_init_basis", "etdm_energy_grad",
           "etdm_energy_grad_host", "etdm_precondition", "etdm_lbfgs_step",
           "etdm_lbfgs_reset", "etdm_minimize", "etdm_check", "etdm_layout",
           "etdm_array_bytes", "etdm_get_array", "etdm_set_profiling",
           "etdm_stage_times", "etdm_last_error", "etdm_free",
           "etdm_lbfgs_direction_noalloc", "etdm_lbfgs_direction_noalloc_status",
           "etdm_init_batch", "etdm_num_systems", "etdm_system_layout", "etdm_system_handle",
           "etdm_set_active", "etdm_minimize_converge", "etdm_pair_gemm",
           "etdm_set_reference"]
STAGES = ["dense_fwd", "rho", "potential", "vmat", "dense_rev", "lbfgs", "eig"]


class EtdmSystem(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32),
                ("pos", ctypes.POINTER(ctypes.c_double)),
                ("Z", ctypes.POINTER(ctypes.c_double)),
                ("n_basis", ctypes.c_int32),
                ("bf_atom", ctypes.POINTER(ctypes.c_int32)),
                ("bf_exp", ctypes.POINTER(ctypes.c_double)),
                ("bf_rcut", ctypes.POINTER(ctypes.c_double)),
                ("box", ctypes.c_double * 3),
                ("grid", ctypes.c_int32 * 3),
                ("ion_sigma", ctypes.c_double),
                ("n_electrons", ctypes.c_int32),
                ("n_k", ctypes.c_int32),
                ("k_frac", ctypes.POINTER(ctypes.c_double)),
                ("k_w", ctypes.POINTER(ctypes.c_double)),
                ("kT", ctypes.c_double)]


class EtdmOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32),
                ("lbfgs_m", ctypes.c_int32),
                ("gamma", ctypes.c_double),
                ("beta0", ctypes.c_double),
                ("device", ctypes.c_int32),
                ("dense_blocks", ctypes.c_int32),
                ("dense_tc", ctypes.c_int32),
                ("param", ctypes.c_int32),
                ("expm", ctypes.c_int32),
                ("ref_update", ctypes.c_int32),
                ("vgroup", ctypes.c_int32),
                ("functional", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libetdm.so and declare the C ABI.  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2101_12597_gb300.build`")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.etdm_default_options.argtypes = [ctypes.POINTER(EtdmOptions)]
    lib.etdm_default_options.restype = None
    lib.etdm_init_basis.argtypes = [ctypes.POINTER(EtdmSystem), ctypes.POINTER(EtdmOptions),
                                    ctypes.POINTER(P)]
    lib.etdm_energy_grad.argtypes = [P, P, P, P, P]
    lib.etdm_energy_grad_host.argtypes = [P, dp, dp, dp]
    lib.etdm_precondition.argtypes = [P, P, P, P]
    lib.etdm_lbfgs_step.argtypes = [P, P, P, P, P]
    lib.etdm_lbfgs_reset.argtypes = [P]
    lib.etdm_minimize.argtypes = [P, P, ctypes.c_int32, dp, dp,
                                  ctypes.POINTER(ctypes.c_int32), P]
    lib.etdm_minimize_converge.argtypes = [P, P, ctypes.c_int32, ctypes.c_double, dp, dp,
                                           ctypes.POINTER(ctypes.c_int32), dp,
                                           ctypes.POINTER(ctypes.c_int32), P]
    lib.etdm_pair_gemm.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_int32, P]
    lib.etdm_check.argtypes = [P, P]
    lib.etdm_layout.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.etdm_array_bytes.argtypes = [P, ctypes.c_int32]
    lib.etdm_array_bytes.restype = ctypes.c_int64
    lib.etdm_get_array.argtypes = [P, ctypes.c_int32, P, ctypes.c_int64]
    lib.etdm_set_profiling.argtypes = [P, ctypes.c_int]
    lib.etdm_stage_times.argtypes = [P, dp, ctypes.POINTER(ctypes.c_int64)]
    lib.etdm_lbfgs_direction_noalloc.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_int64,
                                                 P, P, P]
    lib.etdm_lbfgs_direction_noalloc_status.argtypes = [P]
    lib.etdm_init_batch.argtypes = [ctypes.POINTER(EtdmSystem), ctypes.c_int32,
                                    ctypes.POINTER(EtdmOptions), ctypes.POINTER(P)]
    lib.etdm_num_systems.argtypes = [P]
    lib.etdm_num_systems.restype = ctypes.c_int32
    lib.etdm_system_layout.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64)]
    lib.etdm_system_handle.argtypes = [P, ctypes.c_int32]
    lib.etdm_system_handle.restype = P
    lib.etdm_set_active.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.etdm_set_reference.argtypes = [P, ctypes.c_int32, dp, dp]
    lib.etdm_last_error.argtypes = [P]
    lib.etdm_last_error.restype = ctypes.c_char_p
    lib.etdm_free.argtypes = [P]
    lib.etdm_free.restype = None
    for name in EXPORTS:
        if name not in ("etdm_default_options", "etdm_last_error", "etdm_free",
                        "etdm_array_bytes", "etdm_num_systems", "etdm_system_handle"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class EtdmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ETDM_ERR_{STATUS.get(code, code)}: {msg}")
        self.code = code


def _require(t, dev, name, shape=None, numel=None):
    """ValueError unless t is a contiguous float64 tensor on the device dev, of
    the given shape (or element count): the library receives raw pointers and
    sizes, so nothing past this point can check them."""
    import torch
    ok = (isinstance(t, torch.Tensor) and t.dtype == torch.float64 and t.is_contiguous()
          and t.device == dev and (shape is None or tuple(t.shape) == tuple(shape))
          and (numel is None or t.numel() == numel))
    if not ok:
        want = f"shape {tuple(shape)}" if shape is not None else f"{numel} elements"
        got = (f"{tuple(t.shape)} {t.dtype} on {t.device}, contiguous={t.is_contiguous()}"
               if isinstance(t, torch.Tensor) else type(t).__name__)
        raise ValueError(f"{name}: expected a contiguous float64 tensor of {want} on {dev}; "
                         f"got {got}")


def _noalloc_shapes(g, S, Y, h0, out):
    """(m, n) of an allocation-free direction call after checking that every
    tensor sits on g's device with consistent sizes: S and Y of shape (m, n)
    (both None for m = 0), g, h0 and out of n elements."""
    n = g.numel()
    dev = g.device
    _require(g, dev, "g", numel=n)
    _require(h0, dev, "h0", numel=n)
    _require(out, dev, "out", numel=n)
    if (S is None) != (Y is None):
        raise ValueError("S and Y: give both or neither")
    if S is None:
        return 0, n
    m = S.shape[0] if S.dim() == 2 else -1
    _require(S, dev, "S", shape=(m, n))
    _require(Y, dev, "Y", shape=(m, n))
    return m, n


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream_ptr(stream, dev):
    """The cudaStream_t of `stream` for a call on the device dev (default: dev's
    current stream).  A stream of another device is refused: the library runs
    the call on dev and would queue it on a stream it cannot use there."""
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    if stream.device != dev:
        raise ValueError(f"stream is on {stream.device}, not {dev}")
    return ctypes.c_void_p(stream.cuda_stream)


def _system_struct(sysd, s=None):
    """An EtdmSystem for the system dict sysd (etdm_synth's layout) and the
    arrays it points into (keep them alive while the struct is used)."""
    keep = dict(
        pos=np.ascontiguousarray(sysd["pos"], dtype=np.float64),
        Z=np.ascontiguousarray(sysd["Z"], dtype=np.float64),
        bf_atom=np.ascontiguousarray(sysd["bf_atom"], dtype=np.int32),
        bf_exp=np.ascontiguousarray(sysd["bf_exp"], dtype=np.float64),
        bf_rcut=np.ascontiguousarray(sysd["bf_rcut"], dtype=np.float64))
    s = EtdmSystem() if s is None else s
    s.n_atoms = len(keep["Z"])
    s.pos = _dptr(keep["pos"])
    s.Z = _dptr(keep["Z"])
    s.n_basis = len(keep["bf_exp"])
    s.bf_atom = keep["bf_atom"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    s.bf_exp = _dptr(keep["bf_exp"])
    s.bf_rcut = _dptr(keep["bf_rcut"])
    for a in range(3):
        s.box[a] = float(sysd["box"][a])
        s.grid[a] = int(sysd["grid"][a])
    s.ion_sigma = float(sysd["ion_sigma"])
    s.n_electrons = int(sysd["n_electrons"])
    if sysd.get("kpts") is not None:  # k-points: the full-A path
        keep["k_frac"] = np.ascontiguousarray(np.atleast_2d(sysd["kpts"]), dtype=np.float64)
        keep["k_w"] = np.ascontiguousarray(sysd["kw"], dtype=np.float64)
        s.n_k = len(keep["k_w"])
        s.k_frac = _dptr(keep["k_frac"])
        s.k_w = _dptr(keep["k_w"])
        s.kT = float(sysd["kT"])
    else:
        s.n_k = 0
        s.kT = float(sysd.get("kT", 0.0))
    return s, keep


def _options(lib, precision, lbfgs_m, gamma, beta0, device, dense_blocks, dense_tc=0,
             param="occvirt", expm="eig", ref_update=0, vgroup=0, functional="ks"):
    o = EtdmOptions()
    lib.etdm_default_options(ctypes.byref(o))
    o.precision = PRECISION[precision]
    o.lbfgs_m = lbfgs_m
    o.gamma = gamma
    o.beta0 = beta0
    o.device = device
    o.dense_blocks = dense_blocks
    o.dense_tc = dense_tc
    o.param = PARAM[param]
    o.expm = EXPM[expm]
    o.ref_update = ref_update
    o.vgroup = vgroup
    o.functional = FUNCTIONAL[functional]
    return o


class ETDM:
    """One system on one GPU: the handle of etdm_init_basis.  A system dict
    with "kpts" (with "kw" and "kT"), or param="full", selects the full-A path:
    the variables are then a flat vector of n_k M^2 reals (Re a_ij for i < j,
    then Im a_ij for i <= j, per k-point).  On that path expm="ss" evaluates
    exp(A) by scaling and squaring with the approximate gradient G ~ L^T, and
    ref_update (n > 0: every n steps, -1: the |L| < 3 |[A, L]| test) makes
    minimize() move the reference, C0 <- C0 exp(A), A <- 0; functional="pzsic"
    adds the Perdew-Zunger self-interaction correction (Gamma point, kT = 0).
    vgroup (mixed path) sets the tiles per V group of the grid -> basis pass
    (0: the default of 2)."""

    def __init__(self, sysd, precision="fp64", lbfgs_m=3, gamma=0.25, beta0=1.0,
                 device=0, dense_blocks=0, dense_tc=0, param=None, expm="eig", ref_update=0,
                 functional="ks", vgroup=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("ETDM needs a CUDA GPU; there is no CPU fallback")
        self.lib = load_library()
        self.device = device
        s, self._keep = _system_struct(sysd)
        if param is None:
            param = "full" if sysd.get("kpts") is not None else "occvirt"
        self.full = param == "full"
        o = _options(self.lib, precision, lbfgs_m, gamma, beta0, device, dense_blocks, dense_tc,
                     param, expm, ref_update, vgroup=vgroup, functional=functional)
        torch.cuda.init()
        h = ctypes.c_void_p()
        rc = self.lib.etdm_init_basis(ctypes.byref(s), ctypes.byref(o), ctypes.byref(h))
        if rc != ETDM_OK:
            raise EtdmError(rc, self.lib.etdm_last_error(None).decode())
        self.h = h
        self._borrowed = False
        self._read_dims()
        self.dev = torch.device("cuda", device)

    @classmethod
    def _view(cls, lib, h, dev):
        """A system of a batch: inspection through its borrowed handle."""
        v = object.__new__(cls)
        v.lib, v.h, v.dev, v.device, v._borrowed = lib, h, dev, dev.index, True
        v._read_dims()
        return v

    def _read_dims(self):
        dims = (ctypes.c_int64 * 12)()
        self.lib.etdm_layout(self.h, dims)
        self.dims = dict(zip(DIM_NAMES, [int(x) for x in dims]))
        self.M, self.N, self.V = self.dims["M"], self.dims["N"], self.dims["V"]
        off, ln = ctypes.c_int64(), ctypes.c_int64()
        self.lib.etdm_system_layout(self.h, 0, ctypes.byref(off), ctypes.byref(ln))
        self.nvar = int(ln.value)

    @property
    def var_shape(self):
        """Shape of a and g: N x V (occupied-virtual) or a flat n_k M^2 vector (full A)."""
        return (self.nvar,) if getattr(self, "full", False) else (self.N, self.V)

    # -- helpers ----------------------------------------------------------------
    def _raise(self, rc):
        if rc != ETDM_OK:
            raise EtdmError(rc, self.lib.etdm_last_error(self.h).decode())

    def _check_tensor(self, t, shape, name="a"):
        _require(t, self.dev, name, shape=shape)

    # -- entry points -------------------------------------------------------------
    def energy_grad(self, a, want_grad=True, E=None, g=None, stream=None):
        """E and dE/dA_ov for a (N x V) on the device; returns (E[1], g or None)."""
        import torch
        self._check_tensor(a, self.var_shape)
        if E is None:
            E = torch.empty(1, dtype=torch.float64, device=self.dev)
        _require(E, self.dev, "E", numel=1)
        if want_grad and g is None:
            g = torch.empty(self.var_shape, dtype=torch.float64, device=self.dev)
        if want_grad:
            self._check_tensor(g, self.var_shape, "g")
        rc = self.lib.etdm_energy_grad(self.h, ctypes.c_void_p(a.data_ptr()),
                                       ctypes.c_void_p(E.data_ptr()),
                                       ctypes.c_void_p(g.data_ptr()) if want_grad else None,
                                       _stream_ptr(stream, self.dev))
        self._raise(rc)
        return E, (g if want_grad else None)

    def energy_grad_host(self, a, want_grad=True):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != self.var_shape:
            raise ValueError(f"a: expected shape {self.var_shape}, got {a.shape}")
        E = np.zeros(1)
        g = np.zeros(self.var_shape) if want_grad else None
        rc = self.lib.etdm_energy_grad_host(self.h, _dptr(a), _dptr(E),
                                            _dptr(g) if want_grad else None)
        self._raise(rc)
        return float(E[0]), g

    def precondition(self, g, out=None, stream=None):
        """P^(k) o g (Eq. 33) with the current beta^(k) (Eq. 34): g (N x V) on the
        device; returns `out` (created when None)."""
        import torch
        self._check_tensor(g, self.var_shape, "g")
        out = torch.empty_like(g) if out is None else out
        self._check_tensor(out, self.var_shape, "out")
        self._raise(self.lib.etdm_precondition(self.h, ctypes.c_void_p(g.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()),
                                               _stream_ptr(stream, self.dev)))
        return out

    def lbfgs_step(self, a, g, out=None, stream=None):
        """L-BFGS direction p = -H g at the point a (Sec. 3.1): stores the pair
        (a - a_prev, g - g_prev) when its curvature is positive, updates beta
        (Eq. 34) and runs the two-loop recursion with H0 = P^(k).  Returns `out`."""
        import torch
        self._check_tensor(a, self.var_shape)
        self._check_tensor(g, self.var_shape, "g")
        out = torch.empty_like(g) if out is None else out
        self._check_tensor(out, self.var_shape, "out")
        self._raise(self.lib.etdm_lbfgs_step(self.h, ctypes.c_void_p(a.data_ptr()),
                                             ctypes.c_void_p(g.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()),
                                             _stream_ptr(stream, self.dev)))
        return out

    def lbfgs_reset(self):
        """Erase the L-BFGS memory (no pairs, no previous point, beta = beta0)."""
        self._raise(self.lib.etdm_lbfgs_reset(self.h))

    def set_reference(self, C0, occ=None):
        """Replace the reference orbitals (Eq. 6-7) and, on the full-A path,
        optionally the occupations; re-derives the Eq. 33 orbital energies and
        erases the L-BFGS memory.  C0: (M, M) real (occupied-virtual) or
        (n_k, M, M) complex (full A), columns are orbitals; occ: (n_k, M)."""
        if self.full:
            C0 = np.ascontiguousarray(C0, dtype=np.complex128)
            want = (self.nvar // (self.M * self.M), self.M, self.M)
        else:
            C0 = np.ascontiguousarray(C0, dtype=np.float64)
            want = (self.M, self.M)
        if C0.shape != want:
            raise ValueError(f"C0: expected shape {want}, got {C0.shape}")
        ov = None
        if occ is not None:
            ov = np.ascontiguousarray(occ, dtype=np.float64)
            if not self.full or ov.shape != want[:2]:
                raise ValueError("occ: only on the full-A path, shape (n_k, M)")
        self._raise(self.lib.etdm_set_reference(
            self.h, 0, C0.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            _dptr(ov) if ov is not None else None))

    def minimize(self, a, n_steps, stream=None):
        """Runs n_steps ETDM iterations in place on a; returns (E, alpha, trials)."""
        self._check_tensor(a, self.var_shape)
        E = np.zeros(n_steps + 1)
        al = np.zeros(n_steps + 1)
        tr = np.zeros(n_steps + 1, dtype=np.int32)
        self._raise(self.lib.etdm_minimize(self.h, ctypes.c_void_p(a.data_ptr()), n_steps,
                                           _dptr(E), _dptr(al),
                                           tr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                           _stream_ptr(stream, self.dev)))
        return E, al, tr

    def minimize_converge(self, a, max_steps=333, tol=1e-10 / 27.211386245988 ** 2,
                          stream=None):
        """ETDM iterations in place on a until the Eq. 45 residual is at most tol
        (Hartree^2; default the paper's 1e-10 eV^2) or max_steps; returns
        (steps, E, alpha, trials, residual), the histories cut to steps + 1."""
        self._check_tensor(a, self.var_shape)
        K = max_steps + 1
        E, al, res = np.zeros(K), np.zeros(K), np.zeros(K)
        tr = np.zeros(K, dtype=np.int32)
        done = ctypes.c_int32(0)
        self._raise(self.lib.etdm_minimize_converge(
            self.h, ctypes.c_void_p(a.data_ptr()), max_steps, tol, _dptr(E), _dptr(al),
            tr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(res), ctypes.byref(done),
            _stream_ptr(stream, self.dev)))
        k = int(done.value)
        return k, E[:k + 1], al[:k + 1], tr[:k + 1], res[:k + 1]

    def check(self, stream=None):
        """Wait for `stream` and raise EtdmError on a deferred device-side error."""
        self._raise(self.lib.etdm_check(self.h, _stream_ptr(stream, self.dev)))

    def get_array(self, name):
        """A copy of an internal array (names in ARRAYS: S, T, C0, rho, H, ...)."""
        which, dt = ARRAYS[name]
        nb = self.lib.etdm_array_bytes(self.h, which)
        if nb < 0:
            raise ValueError(f"array {name!r} does not exist on this handle's path "
                             "(full A, occupied-virtual or a batch)")
        out = np.zeros(nb // np.dtype(dt).itemsize, dtype=dt)
        self._raise(self.lib.etdm_get_array(self.h, which, out.ctypes.data_as(ctypes.c_void_p),
                                            nb))
        return out

    def set_profiling(self, on=True):
        """Record CUDA events around each stage (read with stage_times)."""
        self._raise(self.lib.etdm_set_profiling(self.h, 1 if on else 0))

    def stage_times(self):
        """(ms per stage, launches per stage, total kernel launches) since the last call."""
        ms = np.zeros(8)
        cnt = np.zeros(8, dtype=np.int64)
        self._raise(self.lib.etdm_stage_times(self.h, _dptr(ms),
                                              cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return (dict(zip(STAGES, ms[:len(STAGES)].tolist())),
                dict(zip(STAGES, cnt[:len(STAGES)].tolist())), int(cnt[-1]))

    def close(self):
        """Release the handle's device memory (the object is unusable afterwards);
        a system of a batch is released with its batch."""
        if getattr(self, "h", None):
            if not getattr(self, "_borrowed", False):
                self.lib.etdm_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ETDMBatch:
    """Many systems in one handle (etdm_init_batch): packed variable vectors,
    one energy per system, one graph per evaluation on the mixed path.
    vgroup = 0 lets the set-up time V groups of 2, 4 and 8 tiles and keep the
    fastest (tune() reports it); 1..8 fixes the group size."""

    def __init__(self, systems, precision="mixed", lbfgs_m=3, gamma=0.25, beta0=1.0,
                 device=0, dense_blocks=0, vgroup=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("ETDMBatch needs a CUDA GPU; there is no CPU fallback")
        self.lib = load_library()
        n = len(systems)
        if n < 1:
            raise ValueError("need at least one system")
        arr = (EtdmSystem * n)()
        self._keep = [_system_struct(d, arr[i])[1] for i, d in enumerate(systems)]
        o = _options(self.lib, precision, lbfgs_m, gamma, beta0, device, dense_blocks,
                     vgroup=vgroup)
        torch.cuda.init()
        h = ctypes.c_void_p()
        rc = self.lib.etdm_init_batch(arr, n, ctypes.byref(o), ctypes.byref(h))
        if rc != ETDM_OK:
            raise EtdmError(rc, self.lib.etdm_last_error(None).decode())
        self.h = h
        self.n = n
        self.dev = torch.device("cuda", device)
        off, ln = ctypes.c_int64(), ctypes.c_int64()
        self.offsets = []
        for i in range(n):
            self._raise(self.lib.etdm_system_layout(self.h, i, ctypes.byref(off), ctypes.byref(ln)))
            self.offsets.append((int(off.value), int(ln.value)))
        self.nvar = self.offsets[-1][0] + self.offsets[-1][1]
        self.systems = [ETDM._view(self.lib, self.lib.etdm_system_handle(self.h, i), self.dev)
                        for i in range(n)]
        self.shapes = [(m.N, m.V) for m in self.systems]

    def _raise(self, rc):
        if rc != ETDM_OK:
            raise EtdmError(rc, self.lib.etdm_last_error(self.h).decode())

    def tune(self):
        """(tiles per V group in use, {tiles: ms per batched evaluation} timed at set-up)."""
        t = np.zeros(8)
        self._raise(self.lib.etdm_get_array(self.h, ARRAYS["tune"][0],
                                            t.ctypes.data_as(ctypes.c_void_p), 64))
        return int(t[0]), {int(t[1 + 2 * i]): float(t[2 + 2 * i]) for i in range(3) if t[1 + 2 * i]}

    def pack(self, arrays):
        """One packed float64 vector from the per-system (N_i, V_i) arrays."""
        return np.concatenate([np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
                               for x in arrays])

    def split(self, x):
        """Per-system (N_i, V_i) views of a packed vector (numpy or torch)."""
        return [x[o:o + ln].reshape(shp) for (o, ln), shp in zip(self.offsets, self.shapes)]

    def energy_grad(self, a, E=None, g=None, stream=None):
        """E [n] and the packed gradient for the packed point a (on the device)."""
        import torch
        _require(a, self.dev, "a", numel=self.nvar)
        E = torch.empty(self.n, dtype=torch.float64, device=self.dev) if E is None else E
        g = torch.empty_like(a) if g is None else g
        _require(E, self.dev, "E", numel=self.n)
        _require(g, self.dev, "g", numel=self.nvar)
        self._raise(self.lib.etdm_energy_grad(self.h, ctypes.c_void_p(a.data_ptr()),
                                              ctypes.c_void_p(E.data_ptr()),
                                              ctypes.c_void_p(g.data_ptr()), _stream_ptr(stream, self.dev)))
        return E, g

    def energy_grad_host(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        if a.size != self.nvar:
            raise ValueError(f"a: expected {self.nvar} packed variables, got {a.size}")
        E = np.zeros(self.n)
        g = np.zeros(self.nvar)
        self._raise(self.lib.etdm_energy_grad_host(self.h, _dptr(a), _dptr(E), _dptr(g)))
        return E, g

    def set_active(self, mask):
        m = np.ascontiguousarray(mask, dtype=np.int32).reshape(-1)
        if m.size != self.n:
            raise ValueError(f"mask: expected {self.n} entries")
        self._raise(self.lib.etdm_set_active(self.h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))

    def minimize(self, a, n_steps, stream=None):
        """n_steps ETDM iterations of every system, in place on the packed a;
        returns (E, alpha, trials), each [n, n_steps + 1]."""
        _require(a, self.dev, "a", numel=self.nvar)
        E = np.zeros((self.n, n_steps + 1))
        al = np.zeros((self.n, n_steps + 1))
        tr = np.zeros((self.n, n_steps + 1), dtype=np.int32)
        self._raise(self.lib.etdm_minimize(self.h, ctypes.c_void_p(a.data_ptr()), n_steps,
                                           _dptr(E), _dptr(al),
                                           tr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                           _stream_ptr(stream, self.dev)))
        return E, al, tr

    def lbfgs_reset(self):
        self._raise(self.lib.etdm_lbfgs_reset(self.h))

    def check(self, stream=None):
        self._raise(self.lib.etdm_check(self.h, _stream_ptr(stream, self.dev)))

    def launches(self):
        """Kernel launches (graph kernel nodes included) since the last call."""
        ms = np.zeros(8)
        cnt = np.zeros(8, dtype=np.int64)
        self._raise(self.lib.etdm_stage_times(self.h, _dptr(ms),
                                              cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return int(cnt[-1])

    def close(self):
        if getattr(self, "h", None):
            for m in getattr(self, "systems", []):
                m.h = None
            self.lib.etdm_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pair_gemm(A, B, ta=False, tb=False, stream=None):
    """C = op(A) op(B) of FP64 CUDA matrices through the tensor-core product of
    the mixed-precision dense chains (exact BF16 slices, about 2^-39 relative)."""
    import torch
    lib = load_library()
    if not (isinstance(A, torch.Tensor) and A.is_cuda and A.dim() == 2):
        raise ValueError("A: expected a 2-D CUDA tensor")
    if not (isinstance(B, torch.Tensor) and B.dim() == 2):
        raise ValueError("B: expected a 2-D CUDA tensor")
    m, k = (A.shape[1], A.shape[0]) if ta else (A.shape[0], A.shape[1])
    k2, n = (B.shape[1], B.shape[0]) if tb else (B.shape[0], B.shape[1])
    if k != k2:
        raise ValueError(f"inner dimensions differ: {k} and {k2}")
    _require(A, A.device, "A", shape=tuple(A.shape))
    _require(B, A.device, "B", shape=tuple(B.shape))
    if stream is not None and stream.device != A.device:
        raise ValueError(f"stream is on {stream.device}, not {A.device}")
    C = torch.empty((m, n), dtype=torch.float64, device=A.device)
    with torch.cuda.device(A.device):
        st = stream if stream is not None else torch.cuda.current_stream(A.device)
        rc = lib.etdm_pair_gemm(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                ctypes.c_void_p(C.data_ptr()), m, n, k, int(bool(ta)),
                                int(bool(tb)), ctypes.c_void_p(st.cuda_stream))
    if rc != ETDM_OK:
        raise EtdmError(rc, lib.etdm_last_error(None).decode())
    return C


def _storage_span(t):
    """Byte range [lo, hi) of the storage a tensor's elements occupy."""
    lo = t.data_ptr()
    return lo, lo + t.numel() * t.element_size()


def _overlaps(x, y):
    (a0, a1), (b0, b1) = _storage_span(x), _storage_span(y)
    return a0 < b1 and b0 < a1


def _noalloc_checks(g, S, Y, h0, out, stream):
    """(m, n) after every check an allocation-free direction call needs before
    its pointers reach the library: shapes and device (_noalloc_shapes), an
    output that overlaps no input, and a stream on the tensors' device."""
    m, n = _noalloc_shapes(g, S, Y, h0, out)
    for name, t in (("g", g), ("h0", h0), ("S", S), ("Y", Y)):
        if t is not None and t.numel() and out.numel() and _overlaps(out, t):
            raise ValueError(f"out may not overlap {name}")
    if stream is not None and stream.device != g.device:
        raise ValueError(f"stream is on {stream.device}, the tensors on {g.device}")
    return m, n


def lbfgs_direction_noalloc(g, S, Y, h0, out=None, stream=None):
    """p = -H g by the L-BFGS two-loop recursion over the pairs S[i], Y[i]
    (oldest first) with the diagonal initial inverse Hessian h0, through the
    allocation-free entry point: for callers that cannot allocate device
    memory where they need a direction.  All tensors are contiguous CUDA FP64
    on one device; S and Y have shape (m, n) with m <= 16; `out` may not
    overlap the inputs.  `out` must be preallocated by such callers (here it
    is created when None).  The call runs with g's device current, on
    `stream` (default: that device's current stream); a device-side failure
    is reported by lbfgs_direction_noalloc_status(stream)."""
    import torch
    lib = load_library()
    if not (isinstance(g, torch.Tensor) and g.is_cuda):
        raise ValueError("g: expected a CUDA tensor")
    out = torch.empty_like(g) if out is None else out
    m, n = _noalloc_checks(g, S, Y, h0, out, stream)
    with torch.cuda.device(g.device):
        st = stream if stream is not None else torch.cuda.current_stream(g.device)
        rc = lib.etdm_lbfgs_direction_noalloc(
            ctypes.c_void_p(g.data_ptr()),
            ctypes.c_void_p(S.data_ptr()) if m else None,
            ctypes.c_void_p(Y.data_ptr()) if m else None,
            m, n, ctypes.c_void_p(h0.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(st.cuda_stream))
    if rc != ETDM_OK:
        raise EtdmError(rc, lib.etdm_last_error(None).decode())
    return out


def lbfgs_direction_noalloc_status(device=None, stream=None):
    """Waits for `stream` (default: the device's current stream) and raises
    EtdmError when the last allocation-free direction on `device` failed on
    the GPU (a grid barrier that gave up, a pair with y.s <= 0); its output is
    then incomplete."""
    import torch
    lib = load_library()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None \
        else torch.device(device)
    if stream is not None and stream.device != dev:
        raise ValueError(f"stream is on {stream.device}, not {dev}")
    with torch.cuda.device(dev):
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        rc = lib.etdm_lbfgs_direction_noalloc_status(ctypes.c_void_p(st.cuda_stream))
    if rc != ETDM_OK:
        raise EtdmError(rc, lib.etdm_last_error(None).decode())


def energy_function():
    """torch.autograd.Function E(A_ov): forward evaluates the energy only;
    backward re-runs the density (no grid is stored between the two) and the
    analytic adjoint, and scales dE/dA_ov by grad_output."""
    import torch

    class ETDMEnergy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a, solver):
            E, _ = solver.energy_grad(a.contiguous(), want_grad=False)
            ctx.solver = solver
            ctx.save_for_backward(a)
            return E[0].clone()

        @staticmethod
        def backward(ctx, grad_out):
            (a,) = ctx.saved_tensors
            _, g = ctx.solver.energy_grad(a.contiguous(), want_grad=True)
            return grad_out * g, None

    return ETDMEnergy
