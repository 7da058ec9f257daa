"""Argument checks of the Python binding, which run before any pointer reaches
the library (no GPU needed: the checks are exercised with CPU tensors against a
CPU device, which is the only difference from their use on the GPU)."""
import numpy as np
import pytest
import torch

from paper_2101_12597_gb300 import etdm
from paper_2101_12597_gb300.etdm import _noalloc_checks, _noalloc_shapes, _require

CPU = torch.device("cpu")


def _t(*shape, dtype=torch.float64):
    return torch.zeros(shape, dtype=dtype)


def test_require_accepts_the_contract():
    _require(_t(3, 5), CPU, "a", shape=(3, 5))
    _require(_t(1), CPU, "E", numel=1)
    _require(_t(15), CPU, "g", numel=15)


@pytest.mark.parametrize("bad,frag", [
    (_t(5, 3), "shape (3, 5)"),                      # transposed shape
    (_t(3, 5, dtype=torch.float32), "float32"),       # wrong dtype
    (_t(5, 3).t(), "contiguous=False"),               # a transposed view
    (np.zeros((3, 5)), "ndarray"),                    # not a tensor
])
def test_require_rejects_with_a_message(bad, frag):
    with pytest.raises(ValueError) as ei:
        _require(bad, CPU, "a", shape=(3, 5))
    assert str(ei.value).startswith("a: ") and frag in str(ei.value)


def test_require_rejects_another_device():
    with pytest.raises(ValueError, match="on meta"):
        _require(torch.empty((3, 5), dtype=torch.float64, device="meta"), CPU, "a",
                 shape=(3, 5))


def test_noalloc_shapes():
    n = 12
    g, h0, out = _t(3, 4), _t(n), _t(n)
    assert _noalloc_shapes(g, None, None, h0, out) == (0, n)
    assert _noalloc_shapes(g, _t(2, n), _t(2, n), h0, out) == (2, n)
    assert _noalloc_shapes(g, _t(0, n), _t(0, n), h0, out) == (0, n)
    # the limit m <= 16 is the library's to enforce (with its own message)
    assert _noalloc_shapes(g, _t(17, n), _t(17, n), h0, out) == (17, n)
    for S, Y, frag in [(_t(2, n), None, "both or neither"),
                       (_t(2, n + 1), _t(2, n + 1), "S:"),
                       (_t(2, n), _t(3, n), "Y:"),
                       (_t(2 * n), _t(2 * n), "S:")]:
        with pytest.raises(ValueError, match=frag):
            _noalloc_shapes(g, S, Y, h0, out)
    with pytest.raises(ValueError, match="h0:"):
        _noalloc_shapes(g, None, None, _t(n - 1), out)
    with pytest.raises(ValueError, match="out:"):
        _noalloc_shapes(g, None, None, h0, _t(n, dtype=torch.float32))


def test_noalloc_output_may_not_overlap_an_input():
    n = 12
    buf = _t(3 * n)
    g, h0 = buf[:n], buf[n:2 * n]
    S = Y = _t(2, n)
    assert _noalloc_checks(g, S, Y, h0, buf[2 * n:], None) == (2, n)
    with pytest.raises(ValueError, match="overlap g"):
        _noalloc_checks(g, S, Y, h0, g, None)
    with pytest.raises(ValueError, match="overlap h0"):
        _noalloc_checks(g, S, Y, h0, buf[n + 1:2 * n + 1], None)
    with pytest.raises(ValueError, match="overlap S"):
        _noalloc_checks(g, S, Y, h0, S[1], None)


def test_noalloc_stream_must_be_on_the_tensors_device():
    class Stream:
        def __init__(self, dev):
            self.device = torch.device(dev)
            self.cuda_stream = 0

    n = 6
    g, h0, out = _t(n), _t(n), _t(n)
    assert _noalloc_checks(g, None, None, h0, out, Stream("cpu")) == (0, n)
    with pytest.raises(ValueError, match="stream is on meta"):
        _noalloc_checks(g, None, None, h0, out, Stream("meta"))


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU behaviour")
def test_no_cpu_fallback():
    import etdm_synth as synth
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        etdm.ETDM(synth.tiny())
    from paper_2101_12597_gb300 import build
    build.build()
    with pytest.raises(ValueError, match="CUDA tensor"):
        etdm.lbfgs_direction_noalloc(_t(4), None, None, _t(4))


class _StubLib:
    """Records the arguments of each entry point and returns ETDM_OK."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if not name.startswith("etdm_"):
            raise AttributeError(name)

        def f(*args):
            self.calls.append((name, args))
            return 0
        return f


def _stub_solver(N=3, V=5):
    s = object.__new__(etdm.ETDM)
    s.lib, s.h, s.dev, s.N, s.V, s.M = _StubLib(), None, CPU, N, V, N + V
    return s


def test_marshalling_with_a_stub_library():
    class Stream:  # a caller-owned stream: only its handle is passed on
        cuda_stream = 0
        device = CPU

    st = Stream()
    s = _stub_solver()
    a = _t(3, 5)
    E, g = s.energy_grad(a, stream=st)
    name, args = s.lib.calls[-1]
    assert name == "etdm_energy_grad"
    assert [x.value for x in args[1:4]] == [a.data_ptr(), E.data_ptr(), g.data_ptr()]
    E2, g2 = s.energy_grad(a, want_grad=False, stream=st)
    assert g2 is None and s.lib.calls[-1][1][3] is None
    out = _t(3, 5)
    assert s.precondition(g, out=out, stream=st) is out
    assert s.lbfgs_step(a, g, out=out, stream=st) is out
    assert s.lib.calls[-1][0] == "etdm_lbfgs_step"
    assert [x.value for x in s.lib.calls[-1][1][1:4]] == [a.data_ptr(), g.data_ptr(),
                                                          out.data_ptr()]
    n_calls = len(s.lib.calls)
    for bad in [dict(E=_t(2)), dict(g=_t(5, 3)), dict(g=_t(3, 5, dtype=torch.float32))]:
        with pytest.raises(ValueError):
            s.energy_grad(a, stream=st, **bad)
    with pytest.raises(ValueError, match="out:"):
        s.precondition(g, out=_t(15), stream=st)
    with pytest.raises(ValueError, match="a:"):
        s.lbfgs_step(_t(5, 3), g, stream=st)
    with pytest.raises(ValueError):
        s.energy_grad(a.t().contiguous().t(), stream=st)  # a non-contiguous view
    assert len(s.lib.calls) == n_calls  # none of these reached the library
    with pytest.raises(ValueError, match="a: expected shape"):
        s.energy_grad_host(np.zeros((5, 3)))
    E, gh = s.energy_grad_host(np.zeros((3, 5)))
    assert gh.shape == (3, 5) and s.lib.calls[-1][0] == "etdm_energy_grad_host"


def test_handle_calls_refuse_a_stream_of_another_device():
    """A caller's stream must belong to the handle's device: the check runs
    before the library is called."""
    class Stream:
        cuda_stream = 0
        device = torch.device("meta")

    s = _stub_solver()
    a = _t(3, 5)
    with pytest.raises(ValueError, match="stream is on meta"):
        s.energy_grad(a, stream=Stream())
    with pytest.raises(ValueError, match="stream is on meta"):
        s.lbfgs_step(a, _t(3, 5), stream=Stream())
    assert s.lib.calls == []


def test_get_array_of_another_path_is_a_clear_error():
    """etdm_array_bytes returns -1 for an array the handle's path does not
    have (e.g. Uocc on the full-A path); the binding says so instead of
    allocating a negative size."""
    s = _stub_solver()
    s.lib.etdm_array_bytes = lambda h, which: -1
    with pytest.raises(ValueError, match="'Uocc' does not exist"):
        s.get_array("Uocc")
    assert s.lib.calls == []
