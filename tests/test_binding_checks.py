"""Argument checks of the Python binding, which run before any pointer reaches
the library (no GPU needed: the checks are exercised with CPU tensors against a
CPU device, which is the only difference from their use on the GPU)."""
import numpy as np
import pytest
import torch

from paper_2101_12597_gb300 import etdm
from paper_2101_12597_gb300.etdm import _noalloc_shapes, _require

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


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU behaviour")
def test_no_cpu_fallback():
    import etdm_synth as synth
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        etdm.ETDM(synth.tiny())
    from paper_2101_12597_gb300 import build
    build.build()
    with pytest.raises(ValueError, match="CUDA tensor"):
        etdm.lbfgs_direction_noalloc(_t(4), None, None, _t(4))
