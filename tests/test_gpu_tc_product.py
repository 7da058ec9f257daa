"""The tensor-core product of the mixed path's dense chains (etdm_pair_gemm:
exact BF16 slices of float pairs, per-order accumulators in tensor memory)
against FP64 products, over shapes that take every path of it: one K step,
several exact K chunks, several output tiles in both directions, ragged
edges, transposed operands, and rows of very different scale."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


@pytest.mark.parametrize("m,n,k,ta,tb", [
    (1, 1, 3, 0, 0), (4, 4, 12, 0, 1), (16, 4, 16, 0, 0), (128, 64, 16, 0, 0),
    (130, 70, 17, 0, 0), (128, 64, 240, 0, 0), (128, 64, 241, 0, 0), (300, 300, 300, 0, 0),
    (300, 200, 600, 1, 0), (257, 129, 500, 1, 1), (600, 300, 600, 0, 1)])
def test_pair_gemm_against_fp64(m, n, k, ta, tb):
    torch = _torch()
    from paper_2101_12597_gb300.etdm import pair_gemm
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.normal(size=(k, m) if ta else (m, k)) * np.exp(rng.normal(size=(1 if ta else m, m if ta else 1)))
    B = rng.normal(size=(n, k) if tb else (k, n))
    C = pair_gemm(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), ta, tb)
    torch.cuda.synchronize()
    opA = A.T if ta else A
    opB = B.T if tb else B
    ref = opA @ opB
    # the slices resolve each row of op(A) and column of op(B) to about 2^-39 of
    # its largest entry; the bound per entry: 2^-36 of k max|A_i.| max|B_.j|
    scale = k * np.abs(opA).max(1)[:, None] * np.abs(opB).max(0)[None, :]
    err = float(np.max(np.abs(C.cpu().numpy() - ref) / scale))
    print(f"{m}x{n}x{k} ta={ta} tb={tb}: max error {err:.2e} of k max|A_i.| max|B_.j|")
    assert err < 2.0 ** -36
