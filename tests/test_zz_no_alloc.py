"""The allocation-free L-BFGS entry point against the oracle's two-loop
recursion and against the handle entry point etdm_lbfgs_step.  It serves
callers that cannot allocate device memory where they need a direction (stream
capture with a frozen pool, pre-registered buffers only); the checks are that,
fed the same pair history and initial inverse Hessian, it returns the oracle's
direction and the handle's, on two calls in a row that share its fixed scratch
array, and that a failure on the device (a pair without positive curvature)
comes back through the status call.  This file sorts last so that a run
stopping at the first failure has run every other test before it."""
import numpy as np
import pytest

from oracle.etdm_oracle import LBFGS

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def test_noalloc_direction_matches_oracle():
    torch = _torch()
    from paper_2101_12597_gb300.etdm import (EtdmError, lbfgs_direction_noalloc,
                                             lbfgs_direction_noalloc_status)
    n = 4 * 12 + 1  # not a multiple of anything the kernel tiles by
    rng = np.random.default_rng(17)
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)           # SPD quadratic model, gradient A x
    h0 = 1.0 / (1.0 + rng.uniform(size=n))  # a positive diagonal H0
    lb = LBFGS(lambda beta: h0, m=3)
    x = rng.normal(size=n)
    dev = torch.device("cuda", 0)
    h0_d = torch.tensor(h0, device=dev)
    for k in range(7):
        g = A @ x
        p_ref = lb.step(x, g)  # stores the pair (x - x_prev, g - g_prev), keeps 3
        S = torch.tensor(np.array(lb.s), device=dev) if lb.s else None
        Y = torch.tensor(np.array(lb.y), device=dev) if lb.y else None
        gt = torch.tensor(g, device=dev)
        outs = []
        for _ in range(2):  # two calls in a row share the scratch array
            out = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
            lbfgs_direction_noalloc(gt, S, Y, h0_d, out=out)
            lbfgs_direction_noalloc_status(dev)
            outs.append(out.cpu().numpy())
        for o in outs:
            np.testing.assert_allclose(o, p_ref, rtol=1e-11, atol=1e-13 * np.abs(p_ref).max())
        x = x + 0.7 * p_ref
    # a pair without positive curvature: reported by the status call, then
    # cleared by the next call
    s_bad = torch.tensor(rng.normal(size=(1, n)), device=dev)
    out = torch.zeros(n, dtype=torch.float64, device=dev)
    lbfgs_direction_noalloc(gt, s_bad, -s_bad, h0_d, out=out)
    with pytest.raises(EtdmError) as ei:
        lbfgs_direction_noalloc_status(dev)
    assert ei.value.code == -7 and "y.s <= 0" in str(ei.value)
    lbfgs_direction_noalloc(gt, None, None, h0_d, out=out)
    lbfgs_direction_noalloc_status(dev)
    np.testing.assert_allclose(out.cpu().numpy(), -h0 * g, rtol=1e-15)
    # sizes beyond the scratch limit are rejected with a message
    g1 = torch.zeros(n, dtype=torch.float64, device=dev)
    S17 = torch.zeros((17, n), dtype=torch.float64, device=dev)
    with pytest.raises(EtdmError) as ei:
        lbfgs_direction_noalloc(g1, S17, S17, g1, out=torch.empty_like(g1))
    assert ei.value.code == -1 and "scratch limit" in str(ei.value)


def test_noalloc_direction_matches_lbfgs_step():
    """The allocation-free direction against the existing entry point: a handle
    of the 8-atom molecule runs etdm_lbfgs_step along a sequence of points and
    gradients of an SPD quadratic (it stores each pair and updates beta), and
    the allocation-free call, given the same three newest pairs and the
    handle's Eq. 33 diagonal at its current beta (etdm_precondition of a
    vector of ones), returns the handle's direction on two calls in a row, at
    the tolerance of the L-BFGS parity tests."""
    torch = _torch()
    import etdm_synth as synth
    from paper_2101_12597_gb300.etdm import (ETDM, lbfgs_direction_noalloc,
                                             lbfgs_direction_noalloc_status)
    dev = torch.device("cuda", 0)
    s = ETDM(synth.config_small_molecule(), precision="fp64")
    shape = s.var_shape
    n = int(np.prod(shape))
    rng = np.random.default_rng(23)
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)
    x = rng.normal(size=n)
    ones = torch.ones(shape, dtype=torch.float64, device=dev)
    pairs, prev = [], None
    s.lbfgs_reset()
    for k in range(7):
        g = A @ x
        if prev is not None:  # the pair the handle stores (curvature > 0 here)
            pairs = (pairs + [(x - prev[0], g - prev[1])])[-3:]
        prev = (x.copy(), g.copy())
        gt = torch.tensor(g.reshape(shape), device=dev)
        p_step = s.lbfgs_step(torch.tensor(x.reshape(shape), device=dev), gt)
        h0 = s.precondition(ones).reshape(-1)
        S = torch.tensor(np.array([p[0] for p in pairs]), device=dev) if pairs else None
        Y = torch.tensor(np.array([p[1] for p in pairs]), device=dev) if pairs else None
        want = p_step.cpu().numpy().ravel()
        for _ in range(2):  # two calls in a row share the scratch array
            out = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
            lbfgs_direction_noalloc(gt.reshape(-1), S, Y, h0, out=out)
            lbfgs_direction_noalloc_status(dev)
            np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-11,
                                       atol=1e-13 * np.abs(want).max())
        x = x + 0.7 * want
    s.lbfgs_reset()
    s.close()
