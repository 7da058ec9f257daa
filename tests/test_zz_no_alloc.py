"""The allocation-free L-BFGS entry point against the handle's own
etdm_lbfgs_step.  It serves callers that cannot allocate device memory where
they need a direction (stream capture with a frozen pool, pre-registered
buffers only); the check is that, fed the same pair history and the same
initial inverse Hessian, it returns the handle's direction, on two calls in a
row that share its fixed scratch array.  This file sorts last so that a run
stopping at the first failure has run every other test before it."""
import numpy as np
import pytest

import etdm_synth as synth

pytestmark = pytest.mark.gpu


def test_noalloc_direction_matches_handle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2101_12597_gb300.etdm import ETDM, EtdmError, lbfgs_direction_noalloc
    d = synth.config_small_molecule()
    solver = ETDM(d)
    solver.lbfgs_reset()
    N, V = solver.N, solver.V
    n = N * V
    rng = np.random.default_rng(17)
    Q = rng.normal(size=(n, n))
    A = Q @ Q.T + n * np.eye(n)
    x = rng.normal(size=n)
    hist = []  # accepted pairs, oldest first (the handle keeps the newest 3)
    a_prev = g_prev = None
    ones = torch.ones((N, V), dtype=torch.float64, device="cuda")
    for k in range(7):
        g = A @ x
        if a_prev is not None:
            s, y = x - a_prev, g - g_prev
            if s @ y > 1e-30:
                hist.append((s, y))
        a_prev, g_prev = x.copy(), g.copy()
        at = torch.tensor(x.reshape(N, V), device="cuda")
        gt = torch.tensor(g.reshape(N, V), device="cuda")
        p_ref = solver.lbfgs_step(at, gt)
        h0 = solver.precondition(ones)  # Eq. 33 with the beta the step just set
        pairs = hist[-3:]
        S = torch.tensor(np.array([p[0] for p in pairs]), device="cuda") if pairs else None
        Y = torch.tensor(np.array([p[1] for p in pairs]), device="cuda") if pairs else None
        outs = []
        for _ in range(2):  # two calls in a row share the scratch array
            out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            lbfgs_direction_noalloc(gt.reshape(-1), S, Y, h0.reshape(-1), out=out)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
        pr = p_ref.reshape(-1).cpu().numpy()
        for o in outs:
            np.testing.assert_allclose(o, pr, rtol=1e-11, atol=1e-13 * np.abs(pr).max())
        x = x + 0.7 * pr
    # sizes beyond the scratch limit are rejected with a message
    g1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    S17 = torch.zeros((17, n), dtype=torch.float64, device="cuda")
    with pytest.raises(EtdmError) as ei:
        lbfgs_direction_noalloc(g1, S17, S17, g1, out=torch.empty_like(g1))
    assert ei.value.code == -1 and "scratch limit" in str(ei.value)
    solver.close()
