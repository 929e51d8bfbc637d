"""GPU training kernels of the position model against the fp64 CPU oracle:
forward pass, loss and gradient (backward pass), Adam step."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2112_03229_gb300 as m
    return m


def case(seed, B):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(65) * 0.5).astype(np.float32)
    x = rng.uniform(0, 1, (B, 2)).astype(np.float32)
    y = rng.uniform(0, 1, B).astype(np.float32)
    return p, x, y


@pytest.mark.parametrize("B", [1, 7, 512, 513, 100_000])
def test_forward_and_gradient_match_oracle(ss, B):
    p, x, y = case(B, B)
    dev = lambda a: torch.as_tensor(a).cuda()
    yf = ss.mlp_forward(dev(p), dev(x)).cpu().numpy()
    np.testing.assert_allclose(yf, oracle.mlp_forward(p.astype(np.float64), x.astype(np.float64)), rtol=1e-5, atol=1e-5)
    loss, grad = ss.mlp_loss_grad(dev(p), dev(x), dev(y))
    wl, wg = oracle.mlp_loss_grad(p.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
    assert abs(loss.item() - wl) <= 1e-4 * max(wl, 1e-6)
    g = grad.cpu().numpy().astype(np.float64)
    scale = np.abs(wg).max()
    np.testing.assert_allclose(g, wg, rtol=1e-4, atol=1e-5 * scale)


def test_gradient_matches_finite_differences(ss):
    # GPU analytic gradient vs central differences of the fp64 oracle loss
    p, x, y = case(11, 4096)
    _, grad = ss.mlp_loss_grad(torch.as_tensor(p).cuda(), torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda())
    g = grad.cpu().numpy()
    pd, xd, yd = p.astype(np.float64), x.astype(np.float64), y.astype(np.float64)
    for k in range(65):
        q = pd.copy(); q[k] += 1e-6
        lp, _ = oracle.mlp_loss_grad(q, xd, yd)
        q[k] -= 2e-6
        lm, _ = oracle.mlp_loss_grad(q, xd, yd)
        fd = (lp - lm) / 2e-6
        assert abs(g[k] - fd) <= 1e-4 * max(1.0, abs(fd)), (k, g[k], fd)


def test_adam_step_matches_oracle(ss):
    rng = np.random.default_rng(2)
    p = rng.standard_normal(65)
    g = rng.standard_normal(65)
    m1 = rng.standard_normal(65) * 0.1
    m2 = np.abs(rng.standard_normal(65)) * 0.1
    tp, tg, t1, t2 = (torch.as_tensor(a, dtype=torch.float32).cuda() for a in (p, g, m1, m2))
    ss.mlp_adam_step(tp, tg, t1, t2, step=3, lr=1e-2)
    po, m1o, m2o = p.copy(), m1.copy(), m2.copy()
    oracle.adam_step(po, g, m1o, m2o, 3, 1e-2)
    np.testing.assert_allclose(tp.cpu().numpy(), po, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(t1.cpu().numpy(), m1o, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(t2.cpu().numpy(), m2o, rtol=1e-5, atol=1e-7)
