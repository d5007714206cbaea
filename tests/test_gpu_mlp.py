"""The network kernels (BF16 tensor-core products, FP32 accumulation) against
the FP64 oracle that rounds the same operands to BF16."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dcd():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1904_08553_gb300 import dcd as m

    return m


def data(rng, n, scale=1.0):
    X = (rng.standard_normal((n, 12)) * scale).astype(np.float32)
    y = (rng.random(n) < 0.35).astype(np.float32)
    return X, y


@pytest.mark.parametrize("n", [1, 15, 64, 100, 1000, 4099])
def test_forward_matches_oracle(dcd, orc, n):
    import torch

    rng = np.random.default_rng(20 + n)
    X, y = data(rng, n)
    P = (rng.standard_normal(dcd.MLP_PARAMS) * 0.3).astype(np.float32)
    m = dcd.Mlp(seed=1)
    m.params = P
    dX = torch.from_numpy(X).cuda()
    dp = torch.empty(n, dtype=torch.float32, device="cuda")
    m.forward(dX, n, dp)
    p_ref, _ = orc.mlp_forward(P, X)
    assert np.max(np.abs(dp.cpu().numpy() - p_ref)) < 2e-2


@pytest.mark.parametrize("n", [64, 1000, 4099])
def test_gradients_match_oracle(dcd, orc, n):
    import torch

    rng = np.random.default_rng(30 + n)
    X, y = data(rng, n)
    P = (rng.standard_normal(dcd.MLP_PARAMS) * 0.3).astype(np.float32)
    m = dcd.Mlp(seed=2)
    m.params = P
    G, loss = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), n)
    Gr, lr = orc.mlp_grad(P, X, y)
    assert abs(loss - lr) <= 2e-2 * abs(lr)
    sl = {"W1": slice(0, 768), "b1": slice(768, 832), "W2": slice(832, 4928), "b2": slice(4928, 4992),
          "W3": slice(4992, 5056), "b3": slice(5056, 5057)}
    for name, s in sl.items():
        g, r = G[s].astype(np.float64), Gr[s]
        rel = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-12)
        assert rel <= 2e-2, (name, rel)
        if r.size > 1:
            cos = g @ r / max(np.linalg.norm(g) * np.linalg.norm(r), 1e-30)
            assert cos >= 0.999, (name, cos)
        # element by element: within 2e-2 of the tensor's largest magnitude
        # (both sides round the same operands to BF16; what is left is the
        # FP32 accumulation order and the BF16 re-rounding of hidden
        # activations that a one-ulp accumulation difference can flip)
        bound = 2e-2 * max(np.max(np.abs(r)), 1e-12)
        worst = np.max(np.abs(g - r))
        assert worst <= bound, (name, worst, bound)


def test_gradient_is_deterministic(dcd):
    import torch

    rng = np.random.default_rng(40)
    X, y = data(rng, 5000)
    m = dcd.Mlp(seed=3)
    dX, dy = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    g1, l1 = m.grad(dX, dy, 5000)
    g2, l2 = m.grad(dX, dy, 5000)
    assert np.array_equal(g1, g2) and l1 == l2


def test_training_fits_a_separable_rule(dcd):
    import torch

    rng = np.random.default_rng(41)
    n = 20000
    X = rng.standard_normal((n, 12)).astype(np.float32)
    y = ((X[:, 0] + 0.5 * X[:, 3] - 0.3 * X[:, 7]) > 0.2).astype(np.float32)
    m = dcd.Mlp(seed=4)
    dX, dy = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    _, l0 = m.grad(dX, dy, n)
    m.train(dX, dy, n, batch=1024, epochs=8, lr=3e-3)
    _, l1 = m.grad(dX, dy, n)
    assert l1 < 0.25 * l0
    dp = torch.empty(n, device="cuda")
    m.forward(dX, n, dp)
    acc = ((dp.cpu().numpy() > 0.5) == (y > 0.5)).mean()
    assert acc > 0.95
