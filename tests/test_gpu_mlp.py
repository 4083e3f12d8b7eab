"""GPU tests of the learned-correction network kernels (BF16 tensor-core
GEMMs with FP32 accumulation) against the FP64 numpy oracle evaluated on the
same bfloat16-rounded inputs and weights.  Tolerances follow from BF16
activations between layers (8-bit mantissa): ~1e-2 relative."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    c = cgks.Context()
    yield c
    c.close()


def bf16_dev(x):
    return torch.tensor(np.asarray(x, np.float32), device="cuda").to(torch.bfloat16).contiguous()


def case(seed, n):
    rng = np.random.default_rng(seed)
    theta = mlp.init_params(seed) + 0.05 * rng.standard_normal(mlp.N_PARAMS)
    theta = theta.astype(np.float32).astype(np.float64)
    X = rng.standard_normal((n, 68))
    Y = 0.3 * rng.standard_normal((n, 4))
    return theta, X, Y


@pytest.mark.parametrize("n", [1, 37, 1000, 70000])
def test_forward_matches_oracle(ctx, n):
    theta, X, _ = case(1, n)
    ctx.cgks_mlp_set_params(theta)
    Xd = bf16_dev(X)
    P = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    ctx.cgks_mlp_forward(Xd, P)
    torch.cuda.synchronize()
    Xb = mlp.to_bf16(X)
    W = mlp.to_bf16(theta)
    # keep the biases in FP32 as the kernels do
    for (o, i), start in zip(mlp.SIZES, (0, 64 * 68 + 64, 64 * 68 + 64 + 64 * 64 + 64)):
        W[start + o * i:start + o * i + o] = theta[start + o * i:start + o * i + o]
    Po, _ = mlp.forward(W, Xb)
    err = np.abs(P.cpu().numpy() - Po)
    assert np.max(err) <= 2e-2 * (np.max(np.abs(Po)) + 1e-3), np.max(err)


@pytest.mark.parametrize("n", [4096, 16384])
def test_gradient_matches_oracle(ctx, n):
    """Weight gradients with the split-K reduction, up to the training batch size."""
    theta, X, Y = case(2, n)
    ctx.cgks_mlp_set_params(theta)
    g = torch.zeros(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = ctx.cgks_mlp_grad(bf16_dev(X), torch.tensor(Y, dtype=torch.float32, device="cuda"), g)
    go = mlp.grad(theta, mlp.to_bf16(X), Y)
    lo = mlp.loss(theta, mlp.to_bf16(X), Y)
    gg = g.cpu().numpy()
    assert abs(loss - lo) <= 2e-2 * lo
    for a, b in ((0, 64 * 68), (64 * 68, 64 * 68 + 64), (4416, 4416 + 4096), (8576, 8832), (8832, 8836)):
        rel = np.linalg.norm(gg[a:b] - go[a:b]) / (np.linalg.norm(go[a:b]) + 1e-12)
        assert rel < 3e-2, (a, b, rel)


def test_training_reduces_loss(ctx):
    """Fit a smooth synthetic map: the loss falls by more than 10x."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((20000, 68)).astype(np.float32)
    A = rng.standard_normal((68, 4)) / 8.0
    Y = np.tanh(X @ A).astype(np.float32)
    ctx.cgks_mlp_dataset_clear()
    ctx.cgks_mlp_dataset_append(bf16_dev(X), torch.tensor(Y, device="cuda"))
    assert ctx.cgks_mlp_dataset_size() == 20000
    ctx.cgks_mlp_set_params(mlp.init_params(7))
    losses = ctx.cgks_mlp_train(400, 1024, 2e-3, seed=11)
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.1 * losses[:5].mean()
    th = ctx.cgks_mlp_get_params()
    assert th.shape == (8836,) and np.all(np.isfinite(th))
