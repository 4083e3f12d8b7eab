"""GPU tests of the learned-correction network kernels (BF16 tensor-core
products with FP32 accumulation) against the FP64 numpy oracle evaluated on
the same bfloat16-rounded inputs and weights, for both forward
implementations: the fused tcgen05 kernel (accumulators in tensor memory,
impl 0, the default) and the mma.sync GEMM chain (impl 1).  Tolerances follow
from BF16 activations between layers (8-bit mantissa): ~1e-2 relative."""
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
    X = rng.standard_normal((n, 76))
    Y = 0.3 * rng.standard_normal((n, 4))
    return theta, X, Y


@pytest.mark.parametrize("impl", [0, 1])
@pytest.mark.parametrize("n", [1, 37, 1000, 70000])
def test_forward_matches_oracle(ctx, n, impl):
    theta, X, _ = case(1, n)
    ctx.cgks_mlp_set_params(theta)
    ctx.cgks_mlp_select(impl)
    Xd = bf16_dev(X)
    P = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    ctx.cgks_mlp_forward(Xd, P)
    torch.cuda.synchronize()
    Xb = mlp.to_bf16(X)
    W = mlp.to_bf16(theta)
    # keep the biases in FP32 as the kernels do
    for (o, i), start in zip(mlp.SIZES, (0, 64 * 76 + 64, 64 * 76 + 64 + 64 * 64 + 64)):
        W[start + o * i:start + o * i + o] = theta[start + o * i:start + o * i + o]
    Po, _ = mlp.forward(W, Xb)
    ctx.cgks_synchronize()  # raises if the tensor-core kernel gave up waiting
    ctx.cgks_mlp_select(0)
    err = np.abs(P.cpu().numpy() - Po)
    assert np.max(err) <= 2e-2 * (np.max(np.abs(Po)) + 1e-3), np.max(err)


@pytest.mark.parametrize("n", [128, 1000, 65536])
def test_tcgen05_forward_matches_mma_sync(ctx, n):
    """The two forward implementations on the same rows: both take BF16
    operands and FP32 sums, and round the hidden activations to BF16, so they
    differ only where the order of the FP32 sums flips a BF16 rounding."""
    theta, X, _ = case(3, n)
    ctx.cgks_mlp_set_params(theta)
    Xd = bf16_dev(X)
    out = []
    for impl in (0, 1):
        ctx.cgks_mlp_select(impl)
        P = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
        ctx.cgks_mlp_forward(Xd, P)
        ctx.cgks_synchronize()
        out.append(P.cpu().numpy())
    ctx.cgks_mlp_select(0)
    d = np.abs(out[0] - out[1])
    scale = np.max(np.abs(out[1]))
    print(f"\ntcgen05 vs mma.sync forward, {n} rows: max |dP| {d.max():.2e} (scale {scale:.2e}), "
          f"median {np.median(d):.2e}")
    assert np.all(np.isfinite(out[0]))
    assert d.max() <= 1e-2 * scale
    assert np.median(d) <= 1e-5 * scale


@pytest.mark.parametrize("impl", [0, 1])
@pytest.mark.parametrize("n", [4096, 16384])
def test_gradient_matches_oracle(ctx, n, impl):
    """Weight gradients with the split-K reduction, up to the training batch
    size, after the forward pass of either implementation."""
    theta, X, Y = case(2, n)
    ctx.cgks_mlp_set_params(theta)
    ctx.cgks_mlp_select(impl)
    g = torch.zeros(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = ctx.cgks_mlp_grad(bf16_dev(X), torch.tensor(Y, dtype=torch.float32, device="cuda"), g)
    go = mlp.grad(theta, mlp.to_bf16(X), Y)
    lo = mlp.loss(theta, mlp.to_bf16(X), Y)
    gg = g.cpu().numpy()
    ctx.cgks_mlp_select(0)
    assert abs(loss - lo) <= 2e-2 * lo
    o2 = 64 * 76 + 64
    for a, b in ((0, 64 * 76), (64 * 76, o2), (o2, o2 + 4096), (o2 + 4160, o2 + 4416), (o2 + 4416, o2 + 4420)):
        rel = np.linalg.norm(gg[a:b] - go[a:b]) / (np.linalg.norm(go[a:b]) + 1e-12)
        assert rel < 3e-2, (a, b, rel)


def test_training_reduces_loss(ctx):
    """Fit a smooth synthetic map: the loss falls by more than 10x."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((20000, 76)).astype(np.float32)
    A = rng.standard_normal((76, 4)) / 8.0
    Y = np.tanh(X @ A).astype(np.float32)
    ctx.cgks_mlp_dataset_clear()
    ctx.cgks_mlp_dataset_append(bf16_dev(X), torch.tensor(Y, device="cuda"))
    assert ctx.cgks_mlp_dataset_size() == 20000
    ctx.cgks_mlp_set_params(mlp.init_params(7))
    losses = ctx.cgks_mlp_train(400, 1024, 2e-3, seed=11)
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.1 * losses[:5].mean()
    th = ctx.cgks_mlp_get_params()
    assert th.shape == (9348,) and np.all(np.isfinite(th))


def test_nonfinite_rows_take_no_part_in_training(ctx):
    """Rows collected from a diverging mesh carry non-finite inputs or targets.
    Appended to the training set they add neither loss nor gradient, so
    training on a set with such rows stays finite and still fits; and a NaN
    target excludes its row from the gradient: the gradient equals the one
    without that row, times (n - 1) / n for the mean's count, up to the BF16
    rounding of the output gradient (whose scale differs by that factor)."""
    rng = np.random.default_rng(8)
    n = 512
    X = rng.standard_normal((n, 76)).astype(np.float32)
    A = rng.standard_normal((76, 4)) / 8.0
    Y = np.tanh(X @ A).astype(np.float32)
    ctx.cgks_mlp_set_params(mlp.init_params(9))
    # the gradient with one NaN target against the gradient without that row
    Yn = Y.copy()
    Yn[7] = np.nan
    g1 = torch.zeros(9348, dtype=torch.float32, device="cuda")
    g2 = torch.zeros(9348, dtype=torch.float32, device="cuda")
    ctx.cgks_mlp_grad(bf16_dev(X), torch.tensor(Yn, device="cuda"), g1)
    keep = np.arange(n) != 7
    ctx.cgks_mlp_grad(bf16_dev(X[keep]), torch.tensor(Y[keep], device="cuda"), g2)
    a, b = g1.cpu().numpy(), g2.cpu().numpy() * (n - 1) / n
    assert np.all(np.isfinite(a))
    assert np.max(np.abs(a - b)) <= 2e-3 * np.max(np.abs(b))
    # training on a set with rows of NaN inputs and infinite targets
    Xp, Yp = X.copy(), Y.copy()
    Xp[3, 5] = np.nan
    Yp[11, 2] = np.inf
    ctx.cgks_mlp_dataset_clear()
    ctx.cgks_mlp_dataset_append(bf16_dev(Xp), torch.tensor(Yp, device="cuda"))
    ctx.cgks_mlp_set_params(mlp.init_params(9))
    losses = ctx.cgks_mlp_train(200, 256, 2e-3, seed=3)
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.5 * losses[:5].mean()
    assert np.all(np.isfinite(ctx.cgks_mlp_get_params()))
