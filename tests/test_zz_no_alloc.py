"""GPU test of cgks_residual_coarse_noalloc, the coarse KFVS residual for
callers that cannot let a call allocate device memory (memory planned up
front, or latency-critical loops that must avoid the implicit synchronisation
of cudaMalloc/cudaFree).  Its output must match cgks_residual, the ordinary
entry point, on two calls in a row (the fixed face-flux buffer is reused),
and both must match the FP64 oracle's KFVS residual of the same state.

The context is created on torch's current stream, so the torch work that
fills the input and output buffers and the library's kernels are ordered on
one stream (the entry point does not synchronise)."""
import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GAMMA = 1.4


def perturbed(w, n, dim, rng):
    rho0 = w[0]
    u0 = w[1:1 + dim] / rho0
    p0 = (GAMMA - 1) * (w[-1] - 0.5 * rho0 * u0 @ u0)
    rho = rho0 * (1 + 0.05 * rng.random(n))
    u = u0 + 0.2 * rng.standard_normal((n, dim))
    p = p0 * (1 + 0.1 * rng.random(n))
    W = np.zeros((n, dim + 2))
    W[:, 0] = rho
    W[:, 1:1 + dim] = rho[:, None] * u
    W[:, -1] = p / (GAMMA - 1) + 0.5 * rho * np.sum(u * u, 1)
    return W


def flux_scale(W, dim):
    u = W[:, 1:1 + dim] / W[:, :1]
    p = (GAMMA - 1) * (W[:, -1] - 0.5 * W[:, 0] * np.sum(u * u, 1))
    c = np.sqrt(GAMMA * p / W[:, 0])
    return float(np.max((np.abs(W[:, -1]) + p) * (np.linalg.norm(u, axis=1) + c)))


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    return cgks


@pytest.mark.parametrize("name", ["cylinder", "sphere"])
def test_noalloc_matches_residual_twice(cg, name):
    if name == "cylinder":
        m = synth.cylinder_mesh(n_theta=32, n_r=16, ratio=1.05 ** 2, n_refine=2)
        w = synth.freestream(4.0, angle_deg=10.0)
    else:
        m = synth.sphere_mesh(n_panel=8, n_r=8)
        w = synth.freestream(3.0, dim=3, angle_deg=10.0)
    dim, nv = m["dim"], m["dim"] + 2
    ctx = cg.Context(stream=torch.cuda.current_stream().cuda_stream)
    ctx.setup(3, m, w, synth.uniform_state(m, w))
    info = ctx.cgks_mesh_info(3)
    om = oracle.OracleMesh(m)
    cfg = oracle.cfg_vector(dim, winf=w)
    rng = np.random.default_rng(42)
    for lev in (1, 2):
        nl = info[lev]["cells"]
        Smax = float(np.max(om.faces(lev)["S"]))
        for call in range(2):
            W = perturbed(w, nl, dim, rng)
            R_ref = np.zeros((nl, nv))
            ctx.cgks_residual(3, lev, W, R_ref)
            Wd = torch.tensor(W, dtype=torch.float64, device="cuda")
            Rd = torch.full((nl, nv), float("nan"), dtype=torch.float64, device="cuda")
            ctx.cgks_residual_coarse_noalloc(3, lev, Wd, Rd)
            ctx.cgks_synchronize()
            R = Rd.cpu().numpy()
            atol = 1e-12 * flux_scale(W, dim) * Smax
            np.testing.assert_allclose(R, R_ref, rtol=0, atol=atol)
            np.testing.assert_allclose(R, om.kfvs_residual(cfg, W, lev), rtol=0, atol=atol)
    ctx.close()


def test_noalloc_rejects_oversized_level(cg):
    """A level with more faces than the fixed buffer holds is refused with a
    clear error instead of writing past the buffer."""
    m = synth.sphere_mesh(n_panel=24, n_r=24)
    w = synth.freestream(3.0, dim=3)
    ctx = cg.Context(stream=torch.cuda.current_stream().cuda_stream)
    ctx.setup(4, m, w, synth.uniform_state(m, w))
    info = ctx.cgks_mesh_info(4)
    assert info[1]["faces"] > 131072
    nl = info[1]["cells"]
    Wd = torch.tensor(np.tile(w, (nl, 1)), dtype=torch.float64, device="cuda")
    Rd = torch.zeros((nl, 5), dtype=torch.float64, device="cuda")
    rc = ctx.cgks_residual_coarse_noalloc(4, 1, Wd, Rd, check=False)
    assert rc == -1
    assert "131072" in ctx._L.cgks_last_error(ctx.h).decode()
    ctx.close()
