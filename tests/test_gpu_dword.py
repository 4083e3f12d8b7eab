"""GPU parity of the double-word gas-kinetic flux (flux_precision = 1: the flux
arithmetic in two-float words on the FP32 pipes) against the FP64 oracle.

Tolerance: a double-word carries 48 significant bits (unit roundoff 2^-48)
against FP64's 53 (2^-53), so every rounding error, and its amplification by
cancellation, is up to 32 times larger.  The FP64 path's bounds are therefore
scaled by 32: residuals and slopes within 32e-12 of the flux scale, DF factors
within 32e-12 relative.  Whole V-cycles keep the FP64 bounds (norms 1e-8,
state 1e-9).  Measured: about 1e-14 of the flux scale on the small meshes and
the sampled sphere cells, but 1.3e-12 at the worst of the 65,536 cylinder
cells (DF 6e-13), so the FP64 bound of 1e-12 does not hold everywhere.  Covered: small 2-D and 3-D meshes, whole V-cycles, every cell of
the 65,536-cell cylinder, and sampled cells of the 1.18M-tet sphere shell."""
import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth
import test_gpu_parity as tp
from test_gpu_fullsize import smooth_physical_state

pytestmark = pytest.mark.gpu

TOL = 32 * 1e-12  # FP64 tolerance x 2^-48 / 2^-53

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    c = cgks.Context(flux_precision=1)
    yield c
    c.close()


@pytest.mark.parametrize("name", list(tp.MESHES))
def test_fine_residual_dword(ctx, name):
    rng = np.random.default_rng(8)
    m, om, W, G, w = tp.setup(ctx, 31, name, rng)
    dim, nv, n = m["dim"], m["dim"] + 2, len(W)
    R, Gn, al = np.zeros((n, nv)), np.zeros((n, nv, dim)), np.zeros(n)
    ctx.cgks_residual(31, 0, None, R, Gn, al)
    ro = om.residual(oracle.cfg_vector(dim, winf=w), W, G, np.ones(n))
    Fs = tp.flux_scale(W, dim)
    Smax = float(np.max(om.faces(0)["S"]))
    err = np.max(np.abs(R - ro["R"])) / (Fs * Smax)
    print(f"\n{name}: max residual error / (flux scale x max face) = {err:.2e}")
    np.testing.assert_allclose(R, ro["R"], rtol=0, atol=TOL * Fs * Smax)
    vol = om.cells(0)[0]
    np.testing.assert_allclose(Gn * vol[:, None, None], ro["grad"] * vol[:, None, None], rtol=0,
                               atol=TOL * np.max(np.abs(W)) * Smax)
    np.testing.assert_allclose(al, ro["alpha"], rtol=TOL, atol=32e-14)


@pytest.mark.parametrize("name,ncyc", [("vortex", 6), ("cylinder", 6), ("sphere", 3)])
def test_vcycle_dword(ctx, name, ncyc):
    rng = np.random.default_rng(11)
    m, om, W, G, w = tp.setup(ctx, 32, name, rng)
    dim, nv, n = m["dim"], m["dim"] + 2, len(W)
    norms = np.zeros((ncyc, nv, 2))
    ctx.cgks_vcycle([32], ncyc, 0, norms)
    Wd, ad = np.zeros_like(W), np.zeros(n)
    ctx.cgks_get_state(32, Wd, None, ad)
    out = om.vcycle(oracle.cfg_vector(dim, winf=w), W, G, np.ones(n), ncyc)
    np.testing.assert_allclose(norms, out["norms"], rtol=1e-8)
    np.testing.assert_allclose(Wd, out["W"], rtol=0, atol=1e-9 * np.max(np.abs(W)))
    np.testing.assert_allclose(ad, out["alpha"], rtol=0, atol=1e-8)


def test_fullsize_cylinder_residual_dword(ctx):
    m = synth.cylinder_mesh(64, 32, 1.05, n_refine=2)
    w = synth.freestream(5.0)
    rng = np.random.default_rng(2509063470 + 1)
    W, G = smooth_physical_state(rng, m, w)
    n = len(W)
    ctx.setup(33, m, w, W, G)
    R, Gn, al = np.zeros((n, 4)), np.zeros((n, 4, 2)), np.zeros(n)
    ctx.cgks_residual(33, 0, None, R, Gn, al)
    om = oracle.OracleMesh(m, levels=1)
    ro = om.residual(oracle.cfg_vector(2, winf=w), W, G, np.ones(n))
    Fs = tp.flux_scale(W, 2)
    Smax = float(np.max(om.faces(0)["S"]))
    print(f"\ncylinder, every cell: max residual error / (flux scale x max face) = "
          f"{np.max(np.abs(R - ro['R'])) / (Fs * Smax):.2e}, max DF error {np.max(np.abs(al - ro['alpha'])):.2e}")
    np.testing.assert_allclose(R, ro["R"], rtol=0, atol=TOL * Fs * Smax)
    np.testing.assert_allclose(al, ro["alpha"], rtol=TOL, atol=32e-14)


def test_fullsize_sphere_residual_sampled_dword(ctx):
    from helpers import ring_submesh
    m = synth.sphere_mesh(32, 32, 1.08)
    w = synth.freestream(6.0, dim=3)
    rng = np.random.default_rng(2509063470 + 2)
    W, G = smooth_physical_state(rng, m, w)
    n = len(W)
    ctx.setup(34, m, w, W, G)
    R, Gn, al = np.zeros((n, 5)), np.zeros((n, 5, 3)), np.zeros(n)
    ctx.cgks_residual(34, 0, None, R, Gn, al)
    seeds = np.unique(rng.choice(n, 40, replace=False))
    sub, cells, sp = ring_submesh(m, seeds, rings=3)
    om = oracle.OracleMesh(sub, levels=1)
    ro = om.residual(oracle.cfg_vector(3, winf=w), W[cells], G[cells], np.ones(len(cells)))
    Fs = tp.flux_scale(W, 3)
    Smax = float(np.max(om.faces(0)["S"]))
    print(f"\nsphere, sampled cells: max residual error / (flux scale x max face) = "
          f"{np.max(np.abs(R[seeds] - ro['R'][sp])) / (Fs * Smax):.2e}")
    np.testing.assert_allclose(R[seeds], ro["R"][sp], rtol=0, atol=TOL * Fs * Smax)
    np.testing.assert_allclose(al[seeds], ro["alpha"][sp], rtol=TOL, atol=32e-14)


def test_dword_arithmetic_error_bounds(ctx):
    """The double-word operations against extended-precision references on the
    same split inputs (x = hi + lo, the float32 split of each double), within
    small multiples of u^2 = 2^-48: sum and difference normwise, product,
    quotient and root relative; exp and erfc relative with the FP64 function's
    own error added, and an absolute 2^-149 where the result leaves the float
    range."""
    rng = np.random.default_rng(17)
    n = 20000
    a = 10.0 ** rng.uniform(-6, 6, n)
    b = 10.0 ** rng.uniform(-6, 6, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    # include cancellation and exact cases
    b[:500] = -a[:500] * (1 + 1e-9 * rng.standard_normal(500))
    b[500:600] = 1.0
    out = ctx.cgks_dword_selftest(a, b)

    def split(v):
        hi = v.astype(np.float32)
        lo = (v - hi.astype(np.float64)).astype(np.float32)
        return hi.astype(np.longdouble) + lo.astype(np.longdouble)

    x, y = split(a), split(b)
    u2 = np.longdouble(2.0) ** -48
    got = out.astype(np.longdouble)
    np.testing.assert_array_less(np.abs(got[:, 0] - (x + y)), 4 * u2 * (np.abs(x) + np.abs(y)))
    np.testing.assert_array_less(np.abs(got[:, 1] - (x - y)), 4 * u2 * (np.abs(x) + np.abs(y)))
    np.testing.assert_array_less(np.abs(got[:, 2] - x * y), 8 * u2 * np.abs(x * y))
    np.testing.assert_array_less(np.abs(got[:, 3] - x / y), 16 * u2 * np.abs(x / y))
    np.testing.assert_array_less(np.abs(got[:, 4] - np.sqrt(x)), 8 * u2 * np.sqrt(x))
    # results below the float range keep an absolute error under the smallest
    # float subnormal, 2^-149
    tiny = np.longdouble(2.0) ** -149
    ex = np.exp(-x)
    np.testing.assert_array_less(np.abs(got[:, 5] - ex), 8 * u2 * ex + tiny)
    import math
    ec = np.array([math.erfc(float(t)) for t in y], dtype=np.longdouble)
    np.testing.assert_array_less(np.abs(got[:, 6] - ec), 8 * u2 * ec + 4e-16 * ec + tiny)
