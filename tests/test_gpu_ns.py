"""Navier-Stokes (Sec 2.1: tau = mu / p, Pr = 1; no-slip adiabatic walls;
the characteristic far field) through the C ABI against the oracle: the point
flux and point value at random interface states, the fine residual with its
slopes and DF factors on the cylinder and sphere meshes with their walls made
no-slip and either far field, and whole plain-FP64 V-cycles.  Tolerances as
for the Euler path (1e-12 of the flux scale; V-cycle norms 1e-8, states
1e-9)."""
import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth
import test_gpu_parity as tp
from helpers import GAMMA

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MU = 0.02


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    return cgks


def noslip(m, farfield=synth.TAG_FARFIELD):
    m = dict(m)
    t = np.asarray(m["bface_tag"]).copy()
    t[t == synth.TAG_FARFIELD] = farfield
    t[t == synth.TAG_WALL] = synth.TAG_NOSLIP_WALL
    m["bface_tag"] = t
    return m


@pytest.mark.parametrize("dim", [2, 3])
def test_ns_point_flux(cg, dim):
    rng = np.random.default_rng(200 + dim)
    n, nv = 300, dim + 2
    Wl, Wr = np.zeros((n, nv)), np.zeros((n, nv))
    for W in (Wl, Wr):
        rho = rng.uniform(0.3, 3.0, n)
        u = rng.uniform(-1.5, 1.5, (n, dim))
        p = rng.uniform(0.2, 5.0, n)
        W[:, 0] = rho
        W[:, 1:1 + dim] = rho[:, None] * u
        W[:, -1] = p / (GAMMA - 1) + 0.5 * rho * np.sum(u * u, 1)
    Gl, Gr = rng.standard_normal((n, dim, nv)), rng.standard_normal((n, dim, nv))
    dt = 10 ** rng.uniform(-3, 0, n)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    F, Wt, al = (torch.zeros((n, nv), dtype=torch.float64, device="cuda"),
                 torch.zeros((n, nv), dtype=torch.float64, device="cuda"),
                 torch.zeros(n, dtype=torch.float64, device="cuda"))
    ctx = cg.Context(mu=MU)
    try:
        ctx.cgks_gks_points(dim, dev(Wl), dev(Gl), dev(Wr), dev(Gr), dev(dt), F, Wt, al)
        ctx.cgks_synchronize()
    finally:
        ctx.close()
    F, Wt = F.cpu().numpy(), Wt.cpu().numpy()
    cfg = oracle.cfg_vector(dim, mu=MU)
    for i in range(n):
        Fo, Wo, _ = oracle.gks_point(dim, cfg, Wl[i], Gl[i], Wr[i], Gr[i], dt[i])
        sF = max(tp.flux_scale(np.stack([Wl[i], Wr[i]]), dim), np.max(np.abs(Fo)))
        sW = max(np.max(np.abs(Wl[i])), np.max(np.abs(Wr[i])))
        assert np.max(np.abs(F[i] - Fo)) <= 1e-12 * sF, (i, F[i], Fo)
        assert np.max(np.abs(Wt[i] - Wo)) <= 1e-12 * sW, (i, Wt[i], Wo)


@pytest.mark.parametrize("far", [synth.TAG_FARFIELD, synth.TAG_FARFIELD_RIEMANN])
@pytest.mark.parametrize("name", ["cylinder", "sphere"])
def test_ns_residual_noslip(cg, name, far):
    m = noslip(tp.MESHES[name], far)
    rng = np.random.default_rng(31)
    W, G, w = tp.state_for(name, m, rng)
    dim, nv, n = m["dim"], m["dim"] + 2, len(W)
    ctx = cg.Context(mu=MU)
    try:
        ctx.setup(1, m, w, W, G)
        R, Gn, al = np.zeros((n, nv)), np.zeros((n, nv, dim)), np.zeros(n)
        ctx.cgks_residual(1, 0, None, R, Gn, al)
    finally:
        ctx.close()
    om = oracle.OracleMesh(m)
    ro = om.residual(oracle.cfg_vector(dim, winf=w, mu=MU), W, G, np.ones(n))
    Smax = float(np.max(om.faces(0)["S"]))
    np.testing.assert_allclose(R, ro["R"], rtol=0, atol=1e-12 * tp.flux_scale(W, dim) * Smax)
    vol = om.cells(0)[0]
    np.testing.assert_allclose(Gn * vol[:, None, None], ro["grad"] * vol[:, None, None], rtol=0,
                               atol=1e-12 * np.max(np.abs(W)) * Smax)
    np.testing.assert_allclose(al, ro["alpha"], rtol=1e-12, atol=1e-14)
    # the viscous terms act: the residual differs from the inviscid one
    ri = om.residual(oracle.cfg_vector(dim, winf=w), W, G, np.ones(n))["R"]
    assert np.max(np.abs(ri - ro["R"])) > 1e-6 * np.max(np.abs(ro["R"]))


@pytest.mark.parametrize("far", [synth.TAG_FARFIELD, synth.TAG_FARFIELD_RIEMANN])
@pytest.mark.parametrize("name,ncyc", [("cylinder", 4), ("sphere", 2)])
def test_ns_vcycle_noslip(cg, name, ncyc, far):
    m = noslip(tp.MESHES[name], far)
    W, G, w = tp.state_for(name, m, np.random.default_rng(32))
    dim, nv, n = m["dim"], m["dim"] + 2, len(W)
    ctx = cg.Context(mu=MU)
    try:
        ctx.setup(1, m, w, W, G)
        norms = np.zeros((ncyc, nv, 2))
        ctx.cgks_vcycle([1], ncyc, cg.PLAIN_FP64, norms)
        Wd = np.zeros_like(W)
        ctx.cgks_get_state(1, Wd)
    finally:
        ctx.close()
    out = oracle.OracleMesh(m).vcycle(oracle.cfg_vector(dim, winf=w, mu=MU), W, G, np.ones(n), ncyc)
    np.testing.assert_allclose(norms, out["norms"], rtol=1e-8)
    np.testing.assert_allclose(Wd, out["W"], rtol=0, atol=1e-9 * np.max(np.abs(W)))


def test_mu_rejected_when_negative(cg):
    with pytest.raises(cg.CgksError):
        cg.Context(mu=-1.0)
