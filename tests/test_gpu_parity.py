"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances: FP64 results within 1e-12 relative to the
natural scale of each quantity (flux magnitude for residuals), colourings and
sizes bit-exact."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth
from helpers import GAMMA, physical_quadratic_state

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


def meshes():
    return {
        "vortex": synth.vortex_mesh(n_coarse=8, n_refine=2),
        "cylinder": synth.cylinder_mesh(n_theta=16, n_r=8, n_refine=2),
        "sphere": synth.sphere_mesh(n_panel=4, n_r=4),
    }


MESHES = meshes()


def flux_scale(W, dim):
    u = W[:, 1:1 + dim] / W[:, :1]
    p = (GAMMA - 1) * (W[:, -1] - 0.5 * W[:, 0] * np.sum(u * u, 1))
    c = np.sqrt(GAMMA * p / W[:, 0])
    return float(np.max((np.abs(W[:, -1]) + p) * (np.linalg.norm(u, axis=1) + c)))


def perturbed_states(w, n, dim, rng):
    """Physical states near w: density, velocity and pressure perturbed."""
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


def state_for(name, m, rng):
    dim = m["dim"]
    if name == "vortex":
        W, G = synth.vortex_state(m)
        W = W.copy()
        W[:, 1] += 0.3 * W[:, 0]
        W[:, 3] += 0.5 * 0.09 * W[:, 0]
        w = np.array([1.0, 0.3, 0.0, 1.0 / (GAMMA * (GAMMA - 1)) + 0.045])
        return W, G, w
    w = synth.freestream(3.0 if name == "cylinder" else 2.0, dim=dim, angle_deg=10.0)
    Wq, Gq, _, _ = physical_quadratic_state(rng, dim, m["cell_xyz"], scale=0.05)
    W = synth.uniform_state(m, w) + Wq - Wq.mean(0)
    return W, Gq, w


def setup(ctx, mid, name, rng, levels=None):
    m = MESHES[name]
    W, G, w = state_for(name, m, rng)
    ctx.setup(mid, m, w, W, G, levels=levels)
    om = oracle.OracleMesh(m, levels=levels)
    return m, om, W, G, w


@pytest.mark.parametrize("dim", [2, 3])
def test_gks_point_flux(ctx, dim):
    """The device gas-kinetic flux, point value and DF factor at random
    interface states against the oracle's polynomial-moment evaluation."""
    rng = np.random.default_rng(100 + dim)
    n, nv = 400, dim + 2
    Wl = np.zeros((n, nv))
    Wr = np.zeros((n, nv))
    for W in (Wl, Wr):
        rho = rng.uniform(0.3, 3.0, n)
        u = rng.uniform(-3.0, 3.0, (n, dim))
        p = rng.uniform(0.2, 5.0, n)
        W[:, 0] = rho
        W[:, 1:1 + dim] = rho[:, None] * u
        W[:, -1] = p / (GAMMA - 1) + 0.5 * rho * np.sum(u * u, 1)
    # a few interfaces separating into vacuum (collisionless fallback)
    for i in range(0, 40, 4):
        rho, p = 10 ** rng.uniform(-4, -1), 10 ** rng.uniform(-5, -2)
        u = np.zeros(dim)
        u[0] = -rng.uniform(3.0, 8.0) * np.sqrt(GAMMA * p / rho)
        Wl[i] = np.concatenate([[rho], rho * u, [p / (GAMMA - 1) + 0.5 * rho * u @ u]])
        Wr[i] = Wl[i].copy()
        Wr[i, 1] = -Wl[i, 1]
    Gl = rng.standard_normal((n, dim, nv))
    Gr = rng.standard_normal((n, dim, nv))
    Gl[0:40:4] = 0.0  # the separating pairs carry no slopes
    Gr[0:40:4] = 0.0
    dt = 10 ** rng.uniform(-3, 0, n)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    F, Wt, al = (torch.zeros((n, nv), dtype=torch.float64, device="cuda"),
                 torch.zeros((n, nv), dtype=torch.float64, device="cuda"),
                 torch.zeros(n, dtype=torch.float64, device="cuda"))
    ctx.cgks_gks_points(dim, dev(Wl), dev(Gl), dev(Wr), dev(Gr), dev(dt), F, Wt, al)
    ctx.cgks_synchronize()
    F, Wt, al = F.cpu().numpy(), Wt.cpu().numpy(), al.cpu().numpy()
    cfg = oracle.cfg_vector(dim)
    for i in range(n):
        Fo, Wo, _ = oracle.gks_point(dim, cfg, Wl[i], Gl[i], Wr[i], Gr[i], dt[i])
        # the flux is a difference of O(|W| (|u| + c)) terms: scale by the states
        sF = max(flux_scale(np.stack([Wl[i], Wr[i]]), dim), np.max(np.abs(Fo)))
        sW = max(np.max(np.abs(Wl[i])), np.max(np.abs(Wr[i])))
        assert np.max(np.abs(F[i] - Fo)) <= 1e-12 * sF, (i, F[i], Fo)
        assert np.max(np.abs(Wt[i] - Wo)) <= 1e-12 * sW, (i, Wt[i], Wo)
        assert abs(al[i] - oracle.df_point(dim, GAMMA, Wl[i], Wr[i])) <= 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_kfvs_point_flux(ctx, dim):
    rng = np.random.default_rng(200 + dim)
    n, nv = 300, dim + 2
    W = []
    for _ in range(2):
        rho = rng.uniform(0.3, 3.0, n)
        u = rng.uniform(-4.0, 4.0, (n, dim))
        p = rng.uniform(0.2, 5.0, n)
        A = np.zeros((n, nv))
        A[:, 0] = rho
        A[:, 1:1 + dim] = rho[:, None] * u
        A[:, -1] = p / (GAMMA - 1) + 0.5 * rho * np.sum(u * u, 1)
        W.append(A)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    F = torch.zeros((n, nv), dtype=torch.float64, device="cuda")
    ctx.cgks_kfvs_points(dim, dev(W[0]), dev(W[1]), F)
    ctx.cgks_synchronize()
    F = F.cpu().numpy()
    for i in range(n):
        Fo = oracle.kfvs_point(dim, GAMMA, W[0][i], W[1][i])
        assert np.max(np.abs(F[i] - Fo)) <= 1e-12 * flux_scale(np.stack([W[0][i], W[1][i]]), dim)


@pytest.mark.parametrize("name", list(MESHES))
def test_hierarchy_and_coloring_bit_exact(ctx, name):
    """Level sizes, face counts and every level's colouring equal the oracle's."""
    m = MESHES[name]
    mid = 10 + list(MESHES).index(name)
    ctx.cgks_upload_mesh(mid, m)
    ctx.cgks_upload_hierarchy(mid, m["parents"])
    info = ctx.cgks_mesh_info(mid)
    om = oracle.OracleMesh(m)
    assert len(info) == om.n_levels
    for l, lv in enumerate(info):
        assert lv["cells"] == om.n_cells(l)
        assert lv["faces"] == len(om.faces(l)["S"])
        assert lv["colors"] == om.n_colors(l)
        colors = om.colors(l)
        np.testing.assert_array_equal(ctx.cgks_get_coloring(mid, l, lv["cells"]), colors)
        # stored order: colour-major, original order within a colour; parents as uploaded
        last = l == len(info) - 1
        order, parent = ctx.cgks_get_hierarchy(mid, l, lv["cells"], with_parent=not last)
        np.testing.assert_array_equal(order, np.argsort(colors, kind="stable"))
        if not last:
            np.testing.assert_array_equal(parent, np.asarray(m["parents"][l]))


@pytest.mark.parametrize("name", list(MESHES))
def test_reconstruction(ctx, name):
    """Reconstructed polynomials and local time steps (Sec 3)."""
    rng = np.random.default_rng(7)
    m, om, W, G, w = setup(ctx, 20, name, rng)
    dim, nv, n = m["dim"], m["dim"] + 2, len(W)
    nc = 6 if dim == 2 else 10
    coef, dte, dti = np.zeros((n, nv, nc)), np.zeros(n), np.zeros(n)
    ctx.cgks_reconstruct(20, coef, dte, dti)
    cfg = oracle.cfg_vector(dim, winf=w)
    Po, _ = om.reconstruct(cfg, W, G, np.ones(n))
    de, di = om.time_steps(cfg, W)
    np.testing.assert_allclose(dte, de, rtol=1e-13)
    np.testing.assert_allclose(dti, di, rtol=1e-13)
    # compare polynomial values/gradients at cell-scale offsets, relative to |W|
    h = (om.cells(0)[0] ** (1.0 / dim))[:, None]
    scale = np.max(np.abs(W), axis=0)
    np.testing.assert_allclose(coef[:, :, 0], Po[:, :, 0], rtol=0, atol=1e-12 * scale.max())
    np.testing.assert_allclose(coef[:, :, 1:1 + dim] * h[:, None], Po[:, :, 1:1 + dim] * h[:, None],
                               rtol=0, atol=1e-11 * scale.max())
    np.testing.assert_allclose(coef[:, :, 1 + dim:] * h[:, None] ** 2, Po[:, :, 1 + dim:] * h[:, None] ** 2,
                               rtol=0, atol=1e-11 * scale.max())


@pytest.mark.parametrize("name", list(MESHES))
def test_fine_residual(ctx, name):
    """Residual R_i, evolved slopes and DF factors of the third-order scheme."""
    rng = np.random.default_rng(8)
    m, om, W, G, w = setup(ctx, 21, name, rng)
    dim, nv, n = m["dim"], m["dim"] + 2, len(W)
    R, Gn, al = np.zeros((n, nv)), np.zeros((n, nv, dim)), np.zeros(n)
    ctx.cgks_residual(21, 0, None, R, Gn, al)
    ro = om.residual(oracle.cfg_vector(dim, winf=w), W, G, np.ones(n))
    Fs = flux_scale(W, dim)
    Smax = float(np.max(om.faces(0)["S"]))
    np.testing.assert_allclose(R, ro["R"], rtol=0, atol=1e-12 * Fs * Smax)
    vol = om.cells(0)[0]
    np.testing.assert_allclose(Gn * vol[:, None, None], ro["grad"] * vol[:, None, None], rtol=0,
                               atol=1e-12 * np.max(np.abs(W)) * Smax)
    np.testing.assert_allclose(al, ro["alpha"], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("lev", [1, 2])
def test_coarse_kfvs_residual(ctx, name, lev):
    rng = np.random.default_rng(9)
    m, om, W, G, w = setup(ctx, 22, name, rng)
    dim, nv = m["dim"], m["dim"] + 2
    nl = om.n_cells(lev)
    Wc = perturbed_states(w, nl, dim, rng)
    R = np.zeros((nl, nv))
    ctx.cgks_residual(22, lev, Wc, R)
    Ro = om.kfvs_residual(oracle.cfg_vector(dim, winf=w), Wc, lev)
    Fs = flux_scale(Wc, dim)
    Smax = float(np.max(om.faces(lev)["S"]))
    np.testing.assert_allclose(R, Ro, rtol=0, atol=1e-12 * Fs * Smax)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("lev", [0, 1])
def test_lusgs_step(ctx, name, lev):
    """One DF-relaxed multi-colour LU-SGS step (FP64) and its FP32 version."""
    rng = np.random.default_rng(10)
    m, om, W, G, w = setup(ctx, 23, name, rng)
    dim, nv = m["dim"], m["dim"] + 2
    nl = om.n_cells(lev)
    Wl = perturbed_states(w, nl, dim, rng)
    cfg = oracle.cfg_vector(dim, winf=w)
    dte, dti = om.time_steps(cfg, Wl, lev)
    alpha = rng.uniform(0.0, 1.0, nl)
    rhs = 1e-2 * rng.standard_normal((nl, nv)) * (om.cells(lev)[0] / dte)[:, None] * np.max(np.abs(w))
    Wo, dWo = om.lusgs(cfg, Wl, rhs, alpha, dte, dti, lev)
    for mode, tol in ((0, 1e-12), (1, 2e-5)):
        Wg, dWg = Wl.copy(), np.zeros((nl, nv))
        ctx.cgks_lusgs(23, lev, mode, Wg, rhs, alpha, dte, dti, dWg)
        sc = np.max(np.abs(dWo))
        np.testing.assert_allclose(dWg, dWo, rtol=0, atol=tol * sc)
        np.testing.assert_allclose(Wg, Wo, rtol=0, atol=tol * sc + 1e-15 * np.max(np.abs(Wl)))


def test_freestream_preserved_on_device(ctx):
    m = MESHES["vortex"]
    w = np.array([1.1, 0.44, -0.33, 2.0])
    W = synth.uniform_state(m, w)
    ctx.setup(24, m, w, W)
    n = len(W)
    R, al = np.zeros((n, 4)), np.zeros(n)
    ctx.cgks_residual(24, 0, None, R, None, al)
    assert np.max(np.abs(R)) < 1e-13 * 10.0
    assert np.all(al == 1.0)
    norms = np.zeros((2, 4, 2))
    ctx.cgks_vcycle([24], 2, 0, norms)
    Wd = np.zeros_like(W)
    ctx.cgks_get_state(24, Wd)
    np.testing.assert_allclose(Wd, W, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("name,ncyc", [("vortex", 6), ("cylinder", 6), ("sphere", 3)])
def test_vcycle_matches_oracle(ctx, name, ncyc):
    """Whole V-cycles (plain FP64): state and per-cycle residual norms."""
    rng = np.random.default_rng(11)
    m, om, W, G, w = setup(ctx, 25, name, rng)
    dim, nv, n = m["dim"], m["dim"] + 2, len(W)
    norms = np.zeros((ncyc, nv, 2))
    ctx.cgks_vcycle([25], ncyc, 0, norms)
    Wd, Gd, ad = np.zeros_like(W), np.zeros((n, nv, dim)), np.zeros(n)
    ctx.cgks_get_state(25, Wd, Gd, ad)
    out = om.vcycle(oracle.cfg_vector(dim, winf=w), W, G, np.ones(n), ncyc)
    np.testing.assert_allclose(norms, out["norms"], rtol=1e-8)
    np.testing.assert_allclose(Wd, out["W"], rtol=0, atol=1e-9 * np.max(np.abs(W)))
    np.testing.assert_allclose(ad, out["alpha"], rtol=0, atol=1e-8)
    c = ctx.cgks_counters(25)
    assert int(c[3]) == 0


@pytest.mark.parametrize("name", ["vortex", "cylinder", "sphere"])
def test_mixed_vcycle_error_against_oracle(ctx, name):
    """MIXED V-cycles (FP32 LU-SGS sweeps as a defect correction; FP64
    residuals, DF factor and state) against the FP64 oracle: the FP32 sweeps
    give each increment a relative error of order 1e-6, so after three cycles
    the state agrees to 1e-5 of its scale and the residual norms to 1e-3
    relative."""
    from paper_2509_06347_b300 import cgks
    rng = np.random.default_rng(11)
    m, om, W, G, w = setup(ctx, 26, name, rng)
    dim, nv, n = m["dim"], m["dim"] + 2, len(W)
    ncyc = 3
    norms = np.zeros((ncyc, nv, 2))
    ctx.cgks_vcycle([26], ncyc, cgks.MIXED, norms)
    Wd = np.zeros_like(W)
    ctx.cgks_get_state(26, Wd)
    out = om.vcycle(oracle.cfg_vector(dim, winf=w), W, G, np.ones(n), ncyc)
    scale = np.max(np.abs(W), axis=0)
    err = np.max(np.abs(Wd - out["W"]) / scale)
    moved = np.max(np.abs(out["W"] - W) / scale)
    print(f"\n{name}: MIXED state error {err:.2e} (state moved {moved:.2e})")
    assert err <= 1e-5
    np.testing.assert_allclose(norms, out["norms"], rtol=1e-3)


SWITCHES = {
    "fully_implicit": (dict(df_relax=0), dict(relax=1.0)),
    "fixed_factor_0.5": (dict(df_relax=2, relax_beta=0.5), dict(relax=0.5)),
    "plain_injection": (dict(df_prolong=0), dict(df_prolong=0)),
    "explicit_fine_smoother": (dict(fine_smoother=1), dict(fine_smoother=1)),
    "relaxed_slopes_and_df": (dict(slope_relax=0.5, alpha_relax=0.3), dict(slope_relax=0.5, alpha_relax=0.3)),
}


@pytest.mark.parametrize("switch", list(SWITCHES))
@pytest.mark.parametrize("name", ["vortex", "cylinder"])
def test_vcycle_switches_match_oracle(name, switch):
    """V-cycles (plain FP64) with the relaxation and prolongation switches of
    the ablations: LU-SGS relaxed by 1 or by a fixed factor instead of DF,
    plain injection instead of the DF-scaled prolongation, and the explicit
    fine smoother, and the pseudo-time under-relaxation of the slope update and
    of a rising DF factor; state, slopes, DF and norms against the oracle with
    the same switch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    lib_kw, ora_kw = SWITCHES[switch]
    c = cgks.Context(**lib_kw)
    try:
        m = MESHES[name]
        W, G, w = state_for(name, m, np.random.default_rng(13))
        c.setup(1, m, w, W, G)
        dim, nv, n = m["dim"], m["dim"] + 2, len(W)
        ncyc = 3
        norms = np.zeros((ncyc, nv, 2))
        c.cgks_vcycle([1], ncyc, cgks.PLAIN_FP64, norms)
        Wd, Gd, ad = np.zeros_like(W), np.zeros((n, nv, dim)), np.zeros(n)
        c.cgks_get_state(1, Wd, Gd, ad)
    finally:
        c.close()
    out = oracle.OracleMesh(m).vcycle(oracle.cfg_vector(dim, winf=w, **ora_kw), W, G, np.ones(n), ncyc)
    np.testing.assert_allclose(norms, out["norms"], rtol=1e-8)
    np.testing.assert_allclose(Wd, out["W"], rtol=0, atol=1e-9 * np.max(np.abs(W)))
    np.testing.assert_allclose(Gd, out["grad"], rtol=0, atol=1e-8 * np.max(np.abs(out["grad"])))
    np.testing.assert_allclose(ad, out["alpha"], rtol=0, atol=1e-8)
