"""Pins of the oracle's reconstruction (Sec 3), residual (Sec 2.2-2.4),
LU-SGS (Sec 4.2-4.3) and multigrid transfer (Sec 5.2)."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth
from helpers import GAMMA, cell_average, physical_quadratic_state, small_meshes

MESHES = small_meshes()


def interior_cells(om):
    """Cells whose whole von Neumann stencil consists of real cells."""
    cnt, nb = om.neighbors(0)
    return np.array([c for c in range(len(cnt)) if np.all(nb[c, :cnt[c]] >= 0)])


def eval_poly(dim, coef, X):
    """P(X) = c0 + c_d X_d + sum_{d<=e} c_de X_d X_e, quadratic terms in the
    order xx, xy, yy (2-D) / xx, xy, xz, yy, yz, zz (3-D)."""
    out = coef[..., 0] + np.einsum("...d,...d->...", coef[..., 1:1 + dim], X)
    pairs = [(d, e) for d in range(dim) for e in range(d, dim)]
    for k, (d, e) in enumerate(pairs):
        out = out + coef[..., 1 + dim + k] * X[..., d] * X[..., e]
    return out


@pytest.mark.parametrize("name", ["cylinder", "sphere"])
def test_p2_reproduces_global_quadratics(name):
    """With the linear weight of the large stencil set to 1 the reconstruction is
    p2 alone, which must reproduce any global quadratic from its exact cell
    averages and mean slopes (Sec 3.1) on cells with a full real stencil."""
    m = MESHES[name]
    dim = m["dim"]
    om = oracle.OracleMesh(m, levels=1)
    rng = np.random.default_rng(21)
    W, G, q, dq = physical_quadratic_state(rng, dim, m["cell_xyz"])
    cfg = oracle.cfg_vector(dim, weno_gamma_high=1.0)
    P, nb = om.reconstruct(cfg, W, G, np.ones(len(W)))
    assert nb == 0
    _, cen, _ = om.cells(0)
    cells = interior_cells(om)
    # compare the polynomials at random points around each centroid
    pts = cen[cells][:, None, :] + 0.3 * rng.standard_normal((len(cells), 5, dim))
    X = pts - cen[cells][:, None, :]
    got = np.stack([eval_poly(dim, P[cells][:, None, v, :], X) for v in range(dim + 2)], -1)
    np.testing.assert_allclose(got, q(pts), rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("name", list(MESHES))
def test_constant_data_reconstructs_constant(name):
    m = MESHES[name]
    dim = m["dim"]
    om = oracle.OracleMesh(m, levels=1)
    w = np.zeros(dim + 2)
    w[0], w[-1] = 1.3, 2.7
    W = synth.uniform_state(m, w)
    cfg = oracle.cfg_vector(dim, winf=w)
    P, _ = om.reconstruct(cfg, W, np.zeros((len(W), dim + 2, dim)), np.ones(len(W)))
    np.testing.assert_allclose(P[:, :, 0], W, rtol=1e-14)
    assert np.max(np.abs(P[:, :, 1:])) < 1e-13


def test_flat_subs_stencil_wins():
    """With the sub-stencil gradient switched off (previous DF = 0), beta_1 = 0 and
    the nonlinear weights select the flat p1: P is the cell mean up to a
    relative O(eps / beta_2) share of p2."""
    m = MESHES["cylinder"]
    om = oracle.OracleMesh(m, levels=1)
    rng = np.random.default_rng(4)
    W, G, _, _ = physical_quadratic_state(rng, 2, m["cell_xyz"])
    n = len(W)
    P, _ = om.reconstruct(oracle.cfg_vector(2), W, G, np.zeros(n))
    P2, _ = om.reconstruct(oracle.cfg_vector(2, weno_gamma_high=1.0), W, G, np.zeros(n))
    np.testing.assert_allclose(P[:, :, 0], W, rtol=1e-6)
    assert np.max(np.abs(P[:, :, 1:])) < 1e-6 * np.max(np.abs(P2[:, :, 1:]))


def test_positivity_fallback_is_first_order():
    """On rough data every cell's polynomial either has positive density and
    pressure at all of the cell's face Gauss points or is the cell mean
    (reading R11), and the fallback is actually taken somewhere."""
    m = MESHES["cylinder"]
    om = oracle.OracleMesh(m, levels=1)
    n = m["cell_nodes"].shape[0]
    rng = np.random.default_rng(30)
    rho = np.where(rng.random(n) < 0.5, 1e-3, 1.0)
    p = np.where(rng.random(n) < 0.5, 1e-3, 1.0)
    W = np.stack([rho, 0.1 * rho, -0.2 * rho, p / (GAMMA - 1) + 0.5 * rho * 0.05], -1)
    P, nb = om.reconstruct(oracle.cfg_vector(2, weno_gamma_high=1.0), W, np.zeros((n, 4, 2)), np.ones(n))
    assert nb >= 1
    f = om.faces(0)
    _, cen, _ = om.cells(0)
    const = np.all(P[:, :, 1:] == 0.0, axis=(1, 2)) & np.all(P[:, :, 0] == W, axis=1)
    for side, sgn in (("L", 0.0), ("R", 1.0)):
        idx = f[side]
        ok = idx >= 0
        pts = f["gp"][ok, :2] - sgn * f["shift"][ok][:, None, :]
        X = pts - cen[idx[ok]][:, None, :]
        vals = np.stack([eval_poly(2, P[idx[ok]][:, None, v, :], X) for v in range(4)], -1)
        pr = (GAMMA - 1) * (vals[..., 3] - 0.5 * (vals[..., 1] ** 2 + vals[..., 2] ** 2) / vals[..., 0])
        good = (vals[..., 0] > 0).all(1) & (pr > 0).all(1)
        assert np.all(good | const[idx[ok]])


def test_freestream_preservation_periodic():
    """A uniform moving state on the jittered periodic mesh: R = 0, new slopes 0,
    DF = 1 (no discontinuity), up to round-off."""
    m = MESHES["vortex"]
    om = oracle.OracleMesh(m, levels=1)
    w = np.array([1.1, 1.1 * 0.4, 1.1 * -0.3, 2.0])
    W = synth.uniform_state(m, w)
    n = len(W)
    r = om.residual(oracle.cfg_vector(2), W, np.zeros((n, 4, 2)), np.ones(n))
    f = om.faces(0)
    scale = np.max(f["S"]) * np.max(np.abs(w)) * 3.0
    assert np.max(np.abs(r["R"])) < 1e-13 * scale
    assert np.max(np.abs(r["grad"])) < 1e-12
    assert np.all(r["alpha"] == 1.0)


@pytest.mark.parametrize("name", ["cylinder", "sphere"])
def test_freestream_preservation_farfield(name):
    """The free stream on a mesh whose every boundary is far field."""
    m = dict(MESHES[name])
    m["bface_tag"] = np.full_like(m["bface_tag"], synth.TAG_FARFIELD)
    dim = m["dim"]
    om = oracle.OracleMesh(m, levels=1)
    w = synth.freestream(3.0, dim=dim, angle_deg=20.0)
    W = synth.uniform_state(m, w)
    n = len(W)
    r = om.residual(oracle.cfg_vector(dim, winf=w), W, np.zeros((n, dim + 2, dim)), np.ones(n))
    f = om.faces(0)
    assert np.max(np.abs(r["R"])) < 1e-13 * np.max(f["S"]) * 20.0
    assert np.max(np.abs(r["grad"])) < 1e-11


def test_periodic_conservation():
    """On the periodic mesh every face flux enters one cell and leaves another:
    sum_i R_i = 0 for a non-trivial state."""
    m = MESHES["vortex"]
    om = oracle.OracleMesh(m, levels=1)
    W, G = synth.vortex_state(m)
    W[:, 1] += 0.5 * W[:, 0]
    n = len(W)
    r = om.residual(oracle.cfg_vector(2), W, G, np.ones(n))
    tot = np.abs(r["R"]).sum(axis=0)
    assert np.all(np.abs(r["R"].sum(axis=0)) < 1e-13 * tot)
    assert np.all(r["alpha"] > 0) and np.all(r["alpha"] <= 1)


def test_time_steps_closed_form():
    """dt_i = CFL V_i / sum_f S_f (|u.n| + c) (reading R12)."""
    m = MESHES["sphere"]
    om = oracle.OracleMesh(m, levels=1)
    rng = np.random.default_rng(2)
    W, _, _, _ = physical_quadratic_state(rng, 3, m["cell_xyz"])
    dte, dti = om.time_steps(oracle.cfg_vector(3), W)
    vol, _, _ = om.cells(0)
    f = om.faces(0)
    acc = np.zeros(len(W))
    u = W[:, 1:4] / W[:, :1]
    p = (GAMMA - 1) * (W[:, 4] - 0.5 * W[:, 0] * np.sum(u * u, 1))
    c = np.sqrt(GAMMA * p / W[:, 0])
    for side in ("L", "R"):
        idx = f[side]
        ok = idx >= 0
        np.add.at(acc, idx[ok], f["S"][ok] * (np.abs(np.sum(u[idx[ok]] * f["n"][ok], 1)) + c[idx[ok]]))
    np.testing.assert_allclose(dte, 0.5 * vol / acc, rtol=1e-13)
    np.testing.assert_allclose(dti, 10.0 * vol / acc, rtol=1e-13)


def euler_jacobian(dim, W, n, gamma=GAMMA):
    """Textbook Jacobian dT/dW of the Euler flux T(W).n (conservative variables)."""
    rho = W[0]
    u = W[1:1 + dim] / rho
    E = W[-1]
    q2 = u @ u
    un = u @ n
    g1 = gamma - 1
    H = (E + g1 * (E - 0.5 * rho * q2)) / rho
    A = np.zeros((dim + 2, dim + 2))
    A[0, 1:1 + dim] = n
    for i in range(dim):
        A[1 + i, 0] = 0.5 * g1 * q2 * n[i] - u[i] * un
        for j in range(dim):
            A[1 + i, 1 + j] = u[i] * n[j] - g1 * u[j] * n[i] + (un if i == j else 0.0)
        A[1 + i, -1] = g1 * n[i]
    A[-1, 0] = un * (0.5 * g1 * q2 - H)
    A[-1, 1:1 + dim] = H * n - g1 * un * u
    A[-1, -1] = gamma * un
    return A


@pytest.mark.parametrize("dim", [2, 3])
def test_euler_jacobian_matches_flux(dim):
    rng = np.random.default_rng(1)
    W = np.concatenate([[1.2], rng.uniform(-0.5, 0.5, dim), [3.0]])
    n = rng.standard_normal(dim)
    n /= np.linalg.norm(n)
    A = euler_jacobian(dim, W, n)
    h = 1e-6
    for k in range(dim + 2):
        e = np.zeros(dim + 2)
        e[k] = h
        fd = (oracle.euler_flux(dim, GAMMA, W + e, n) - oracle.euler_flux(dim, GAMMA, W - e, n)) / (2 * h)
        np.testing.assert_allclose(A[:, k], fd, rtol=1e-7, atol=1e-8)


def lusgs_dense_operator(om, cfg, W, alpha, dte, dti, lev=0):
    """Dense (D+L) D^-1 (D+U) of the multi-colour LU-SGS with DF relaxation:
    D_i = alpha_i (V/dt_imp + 1/2 sum S r) + (1-alpha_i) V/dt_exp on the
    diagonal, 1/2 alpha_i S_ij (A_n(W_j) - r_ij I) for colour(j) < colour(i)
    in L and colour(j) > colour(i) in U."""
    dim, nv = om.dim, om.nv
    n = om.n_cells(lev)
    vol, _, _ = om.cells(lev)
    f = om.faces(lev)
    col = om.colors(lev)
    winf = cfg[9:9 + nv]

    def ghost(Wi, nn, tag):
        if tag == 1:
            g = Wi.copy()
            g[1:1 + dim] -= 2 * (Wi[1:1 + dim] @ nn) * nn
            return g
        if winf[1:1 + dim] @ nn < 0:
            return winf.copy()
        return Wi.copy()

    def radius(Wi, Wj, nn):
        mW = 0.5 * (Wi + Wj)
        u = mW[1:1 + dim] / mW[0]
        p = (GAMMA - 1) * (mW[-1] - 0.5 * mW[0] * u @ u)
        return abs(u @ nn) + math.sqrt(GAMMA * p / mW[0])

    Dg = np.zeros(n)
    Lm = np.zeros((n * nv, n * nv))
    Um = np.zeros((n * nv, n * nv))
    sr = np.zeros(n)
    for k in range(len(f["S"])):
        i, j, nn, S = f["L"][k], f["R"][k], f["n"][k], f["S"][k]
        if j < 0:
            sr[i] += S * radius(W[i], ghost(W[i], nn, f["tag"][k]), nn)
            continue
        r = radius(W[i], W[j], nn)
        sr[i] += S * r
        sr[j] += S * r
        for (a, b, nab) in ((i, j, nn), (j, i, -nn)):
            blk = 0.5 * alpha[a] * S * (euler_jacobian(dim, W[b], nab) - r * np.eye(nv))
            tgt = Lm if col[b] < col[a] else Um
            tgt[a * nv:(a + 1) * nv, b * nv:(b + 1) * nv] += blk
    Dg = alpha * (vol / dti + 0.5 * sr) + (1 - alpha) * vol / dte
    D = np.diag(np.repeat(Dg, nv))
    return D, Lm, Um


@pytest.mark.parametrize("name", ["cylinder3", "sphere2"])
def test_lusgs_matches_dense_factorisation(name):
    """The matrix-free sweeps equal (D+U)^-1 D (D+L)^-1 b up to O(|b|^2), the
    nonlinearity of dT; the defect shrinks ~100x when b shrinks 10x."""
    if name == "cylinder3":
        m = synth.cylinder_mesh(n_theta=6, n_r=2, n_refine=0)
    else:
        m = synth.sphere_mesh(n_panel=2, n_r=2)
    dim = m["dim"]
    om = oracle.OracleMesh(m, levels=1)
    rng = np.random.default_rng(8)
    n = om.n_cells(0)
    nv = dim + 2
    w = synth.freestream(2.0, dim=dim, angle_deg=10.0)
    W = synth.uniform_state(m, w) * (1 + 0.1 * rng.random((n, 1)))
    W[:, 1:1 + dim] += 0.2 * rng.standard_normal((n, dim))
    cfg = oracle.cfg_vector(dim, winf=w)
    alpha = rng.uniform(0.2, 1.0, n)
    dte, dti = om.time_steps(cfg, W)
    D, Lm, Um = lusgs_dense_operator(om, cfg, W, alpha, dte, dti)
    b0 = rng.standard_normal((n, nv))
    errs = []
    for eps in (1e-4, 1e-5):
        b = eps * b0
        _, dW = om.lusgs(cfg, W, b, alpha, dte, dti)
        ref = np.linalg.solve(D + Um, D @ np.linalg.solve(D + Lm, b.reshape(-1)))
        errs.append((np.max(np.abs(dW.reshape(-1) - ref)), np.max(np.abs(ref))))
    # relative defect O(|b|), absolute defect O(|b|^2)
    assert errs[0][0] / errs[0][1] < 1e-5
    assert 50 < errs[0][0] / errs[1][0] < 200


def test_lusgs_alpha_zero_is_explicit():
    """alpha = 0 reverts to the explicit update dW = -R dt_exp / V (remark, Sec 4.3)."""
    m = MESHES["cylinder"]
    om = oracle.OracleMesh(m, levels=1)
    n = om.n_cells(0)
    rng = np.random.default_rng(3)
    w = synth.freestream(2.0)
    W = synth.uniform_state(m, w) * (1 + 0.05 * rng.random((n, 1)))
    cfg = oracle.cfg_vector(2, winf=w)
    dte, dti = om.time_steps(cfg, W)
    R = 1e-3 * rng.standard_normal((n, 4))
    vol, _, _ = om.cells(0)
    _, dW = om.lusgs(cfg, W, -R, np.zeros(n), dte, dti)
    np.testing.assert_allclose(dW, -R * (dte / vol)[:, None], rtol=1e-14, atol=1e-18)


def test_fas_zero_forcing_leaves_coarse_state():
    """If the restricted fine residual is zero, the coarse problem is solved by
    the restricted state itself: the FAS-consistent sign (reading R18) gives a
    zero coarse correction; the literal sign would not."""
    m = MESHES["cylinder"]
    om = oracle.OracleMesh(m)
    rng = np.random.default_rng(6)
    n1 = om.n_cells(1)
    w = synth.freestream(3.0)
    W0 = np.tile(w, (n1, 1)) * (1 + 0.1 * rng.random((n1, 1)))
    W0[:, 2] += 0.3 * rng.standard_normal(n1)
    cfg = oracle.cfg_vector(2, winf=w)
    W = om.coarse_solve(cfg, 1, W0, np.zeros_like(W0), rng.uniform(0.5, 1, n1))
    assert np.array_equal(W, W0)
    # and a non-zero forcing does move it
    W2 = om.coarse_solve(cfg, 1, W0, 1e-3 * rng.standard_normal(W0.shape), np.ones(n1))
    assert np.max(np.abs(W2 - W0)) > 0


def test_restriction_and_prolongation():
    """Volume-weighted restriction keeps a uniform state; the residual
    restriction is a plain sum; DF = 0 prolongation is the identity and DF = 1
    adds the coarse correction by injection (Eq. prolongation)."""
    m = MESHES["vortex"]
    om = oracle.OracleMesh(m)
    rng = np.random.default_rng(12)
    n0, n1 = om.n_cells(0), om.n_cells(1)
    w = np.array([1.0, 0.2, 0.1, 2.6])
    Wc, ac, Rc = om.restrict(0, np.tile(w, (n0, 1)), rng.random(n0), rng.standard_normal((n0, 4)))
    np.testing.assert_allclose(Wc, np.tile(w, (n1, 1)), rtol=1e-15)
    Rf = rng.standard_normal((n0, 4))
    af = rng.random(n0)
    _, ac, Rc = om.restrict(0, np.tile(w, (n0, 1)), af, Rf)
    par = m["parents"][0]
    for v in range(4):
        np.testing.assert_allclose(Rc[:, v], np.bincount(par, weights=Rf[:, v], minlength=n1), rtol=1e-14)
    np.testing.assert_array_equal(ac, [af[par == I].min() for I in range(n1)])
    Wf = np.tile(w, (n0, 1))
    Wc1 = Wc + 1e-3 * rng.standard_normal(Wc.shape)
    cfg = oracle.cfg_vector(2)
    np.testing.assert_array_equal(om.prolong(cfg, 0, Wf, np.zeros(n0), Wc1, Wc), Wf)
    np.testing.assert_allclose(om.prolong(cfg, 0, Wf, np.ones(n0), Wc1, Wc), Wf + (Wc1 - Wc)[par], rtol=1e-15)


def test_vcycle_preserves_freestream():
    """One V-cycle leaves a uniform periodic state unchanged (to 1e-14)."""
    m = MESHES["vortex"]
    om = oracle.OracleMesh(m)
    w = np.array([1.0, 0.3, -0.2, 2.6])
    W = synth.uniform_state(m, w)
    n = len(W)
    out = om.vcycle(oracle.cfg_vector(2), W, np.zeros((n, 4, 2)), np.ones(n), 2)
    np.testing.assert_allclose(out["W"], W, rtol=1e-14, atol=1e-14)
    assert np.all(out["stats"] == 0)


@pytest.mark.parametrize("switch", [dict(), dict(relax=1.0), dict(relax=0.5), dict(df_prolong=0),
                                    dict(fine_smoother=1)])
def test_vcycle_is_its_steps(switch):
    """A two-level V-cycle equals its steps run one by one (Sec 5.2): the
    third-order residual with the DF slope update, the fine smoothing (an
    LU-SGS step relaxed by DF, by a constant for the fully implicit (1) and
    fixed-factor (0.5) schemes, or the explicit update of Eq. smo), the
    residual at the smoothed state, restriction, the coarse FAS solve relaxed
    the same way, and prolongation scaled by DF or plain injection."""
    m = MESHES["cylinder"]
    om = oracle.OracleMesh(m, levels=2)
    rng = np.random.default_rng(31)
    w = synth.freestream(2.0, angle_deg=10.0)
    Wq, Gq, _, _ = physical_quadratic_state(rng, 2, m["cell_xyz"], scale=0.05)
    W0 = synth.uniform_state(m, w) + Wq - Wq.mean(0)
    n = len(W0)
    a0 = rng.uniform(0.3, 1.0, n)
    cfg = oracle.cfg_vector(2, winf=w, **switch)
    out = om.vcycle(cfg, W0, Gq, a0, 1)

    relax = switch.get("relax", -1.0)
    r = om.residual(cfg, W0, Gq, a0)
    al = r["alpha"]
    G = al[:, None, None] * r["grad"]
    if switch.get("fine_smoother", 0) == 1:
        vol = om.cells(0)[0]
        W = W0 - (r["dt_exp"] / vol)[:, None] * r["R"]
    else:
        W, _ = om.lusgs(cfg, W0, -r["R"], al if relax < 0 else np.full(n, relax), r["dt_exp"], r["dt_imp"])
    r2 = om.residual(cfg, W, G, al)
    al = r2["alpha"]
    Wc0, ac, Rc = om.restrict(0, W, al, r2["R"])
    Wc = om.coarse_solve(cfg, 1, Wc0, Rc, ac if relax < 0 else np.full(len(ac), relax))
    W = om.prolong(cfg, 0, W, al if switch.get("df_prolong", 1) else np.ones(n), Wc, Wc0)
    np.testing.assert_allclose(out["W"], W, rtol=0, atol=1e-14 * np.max(np.abs(W0)))
    np.testing.assert_allclose(out["grad"], G, rtol=0, atol=1e-14 * np.max(np.abs(G)))
    np.testing.assert_allclose(out["alpha"], al, rtol=0, atol=1e-13)
    # the switches change the result
    if switch:
        base = om.vcycle(oracle.cfg_vector(2, winf=w), W0, Gq, a0, 1)
        assert np.max(np.abs(base["W"] - out["W"])) > 1e-10


def test_vcycle_relaxed_slopes_and_df_are_its_steps():
    """With pseudo-time under-relaxation of the slope update (slope_relax) and
    of a rise of the stored DF (alpha_relax), a two-level V-cycle equals its
    steps: the DF kept after each residual is the Gauss-point product where it
    does not exceed the kept value, else the kept value plus alpha_relax times
    the rise; the slopes move slope_relax of the way to DF times the evolved
    slopes.  A uniform state stays a fixed point."""
    m = MESHES["cylinder"]
    om = oracle.OracleMesh(m, levels=2)
    rng = np.random.default_rng(32)
    w = synth.freestream(2.0, angle_deg=10.0)
    Wq, Gq, _, _ = physical_quadratic_state(rng, 2, m["cell_xyz"], scale=0.05)
    W0 = synth.uniform_state(m, w) + Wq - Wq.mean(0)
    n = len(W0)
    a0 = rng.uniform(0.3, 1.0, n)
    ws, wa = 0.5, 0.3
    cfg = oracle.cfg_vector(2, winf=w, slope_relax=ws, alpha_relax=wa)
    out = om.vcycle(cfg, W0, Gq, a0, 1)

    def kept(prev, prod):
        return np.where(prod > prev, prev + wa * (prod - prev), prod)

    r = om.residual(cfg, W0, Gq, a0)
    al = kept(a0, r["alpha"])
    assert np.any(r["alpha"] > a0) and np.any(r["alpha"] < a0)  # both branches taken
    G = Gq + ws * (al[:, None, None] * r["grad"] - Gq)
    W, _ = om.lusgs(cfg, W0, -r["R"], al, r["dt_exp"], r["dt_imp"])
    r2 = om.residual(cfg, W, G, al)
    al = kept(al, r2["alpha"])
    Wc0, ac, Rc = om.restrict(0, W, al, r2["R"])
    Wc = om.coarse_solve(cfg, 1, Wc0, Rc, ac)
    W = om.prolong(cfg, 0, W, al, Wc, Wc0)
    np.testing.assert_allclose(out["W"], W, rtol=0, atol=1e-14 * np.max(np.abs(W0)))
    np.testing.assert_allclose(out["grad"], G, rtol=0, atol=1e-14 * np.max(np.abs(G)))
    np.testing.assert_allclose(out["alpha"], al, rtol=0, atol=1e-13)
    base = om.vcycle(oracle.cfg_vector(2, winf=w), W0, Gq, a0, 1)
    assert np.max(np.abs(base["W"] - out["W"])) > 1e-10

    mv = MESHES["vortex"]
    omv = oracle.OracleMesh(mv)
    wu = np.array([1.0, 0.3, -0.2, 2.6])
    Wu = synth.uniform_state(mv, wu)
    nu = len(Wu)
    outu = omv.vcycle(oracle.cfg_vector(2, slope_relax=ws, alpha_relax=wa), Wu, np.zeros((nu, 4, 2)),
                      np.ones(nu), 2)
    np.testing.assert_allclose(outu["W"], Wu, rtol=1e-14, atol=1e-14)
