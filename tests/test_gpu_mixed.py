"""GPU parity on mixed-element 3-D meshes (hexahedra, prisms, pyramids; four
Gauss points per quadrilateral face, Sec 2.2): the CUDA path through
cgks_upload_mesh_mixed against the FP64 oracle on the same seeded inputs, on
a box of planar cells and on a cubed-sphere shell of curved ones.
Tolerances as for the simplex meshes: colourings and level sizes bit-exact,
FP64 results within 1e-12 of their natural scale, V-cycle norms within 1e-8
and states within 1e-9 over three cycles; MIXED within 1e-5 of the state
scale."""
import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth
from test_oracle_mixed import quadratic_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GAMMA = 1.4


def meshes():
    return {"box": synth.mixed_box_mesh(4), "shell": synth.mixed_shell_mesh(4, 4)}


MESHES = meshes()


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    c = cgks.Context()
    yield c
    c.close()


def flux_scale(W):
    u = W[:, 1:4] / W[:, :1]
    p = (GAMMA - 1) * (W[:, -1] - 0.5 * W[:, 0] * np.sum(u * u, 1))
    c = np.sqrt(GAMMA * p / W[:, 0])
    return float(np.max((np.abs(W[:, -1]) + p) * (np.linalg.norm(u, axis=1) + c)))


def state_for(name, m, rng):
    """A quadratic perturbation of a free stream at an angle (Mach 2; the
    shell's wall stays a slip wall, its outer boundary far field)."""
    w = synth.freestream(2.0, dim=3, angle_deg=15.0)
    Wq, Gq, _ = quadratic_state(rng, m, scale=0.05)
    W = np.tile(w, (len(Wq), 1)) + Wq - Wq.mean(0)
    return W, Gq, w


def setup(ctx, mid, name, rng):
    m = MESHES[name]
    W, G, w = state_for(name, m, rng)
    ctx.setup(mid, m, w, W, G)
    return m, oracle.OracleMesh(m), W, G, w


@pytest.mark.parametrize("name", list(MESHES))
def test_levels_and_colourings_bit_exact(ctx, name):
    m = MESHES[name]
    ctx.cgks_upload_mesh_mixed(30, m)
    ctx.cgks_upload_hierarchy(30, m["parents"])
    info = ctx.cgks_mesh_info(30)
    om = oracle.OracleMesh(m)
    assert len(info) == om.n_levels == 3
    for lev, lv in enumerate(info):
        assert lv["cells"] == om.n_cells(lev)
        assert lv["faces"] == len(om.faces(lev)["S"])
        assert lv["colors"] == om.n_colors(lev)
        np.testing.assert_array_equal(ctx.cgks_get_coloring(30, lev, lv["cells"]), om.colors(lev))


@pytest.mark.parametrize("name", list(MESHES))
def test_reconstruction(ctx, name):
    rng = np.random.default_rng(7)
    m, om, W, G, w = setup(ctx, 31, name, rng)
    n = len(W)
    coef, dte, dti = np.zeros((n, 5, 10)), np.zeros(n), np.zeros(n)
    ctx.cgks_reconstruct(31, coef, dte, dti)
    cfg = oracle.cfg_vector(3, winf=w)
    Po, nb = om.reconstruct(cfg, W, G, np.ones(n))
    de, di = om.time_steps(cfg, W)
    np.testing.assert_allclose(dte, de, rtol=1e-13)
    np.testing.assert_allclose(dti, di, rtol=1e-13)
    h = (om.cells(0)[0] ** (1.0 / 3.0))[:, None]
    sc = np.max(np.abs(W))
    np.testing.assert_allclose(coef[:, :, 0], Po[:, :, 0], rtol=0, atol=1e-12 * sc)
    np.testing.assert_allclose(coef[:, :, 1:4] * h[:, None], Po[:, :, 1:4] * h[:, None], rtol=0, atol=1e-11 * sc)
    np.testing.assert_allclose(coef[:, :, 4:] * h[:, None] ** 2, Po[:, :, 4:] * h[:, None] ** 2, rtol=0,
                               atol=1e-11 * sc)


@pytest.mark.parametrize("name", list(MESHES))
def test_fine_residual(ctx, name):
    """Residual, evolved slopes and DF factors: every cell type, every face
    kind (triangles with 3 points, quadrilaterals with 4 weighted points)."""
    rng = np.random.default_rng(8)
    m, om, W, G, w = setup(ctx, 32, name, rng)
    n = len(W)
    R, Gn, al = np.zeros((n, 5)), np.zeros((n, 5, 3)), np.zeros(n)
    ctx.cgks_residual(32, 0, None, R, Gn, al)
    ro = om.residual(oracle.cfg_vector(3, winf=w), W, G, np.ones(n))
    Fs = flux_scale(W)
    Smax = float(np.max(om.faces(0)["S"]))
    np.testing.assert_allclose(R, ro["R"], rtol=0, atol=1e-12 * Fs * Smax)
    vol = om.cells(0)[0]
    np.testing.assert_allclose(Gn * vol[:, None, None], ro["grad"] * vol[:, None, None], rtol=0,
                               atol=1e-12 * np.max(np.abs(W)) * Smax)
    np.testing.assert_allclose(al, ro["alpha"], rtol=1e-12, atol=1e-14)
    assert np.max(np.abs(R)) > 1e-3 * Fs * Smax  # a non-trivial residual


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("lev", [1, 2])
def test_coarse_kfvs_residual(ctx, name, lev):
    rng = np.random.default_rng(9)
    m, om, W, G, w = setup(ctx, 33, name, rng)
    nl = om.n_cells(lev)
    Wc = np.tile(w, (nl, 1)) * (1.0 + 0.05 * rng.random((nl, 1)))
    R = np.zeros((nl, 5))
    ctx.cgks_residual(33, lev, Wc, R)
    Ro = om.kfvs_residual(oracle.cfg_vector(3, winf=w), Wc, lev)
    Smax = float(np.max(om.faces(lev)["S"]))
    np.testing.assert_allclose(R, Ro, rtol=0, atol=1e-12 * flux_scale(Wc) * Smax)


@pytest.mark.parametrize("name", list(MESHES))
def test_vcycles_match_oracle(ctx, name):
    """Three whole V-cycles (plain FP64) against the oracle; MIXED stated
    against the same oracle run."""
    from paper_2509_06347_b300 import cgks
    rng = np.random.default_rng(13)
    m, om, W, G, w = setup(ctx, 34, name, rng)
    n = len(W)
    ncyc = 3
    out = om.vcycle(oracle.cfg_vector(3, winf=w), W, G, np.ones(n), ncyc)
    for mode, tol_state in ((cgks.PLAIN_FP64, 1e-9), (cgks.MIXED, 1e-5)):
        ctx.cgks_init_state(34, W, G)
        norms = np.zeros((ncyc, 5, 2))
        ctx.cgks_vcycle([34], ncyc, mode, norms)
        Wd = np.zeros_like(W)
        ctx.cgks_get_state(34, Wd)
        if mode == cgks.PLAIN_FP64:
            np.testing.assert_allclose(norms, out["norms"], rtol=1e-8)
        else:
            np.testing.assert_allclose(norms, out["norms"], rtol=1e-3)
        scale = np.max(np.abs(W), axis=0)
        err = np.max(np.abs(Wd - out["W"]) / scale)
        moved = np.max(np.abs(out["W"] - W) / scale)
        print(f"\n{name} mode {mode}: state error {err:.2e} (moved {moved:.2e})")
        assert err <= tol_state


def test_uniform_flow_is_steady_on_gpu(ctx):
    from paper_2509_06347_b300 import cgks
    m = dict(MESHES["shell"])
    m["bface_tag"] = np.full_like(m["bface_tag"], synth.TAG_FARFIELD)
    w = synth.freestream(3.0, dim=3, angle_deg=30.0)
    W = synth.uniform_state(m, w)
    ctx.setup(35, m, w, W)
    R = np.zeros_like(W)
    ctx.cgks_residual(35, 0, None, R)
    assert np.max(np.abs(R)) <= 1e-13 * flux_scale(W) * 20.0
    ctx.cgks_vcycle([35], 2, cgks.MIXED, np.zeros((2, 5, 2)))
    Wd = np.zeros_like(W)
    ctx.cgks_get_state(35, Wd)
    np.testing.assert_allclose(Wd, W, rtol=1e-13, atol=1e-13)


def test_mixed_upload_errors(ctx):
    """An open face, an unknown cell type and the double-word flux are
    refused with status codes; the context stays usable."""
    from paper_2509_06347_b300 import cgks
    m = MESHES["box"]
    bad = dict(m)
    bad["bface_node_off"] = m["bface_node_off"][:-1]
    bad["bface_tag"] = m["bface_tag"][:-1]
    with pytest.raises(cgks.CgksError) as e:
        ctx.cgks_upload_mesh_mixed(36, bad)
    assert e.value.code == -2
    bad = dict(m)
    bad["cell_type"] = m["cell_type"].copy()
    bad["cell_type"][0] = 7
    with pytest.raises(cgks.CgksError) as e:
        ctx.cgks_upload_mesh_mixed(36, bad)
    assert e.value.code == -2
    c2 = cgks.Context(flux_precision=1)
    with pytest.raises(cgks.CgksError) as e:
        c2.cgks_upload_mesh_mixed(1, m)
    assert e.value.code == -1
    c2.close()
    ctx.cgks_upload_mesh_mixed(36, m)
