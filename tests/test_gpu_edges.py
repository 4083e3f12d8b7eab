"""Edge cases through the C ABI on the GPU: empty point batches, zero V-cycles,
invalid arguments and out-of-order calls reported as status codes, an open
mesh rejected, a one-triangle mesh and a ragged-size mesh against the oracle,
and the two DF limits of the LU-SGS step (alpha = 0: the explicit update;
alpha = 1: fully implicit)."""
import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth
import test_gpu_parity as tp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    return cgks


def test_empty_point_batches(cg):
    ctx = cg.Context()
    try:
        for dim in (2, 3):
            nv = dim + 2
            e = np.zeros((0, nv))
            g = np.zeros((0, dim, nv))
            ctx.cgks_gks_points(dim, e, g, e, g, np.zeros(0), np.zeros((0, nv)), np.zeros((0, nv)), np.zeros(0))
            ctx.cgks_kfvs_points(dim, e, e, np.zeros((0, nv)))
        assert ctx.cgks_dword_selftest(np.zeros(0), np.zeros(0)).shape == (0, 7)
    finally:
        ctx.close()


def test_zero_cycles_leave_the_state(cg):
    m = tp.MESHES["cylinder"]
    rng = np.random.default_rng(3)
    W, G, w = tp.state_for("cylinder", m, rng)
    ctx = cg.Context()
    try:
        ctx.setup(1, m, w, W, G)
        ctx.cgks_vcycle([1], 0, cg.MIXED)
        Wd = np.zeros_like(W)
        ctx.cgks_get_state(1, Wd)
        np.testing.assert_array_equal(Wd, W)
    finally:
        ctx.close()


def test_errors_are_status_codes(cg):
    ctx = cg.Context()
    try:
        with pytest.raises(cg.CgksError) as e:
            ctx.cgks_counters(99)  # unknown mesh id
        assert e.value.code == -1
        m = tp.MESHES["vortex"]
        ctx.cgks_upload_mesh(5, m)
        with pytest.raises(cg.CgksError) as e:
            ctx.cgks_vcycle([5], 1, cg.MIXED)  # no hierarchy, free stream or state yet
        assert e.value.code in (-1, -7)
        W, G, w = tp.state_for("vortex", m, np.random.default_rng(1))
        ctx.cgks_upload_hierarchy(5, m["parents"])
        ctx.cgks_set_freestream(5, w)
        ctx.cgks_init_state(5, W, G)
        with pytest.raises(cg.CgksError) as e:
            ctx.cgks_vcycle([5], 1, 9)  # no such mode
        assert e.value.code == -1
        with pytest.raises(cg.CgksError) as e:
            ctx.cgks_vcycle([5], -1, cg.MIXED)
        assert e.value.code == -1
        # the context stays usable after the errors
        ctx.cgks_vcycle([5], 1, cg.PLAIN_FP64)
    finally:
        ctx.close()
    with pytest.raises(cg.CgksError):
        cg.Context(n_pre=2)  # only one pre-smoothing step is supported
    with pytest.raises(cg.CgksError):
        cg.Context(df_relax=3)  # no such relaxation scheme
    with pytest.raises(cg.CgksError):
        cg.Context(df_relax=2, relax_beta=1.5)  # the fixed factor lies in [0, 1]
    with pytest.raises(cg.CgksError):
        cg.Context(tau_c1=0.0)  # the collision time must stay positive
    with pytest.raises(cg.CgksError):
        cg.Context(tau_c2=-1.0)


def test_open_mesh_is_rejected(cg):
    m = dict(synth.vortex_mesh(4, 1))
    m["cell_nodes"] = m["cell_nodes"][1:].copy()  # drop one cell of the periodic box: an open mesh
    m["cell_xyz"] = m["cell_xyz"][1:].copy()
    m["parents"] = []
    ctx = cg.Context()
    try:
        with pytest.raises(cg.CgksError) as e:
            ctx.cgks_upload_mesh(1, m)
        assert e.value.code == -2
    finally:
        ctx.close()


def test_one_triangle_mesh(cg):
    """One cell, three far-field faces: the free stream is preserved and a
    perturbed state gives the oracle's residual."""
    m = dict(dim=2, cell_nodes=np.array([[0, 1, 2]], np.int32),
             cell_xyz=np.array([[[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]]),
             bface_nodes=np.array([[1, 2], [2, 0], [0, 1]], np.int32),
             bface_tag=np.full(3, synth.TAG_FARFIELD, np.int32), parents=[])
    w = synth.freestream(2.0, angle_deg=20.0)
    ctx = cg.Context()
    try:
        ctx.setup(1, m, w, synth.uniform_state(m, w), levels=1)
        R = np.zeros((1, 4))
        ctx.cgks_residual(1, 0, None, R)
        assert np.max(np.abs(R)) < 1e-13 * np.max(np.abs(w))
        W = synth.uniform_state(m, w) * np.array([[1.1, 0.9, 1.05, 1.02]])
        G = 0.1 * np.ones((1, 4, 2))
        ctx.cgks_init_state(1, W, G)
        ctx.cgks_residual(1, 0, None, R)
        ro = oracle.OracleMesh(m, levels=1).residual(oracle.cfg_vector(2, winf=w), W, G, np.ones(1))
        np.testing.assert_allclose(R, ro["R"], rtol=0, atol=1e-12 * tp.flux_scale(W, 2))
    finally:
        ctx.close()


def test_ragged_mesh_size(cg):
    """360 cells on 2 levels: no launch dimension is a multiple of a warp."""
    m = synth.cylinder_mesh(9, 5, n_refine=1)
    n = m["cell_nodes"].shape[0]
    assert n % 32 != 0
    W, G, w = tp.state_for("cylinder", m, np.random.default_rng(4))
    ctx = cg.Context()
    try:
        ctx.setup(1, m, w, W, G)
        R = np.zeros((n, 4))
        ctx.cgks_residual(1, 0, None, R)
        om = oracle.OracleMesh(m, levels=1)
        ro = om.residual(oracle.cfg_vector(2, winf=w), W, G, np.ones(n))
        Smax = float(np.max(om.faces(0)["S"]))
        np.testing.assert_allclose(R, ro["R"], rtol=0, atol=1e-12 * tp.flux_scale(W, 2) * Smax)
    finally:
        ctx.close()


@pytest.mark.parametrize("a", [0.0, 1.0])
def test_lusgs_df_limits(cg, a):
    """alpha = 0 makes the step the explicit update dW = -R dt_exp / V exactly;
    alpha = 1 is the fully implicit step; both against the oracle."""
    m = tp.MESHES["cylinder"]
    rng = np.random.default_rng(10)
    W, G, w = tp.state_for("cylinder", m, rng)
    ctx = cg.Context()
    try:
        ctx.setup(1, m, w, W, G)
        om = oracle.OracleMesh(m)
        nv, n = 4, len(W)
        Wl = tp.perturbed_states(w, n, 2, rng)
        cfg = oracle.cfg_vector(2, winf=w)
        dte, dti = om.time_steps(cfg, Wl, 0)
        alpha = np.full(n, a)
        V = om.cells(0)[0]
        rhs = 1e-2 * rng.standard_normal((n, nv)) * (V / dte)[:, None] * np.max(np.abs(w))
        Wo, dWo = om.lusgs(cfg, Wl, rhs, alpha, dte, dti, 0)
        Wg, dWg = Wl.copy(), np.zeros((n, nv))
        ctx.cgks_lusgs(1, 0, 0, Wg, rhs, alpha, dte, dti, dWg)
        sc = np.max(np.abs(dWo))
        np.testing.assert_allclose(dWg, dWo, rtol=0, atol=1e-12 * sc)
        if a == 0.0:
            # rhs is -R: the explicit update (unless the positivity guard acted)
            np.testing.assert_allclose(dWg, rhs * (dte / V)[:, None], rtol=1e-12, atol=1e-15 * sc)
    finally:
        ctx.close()


def test_checkpoint_resume_is_exact(cg):
    """get_state / set_state of (W, slopes, DF): 3 cycles, checkpoint, 3 more
    cycles equal 6 cycles in one go, bit for bit (deterministic kernels)."""
    m = tp.MESHES["cylinder"]
    W0, G0, w = tp.state_for("cylinder", m, np.random.default_rng(5))
    n = len(W0)
    ctx = cg.Context()
    try:
        ctx.setup(1, m, w, W0, G0)
        ctx.cgks_vcycle([1], 6, cg.MIXED, check=False)
        Wa = np.zeros_like(W0)
        ctx.cgks_get_state(1, Wa)
        ctx.setup(2, m, w, W0, G0)
        ctx.cgks_vcycle([2], 3, cg.MIXED, check=False)
        Wc, Gc, ac = np.zeros_like(W0), np.zeros((n, 4, 2)), np.zeros(n)
        ctx.cgks_get_state(2, Wc, Gc, ac)
        ctx.setup(3, m, w, W0, G0)  # a fresh mesh slot, then resume from the checkpoint
        ctx.cgks_set_state(3, Wc, Gc, ac)
        ctx.cgks_vcycle([3], 3, cg.MIXED, check=False)
        Wb = np.zeros_like(W0)
        ctx.cgks_get_state(3, Wb)
        np.testing.assert_array_equal(Wb, Wa)
    finally:
        ctx.close()


def test_divergence_is_reported(cg):
    """A run that blows up (Mach 5 from the free stream, no DF relaxation, CFL
    1000) ends with CGKS_ERR_DIVERGED, found on the host from the residual
    history and the non-finite counter, and the context stays usable."""
    m = synth.cylinder_mesh(16, 8, n_refine=2)
    w = synth.freestream(5.0)
    W = synth.uniform_state(m, w)
    ctx = cg.Context(df_relax=0, cfl_imp=1000.0)
    try:
        ctx.setup(1, m, w, W)
        rc = ctx.cgks_vcycle([1], 200, cg.MIXED, check=False)
        assert rc == -4
        ctx.cgks_init_state(1, W)  # reset and run a sane single cycle
        ctx.cgks_vcycle([1], 1, cg.PLAIN_FP64, check=False)
    finally:
        ctx.close()
