"""GPU tests of batched solves (several meshes of different sizes and Mach
numbers advanced together in one V-cycle graph) and of the block-size
autotuner."""
import numpy as np
import pytest

from paper_2509_06347_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    return cgks


SPECS = [dict(n_theta=16, n_r=8, ratio=1.05 ** 4, mach=2.0),
         dict(n_theta=24, n_r=12, ratio=1.05 ** (32 / 12), mach=3.5),
         dict(n_theta=8, n_r=4, ratio=1.05 ** 8, mach=6.0)]


def run_single(cg, spec, ncyc, mode):
    m = synth.cylinder_mesh(spec["n_theta"], spec["n_r"], spec["ratio"], n_refine=2)
    w = synth.freestream(spec["mach"])
    ctx = cg.Context()
    ctx.setup(1, m, w, synth.uniform_state(m, w))
    ctx.cgks_vcycle([1], ncyc, mode)
    W = np.zeros((m["cell_nodes"].shape[0], 4))
    ctx.cgks_get_state(1, W)
    ctx.close()
    return W


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_equals_individual_solves(cg, mode):
    """Each member of the union advances exactly as when solved alone: same
    colouring per component, same per-cell arithmetic (only the norm sums are
    grouped differently)."""
    ncyc = 4
    union, grp, winf, W0 = synth.batch_cylinders(SPECS)
    ctx = cg.Context()
    ctx.setup(7, union, winf[0], W0)
    ctx.cgks_set_groups(7, grp, winf)
    norms = np.zeros((ncyc, len(SPECS), 4, 2))
    conv, done, rc = ctx.cgks_vcycle_groups(7, ncyc, mode, norms)
    assert done == ncyc and rc == 0
    W = np.zeros_like(W0)
    ctx.cgks_get_state(7, W)
    for g, spec in enumerate(SPECS):
        Ws = run_single(cg, spec, ncyc, mode)
        np.testing.assert_allclose(W[grp == g], Ws, rtol=1e-13, atol=1e-13)
    assert np.all(norms[:, :, 0, 0] > 0)
    ctx.close()


def test_converged_members_are_frozen(cg):
    """With a loose tolerance, members stop at their own cycle and their state
    no longer changes while the others continue."""
    union, grp, winf, W0 = synth.batch_cylinders(SPECS)
    cfg = cg.default_config(tol=0.9, check_every=1)
    ctx = cg.Context(cfg)
    ctx.setup(8, union, winf[0], W0)
    ctx.cgks_set_groups(8, grp, winf)
    ncyc = 40
    norms = np.zeros((ncyc, len(SPECS), 4, 2))
    conv, done, rc = ctx.cgks_vcycle_groups(8, ncyc, 0, norms)
    assert rc == 0
    assert np.all(conv > 0), conv
    W1 = np.zeros_like(W0)
    ctx.cgks_get_state(8, W1)
    # a frozen member that converged before the end saw identical norms afterwards
    g0 = int(np.argmin(conv))
    if conv[g0] < done:
        k = conv[g0]
        assert np.all(norms[k:done, g0, 0, 0] == norms[k, g0, 0, 0])
    ctx.close()


def test_diverged_member_is_frozen_and_others_run_on(cg):
    """A member whose residual grows past diverge_factor is frozen and
    reported (cycles_to_tol -2, status DIVERGED) while the others run to the
    end unaffected: they share no faces with it.  The factor is set between
    the members' largest residual growths of a reference run, so that some
    members cross it and some do not."""
    union, grp, winf, W0 = synth.batch_cylinders(SPECS)
    ncyc = 40
    G = len(SPECS)

    def run(factor):
        ctx = cg.Context(cg.default_config(tol=1e-30, check_every=1, diverge_factor=factor))
        ctx.setup(8, union, winf[0], W0)
        ctx.cgks_set_groups(8, grp, winf)
        norms = np.zeros((ncyc, G, 4, 2))
        conv, done, rc = ctx.cgks_vcycle_groups(8, ncyc, 0, norms, check=False)
        W = np.zeros_like(W0)
        ctx.cgks_get_state(8, W)
        ctx.close()
        return conv, done, rc, norms, W

    conv0, done0, rc0, norms0, W0ref = run(1e6)
    assert rc0 == 0 and done0 == ncyc and np.all(conv0 == -1)
    growth = norms0[:, :, 0, 0].max(axis=0) / norms0[0, :, 0, 0]
    factor = float(np.median(growth))
    conv, done, rc, norms, W = run(factor)
    hit = conv == -2
    print(f"\nresidual growth per member {np.round(growth, 4)}, factor {factor:.4f}, frozen as diverged: {hit}")
    assert hit.any() and (~hit).any()
    assert rc == -4 and done == ncyc  # CGKS_ERR_DIVERGED
    for q in range(G):
        rows = grp == q
        if hit[q]:
            # frozen: from the cycle after the one that crossed the factor on,
            # the state and so its residual no longer change
            k = int(np.argmax(norms[:, q, 0, 0] > factor * norms[0, q, 0, 0]))
            assert np.all(norms[k + 1:, q, 0, 0] == norms[k + 1, q, 0, 0])
        else:
            np.testing.assert_array_equal(W[rows], W0ref[rows])
            np.testing.assert_array_equal(norms[:, q], norms0[:, q])


def test_autotune_keeps_results(cg):
    """Block sizes change only the launch shape: the state after three cycles
    is bit-identical with and without autotuning."""
    m = synth.cylinder_mesh(32, 16, 1.05 ** 2, n_refine=2)
    w = synth.freestream(3.0)
    W0 = synth.uniform_state(m, w)
    res = []
    for tune in (False, True):
        ctx = cg.Context()
        ctx.setup(9, m, w, W0)
        if tune:
            blocks = ctx.cgks_autotune(9)
            assert set(blocks.tolist()) <= {64, 128, 256}
        ctx.cgks_vcycle([9], 3, 1)
        W = np.zeros_like(W0)
        ctx.cgks_get_state(9, W)
        res.append(W)
        ctx.close()
    np.testing.assert_array_equal(res[0], res[1])


@pytest.mark.parametrize("mode", [0, 1])
def test_coarse_cluster_step_keeps_results(cg, mode):
    """The coarse smoothing step in one thread-block cluster (cell residual,
    colour-0 forward step and both sweep phases separated by cluster barriers)
    does each cell's work of the three kernels it replaces: states and norms
    after ten cycles are bit-identical with it on both coarse levels, on level
    2 only and off, and it takes fewer launches per cycle."""
    m = synth.cylinder_mesh(32, 16, 1.05 ** 2, n_refine=2)  # 16,384 / 4,096 / 1,024 cells
    w = synth.freestream(3.0)
    W0 = synth.uniform_state(m, w)
    res, launches = [], []
    for mc in (0, 2000, 5000):
        ctx = cg.Context(coarse_cluster_max_cells=mc)
        ctx.setup(9, m, w, W0)
        norms = np.zeros((10, 4, 2))
        ctx.cgks_vcycle([9], 10, mode, norms)
        W = np.zeros_like(W0)
        ctx.cgks_get_state(9, W)
        res.append((W, norms))
        launches.append(ctx.cgks_launch_count(9, mode))
        ctx.close()
    for W, norms in res[1:]:
        np.testing.assert_array_equal(W, res[0][0])
        np.testing.assert_array_equal(norms, res[0][1])
    assert launches[0] > launches[1] > launches[2]
