"""GPU tests of the learned coarse-grid correction inside the V-cycle:
trajectory collection, the DF gate, the judge and fallback policy, and a
measurement of what a trained network gains over the plain V-cycle."""
import numpy as np
import pytest

from oracle import mlp
from paper_2509_06347_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GAMMA = 1.4


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    return cgks


def mesh():
    return synth.cylinder_mesh(16, 8, 1.05 ** 4, n_refine=2)


def run(cg, mach, ncyc, mode, levels=None, theta=None, **cfg):
    m = mesh()
    w = synth.freestream(mach)
    ctx = cg.Context(cg.default_config(**cfg))
    if theta is not None:
        ctx.cgks_mlp_set_params(theta)
    ctx.setup(1, m, w, synth.uniform_state(m, w), levels=levels)
    norms = np.zeros((ncyc, 4, 2))
    done = np.zeros(1, np.int32)
    rc = ctx.cgks_vcycle([1], ncyc, mode, norms, done, check=False)
    W = np.zeros((m["cell_nodes"].shape[0], 4))
    ctx.cgks_get_state(1, W)
    stats = ctx.cgks_learned_stats(1) if mode == cg.LEARNED else None
    ctx.close()
    return rc, W, norms[:done[0]], stats


def constant_net(delta):
    """Network whose output is the constant delta (last layer weights zero)."""
    th = mlp.init_params(3)
    th[-4:] = delta
    th[-4 - 4 * 64:-4] = 0.0
    return th


def test_collect_fills_training_set(cg):
    m = mesh()
    w = synth.freestream(3.0)
    ctx = cg.Context()
    ctx.cgks_mlp_set_params(mlp.init_params(0))
    ctx.setup(1, m, w, synth.uniform_state(m, w))
    ctx.cgks_mlp_dataset_clear()
    ctx.cgks_mlp_collect(1, 3, 1)
    assert ctx.cgks_mlp_dataset_size() == 3 * m["cell_nodes"].shape[0]
    ctx.close()


def test_closed_gate_is_fine_smoothing_only(cg):
    """With the gate above any DF value and no judge cycles, the first learned
    cycle changes the state exactly as a one-level V-cycle (fine steps only).
    (Later cycles differ: the learned cycle also evaluates the residual after
    smoothing, whose DF factor feeds the next cycle's sub-stencil.)"""
    th = constant_net(np.array([0.1, 0.0, 0.0, 0.1]))
    _, Wl, _, st = run(cg, 3.0, 1, cg.LEARNED, theta=th, df_gate=2.0, learned_judge_every=0)
    _, W1, _, _ = run(cg, 3.0, 1, cg.MIXED, levels=1)
    np.testing.assert_array_equal(Wl, W1)
    assert st["learned"] == 1 and st["judge"] == 0


def test_open_gate_adds_the_prediction(cg):
    """With every cell gated in, one learned cycle adds the (constant)
    prediction times the free-stream scales to the one-level result."""
    d = np.array([1e-3, 2e-3, -1e-3, 3e-3])
    th = constant_net(d)
    _, Wl, _, _ = run(cg, 3.0, 1, cg.LEARNED, theta=th, df_gate=-1.0, learned_judge_every=0)
    _, W1, _, _ = run(cg, 3.0, 1, cg.MIXED, levels=1)
    w = synth.freestream(3.0)
    rho, c = w[0], 1.0
    sc = np.array([rho, rho * c, rho * c, rho * c * c])
    np.testing.assert_allclose(Wl - W1, np.tile(d * sc, (len(W1), 1)), rtol=1e-2, atol=1e-7)


def test_open_gate_scales_with_the_residual_norm(cg):
    """learned_scale = 1: the prediction is multiplied by the cell's defect
    scale as well, dt_imp at the smoothed state times the RMS over the
    variables of the cycle's fine residual norms in free-stream units."""
    d = np.array([1e-3, 2e-3, -1e-3, 3e-3])
    th = constant_net(d)
    m = mesh()
    w = synth.freestream(3.0)
    W0 = synth.uniform_state(m, w)
    n = len(W0)
    ctx = cg.Context(cg.default_config(df_gate=-1.0, learned_judge_every=0, learned_scale=1))
    ctx.cgks_mlp_set_params(th)
    ctx.setup(1, m, w, W0)
    norms = np.zeros((1, 4, 2))
    assert ctx.cgks_vcycle([1], 1, cg.LEARNED, norms, check=False) == 0
    Wl = np.zeros_like(W0)
    ctx.cgks_get_state(1, Wl)
    ctx.close()
    _, W1, _, _ = run(cg, 3.0, 1, cg.MIXED, levels=1)
    c1 = cg.Context()
    c1.setup(1, m, w, W1)
    dte, dti = np.zeros(n), np.zeros(n)
    c1.cgks_reconstruct(1, None, dte, dti)
    c1.close()
    sc = np.array([w[0], w[0], w[0], w[0]])  # rho = 1, c = 1
    sigma = np.sqrt(np.mean((norms[0, :, 0] / sc) ** 2))
    s = (Wl - W1) / (d * sc)
    np.testing.assert_allclose(s, np.tile((dti * sigma)[:, None], (1, 4)), rtol=1e-4)


def test_per_variable_judge_errors_bracket_the_total(cg):
    """The judge's error over all variables is the correction-weighted mean of
    the per-variable squared errors, so it lies between their extremes."""
    th = constant_net(np.array([0.5, -0.5, 0.5, 2.0]))
    for ls in (0, 1):
        rc, _, _, st = run(cg, 3.0, 2, cg.LEARNED, theta=th, learned_scale=ls)
        pv = np.array(st["judge_error_per_variable"])
        assert rc == 0 and st["judge"] == 1 and np.all(pv >= 0)
        assert pv.min() * (1 - 1e-12) <= st["judge_error"] <= pv.max() * (1 + 1e-12)


def test_bad_network_is_disabled_by_the_judge(cg):
    """A network predicting nonsense fails the first judge cycle and the run
    then follows the plain V-cycle exactly."""
    th = constant_net(np.array([0.5, -0.5, 0.5, 2.0]))
    rc, Wl, nl, st = run(cg, 3.0, 6, cg.LEARNED, theta=th)
    _, Wp, np_, _ = run(cg, 3.0, 6, cg.MIXED)
    assert rc == 0 and st["disabled"] and st["learned"] == 0 and st["judge"] == 1
    np.testing.assert_array_equal(Wl, Wp)
    np.testing.assert_array_equal(nl, np_)


@pytest.fixture(scope="module")
def trained(cg):
    """A network trained on trajectories at Mach 2 and 4 (this file's small
    cylinder), for evaluation at the held-out Mach 3."""
    m = mesh()
    ctx = cg.Context()
    ctx.cgks_mlp_set_params(mlp.init_params(1))
    ctx.cgks_mlp_dataset_clear()
    for i, mach in enumerate((2.0, 4.0)):
        w = synth.freestream(mach)
        ctx.setup(10 + i, m, w, synth.uniform_state(m, w))
        ctx.cgks_mlp_collect(10 + i, 60, 1)
    losses = ctx.cgks_mlp_train(1500, 4096, 1e-3, seed=5)
    theta = ctx.cgks_mlp_get_params()
    ctx.close()
    return theta, losses


def test_trained_network_gain_is_measured(cg, trained, capsys):
    """Evaluate the trained network at the held-out Mach 3: report its judge
    error and the residual / time of learned versus plain cycles.  The policy
    must hold either way: a judge error above 0.5 disables the network on the
    first judge cycle and the run then equals the plain MIXED run; otherwise
    learned cycles run."""
    import time
    theta, losses = trained
    assert losses[-50:].mean() < losses[:5].mean()
    out = {}
    for mode in (cg.MIXED, cg.LEARNED):
        torch.cuda.synchronize()
        t0 = time.time()
        rc, W, norms, st = run(cg, 3.0, 200, mode, theta=theta)
        out[mode] = (time.time() - t0, norms[-1, 0, 0] / norms[0, 0, 0], st, norms)
        assert rc == 0
    st = out[cg.LEARNED][2]
    with capsys.disabled():
        print(f"\nlearned-correction gain at held-out Mach 3: plain {out[cg.MIXED][:2]}, "
              f"learned {out[cg.LEARNED][:3]}")
    if st["judge_error"] > 0.5:
        assert st["disabled"] and st["learned"] == 0
        np.testing.assert_array_equal(out[cg.LEARNED][3], out[cg.MIXED][3])
    else:
        assert not st["disabled"] and st["learned"] > 0
    assert out[cg.LEARNED][1] <= 2.0 * out[cg.MIXED][1]


def test_learned_cycles_run_when_not_disabled(cg, trained):
    """With the judge kept from disabling the network, the trained network's
    corrections are applied (learned cycles run; judge cycles at 0, 20 and 40,
    except where a fallback of 10 plain cycles covers one) and the state stays
    finite."""
    theta, _ = trained
    rc, W, norms, st = run(cg, 3.0, 60, cg.LEARNED, theta=theta, learned_max_error=1e30)
    print(f"\nlearned cycles with the judge kept from disabling: {st}")
    assert st["learned"] > 0 and st["judge"] >= 2 and not st["disabled"]
    assert st["learned"] + st["plain"] == 60 and st["plain"] <= st["judge"] + 10 * st["fallbacks"]
    assert np.all(np.isfinite(W)) and np.all(np.isfinite(norms))


@pytest.mark.xfail(strict=False, reason="measured: at held-out Mach the trained per-cell network explains "
                   "about a third of the coarse correction (judge error 0.78-0.83 on the 65,536-cell "
                   "cylinder at Mach 2.5/5.5/7.5), above the 0.5 the judge accepts")
def test_trained_network_passes_the_judge(cg, trained):
    """The goal the learned correction does not reach yet: a trained network
    whose held-out judge error is below the 0.5 that keeps it enabled."""
    theta, _ = trained
    rc, W, norms, st = run(cg, 3.0, 40, cg.LEARNED, theta=theta)
    assert st["judge_error"] <= 0.5 and st["learned"] > 0
