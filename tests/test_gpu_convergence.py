"""Convergence-history parity: whole solves to a 1e-10 drop of the RMS density
residual (Sec 5.2 V-cycle, Sec 6 convergence histories), the CUDA path
against the FP64 oracle on the vortex workload (2,048 jittered periodic
triangles, three levels), and a physical check of a converged Mach-5
cylinder solve.

* FP64: the cycle at which the drop first reaches 1e-10 agrees within 1 %,
  and so do the histories and the converged states.
* MIXED (FP32 sweeps): its converged state is stated against the oracle's.
  The pseudo-time iteration does not keep the vortex: the numerical collision
  time of the flux dissipates it, the iteration (local time steps, LU-SGS)
  does not conserve momentum or energy, and the solve ends at a uniform
  state, which has an exactly zero residual for any velocity.  MIXED and FP64
  take different paths there and stop at slightly different uniform states,
  so their difference is itself uniform; the test checks both facts.
* The Mach-5 cylinder of 65,536 cells (the benchmark's workload) reaches a 1e-10
  drop in FP64 and in MIXED with the convergence settings, MIXED within 1 %
  of FP64's cycle count, and its converged state gives the stagnation-point
  wall pressure of the Rayleigh pitot formula (32.65 free-stream pressures at
  M = 5, gamma = 1.4) within 2 %.
"""
import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-10
CFG = dict(tau_c1=1.0)  # the convergence setting of the vortex solves (reading R4: C1 is a config field)
# the convergence setting of the Mach-5 cylinder solves: collision-time constants and the
# pseudo-time under-relaxation of the slopes and of a rising DF factor
# and the linear weight 0.8 of the large HWENO stencil, with which the drop
# reaches 1e-10 (0.95 leaves it near 2e-7)
CYLINDER_CFG = dict(tau_c1=1.0, tau_c2=5.0, alpha_relax=0.05, slope_relax=0.5, weno_gamma_high=0.8)


def first_drop(hist, tol=TOL):
    d = hist / hist[0]
    k = np.nonzero(d <= tol)[0]
    return int(k[0]) if k.size else None


@pytest.fixture(scope="module")
def solves():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    m = synth.vortex_mesh(n_coarse=8, n_refine=2)
    W0, G0 = synth.vortex_state(m)
    w = np.array([1.0, 0.0, 0.0, 1.0 / 0.4])
    n = len(W0)
    out = {"mesh": m, "W0": W0, "G0": G0}
    cap = 2000
    for name, mode in (("fp64", cgks.PLAIN_FP64), ("mixed", cgks.MIXED)):
        ctx = cgks.Context(stream=torch.cuda.current_stream().cuda_stream, **CFG)
        ctx.setup(1, m, w, W0, G0)
        norms = np.zeros((cap, 4, 2))
        done = np.zeros(1, np.int32)
        ctx.cgks_vcycle([1], cap, mode, norms, done)
        k = int(done[0])
        W, G, a = np.zeros_like(W0), np.zeros((n, 4, 2)), np.zeros(n)
        ctx.cgks_get_state(1, W, G, a)
        ctx.close()
        out[name] = dict(hist=norms[:k, 0, 0], W=W, G=G)
    # the oracle, in chunks, carrying its state, until the same drop
    om = oracle.OracleMesh(m)
    cfg = oracle.cfg_vector(2, winf=w, **CFG)
    Ws, Gs, al = W0.copy(), G0.copy(), np.ones(n)
    hist = []
    while len(hist) < cap:
        r = om.vcycle(cfg, Ws, Gs, al, 50)
        Ws, Gs, al = r["W"], r["grad"], r["alpha"]
        hist.extend(r["norms"][:, 0, 0].tolist())
        if first_drop(np.array(hist)) is not None:
            break
    out["oracle"] = dict(hist=np.array(hist), W=Ws, G=Gs)
    return out


def test_fp64_cycles_to_1e10_match_oracle(solves):
    kg = first_drop(solves["fp64"]["hist"])
    ko = first_drop(solves["oracle"]["hist"])
    print(f"\ncycles to a 1e-10 drop: GPU FP64 {kg}, oracle {ko}, MIXED {first_drop(solves['mixed']['hist'])}")
    assert ko is not None and kg is not None
    assert abs(kg - ko) <= 0.01 * ko
    # the histories agree cycle by cycle while the drop is well above rounding
    k = min(len(solves["fp64"]["hist"]), len(solves["oracle"]["hist"]))
    hg, ho = solves["fp64"]["hist"][:k], solves["oracle"]["hist"][:k]
    big = ho / ho[0] > 1e-6
    np.testing.assert_allclose(hg[big], ho[big], rtol=1e-6)
    # the converged FP64 states agree
    Wg, Wo = solves["fp64"]["W"], solves["oracle"]["W"]
    err = np.max(np.abs(Wg - Wo) / np.max(np.abs(Wo), axis=0))
    print(f"converged FP64 state: max relative difference to the oracle {err:.2e}")
    assert err < 1e-8


def test_mixed_converged_state_against_oracle(solves):
    km = first_drop(solves["mixed"]["hist"])
    ko = first_drop(solves["oracle"]["hist"])
    assert km is not None and abs(km - ko) <= 0.05 * ko
    W0, Wm, Wo = solves["W0"], solves["mixed"]["W"], solves["oracle"]["W"]
    scale = np.max(np.abs(Wo), axis=0)
    # the end state is uniform: the vortex (a density dip of about half the
    # background) is gone
    spread = np.max(np.abs(Wo - Wo.mean(0)) / scale)
    dip = np.max(np.abs(W0 - W0.mean(0)) / np.max(np.abs(W0), axis=0))
    dW = (Wm - Wo) / scale
    err = float(np.max(np.abs(dW)))
    shift = dW.mean(0)
    rest = float(np.max(np.abs(dW - shift)))
    print(f"\nvortex end state: max deviation from uniform {spread:.2e} (initial vortex {dip:.2e}); "
          f"MIXED vs oracle: max relative difference {err:.2e}, of which uniform "
          f"{np.array2string(shift, precision=2)} and non-uniform {rest:.2e}")
    assert spread < 1e-3 * dip
    assert err < 1e-4
    assert rest < 0.05 * err + 1e-9


@pytest.fixture(scope="module")
def cylinder():
    """The 65,536-cell Mach-5 cylinder solved from the free stream to a 1e-10 drop, FP64
    and MIXED (about 11,300 cycles each)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    m = synth.cylinder_mesh(n_theta=64, n_r=32, ratio=1.05, n_refine=2)
    w = synth.freestream(5.0)
    W0 = synth.uniform_state(m, w)
    out = {"mesh": m}
    cap = 14000
    for name, mode in (("fp64", cgks.PLAIN_FP64), ("mixed", cgks.MIXED)):
        ctx = cgks.Context(stream=torch.cuda.current_stream().cuda_stream, **CYLINDER_CFG)
        ctx.setup(1, m, w, W0)
        norms = np.zeros((cap, 4, 2))
        done = np.zeros(1, np.int32)
        rc = ctx.cgks_vcycle([1], cap, mode, norms, done, check=False)
        W = np.zeros_like(W0)
        ctx.cgks_get_state(1, W)
        ctx.close()
        k = int(done[0])
        out[name] = dict(rc=rc, hist=norms[:k, 0, 0], W=W)
    return out


def test_mach5_cylinder_reaches_1e10(cylinder):
    """FP64 and MIXED both reach the 1e-10 drop; the FP32 sweeps change the
    cycle count by under 1 %, and the converged states agree to the size of a
    1e-10 residual's effect on a weakly determined inviscid solution."""
    kf = first_drop(cylinder["fp64"]["hist"])
    km = first_drop(cylinder["mixed"]["hist"])
    Wf, Wm = cylinder["fp64"]["W"], cylinder["mixed"]["W"]
    diff = np.max(np.abs(Wm - Wf) / np.max(np.abs(Wf), axis=0))
    print(f"\nMach-5 cylinder to a 1e-10 drop: FP64 {kf} cycles, MIXED {km}; converged states differ by "
          f"{diff:.2e} of the state scale")
    assert cylinder["fp64"]["rc"] == 0 and cylinder["mixed"]["rc"] == 0
    assert kf is not None and km is not None
    assert abs(km - kf) <= 0.01 * kf
    assert np.all(np.isfinite(Wm)) and np.all(np.isfinite(Wf))


def test_mach5_stagnation_pressure_matches_pitot(cylinder):
    """Converged Mach-5 cylinder (65,536 cells, MIXED, 1e-10 drop): the
    pressure of the wall cells at the front stagnation point against the
    Rayleigh pitot pressure
    p02/p1 = [(g+1)^2 M^2 / (4 g M^2 - 2 (g-1))]^(g/(g-1)) (1 - g + 2 g M^2)/(g+1)."""
    g, M = 1.4, 5.0
    pitot = ((g + 1) ** 2 * M * M / (4 * g * M * M - 2 * (g - 1))) ** (g / (g - 1)) * (1 - g + 2 * g * M * M) / (g + 1)
    assert abs(pitot - 32.653) < 1e-3
    m = cylinder["mesh"]
    W = cylinder["mixed"]["W"]
    hist = cylinder["mixed"]["hist"]
    k = len(hist)
    drop = hist[-1] / hist[0]
    cen = m["cell_xyz"].mean(1)
    r = np.hypot(cen[:, 0], cen[:, 1])
    # the wall-adjacent cells on the stagnation line (two layers, |y| < 0.02;
    # their centroids lie 0.015 and 0.03 from the wall)
    front = (cen[:, 0] < 0) & (np.abs(cen[:, 1]) < 0.02) & (r < 1.05)
    u = W[:, 1:3] / W[:, :1]
    p = (g - 1) * (W[:, 3] - 0.5 * W[:, 0] * np.sum(u * u, 1))
    p_inf = 1.0 / g
    ratio = p[front] / p_inf
    print(f"\nMach-5 cylinder after {k} cycles (drop {drop:.1e}): stagnation wall cells p/p_inf = "
          f"{np.array2string(ratio, precision=3)}, pitot {pitot:.3f}")
    assert drop <= 1e-10
    assert front.sum() == 4
    assert np.all(np.abs(ratio / pitot - 1) < 0.02)
