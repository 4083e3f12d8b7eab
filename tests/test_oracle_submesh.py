"""The sampled full-size parity tests evaluate the oracle on ring submeshes.
Pins of that premise, oracle only: the fine residual of a cell on its 3-ring
submesh, and the coarse residual of a coarse cell on its 1-ring submesh, equal
the same values on the whole mesh."""
import numpy as np

import oracle
from paper_2509_06347_b300 import synth
from helpers import coarse_ring_submesh, physical_quadratic_state, ring_submesh

MESHES = ((lambda: synth.cylinder_mesh(16, 8, n_refine=2), 3.0), (lambda: synth.sphere_mesh(4, 4), 2.0))


def _state(m, mach, seed):
    dim = m["dim"]
    w = synth.freestream(mach, dim=dim, angle_deg=10.0)
    rng = np.random.default_rng(seed)
    Wq, Gq, _, _ = physical_quadratic_state(rng, dim, m["cell_xyz"], scale=0.05)
    return w, synth.uniform_state(m, w) + Wq - Wq.mean(0), Gq, rng


def test_fine_residual_on_ring_submesh_equals_whole_mesh():
    for make, mach in MESHES:
        m = make()
        dim = m["dim"]
        w, W, G, rng = _state(m, mach, 5)
        n = len(W)
        # interior, wall and far-field cells
        seeds = rng.choice(n, 12, replace=False)
        cfg = oracle.cfg_vector(dim, winf=w)
        full = oracle.OracleMesh(m, levels=1).residual(cfg, W, G, np.ones(n))
        sub, cells, sp = ring_submesh(m, seeds, rings=3)
        assert len(cells) < n
        part = oracle.OracleMesh(sub, levels=1).residual(cfg, W[cells], G[cells], np.ones(len(cells)))
        np.testing.assert_allclose(part["R"][sp], full["R"][seeds], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(part["grad"][sp], full["grad"][seeds], rtol=1e-13, atol=1e-15)
        np.testing.assert_array_equal(part["alpha"][sp], full["alpha"][seeds])


def test_ring_of_two_is_not_enough_somewhere():
    """Sanity of the pin above: with one ring the seeds' residuals change
    (the neighbours' reconstructions lose their own neighbours)."""
    m = synth.cylinder_mesh(16, 8, n_refine=2)
    w, W, G, rng = _state(m, 3.0, 5)
    n = len(W)
    seeds = rng.choice(n, 12, replace=False)
    cfg = oracle.cfg_vector(2, winf=w)
    full = oracle.OracleMesh(m, levels=1).residual(cfg, W, G, np.ones(n))
    sub, cells, sp = ring_submesh(m, seeds, rings=1)
    part = oracle.OracleMesh(sub, levels=1).residual(cfg, W[cells], G[cells], np.ones(len(cells)))
    assert np.max(np.abs(part["R"][sp] - full["R"][seeds])) > 1e-8


def test_coarse_residual_on_ring_submesh_equals_whole_mesh():
    for make, mach in MESHES:
        m = make()
        dim = m["dim"]
        w, _, _, rng = _state(m, mach, 6)
        cfg = oracle.cfg_vector(dim, winf=w)
        om = oracle.OracleMesh(m)
        for lev in (1, 2):
            nl = om.n_cells(lev)
            Wc = np.tile(w, (nl, 1)) * (1 + 0.02 * rng.random((nl, 1)))
            full = om.kfvs_residual(cfg, Wc, lev)
            seeds = rng.choice(nl, 6, replace=False)
            sub, ids, sp = coarse_ring_submesh(m, lev, seeds, rings=1)
            sm = oracle.OracleMesh(sub)
            assert sm.n_levels == lev + 1 and sm.n_cells(lev) == len(ids) < nl
            part = sm.kfvs_residual(cfg, Wc[ids], lev)
            np.testing.assert_allclose(part[sp], full[seeds], rtol=1e-13, atol=1e-14)
