"""Pins of the oracle on mixed-element 3-D meshes: hexahedra, prisms and
pyramids (Sec 2.2: a quadrilateral face carries four Gauss points), on a box
of planar cells and on a cubed-sphere shell of curved ones.

* geometry: every cell closes (sum of outward area vectors 0); volumes,
  centroids and second moments equal those integrated here with a degree-2
  tetrahedron rule over the same decomposition (apex at the node mean, each
  quadrilateral as the four triangles around its node mean);
* the four-point rule of a planar quadrilateral integrates bicubic
  polynomials exactly (against a tensor Gauss-Legendre rule of order 6);
* the colouring is valid;
* the reconstruction p2 reproduces a global quadratic exactly on cells whose
  faces all have real neighbours (large-stencil weight 1);
* a uniform free stream gives a zero residual, and V-cycles keep it.
"""
import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth
from helpers import _TET2, mixed_cell_faces, mixed_tets


def meshes():
    return {"box": synth.mixed_box_mesh(4), "shell": synth.mixed_shell_mesh(4, 4)}


MESHES = meshes()


def tet_rule(T, f):
    """Integral of f over tetrahedron T [4][3] by the degree-2 four-point rule."""
    V = abs(np.linalg.det(np.array([T[1] - T[0], T[2] - T[0], T[3] - T[0]]))) / 6.0
    bary, w = _TET2
    pts = bary @ T
    return V * sum(wq * f(p) for wq, p in zip(w, pts)), V


@pytest.mark.parametrize("name", list(MESHES))
def test_cells_close_and_moments_match_quadrature(name):
    m = MESHES[name]
    om = oracle.OracleMesh(m, levels=1)
    vol, cen, m2 = om.cells(0)
    F = om.faces(0)
    n = len(vol)
    acc = np.zeros((n, 3))
    np.add.at(acc, F["L"], F["S"][:, None] * F["n"])
    inner = F["R"] >= 0
    np.add.at(acc, F["R"][inner], -(F["S"][inner, None] * F["n"][inner]))
    assert np.max(np.abs(acc)) <= 1e-13 * np.max(F["S"])
    cells, _ = mixed_cell_faces(m)
    off, xyz = m["cell_node_off"], m["cell_xyz"]
    for c in range(0, n, max(1, n // 97)):
        Xc = xyz[off[c]:off[c + 1]]
        tets = mixed_tets(Xc, [X for _, X in cells[c]]) if len(Xc) != 4 else [Xc]
        V = sum(tet_rule(T, lambda p: 1.0)[0] for T in tets)
        C = sum(tet_rule(T, lambda p: p)[0] for T in tets) / V
        M2 = sum(tet_rule(T, lambda p: np.outer(p - C, p - C))[0] for T in tets) / V
        assert abs(vol[c] - V) <= 1e-12 * V
        np.testing.assert_allclose(cen[c], C, rtol=0, atol=1e-12 * np.max(np.abs(Xc)))
        np.testing.assert_allclose(m2[c], M2, rtol=0, atol=1e-11 * np.max(np.abs(M2)))


def test_quad_rule_integrates_bicubics():
    """On the box every quadrilateral is an axis-aligned square: four points
    with their weights integrate x^a y^b z^c (a, b, c <= 3) exactly."""
    m = MESHES["box"]
    om = oracle.OracleMesh(m, levels=1)
    F = om.faces(0)
    quads = np.nonzero(F["ngp"] == 4)[0]
    assert quads.size > 50 and np.all(F["ngp"][F["ngp"] != 4] == 3)
    np.testing.assert_allclose(F["gw"][quads].sum(1), 1.0, rtol=1e-15)
    x6, w6 = np.polynomial.legendre.leggauss(6)
    rng = np.random.default_rng(3)
    # the axis-aligned squares (the faces between the two prisms of a slot are
    # diagonal rectangles and are left out here)
    square = quads[np.max(np.abs(F["n"][quads]), axis=1) > 1.0 - 1e-14]
    assert square.size > 50
    for f in rng.choice(square, 40, replace=False):
        nrm = np.abs(F["n"][f])
        ax = int(np.argmax(nrm))
        t1, t2 = [a for a in range(3) if a != ax]
        gp = F["gp"][f, :4]
        # the square's extent from its Gauss points: they sit at +-1/sqrt(3) of its half-width
        c0 = gp.mean(0)
        half = np.abs(gp - c0).max(0) * np.sqrt(3.0)
        for a, b, cc in ((1, 0, 0), (3, 2, 0), (0, 3, 1), (2, 2, 3), (3, 3, 3)):
            pw = np.array([a, b, cc])
            fq = lambda P: np.prod(P ** pw, axis=-1)
            got = F["S"][f] * np.sum(F["gw"][f, :4] * fq(gp))
            # tensor rule on the square
            s1 = c0[t1] + half[t1] * x6
            s2 = c0[t2] + half[t2] * x6
            P = np.zeros((6, 6, 3))
            P[..., ax] = c0[ax]
            P[..., t1] = s1[:, None]
            P[..., t2] = s2[None, :]
            ref = half[t1] * half[t2] * np.sum(w6[:, None] * w6[None, :] * fq(P))
            assert abs(got - ref) <= 1e-12 * (abs(ref) + 1e-12), (f, pw, got, ref)


@pytest.mark.parametrize("name", list(MESHES))
def test_coloring_is_valid(name):
    m = MESHES[name]
    om = oracle.OracleMesh(m)
    for lev in range(om.n_levels):
        col = om.colors(lev)
        cnt, nb = om.neighbors(lev)
        assert np.all(col >= 1)
        for c in range(len(col)):
            for k in range(cnt[c]):
                j = nb[c, k]
                if j >= 0:
                    assert col[j] != col[c]


def quadratic_state(rng, mesh, scale=0.05):
    """Cell averages and mean slopes of random global quadratics (kept
    physical), by the degree-2 tetrahedron rule over each cell's
    decomposition (exact for quadratics)."""
    cells, _ = mixed_cell_faces(mesh)
    off, xyz, types = mesh["cell_node_off"], mesh["cell_xyz"], mesh["cell_type"]
    Lr = float(np.max(np.abs(xyz)))
    coef = rng.standard_normal((5, 10))
    coef[:, 1:4] /= Lr
    coef[:, 4:] /= Lr * Lr
    iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]

    def q(p):
        v = coef[:, 0] + coef[:, 1:4] @ p + sum(coef[:, 4 + k] * p[a] * p[b] for k, (a, b) in enumerate(iu))
        return v * scale + np.array([2.0, 0, 0, 0, 12.0])

    def dq(p):
        g = np.array(coef[:, 1:4])
        for k, (a, b) in enumerate(iu):
            g[:, a] += coef[:, 4 + k] * p[b]
            g[:, b] += coef[:, 4 + k] * p[a]
        return g * scale

    n = len(types)
    W, G = np.zeros((n, 5)), np.zeros((n, 5, 3))
    for c in range(n):
        Xc = xyz[off[c]:off[c + 1]]
        tets = mixed_tets(Xc, [X for _, X in cells[c]]) if len(Xc) != 4 else [Xc]
        V = sum(tet_rule(T, lambda p: 1.0)[0] for T in tets)
        W[c] = sum(tet_rule(T, q)[0] for T in tets) / V
        G[c] = sum(tet_rule(T, dq)[0] for T in tets) / V
    return W, G, q


@pytest.mark.parametrize("name", list(MESHES))
def test_p2_reproduces_global_quadratics(name):
    m = MESHES[name]
    om = oracle.OracleMesh(m, levels=1)
    rng = np.random.default_rng(12)
    W, G, q = quadratic_state(rng, m)
    P, nb = om.reconstruct(oracle.cfg_vector(3, weno_gamma_high=1.0), W, G, np.ones(len(W)))
    assert nb == 0
    _, cen, _ = om.cells(0)
    cnt, nbr = om.neighbors(0)
    full = np.array([all(nbr[c, k] >= 0 for k in range(cnt[c])) for c in range(len(W))])
    assert full.sum() > 10
    types = m["cell_type"]
    for t in (5, 6, 8):
        assert np.any(full & (types == t)), t
    worst = 0.0
    for c in np.nonzero(full)[0]:
        for X in 0.3 * rng.standard_normal((4, 3)):
            x = cen[c] + X
            iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
            got = P[c, :, 0] + P[c, :, 1:4] @ X + sum(P[c, :, 4 + k] * X[a] * X[b] for k, (a, b) in enumerate(iu))
            worst = max(worst, float(np.max(np.abs(got - q(x)))))
    assert worst < 1e-10, worst


@pytest.mark.parametrize("name", list(MESHES))
def test_uniform_flow_is_steady(name):
    """Free stream at an angle: zero residual (the shell's wall taken as far
    field) and two V-cycles leave it unchanged."""
    m = dict(MESHES[name])
    m["bface_tag"] = np.full_like(m["bface_tag"], synth.TAG_FARFIELD)
    w = synth.freestream(2.0, dim=3, angle_deg=20.0)
    om = oracle.OracleMesh(m)
    n = len(m["cell_type"])
    W = np.tile(w, (n, 1))
    cfg = oracle.cfg_vector(3, winf=w)
    r = om.residual(cfg, W, np.zeros((n, 5, 3)), np.ones(n))
    F = om.faces(0)
    scale = np.max(F["S"]) * 20.0
    assert np.max(np.abs(r["R"])) <= 1e-13 * scale
    out = om.vcycle(cfg, W, np.zeros((n, 5, 3)), np.ones(n), 2)
    np.testing.assert_allclose(out["W"], W, rtol=1e-13, atol=1e-13)
