"""Pins of the oracle's mesh preprocessing: geometry (Sec 2.2), coarse-cell
agglomeration (Sec 5.1) and the colouring algorithm (Sec 4.1)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2509_06347_b300 import synth
from helpers import cell_average, small_meshes

MESHES = small_meshes()


def closure(om, lev):
    f = om.faces(lev)
    n = om.n_cells(lev)
    acc = np.zeros((n, om.dim))
    tot = np.zeros(n)
    sn = f["S"][:, None] * f["n"]
    np.add.at(acc, f["L"], sn)
    np.add.at(tot, f["L"], f["S"])
    inner = f["R"] >= 0
    np.add.at(acc, f["R"][inner], -sn[inner])
    np.add.at(tot, f["R"][inner], f["S"][inner])
    return acc, tot


@pytest.mark.parametrize("name", list(MESHES))
def test_closed_cells_every_level(name):
    """sum_f S_f n_f = 0 for every fine cell and every agglomerated cell."""
    om = oracle.OracleMesh(MESHES[name])
    for lev in range(om.n_levels):
        acc, tot = closure(om, lev)
        assert np.max(np.linalg.norm(acc, axis=1) / tot) < 1e-14


@pytest.mark.parametrize("name", list(MESHES))
def test_coarse_volume_and_centre(name):
    """V_c = sum V_i and C_c = sum V_i C_i / V_c over children (Sec 5.1)."""
    m = MESHES[name]
    om = oracle.OracleMesh(m)
    for lev in range(om.n_levels - 1):
        vf, cf, _ = om.cells(lev)
        vc, cc, _ = om.cells(lev + 1)
        par = m["parents"][lev]
        np.testing.assert_allclose(np.bincount(par, weights=vf), vc, rtol=1e-14)
        for d in range(om.dim):
            np.testing.assert_allclose(np.bincount(par, weights=vf * cf[:, d]) / vc, cc[:, d], rtol=1e-13, atol=1e-13)


def test_total_areas():
    """Vortex box area is L^2; the cylinder O-mesh area is the difference of the
    inscribed outer and inner polygons (fine wall nodes lie on the circles)."""
    om = oracle.OracleMesh(MESHES["vortex"])
    assert abs(om.cells(0)[0].sum() - 100.0) < 1e-12
    m = MESHES["cylinder"]
    om = oracle.OracleMesh(m)
    N = 16 * 4
    poly = 0.5 * N * math.sin(2 * math.pi / N)
    assert abs(om.cells(0)[0].sum() - poly * (15.0 ** 2 - 1.0)) < 1e-10


@pytest.mark.parametrize("name", list(MESHES))
def test_cell_moments_against_quadrature(name):
    """Volume, centroid and central second moments against a degree-2 quadrature."""
    m = MESHES[name]
    om = oracle.OracleMesh(m)
    vol, cen, m2 = om.cells(0)
    xyz = m["cell_xyz"][:50]
    c_q = cell_average(xyz, lambda p: p)
    np.testing.assert_allclose(cen[:50], c_q, rtol=1e-13, atol=1e-13)
    m_q = cell_average(xyz, lambda p: np.einsum("...d,...e->...de", p, p)) - np.einsum("cd,ce->cde", c_q, c_q)
    np.testing.assert_allclose(m2[:50], m_q, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("name", list(MESHES))
def test_face_gauss_points_and_shifts(name):
    """Gauss points lie on the face plane and integrate the face's degree-3 (2-D)
    or degree-2 (3-D) polynomials exactly; periodic shifts map R's face onto L's."""
    m = MESHES[name]
    om = oracle.OracleMesh(m)
    f = om.faces(0)
    dim = om.dim
    ng = 2 if dim == 2 else 3
    gp = f["gp"][:, :ng]
    _, cen, _ = om.cells(0)
    # on the plane: (x - x_face) . n = 0 with x_face the mean of the points
    xf = gp.mean(axis=1)
    assert np.max(np.abs(np.einsum("fgd,fd->fg", gp - xf[:, None], f["n"]))) < 1e-12
    # normals point from L to R (or outward at boundaries)
    assert np.all(np.einsum("fd,fd->f", xf - cen[f["L"]], f["n"]) > 0)
    if dim == 2:
        # edge endpoints from the Gauss points: x = mid -+ e/(2 sqrt 3)
        e = (gp[:, 1] - gp[:, 0]) * math.sqrt(3.0)
        a, b = xf - 0.5 * e, xf + 0.5 * e
        s, w = np.polynomial.legendre.leggauss(6)
        s = 0.5 * (s + 1)
        w = 0.5 * w
        k = np.array([0.3, -1.2])
        f3 = lambda p: (p @ k) ** 3 + (p @ k) ** 2
        exact = sum(wi * f3(a + si * (b - a)) for si, wi in zip(s, w))
        approx = 0.5 * (f3(gp[:, 0]) + f3(gp[:, 1]))
        np.testing.assert_allclose(approx, exact, rtol=1e-12, atol=1e-12)
    per = f["R"] >= 0
    if name == "vortex":
        sh = f["shift"][per]
        assert set(np.unique(np.round(sh, 12))) <= {-10.0, 0.0, 10.0}
        assert np.any(np.abs(sh) > 0)


def test_golden_strip_coloring():
    """Hand-worked colouring (tests/golden/coloring_strip.txt)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "coloring_strip.txt")
    cells, colors = None, None
    for line in open(path):
        if line.startswith("cells"):
            cells = [list(map(int, c.split())) for c in line[5:].split("|")]
        if line.startswith("colors"):
            colors = list(map(int, line.split()[1:]))
    xy = {0: (0, 0), 1: (1, 0), 2: (2, 0), 3: (0, 1), 4: (1, 1), 5: (2, 1)}
    cn = np.array(cells, np.int32)
    cx = np.array([[xy[v] for v in c] for c in cells], float)
    bnd = [(0, 1), (1, 2), (2, 5), (5, 4), (4, 3), (3, 0)]
    mesh = dict(dim=2, cell_nodes=cn, cell_xyz=cx, bface_nodes=np.array(bnd, np.int32),
                bface_tag=np.full(6, 2, np.int32), parents=[])
    om = oracle.OracleMesh(mesh)
    assert list(om.colors(0)) == colors


@pytest.mark.parametrize("name", list(MESHES))
def test_coloring_valid_every_level(name):
    """No face joins two cells of one colour; colours are 1..Nc, all used;
    Nc <= max degree + 1 (greedy bound)."""
    om = oracle.OracleMesh(MESHES[name])
    for lev in range(om.n_levels):
        col = om.colors(lev)
        f = om.faces(lev)
        inner = f["R"] >= 0
        assert np.all(col[f["L"][inner]] != col[f["R"][inner]])
        nc = om.n_colors(lev)
        assert set(np.unique(col)) == set(range(1, nc + 1))
        cnt, nb = om.neighbors(lev)
        deg = np.array([np.sum(nb[c, :cnt[c]] >= 0) for c in range(len(cnt))])
        assert nc <= deg.max() + 1


@pytest.mark.parametrize("name", list(MESHES))
def test_coloring_is_greedy(name):
    """A cell painted k had painted neighbours of every colour 1..k-1 when it was
    painted (smallest free colour), and colours never change afterwards, so
    every cell of colour k has neighbours of all colours below k."""
    om = oracle.OracleMesh(MESHES[name])
    for lev in range(om.n_levels):
        col = om.colors(lev)
        cnt, nb = om.neighbors(lev)
        for c in range(len(col)):
            nbc = {int(col[j]) for j in nb[c, :cnt[c]] if j >= 0}
            assert set(range(1, int(col[c]))) <= nbc
