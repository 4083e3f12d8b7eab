"""Pins of the agglomeration oracle (Sec 5.1): the hash of Eq. hash value
against hand-worked values, hand-built meshes whose merge decisions follow
from closed forms (a trapezoid in 2D, a bipyramid of two tetrahedra in 3D,
where the virtual centre of Eq. virtual center and the skewness of Eq.
skewness factor are worked out by hand), a strip where the hash collision
decides the pairing, and invariants of the partition on the synthetic
meshes."""
import math

import numpy as np
import pytest

from oracle import agglomerate as oa
from paper_2509_06347_b300 import synth
from helpers import face_neighbours


def test_hash_hand_values():
    # 23 * 22 + 120 = 626 = 6 * 100 + 26.  The paper's worked example quotes 5
    # for these ids; its formula gives 26, which is what is implemented.
    assert oa.hash_value(10, 12, 100) == 26
    assert oa.hash_value(0, 1, 7) == 2          # 23 mod 7
    assert oa.hash_value(3, 5, 50) == 49        # 184 + 15 = 199
    assert oa.hash_value(4, 9, 1) == 0          # one interior face: always kept
    # ids near 2^30 (the largest mesh the library takes): 2^60 + 23 * 2^31
    # - 3 * 2^30 - 67 is 2^30 - 67 modulo 2^31; no overflow in the products
    assert oa.hash_value(2**30 - 2, 2**30 - 1, 2**31) == 2**30 - 67


def _mesh(dim, cells, xyz, bfaces, tags):
    cn = np.array(cells, np.int32)
    return dict(dim=dim, cell_nodes=cn, cell_xyz=np.array([[xyz[v] for v in c] for c in cells], np.float64),
                bface_nodes=np.array(bfaces, np.int32), bface_tag=np.array(tags, np.int32))


def _trapezoid():
    # (0,0), (2,0), (1,1), (0,1) cut along (0,0)-(1,1): areas 1 and 1/2.  Every
    # boundary edge of a triangle has its own tag, so it is a face of its own.
    xyz = {0: (0.0, 0.0), 1: (2.0, 0.0), 2: (1.0, 1.0), 3: (0.0, 1.0)}
    return _mesh(2, [[0, 1, 2], [0, 2, 3]], xyz, [[0, 1], [1, 2], [2, 3], [3, 0]], [1, 2, 1, 2])


def test_trapezoid_skew_closed_form():
    """Virtual centre (7/9, 4/9) (volume-weighted); the slanted edge from (2,0)
    to (1,1) has the smallest sin(alpha) = 14 / sqrt(340) = 0.75926.  An
    unweighted centre (2/3, 1/2) would give 1/sqrt(2) = 0.70711 there, and a
    wrong normal sign a negative value."""
    s = 14.0 / math.sqrt(340.0)
    m = _trapezoid()
    for lim, merged in [(s - 1e-9, True), (s + 1e-9, False), (0.72, True), (-0.5, True)]:
        p = oa.agglomerate(m, n_levels=2, passes=1, min_skew=lim)[0]
        assert list(p) == ([0, 0] if merged else [0, 1]), lim


def _bipyramid(h1, h2):
    r3 = math.sqrt(3.0) / 2.0
    xyz = {0: (1.0, 0.0, 0.0), 1: (-0.5, r3, 0.0), 2: (-0.5, -r3, 0.0), 3: (0.0, 0.0, h1), 4: (0.0, 0.0, -h2)}
    cells = [[0, 1, 2, 3], [0, 1, 2, 4]]
    bf = [[0, 1, 3], [1, 2, 3], [2, 0, 3], [0, 1, 4], [1, 2, 4], [2, 0, 4]]
    return _mesh(3, cells, xyz, bf, [1, 2, 3, 1, 2, 3])


def test_bipyramid_skew_closed_form():
    """Two tetrahedra on an equilateral triangle of circumradius 1, apexes at
    heights h1 and -h2.  Volumes are in the ratio h1 : h2 and centroids at
    z = h1/4 and -h2/4, so the virtual centre is at z_c = (h1 - h2) / 4.  In the
    plane through the axis and a face's centre, the face centre sits at radius
    1/3 and height h/3 and the outward normal is (2h, 1) / sqrt(4h^2 + 1):
    sin(alpha) = (h - z_c) / (sqrt(4h^2 + 1) sqrt(1/9 + (h/3 - z_c)^2)) on the
    upper faces and the mirror image on the lower ones."""
    h1, h2 = 1.0, 0.5
    zc = (h1 - h2) / 4.0
    up = (h1 - zc) / (math.sqrt(4 * h1 * h1 + 1) * math.sqrt(1 / 9 + (h1 / 3 - zc) ** 2))
    lo = (h2 + zc) / (math.sqrt(4 * h2 * h2 + 1) * math.sqrt(1 / 9 + (h2 / 3 + zc) ** 2))
    s = min(up, lo)
    m = _bipyramid(h1, h2)
    assert list(oa.agglomerate(m, 2, 1, s - 1e-9)[0]) == [0, 0]
    assert list(oa.agglomerate(m, 2, 1, s + 1e-9)[0]) == [0, 1]
    # the symmetric bipyramid: 3 / sqrt(10) on every face
    m = _bipyramid(1.0, 1.0)
    s = 3.0 / math.sqrt(10.0)
    assert list(oa.agglomerate(m, 2, 1, s - 1e-9)[0]) == [0, 0]
    assert list(oa.agglomerate(m, 2, 1, s + 1e-9)[0]) == [0, 1]


def test_strip_hash_collision_decides():
    """Four triangles in a 2 x 1 strip, numbered so that the chain of
    neighbours is 0-2-1-3.  Faces (0,2), (1,2), (1,3), N_f = 3: hashes
    46 mod 3 = 1, 71 mod 3 = 2, 95 mod 3 = 2.  (1,3) collides with (1,2) and is
    not collected; (0,2) merges; (1,2) finds cell 2 taken.  So cells 1 and 3
    stay single, where merging every face greedily would have paired them."""
    xyz = {0: (0.0, 0.0), 1: (1.0, 0.0), 2: (2.0, 0.0), 3: (0.0, 1.0), 4: (1.0, 1.0), 5: (2.0, 1.0)}
    cells = [[0, 1, 3], [1, 2, 4], [1, 4, 3], [2, 5, 4]]
    bf = [[0, 1], [1, 2], [2, 5], [5, 4], [4, 3], [3, 0]]
    m = _mesh(2, cells, xyz, bf, [2] * 6)
    assert list(oa.agglomerate(m, 2, 1, 0.5)[0]) == [0, 1, 0, 2]


def test_open_mesh_rejected():
    m = _trapezoid()
    m["bface_nodes"] = m["bface_nodes"][1:]
    m["bface_tag"] = m["bface_tag"][1:]
    with pytest.raises(ValueError):
        oa.agglomerate(m, 2, 1, 0.1)


def _components(members, adj):
    seen, start = set(), members[0]
    stack = [start]
    mset = set(members)
    while stack:
        c = stack.pop()
        if c in seen:
            continue
        seen.add(c)
        stack.extend(j for j in adj[c] if j in mset and j not in seen)
    return len(seen) == len(mset)


@pytest.mark.parametrize("name", ["vortex", "cylinder", "sphere"])
def test_partition_invariants(name):
    """Every level covers each cell of the level above once; ids follow the
    lowest member; an agglomerate has at most 2^passes members and is
    face-connected on the fine mesh and never joins two cells across the
    periodic seam of the vortex box; every level coarsens by more than 1.5:1."""
    m = {"vortex": lambda: synth.vortex_mesh(8, 1), "cylinder": lambda: synth.cylinder_mesh(16, 8, n_refine=1),
         "sphere": lambda: synth.sphere_mesh(4, 4)}[name]()
    passes = 3
    par = oa.agglomerate(m, 3, passes, 0.1)
    n = m["cell_nodes"].shape[0]
    nb, _ = face_neighbours(np.asarray(m["cell_nodes"], np.int64))
    adj = [[int(j) for j in nb[i] if j >= 0] for i in range(n)]
    fine_of = np.arange(n)
    for p in par:
        assert len(p) == int(fine_of.max()) + 1
        k = int(p.max()) + 1
        assert np.array_equal(np.unique(p), np.arange(k))
        first = [int(np.argmax(p == j)) for j in range(k)]
        assert first == sorted(first)
        assert np.bincount(p).max() <= 2 ** passes
        assert len(p) / k > 1.5
        fine_of = p[fine_of]
        for j in range(k):
            members = list(np.nonzero(fine_of == j)[0])
            assert _components(members, adj)
        # two neighbours in one agglomerate see their shared nodes at the same
        # place: no face inside an agglomerate is a periodic image
        cn, cx = np.asarray(m["cell_nodes"]), np.asarray(m["cell_xyz"])
        for i in range(n):
            for j in adj[i]:
                if fine_of[i] == fine_of[j]:
                    shared = set(cn[i]) & set(cn[j])
                    for v in shared:
                        xi = cx[i][list(cn[i]).index(v)]
                        xj = cx[j][list(cn[j]).index(v)]
                        assert np.allclose(xi, xj, rtol=0, atol=1e-12)
