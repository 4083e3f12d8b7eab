"""Oracle of the agglomeration coarsening of Sec 5.1 (hash-selected face
removal with a skewness guard).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path.  Plain
Python over small meshes, FP64 geometry, exact integer hashing.  Every
agglomerate is kept as its set of fine cells and its geometry is summed from
the fine cells and fine faces directly (the definitions of Sec 5.1: V_c = sum
V_i, C_c = sum V_i C_i / V_c; a coarse face is the union of the fine faces
between two agglomerates).

Readings where the paper is open (shared with the library, stated there too):
the hash of Eq. hash value with N_l < N_r the two cell ids and N_f the number
of interior faces of the level; the faces of a level visited in (N_l, N_r)
order; a face kept when its hash is new; pairwise merging, one merge per cell
per pass; the skewness of Eq. skewness factor required above the limit for
every other face of the merged cell, measured from the virtual centre of
Eq. virtual center (d = 0 counts as sin alpha = -1); boundary faces and faces
on a periodic seam never removed; new ids in order of the lowest member; one
level = `passes` passes.

Parity pins (tests/test_oracle_agglomerate.py): the hash against hand-worked
values (the paper's own worked example is inconsistent with its formula); a
trapezoid of two triangles and a bipyramid of two tetrahedra whose merge the
skewness guard allows or refuses at the closed-form angle (which also fixes
the volume weighting of the virtual centre and the normal orientation); a
strip of four triangles where a hash collision decides the pairing; and the
partition invariants (every cell covered once, ids by lowest member,
face-connected agglomerates, none across a periodic seam).
"""
from __future__ import annotations

import math

import numpy as np


def hash_value(nl: int, nr: int, nf: int) -> int:
    """Eq. hash value, h_f = [23 (N_l + N_r) + N_l N_r] mod N_f, in exact integers."""
    return (23 * (nl + nr) + nl * nr) % nf


def _simplex_measure(x: np.ndarray) -> float:
    """Area (2D) or volume (3D) of a simplex from its vertices x [dim+1][dim]."""
    dim = x.shape[1]
    e = [x[i + 1] - x[0] for i in range(dim)]
    return abs(float(np.linalg.det(np.array(e)))) / math.factorial(dim)


def _face_area_vector(pts: np.ndarray) -> np.ndarray:
    """Unoriented area vector of a face from its vertices pts [dim][dim]."""
    if pts.shape[1] == 2:
        t = pts[1] - pts[0]
        return np.array([t[1], -t[0]])
    return 0.5 * np.cross(pts[1] - pts[0], pts[2] - pts[0])


def fine_faces(mesh: dict):
    """Cells (volume, centroid) and faces of the fine mesh.  A face is a dict with
    'cells' (one or two cell ids, ascending), 'tag' (boundary) and, per cell
    side, the outward area vector and the face centre in that cell's own
    coordinates (which differ across a periodic seam)."""
    dim = int(mesh["dim"])
    cn = np.asarray(mesh["cell_nodes"])
    cx = np.asarray(mesh["cell_xyz"], np.float64)
    n = cn.shape[0]
    vol = np.array([_simplex_measure(cx[c]) for c in range(n)])
    cen = np.array([cx[c].sum(axis=0) / (dim + 1) for c in range(n)])
    by_nodes: dict = {}
    for c in range(n):
        for k in range(dim + 1):
            idx = [i for i in range(dim + 1) if i != k]
            pts = cx[c, idx]
            centre = pts.sum(axis=0) / dim
            a = _face_area_vector(pts)
            if a @ (centre - cen[c]) < 0.0:  # outward: away from the cell's centroid
                a = -a
            by_nodes.setdefault(tuple(sorted(int(v) for v in cn[c, idx])), []).append((c, a, centre))
    tags = {tuple(sorted(int(v) for v in r)): int(t)
            for r, t in zip(np.asarray(mesh["bface_nodes"]).reshape(-1, dim), np.asarray(mesh["bface_tag"]))}
    faces = []
    for key, sides in by_nodes.items():
        if len(sides) > 2:
            raise ValueError("face shared by more than two cells")
        if len(sides) == 1 and key not in tags:
            raise ValueError("open face missing from the boundary list")
        sides = sorted(sides, key=lambda s: s[0])
        faces.append(dict(cells=tuple(s[0] for s in sides), tag=tags.get(key, 0),
                          a={s[0]: s[1] for s in sides}, x={s[0]: s[2] for s in sides}))
    return vol, cen, faces


def _level_faces(faces, owner, dim):
    """Faces of the level whose cells are given by owner (fine cell -> id):
    interior pairs (lo, hi) and boundary groups (cell, tag), each with the
    area vector out of each of its cells, the face centre seen from each of
    them (weighted by fine face area) and the seam flag."""
    inner: dict = {}
    bnd: dict = {}
    for f in faces:
        cs = f["cells"]
        if len(cs) == 1:
            c = cs[0]
            g = bnd.setdefault((owner[c], f["tag"]), dict(a=np.zeros(dim), xw=np.zeros(dim), w=0.0))
            wf = float(np.linalg.norm(f["a"][c]))
            g["a"] += f["a"][c]
            g["xw"] += wf * f["x"][c]
            g["w"] += wf
            continue
        c1, c2 = cs
        A, B = owner[c1], owner[c2]
        if A == B:
            continue
        lo, hi = (A, B) if A < B else (B, A)
        clo, chi = (c1, c2) if owner[c1] == lo else (c2, c1)
        g = inner.setdefault((lo, hi), dict(a={lo: np.zeros(dim), hi: np.zeros(dim)},
                                            xw={lo: np.zeros(dim), hi: np.zeros(dim)}, w=0.0, seam=False))
        wf = float(np.linalg.norm(f["a"][clo]))
        g["a"][lo] += f["a"][clo]
        g["a"][hi] += f["a"][chi]
        g["xw"][lo] += wf * f["x"][clo]
        g["xw"][hi] += wf * f["x"][chi]
        g["w"] += wf
        # a periodic image: the two cells see the face at different places
        size = math.sqrt(wf) if dim == 3 else wf
        if float(np.linalg.norm(f["x"][clo] - f["x"][chi])) > 1e-6 * size:
            g["seam"] = True
    return inner, bnd


def merge_pass(vol, cen, faces, owner, n_cur, dim, min_skew, stats=None):
    """One pass of the cell-merge algorithm of Sec 5.1 on the level whose cells
    are owner's ids 0..n_cur-1.  Returns the new id of every current cell."""
    V = np.zeros(n_cur)
    VC = np.zeros((n_cur, dim))
    for c in range(len(owner)):
        V[owner[c]] += vol[c]
        VC[owner[c]] += vol[c] * cen[c]
    C = VC / V[:, None]
    inner, bnd = _level_faces(faces, owner, dim)
    keys = sorted(inner)
    nf = len(keys)
    # faces of each cell of the level: (key, kind)
    around: dict = {i: [] for i in range(n_cur)}
    for k in keys:
        around[k[0]].append(("i", k))
        around[k[1]].append(("i", k))
    for k in bnd:
        around[k[0]].append(("b", k))
    # the collection: faces with a hash value not seen before
    table, collection = set(), []
    for k in keys:
        h = hash_value(k[0], k[1], nf)
        if h not in table:
            table.add(h)
            collection.append(k)
    partner = [-1] * n_cur
    for lo, hi in collection:
        g = inner[(lo, hi)]
        if g["seam"] or partner[lo] >= 0 or partner[hi] >= 0:
            continue
        Cc = (V[lo] * C[lo] + V[hi] * C[hi]) / (V[lo] + V[hi])  # Eq. virtual center
        sins = []
        for cell in (lo, hi):
            for kind, k in around[cell]:
                if kind == "i" and k == (lo, hi):
                    continue  # the face to be removed
                if kind == "i":
                    e = inner[k]
                    a, x = e["a"][cell], e["xw"][cell] / e["w"]
                else:
                    e = bnd[k]
                    a, x = e["a"], e["xw"] / e["w"]
                d = x - Cc
                dn = float(np.linalg.norm(d))
                sins.append(float(d @ a) / (dn * float(np.linalg.norm(a))) if dn > 0.0 else -1.0)
        s = min(sins)
        if stats is not None:
            stats["margin"] = min(stats.get("margin", math.inf), abs(s - min_skew))
            stats["tested"] = stats.get("tested", 0) + 1
        if s > min_skew:
            partner[lo], partner[hi] = hi, lo
    new = [-1] * n_cur
    k = 0
    for i in range(n_cur):
        if new[i] < 0:
            new[i] = k
            if partner[i] >= 0:
                new[partner[i]] = k
            k += 1
    return new


def agglomerate(mesh: dict, n_levels: int = 3, passes: int = 3, min_skew: float = 0.1,
                stats: dict | None = None):
    """Parent arrays of the agglomerated hierarchy, [n_levels - 1] int32 arrays:
    parents[l-1][i] = level-l agglomerate of level-(l-1) cell i.  stats, if
    given, receives the number of skewness tests and the smallest distance of
    a tested sin(alpha) from the limit."""
    dim = int(mesh["dim"])
    vol, cen, faces = fine_faces(mesh)
    n = len(vol)
    owner = list(range(n))  # fine cell -> current id
    n_cur = n
    parents = []
    for _ in range(1, n_levels):
        start = list(range(n_cur))  # level cell -> current id
        for _ in range(passes):
            new = merge_pass(vol, cen, faces, owner, n_cur, dim, min_skew, stats)
            owner = [new[o] for o in owner]
            start = [new[s] for s in start]
            n_cur = max(new) + 1
        parents.append(np.array(start, np.int32))
    return parents
