"""Small test-side utilities: exact quadrature rules written in the tests,
independent of both the oracle and the CUDA path."""
import math

import numpy as np

from paper_2509_06347_b300 import synth

GAMMA = 1.4

# degree-2 rules: triangle edge midpoints; tetrahedron 4-point rule
_TRI2 = (np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]]), np.full(3, 1.0 / 3.0))
_a, _b = 0.5854101966249685, 0.1381966011250105
_TET2 = (np.array([[_a, _b, _b, _b], [_b, _a, _b, _b], [_b, _b, _a, _b], [_b, _b, _b, _a]]), np.full(4, 0.25))


def cell_average(xyz, f):
    """Average of a quadratic f(x[..., dim]) over simplices xyz [n, dim+1, dim]."""
    dim = xyz.shape[-1]
    bary, w = _TRI2 if dim == 2 else _TET2
    pts = np.einsum("qv,cvd->cqd", bary, xyz)
    return np.einsum("q,cq...->c...", w, f(pts))


def physical_quadratic_state(rng, dim, xyz, scale=0.05):
    """Conservative variables given by random global quadratics, kept physical;
    returns (W, grad[n, nv, dim], fn) with fn(points) -> W(points)."""
    nv = dim + 2
    c = rng.standard_normal((nv, 1 + dim + dim * dim))
    Lr = float(np.max(np.abs(xyz)))  # keep the quadratic O(1) over the domain
    c[:, 1:1 + dim] /= Lr
    c[:, 1 + dim:] /= Lr * Lr

    def q(pts):
        out = []
        for v in range(nv):
            lin = c[v, 1:1 + dim]
            H = c[v, 1 + dim:].reshape(dim, dim)
            H = 0.5 * (H + H.T)
            val = c[v, 0] + pts @ lin + 0.5 * np.einsum("...d,de,...e->...", pts, H, pts)
            out.append(val)
        base = np.zeros(nv)
        base[0] = 2.0
        base[-1] = 12.0
        return np.stack(out, -1) * scale + base

    def dq(pts):
        out = []
        for v in range(nv):
            lin = c[v, 1:1 + dim]
            H = c[v, 1 + dim:].reshape(dim, dim)
            H = 0.5 * (H + H.T)
            out.append(lin + pts @ H)
        return np.stack(out, -2) * scale

    W = cell_average(xyz, q)
    G = cell_average(xyz, dq)
    return W, G, q, dq


def small_meshes():
    return {
        "vortex": synth.vortex_mesh(n_coarse=4, n_refine=2),
        "cylinder": synth.cylinder_mesh(n_theta=16, n_r=8, n_refine=2),
        "sphere": synth.sphere_mesh(n_panel=4, n_r=4),
    }


def face_neighbours(cell_nodes):
    """Face adjacency of a simplex mesh from its node ids: nb [n, dim+1] with
    nb[c, k] the cell across the face opposite vertex k (-1 on the boundary),
    and the sorted node key of every cell face [n, dim+1, dim]."""
    n, nvtx = cell_nodes.shape
    faces = np.stack([np.delete(cell_nodes, k, axis=1) for k in range(nvtx)], 1)
    faces = np.sort(faces, axis=2)
    base = int(cell_nodes.max()) + 1
    key = np.zeros(faces.shape[:2], np.int64)
    for d in range(nvtx - 1):
        key = key * base + faces[..., d]
    flat = key.reshape(-1)
    order = np.argsort(flat, kind="stable")
    sk = flat[order]
    nb = -np.ones(n * nvtx, np.int64)
    same = np.nonzero(sk[1:] == sk[:-1])[0]
    a, b = order[same], order[same + 1]
    nb[a] = b // nvtx
    nb[b] = a // nvtx
    return nb.reshape(n, nvtx), faces


def ring_submesh(mesh, seeds, rings=3, adjacency=None):
    """The cells within `rings` face-neighbour steps of the seed cells, as a
    stand-alone mesh: nodes renumbered, original boundary faces kept with their
    tags and cut faces tagged far field.  Returns (submesh, cell ids in the
    original mesh, positions of the seeds in the submesh).  A cell's fine
    residual depends on two rings only, so the seeds' residuals are those of
    the full mesh.  adjacency: face_neighbours(cell_nodes), if already known."""
    cn = np.asarray(mesh["cell_nodes"], np.int64)
    nb, faces = face_neighbours(cn) if adjacency is None else adjacency
    keep = np.zeros(len(cn), bool)
    keep[seeds] = True
    front = np.asarray(seeds)
    for _ in range(rings):
        nxt = nb[front].reshape(-1)
        nxt = nxt[nxt >= 0]
        nxt = nxt[~keep[nxt]]
        keep[nxt] = True
        front = np.unique(nxt)
    cells = np.nonzero(keep)[0]
    pos = -np.ones(len(cn), np.int64)
    pos[cells] = np.arange(len(cells))
    nodes = np.unique(cn[cells])
    nmap = -np.ones(int(cn.max()) + 1, np.int64)
    nmap[nodes] = np.arange(len(nodes))
    # original boundary tags by sorted face key
    bn = np.sort(np.asarray(mesh["bface_nodes"], np.int64), axis=1)
    btag = {tuple(r): int(t) for r, t in zip(bn, mesh["bface_tag"])}
    sub_bn, sub_bt = [], []
    for c in cells:
        for k in range(cn.shape[1]):
            j = nb[c, k]
            if j >= 0 and keep[j]:
                continue
            key = tuple(faces[c, k])
            sub_bn.append([nmap[v] for v in key])
            sub_bt.append(btag.get(key, synth.TAG_FARFIELD) if j < 0 else synth.TAG_FARFIELD)
    sub = dict(dim=mesh["dim"], cell_nodes=np.ascontiguousarray(nmap[cn[cells]], np.int32),
               cell_xyz=np.ascontiguousarray(mesh["cell_xyz"][cells]),
               bface_nodes=np.ascontiguousarray(np.array(sub_bn, np.int32).reshape(-1, mesh["dim"])),
               bface_tag=np.ascontiguousarray(np.array(sub_bt, np.int32)), parents=[])
    return sub, cells, pos[np.asarray(seeds)]


def coarse_ring_submesh(mesh, level, seeds, rings=1):
    """The coarse cells of `level` within `rings` steps of the seeds, with all
    their fine descendants, as a stand-alone mesh with a `level`-deep
    hierarchy.  The first-order coarse residual of a cell depends on its face
    neighbours only, so one ring gives the seeds' full-mesh residuals.
    Returns (submesh, the kept coarse cell ids in the submesh's order, the
    positions of the seeds among them)."""
    cn = np.asarray(mesh["cell_nodes"], np.int64)
    nb, _ = face_neighbours(cn)
    par = [np.asarray(p, np.int64) for p in mesh["parents"][:level]]
    anc = np.arange(len(cn))
    for p in par:
        anc = p[anc]  # fine cell -> its ancestor on `level`
    ncoarse = int(anc.max()) + 1
    fi = np.repeat(np.arange(len(cn)), cn.shape[1])
    fj = nb.reshape(-1)
    ok = fj >= 0
    a, b = anc[fi[ok]], anc[fj[ok]]
    cross = a != b
    a, b = a[cross], b[cross]
    keep = np.zeros(ncoarse, bool)
    keep[seeds] = True
    front = np.asarray(seeds)
    for _ in range(rings):
        sel = np.isin(a, front)
        nxt = np.unique(b[sel])
        nxt = nxt[~keep[nxt]]
        keep[nxt] = True
        front = nxt
    fine = np.nonzero(keep[anc])[0]
    sub, cells, _ = ring_submesh(mesh, fine, rings=0)
    assert np.array_equal(cells, fine)
    parents, cur = [], fine
    for p in par:
        up = p[cur]
        ids = np.unique(up)
        parents.append(np.ascontiguousarray(np.searchsorted(ids, up), np.int32))
        cur = ids
    sub["parents"] = parents
    return sub, cur, np.searchsorted(cur, np.asarray(seeds))


# local faces of the mixed-element cell types (node counts 4, 5, 6, 8), in the
# node order of the mesh generators
MIXED_FACES = {
    4: [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)],
    5: [(0, 1, 2, 3), (0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4)],
    6: [(0, 1, 2), (3, 4, 5), (0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5)],
    8: [(0, 1, 2, 3), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)],
}


def mixed_cell_faces(mesh):
    """For each cell, its faces as (sorted node-id key, local vertex coordinates
    in cyclic order); and the boundary-face keys with their tags."""
    off, nodes, xyz, types = mesh["cell_node_off"], mesh["cell_nodes"], mesh["cell_xyz"], mesh["cell_type"]
    cells = []
    for c in range(len(types)):
        ids = nodes[off[c]:off[c + 1]]
        X = xyz[off[c]:off[c + 1]]
        cells.append([(tuple(sorted(int(ids[v]) for v in f)), X[list(f)]) for f in MIXED_FACES[int(types[c])]])
    boff, bnodes = mesh["bface_node_off"], mesh["bface_nodes"]
    bkeys = {tuple(sorted(int(x) for x in bnodes[boff[b]:boff[b + 1]])): int(mesh["bface_tag"][b])
             for b in range(len(mesh["bface_tag"]))}
    return cells, bkeys


def mixed_tets(Xc, faces):
    """Tetrahedra (4 x 3 arrays) of a cell given the local coordinates of its
    faces: apex at the mean of the cell's nodes, each triangular face as it is
    and each quadrilateral as the 4 triangles around its node mean."""
    xm = np.mean(Xc, axis=0)
    out = []
    for F in faces:
        if len(F) == 3:
            out.append(np.array([xm, F[0], F[1], F[2]]))
        else:
            fc = F.mean(0)
            for i in range(4):
                out.append(np.array([xm, fc, F[i], F[(i + 1) % 4]]))
    return out
