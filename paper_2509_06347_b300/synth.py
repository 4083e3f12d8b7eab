"""Seeded synthetic inputs: meshes, nested hierarchies and initial states.

This module is the only code shared by the CUDA path and the oracle.  It builds
*inputs* (node connectivity, per-cell vertex coordinates, boundary tags, parent
maps, initial cell averages) and holds none of the scheme's arithmetic:
geometry, faces, colouring, reconstruction and fluxes are computed separately
by each side from these raw arrays.

Mesh format (simplices only):
  dim          2 (triangles) or 3 (tetrahedra)
  cell_nodes   int32 [n_cells, dim+1]   topological node ids; periodic images of
                                        a node share one id, so faces match
  cell_xyz     float64 [n_cells, dim+1, dim]  the cell's own (unwrapped) vertex
                                        coordinates; across a periodic boundary a
                                        shared face appears shifted by the period
  bface_nodes  int32 [n_bfaces, dim]    boundary faces (node ids)
  bface_tag    int32 [n_bfaces]         1 = slip wall, 2 = supersonic far field
  parents      list of int32 arrays     parents[l][i] = level-(l+1) parent of
                                        level-l cell i (nested hierarchy)

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).
"""
from __future__ import annotations

import math
import numpy as np

TAG_WALL = 1
TAG_FARFIELD = 2
TAG_NOSLIP_WALL = 3
TAG_FARFIELD_RIEMANN = 4
DEFAULT_SEED = 2509063470

_M64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64: state += golden gamma, then two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


# ----------------------------------------------------------------------------
# 2-D triangle meshes
# ----------------------------------------------------------------------------

def _refine_tri(cell_nodes, cell_s, n_nodes, mapping):
    """One 4-way edge-midpoint split of every triangle.

    cell_s holds each cell's vertex coordinates in a parameter space (unwrapped);
    midpoints are taken there and `mapping` turns parameter coordinates into
    physical ones.  Children of cell p are 4p..4p+3: three corner triangles then
    the middle one, all with the parent's orientation.
    """
    n = cell_nodes.shape[0]
    edge_id = {}
    new_nodes = np.zeros((4 * n, 3), np.int64)
    new_s = np.zeros((4 * n, 3, 2))
    nid = n_nodes
    for c in range(n):
        a, b, cc = (int(v) for v in cell_nodes[c])
        sa, sb, sc = cell_s[c]
        mids = []
        for (p, q, sp, sq) in ((a, b, sa, sb), (b, cc, sb, sc), (cc, a, sc, sa)):
            key = (p, q) if p < q else (q, p)
            if key not in edge_id:
                edge_id[key] = nid
                nid += 1
            mids.append((edge_id[key], 0.5 * (sp + sq)))
        (mab, sab), (mbc, sbc), (mca, sca) = mids
        new_nodes[4 * c + 0] = (a, mab, mca)
        new_s[4 * c + 0] = (sa, sab, sca)
        new_nodes[4 * c + 1] = (mab, b, mbc)
        new_s[4 * c + 1] = (sab, sb, sbc)
        new_nodes[4 * c + 2] = (mca, mbc, cc)
        new_s[4 * c + 2] = (sca, sbc, sc)
        new_nodes[4 * c + 3] = (mab, mbc, mca)
        new_s[4 * c + 3] = (sab, sbc, sca)
    return new_nodes, new_s, nid, edge_id


def _refine_bfaces(bface_nodes, bface_s, edge_id):
    """Split each boundary edge in two, following the cells' edge midpoints."""
    out_nodes, out_s = [], []
    for (p, q), (sp, sq) in zip(bface_nodes, bface_s):
        p, q = int(p), int(q)
        key = (p, q) if p < q else (q, p)
        m = edge_id[key]
        sm = 0.5 * (sp + sq)
        out_nodes += [(p, m), (m, q)]
        out_s += [(sp, sm), (sm, sq)]
    return np.array(out_nodes, np.int64), np.array(out_s)


def _finish(dim, cell_nodes, cell_xyz, bface_nodes, bface_tag, parents, **extra):
    m = dict(dim=dim,
             cell_nodes=np.ascontiguousarray(cell_nodes, np.int32),
             cell_xyz=np.ascontiguousarray(cell_xyz, np.float64),
             bface_nodes=np.ascontiguousarray(bface_nodes, np.int32).reshape(-1, dim),
             bface_tag=np.ascontiguousarray(bface_tag, np.int32),
             parents=[np.ascontiguousarray(p, np.int32) for p in parents])
    m.update(extra)
    return m


def vortex_mesh(n_coarse: int = 8, n_refine: int = 2, jitter: float = 0.1,
                length: float = 10.0, seed: int = DEFAULT_SEED + 0):
    """Jittered periodic triangle mesh of [0, L]^2.

    n_coarse^2 quads, each split along the same diagonal, interior nodes moved
    by a seeded uniform +-jitter*h in x and y independently (boundary nodes are
    kept so periodic edges match), then n_refine 4-way splits.  The hierarchy
    returned is nested: level l+1 cells are the level-l cells before one split.
    """
    h = length / n_coarse
    rng = SplitMix64(seed)
    pos = np.zeros((n_coarse + 1, n_coarse + 1, 2))
    for j in range(n_coarse + 1):
        for i in range(n_coarse + 1):
            pos[i, j] = (i * h, j * h)
    for j in range(1, n_coarse):
        for i in range(1, n_coarse):
            dx = (2.0 * rng.uniform() - 1.0) * jitter * h
            dy = (2.0 * rng.uniform() - 1.0) * jitter * h
            pos[i, j] += (dx, dy)

    def nid(i, j):
        return (i % n_coarse) + n_coarse * (j % n_coarse)

    cells, cs = [], []
    for j in range(n_coarse):
        for i in range(n_coarse):
            q = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
            for tri in ((0, 1, 2), (0, 2, 3)):
                cells.append([nid(*q[t]) for t in tri])
                cs.append([pos[q[t]] for t in tri])
    cell_nodes = np.array(cells, np.int64)
    cell_s = np.array(cs)
    n_nodes = n_coarse * n_coarse
    levels = [(cell_nodes, cell_s)]
    for _ in range(n_refine):
        cell_nodes, cell_s, n_nodes, _e = _refine_tri(cell_nodes, cell_s, n_nodes, None)
        levels.append((cell_nodes, cell_s))
    parents = []
    for lv in range(n_refine):
        nf = levels[n_refine - lv][0].shape[0]
        parents.append(np.arange(nf) // 4)
    return _finish(2, cell_nodes, cell_s, np.zeros((0, 2)), np.zeros(0), parents,
                   name=f"vortex{n_coarse}x{n_coarse}r{n_refine}", length=length,
                   level_sizes=[levels[n_refine - l][0].shape[0] for l in range(n_refine + 1)])


def radial_nodes(n_r: int, r_in: float, r_out: float, ratio: float):
    """First spacing h0 such that n_r layers growing by `ratio` span [r_in, r_out]."""
    return (r_out - r_in) * (ratio - 1.0) / (ratio ** n_r - 1.0)


def cylinder_mesh(n_theta: int = 64, n_r: int = 32, ratio: float = 1.05,
                  r_in: float = 1.0, r_out: float = 15.0, n_refine: int = 2):
    """O-mesh around the unit cylinder, split into triangles and refined.

    Coarse quads (n_theta periodic in theta, n_r radial, radial spacing growing
    by `ratio` from r_in to r_out) are split along a fixed diagonal; refined
    nodes sit at index-space midpoints mapped through (theta, r), so fine wall
    nodes lie on the circle.  Boundary tags: wall at r_in, far field at r_out.
    """
    h0 = radial_nodes(n_r, r_in, r_out, ratio)

    def rmap(s):  # index-space radial coordinate -> radius
        return r_in + h0 * (ratio ** s - 1.0) / (ratio - 1.0)

    def to_xyz(s):
        th = 2.0 * math.pi * s[..., 0] / n_theta
        r = rmap(s[..., 1])
        return np.stack([r * np.cos(th), r * np.sin(th)], axis=-1)

    def nid(i, j):
        return (i % n_theta) + n_theta * j

    cells, cs = [], []
    for j in range(n_r):
        for i in range(n_theta):
            q = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
            for tri in ((0, 1, 2), (0, 2, 3)):
                cells.append([nid(*q[t]) for t in tri])
                cs.append([np.array(q[t], float) for t in tri])
    cell_nodes = np.array(cells, np.int64)
    cell_s = np.array(cs)
    bn, bs, bt = [], [], []
    for i in range(n_theta):
        # wall edge (j = 0) and far-field edge (j = n_r)
        bn.append((nid(i, 0), nid(i + 1, 0)))
        bs.append((np.array((i, 0.0)), np.array((i + 1, 0.0))))
        bt.append(TAG_WALL)
        bn.append((nid(i, n_r), nid(i + 1, n_r)))
        bs.append((np.array((i, float(n_r))), np.array((i + 1, float(n_r)))))
        bt.append(TAG_FARFIELD)
    bface_nodes = np.array(bn, np.int64)
    bface_s = np.array(bs)
    bface_tag = np.array(bt, np.int64)
    n_nodes = n_theta * (n_r + 1)
    sizes = [cell_nodes.shape[0]]
    for _ in range(n_refine):
        cell_nodes, cell_s, n_nodes, edge_id = _refine_tri(cell_nodes, cell_s, n_nodes, None)
        bface_nodes, bface_s = _refine_bfaces(bface_nodes, bface_s, edge_id)
        bface_tag = np.repeat(bface_tag, 2)
        sizes.append(cell_nodes.shape[0])
    parents = [np.arange(sizes[n_refine - lv]) // 4 for lv in range(n_refine)]
    return _finish(2, cell_nodes, to_xyz(cell_s), bface_nodes, bface_tag, parents,
                   name=f"cylinder{n_theta}x{n_r}r{n_refine}", r_in=r_in, r_out=r_out,
                   level_sizes=sizes[::-1])


# ----------------------------------------------------------------------------
# 3-D cubed-sphere tetrahedral mesh
# ----------------------------------------------------------------------------

# Each panel: fixed axis and sign, then the two tangential global axes in
# increasing order, so every seam is parametrised the same way by both panels.
_PANELS = [(0, +1), (0, -1), (1, +1), (1, -1), (2, +1), (2, -1)]

# Kuhn split of a hex: one tet per permutation of the three index axes, each a
# monotone lattice path from corner (0,0,0) to (1,1,1).
_KUHN = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def sphere_mesh(n_panel: int = 32, n_r: int = 32, ratio: float = 1.08,
                r_in: float = 1.0, r_out: float = 15.0):
    """Equiangular cubed-sphere shell of hexes, each split into 6 tets.

    Hierarchy: level 1 = the hexes (6 tets each); level 2 = 2x2x2 hex blocks
    (needs even n_panel and n_r).  Tags: wall at r_in, far field at r_out.
    """
    assert n_panel % 2 == 0 and n_r % 2 == 0
    h0 = radial_nodes(n_r, r_in, r_out, ratio)
    radii = r_in + h0 * (ratio ** np.arange(n_r + 1) - 1.0) / (ratio - 1.0)
    radii[-1] = r_out
    # global node ids of surface nodes, keyed by integer cube-surface coordinates
    key_to_id = {}
    ang = np.tan(0.25 * math.pi * (2.0 * np.arange(n_panel + 1) / n_panel - 1.0))
    surf_dir = []
    panel_ids = np.zeros((6, n_panel + 1, n_panel + 1), np.int64)
    for p, (ax, sg) in enumerate(_PANELS):
        t1, t2 = [a for a in range(3) if a != ax]
        for a in range(n_panel + 1):
            for b in range(n_panel + 1):
                key = [0, 0, 0]
                key[ax] = sg * n_panel
                key[t1] = 2 * a - n_panel
                key[t2] = 2 * b - n_panel
                key = tuple(key)
                if key not in key_to_id:
                    d = np.zeros(3)
                    d[ax] = sg
                    d[t1] = ang[a]
                    d[t2] = ang[b]
                    key_to_id[key] = len(surf_dir)
                    surf_dir.append(d / np.linalg.norm(d))
                panel_ids[p, a, b] = key_to_id[key]
    surf_dir = np.array(surf_dir)
    ns = surf_dir.shape[0]
    n_hex = 6 * n_panel * n_panel * n_r
    # hex corners (di, dj, dk) -> node id / coordinate
    P, A, B, K = np.meshgrid(np.arange(6), np.arange(n_panel), np.arange(n_panel),
                             np.arange(n_r), indexing="ij")
    # hex ordering: level-2 blocks contiguous (8 hexes each), so parents are i // 8
    blk = (((P * (n_panel // 2) + A // 2) * (n_panel // 2) + B // 2) * (n_r // 2) + K // 2)
    sub = ((A % 2) * 2 + (B % 2)) * 2 + (K % 2)
    hex_index = (blk * 8 + sub).ravel()
    order = np.argsort(hex_index, kind="stable")
    Pf, Af, Bf, Kf = (x.ravel()[order] for x in (P, A, B, K))
    cn = np.zeros((n_hex, 6, 4), np.int64)
    cx = np.zeros((n_hex, 6, 4, 3))
    corner_id = {}
    corner_xyz = {}
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                sid = panel_ids[Pf, Af + di, Bf + dj]
                corner_id[(di, dj, dk)] = sid + ns * (Kf + dk)
                corner_xyz[(di, dj, dk)] = surf_dir[sid] * radii[Kf + dk][:, None]
    for t, perm in enumerate(_KUHN):
        c = [0, 0, 0]
        path = [tuple(c)]
        for axis in perm:
            c[axis] = 1
            path.append(tuple(c))
        for v, corner in enumerate(path):
            cn[:, t, v] = corner_id[corner]
            cx[:, t, v] = corner_xyz[corner]
    cell_nodes = cn.reshape(-1, 4)
    cell_xyz = cx.reshape(-1, 4, 3)
    # boundary faces: the two triangles of each hex's inner (k = 0) and outer face
    bn, bt = [], []
    for p in range(6):
        for a in range(n_panel):
            for b in range(n_panel):
                for (k, tag) in ((0, TAG_WALL), (n_r, TAG_FARFIELD)):
                    q00 = panel_ids[p, a, b] + ns * k
                    q10 = panel_ids[p, a + 1, b] + ns * k
                    q11 = panel_ids[p, a + 1, b + 1] + ns * k
                    q01 = panel_ids[p, a, b + 1] + ns * k
                    # the Kuhn split cuts this face along the (0,0)-(1,1) diagonal
                    bn += [(q00, q10, q11), (q00, q11, q01)]
                    bt += [tag, tag]
    parents = [np.arange(6 * n_hex) // 6, np.arange(n_hex) // 8]
    return _finish(3, cell_nodes, cell_xyz, np.array(bn), np.array(bt), parents,
                   name=f"sphere{n_panel}x{n_r}", r_in=r_in, r_out=r_out,
                   level_sizes=[6 * n_hex, n_hex, n_hex // 8])


def batch_cylinder_specs(n_meshes: int = 64, seed: int = DEFAULT_SEED + 3,
                         mach_lo: float = 1.5, mach_hi: float = 8.0):
    """Seeded (n_theta, n_r, ratio, mach) for the batched parametric sweep.

    n_theta uniform in {32, 48, ..., 128}, n_r = n_theta / 2, radial ratio
    1.05^(32 / n_r) so that ratio^n_r matches the 64x32 mesh and the outer
    radius stays 15, Mach uniform in [mach_lo, mach_hi].
    """
    rng = SplitMix64(seed)
    choices = list(range(32, 129, 16))
    specs = []
    for _ in range(n_meshes):
        nt = choices[min(int(rng.uniform() * len(choices)), len(choices) - 1)]
        mach = mach_lo + (mach_hi - mach_lo) * rng.uniform()
        nr = nt // 2
        specs.append(dict(n_theta=nt, n_r=nr, ratio=1.05 ** (32.0 / nr), mach=mach))
    return specs


# ----------------------------------------------------------------------------
# Initial states (conservative variables rho, rho*u, rho*v, [rho*w], rho*E)
# ----------------------------------------------------------------------------

def freestream(mach: float, gamma: float = 1.4, dim: int = 2, angle_deg: float = 0.0):
    """rho = 1, p = 1/gamma (so c = 1), velocity mach along x rotated by angle."""
    rho, p = 1.0, 1.0 / gamma
    a = math.radians(angle_deg)
    vel = [mach * math.cos(a), mach * math.sin(a)] + ([0.0] if dim == 3 else [])
    w = [rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + 0.5 * rho * mach * mach]
    return np.array(w)


def uniform_state(mesh, w):
    n = len(mesh["cell_type"]) if mesh.get("mixed") else mesh["cell_nodes"].shape[0]
    return np.tile(np.asarray(w, float), (n, 1))


def _tri_rule(order_1d: int = 6):
    """Collapsed (Duffy) tensor Gauss rule on the reference triangle.

    Exact for polynomials of degree <= 2*order_1d - 2; returns barycentric
    points and weights summing to 1.
    """
    x, w = np.polynomial.legendre.leggauss(order_1d)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    pts, wts = [], []
    for xi, wi in zip(x, w):
        for yj, wj in zip(x, w):
            s = xi
            t = yj * (1.0 - xi)
            pts.append((1.0 - s - t, s, t))
            wts.append(wi * wj * (1.0 - xi) * 2.0)
    return np.array(pts), np.array(wts)


def vortex_fields(x, y, gamma=1.4, eps=5.0, xc=5.0, yc=5.0):
    """Isentropic vortex with zero mean flow (conservative variables)."""
    xb, yb = x - xc, y - yc
    r2 = xb * xb + yb * yb
    e = np.exp(0.5 * (1.0 - r2))
    du = eps / (2.0 * math.pi) * e * (-yb)
    dv = eps / (2.0 * math.pi) * e * xb
    T = 1.0 - (gamma - 1.0) * eps * eps * e * e / (8.0 * gamma * math.pi ** 2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    E = p / (gamma - 1.0) + 0.5 * rho * (du * du + dv * dv)
    return np.stack([rho, rho * du, rho * dv, E], axis=-1)


def vortex_state(mesh, gamma: float = 1.4, eps: float = 5.0, order_1d: int = 6,
                 edge_pts: int = 8):
    """Cell averages and mean slopes (1/V) \\oint W n ds of the vortex.

    Averages use a degree-10 collapsed Gauss rule per triangle; mean slopes a
    Gauss-Legendre rule with `edge_pts` points per edge.  Returns (W, grad) with
    grad laid out [n_cells, nv, dim].
    """
    xyz = mesh["cell_xyz"]
    L = mesh.get("length", 10.0)
    bary, wts = _tri_rule(order_1d)
    pts = np.einsum("qv,cvd->cqd", bary, xyz)
    f = vortex_fields(pts[..., 0], pts[..., 1], gamma, eps, 0.5 * L, 0.5 * L)
    W = np.einsum("q,cqn->cn", wts, f)
    a = xyz[:, 1] - xyz[:, 0]
    b = xyz[:, 2] - xyz[:, 0]
    area = 0.5 * (a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    s, ws = np.polynomial.legendre.leggauss(edge_pts)
    s = 0.5 * (s + 1.0)
    ws = 0.5 * ws
    grad = np.zeros((xyz.shape[0], 4, 2))
    for (i, j) in ((0, 1), (1, 2), (2, 0)):
        p0, p1 = xyz[:, i], xyz[:, j]
        e = p1 - p0
        # outward normal times length for counter-clockwise cells: (ey, -ex)
        nvec = np.stack([e[:, 1], -e[:, 0]], axis=-1) * np.sign(area)[:, None]
        q = p0[:, None, :] + s[None, :, None] * e[:, None, :]
        fv = vortex_fields(q[..., 0], q[..., 1], gamma, eps, 0.5 * L, 0.5 * L)
        fm = np.einsum("q,cqn->cn", ws, fv)
        grad += fm[:, :, None] * nvec[:, None, :]
    grad /= np.abs(area)[:, None, None]
    return W, grad


def concat_meshes(meshes):
    """Concatenate meshes (same dim, same number of levels) into one
    disconnected mesh.  Node ids, cells, boundary faces and parent maps are
    offset per mesh; returns (union mesh, group_of_cell) where group_of_cell[i]
    is the index of the mesh that fine cell i came from."""
    dim = meshes[0]["dim"]
    nlev = len(meshes[0]["parents"]) + 1
    cn, cx, bn, bt, grp = [], [], [], [], []
    parents = [[] for _ in range(nlev - 1)]
    node_off = 0
    lev_off = [0] * nlev
    for g, m in enumerate(meshes):
        assert m["dim"] == dim and len(m["parents"]) + 1 == nlev
        cn.append(m["cell_nodes"].astype(np.int64) + node_off)
        cx.append(m["cell_xyz"])
        if m["bface_nodes"].size:
            bn.append(m["bface_nodes"].astype(np.int64) + node_off)
            bt.append(m["bface_tag"])
        grp.append(np.full(m["cell_nodes"].shape[0], g, np.int32))
        sizes = [m["cell_nodes"].shape[0]] + [int(p.max()) + 1 for p in m["parents"]]
        for l, p in enumerate(m["parents"]):
            parents[l].append(p.astype(np.int64) + lev_off[l + 1])
        for l in range(nlev):
            lev_off[l] += sizes[l]
        node_off += int(max(m["cell_nodes"].max(), m["bface_nodes"].max() if m["bface_nodes"].size else 0)) + 1
    union = _finish(dim, np.concatenate(cn), np.concatenate(cx),
                    np.concatenate(bn) if bn else np.zeros((0, dim)),
                    np.concatenate(bt) if bt else np.zeros(0),
                    [np.concatenate(p) for p in parents],
                    name=f"batch{len(meshes)}", level_sizes=lev_off)
    return union, np.concatenate(grp)


MLP_LAYERS = ((64, 76), (64, 64), (4, 64))  # (outputs, inputs) of the per-cell network


def mlp_init_params(seed: int = DEFAULT_SEED + 4):
    """Seeded He-style initial weights of the per-cell network, flat
    [W1 (64x76 row-major), b1, W2 (64x64), b2, W3 (4x64), b3] = 9,348 values,
    biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in MLP_LAYERS:
        parts.append(rng.standard_normal(o * i) * math.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)


def batch_cylinders(specs):
    """Meshes, free streams and initial states of a batched cylinder sweep."""
    meshes, winf = [], []
    for s in specs:
        meshes.append(cylinder_mesh(n_theta=s["n_theta"], n_r=s["n_r"], ratio=s["ratio"], n_refine=2))
        winf.append(freestream(s["mach"]))
    union, grp = concat_meshes(meshes)
    W = np.asarray(winf)[grp]
    return union, grp, np.asarray(winf), W


# ----------------------------------------------------------------------------
# 3-D mixed-element meshes (hexahedra, prisms, pyramids)
# ----------------------------------------------------------------------------
# Cell types are given by their node counts.  Local node order:
#   tet (4)      any; face k is opposite node k
#   pyramid (5)  base 0-1-2-3 (cyclic), apex 4
#   prism (6)    bottom triangle 0-1-2, top 3-4-5 (3 above 0, 4 above 1, 5 above 2)
#   hex (8)      bottom 0-1-2-3 (cyclic), top 4-5-6-7 (4 above 0, ...)
CELL_TET, CELL_PYRAMID, CELL_PRISM, CELL_HEX = 4, 5, 6, 8

# hex slot corners (di, dj, dk) in the hex node order above
_HEX_CORNERS = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
# the six quads of a hex, cyclic, in hex node indices
_HEX_FACES = [(0, 1, 2, 3), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7)]
# a prism column splits every slot along the (0,0)-(1,1) diagonal of its (i, j) plane
_PRISM_SPLIT = [(0, 1, 2, 4, 5, 6), (0, 2, 3, 4, 6, 7)]


def _mixed_cells(corner_id, corner_xyz, kind, next_id):
    """Cells of hex slots.  corner_id [ns][8], corner_xyz [ns][8][3] in hex
    node order; kind [ns]: 0 hex, 1 two prisms, 2 six pyramids around a new
    node at the slot's corner average (ids from next_id on).  Returns
    (cell_type, cell_node_off, cell_nodes, cell_xyz, slot of each cell)."""
    types, nodes, xyz, slot = [], [], [], []
    for s in range(len(kind)):
        ids, X = corner_id[s], corner_xyz[s]
        if kind[s] == 0:
            types.append(CELL_HEX)
            nodes.append(list(ids))
            xyz.append(X)
            slot.append(s)
        elif kind[s] == 1:
            for sp in _PRISM_SPLIT:
                types.append(CELL_PRISM)
                nodes.append([ids[v] for v in sp])
                xyz.append(X[list(sp)])
                slot.append(s)
        else:
            apex = next_id
            next_id += 1
            xa = X.mean(0)
            for fc in _HEX_FACES:
                types.append(CELL_PYRAMID)
                nodes.append([ids[v] for v in fc] + [apex])
                xyz.append(np.vstack([X[list(fc)], xa[None, :]]))
                slot.append(s)
    off = np.zeros(len(types) + 1, np.int64)
    off[1:] = np.cumsum([len(t) for t in nodes])
    return (np.array(types, np.int32), off, np.concatenate([np.asarray(t, np.int64) for t in nodes]),
            np.concatenate(xyz), np.array(slot, np.int64))


def _mixed_finish(types, off, nodes, xyz, slot, bnodes, btags, n_slots, **extra):
    boff = np.zeros(len(bnodes) + 1, np.int64)
    boff[1:] = np.cumsum([len(b) for b in bnodes])
    return dict(dim=3, mixed=True,
                cell_type=np.ascontiguousarray(types, np.int32),
                cell_node_off=np.ascontiguousarray(off, np.int64),
                cell_nodes=np.ascontiguousarray(nodes, np.int32),
                cell_xyz=np.ascontiguousarray(xyz, np.float64).reshape(-1, 3),
                bface_node_off=boff,
                bface_nodes=np.ascontiguousarray(np.concatenate([np.asarray(b) for b in bnodes]), np.int32),
                bface_tag=np.ascontiguousarray(btags, np.int32),
                parents=[np.ascontiguousarray(slot, np.int32), np.ascontiguousarray(np.arange(n_slots) // 8, np.int32)],
                **extra)


def _slot_kinds(n_cols, n_layers, prism_frac, pyramid_frac, seed):
    """Seeded slot kinds: whole columns of prisms (their triangular caps meet
    only each other), pyramid sextets elsewhere, hexes otherwise."""
    rng = SplitMix64(seed)
    col_prism = np.array([rng.uniform() < prism_frac for _ in range(n_cols)])
    kind = np.zeros((n_cols, n_layers), np.int64)
    for c in range(n_cols):
        for k in range(n_layers):
            u = rng.uniform()
            kind[c, k] = 1 if col_prism[c] else (2 if u < pyramid_frac else 0)
    return kind


def mixed_shell_mesh(n_panel: int = 8, n_r: int = 8, ratio: float = 1.08, r_in: float = 1.0,
                     r_out: float = 15.0, prism_frac: float = 0.25, pyramid_frac: float = 0.2,
                     seed: int = DEFAULT_SEED + 6):
    """Cubed-sphere shell (as sphere_mesh) of hex slots, each kept as a hex,
    split into two prisms (whole radial columns, seeded) or into six pyramids
    around its centre (seeded).  Faces: quadrilaterals (curved: their corners
    lie on spheres) and triangles.  Hierarchy: level 1 = the slots, level 2 =
    2x2x2 slot blocks.  Tags: wall at r_in, far field at r_out."""
    assert n_panel % 2 == 0 and n_r % 2 == 0
    h0 = radial_nodes(n_r, r_in, r_out, ratio)
    radii = r_in + h0 * (ratio ** np.arange(n_r + 1) - 1.0) / (ratio - 1.0)
    radii[-1] = r_out
    key_to_id, surf_dir = {}, []
    ang = np.tan(0.25 * math.pi * (2.0 * np.arange(n_panel + 1) / n_panel - 1.0))
    panel_ids = np.zeros((6, n_panel + 1, n_panel + 1), np.int64)
    for p, (ax, sg) in enumerate(_PANELS):
        t1, t2 = [a for a in range(3) if a != ax]
        for a in range(n_panel + 1):
            for b in range(n_panel + 1):
                key = [0, 0, 0]
                key[ax] = sg * n_panel
                key[t1] = 2 * a - n_panel
                key[t2] = 2 * b - n_panel
                key = tuple(key)
                if key not in key_to_id:
                    d = np.zeros(3)
                    d[ax], d[t1], d[t2] = sg, ang[a], ang[b]
                    key_to_id[key] = len(surf_dir)
                    surf_dir.append(d / np.linalg.norm(d))
                panel_ids[p, a, b] = key_to_id[key]
    surf_dir = np.array(surf_dir)
    ns_ = surf_dir.shape[0]
    # slots ordered so that 2x2x2 blocks are contiguous
    P, A, B, K = np.meshgrid(np.arange(6), np.arange(n_panel), np.arange(n_panel), np.arange(n_r), indexing="ij")
    blk = (((P * (n_panel // 2) + A // 2) * (n_panel // 2) + B // 2) * (n_r // 2) + K // 2)
    sub = ((A % 2) * 2 + (B % 2)) * 2 + (K % 2)
    order = np.argsort((blk * 8 + sub).ravel(), kind="stable")
    Pf, Af, Bf, Kf = (x.ravel()[order] for x in (P, A, B, K))
    n_slots = len(Pf)
    cid = np.zeros((n_slots, 8), np.int64)
    cxyz = np.zeros((n_slots, 8, 3))
    for v, (di, dj, dk) in enumerate(_HEX_CORNERS):
        sid = panel_ids[Pf, Af + di, Bf + dj]
        cid[:, v] = sid + ns_ * (Kf + dk)
        cxyz[:, v] = surf_dir[sid] * radii[Kf + dk][:, None]
    kinds_cols = _slot_kinds(6 * n_panel * n_panel, n_r, prism_frac, pyramid_frac, seed)
    col = (Pf * n_panel + Af) * n_panel + Bf
    kind = kinds_cols[col, Kf]
    types, off, nodes, xyz, slot = _mixed_cells(cid, cxyz, kind, ns_ * (n_r + 1))
    bn, bt = [], []
    for p in range(6):
        for a in range(n_panel):
            for b in range(n_panel):
                prism = kinds_cols[(p * n_panel + a) * n_panel + b, 0] == 1
                for (k, tag) in ((0, TAG_WALL), (n_r, TAG_FARFIELD)):
                    q = [panel_ids[p, a, b], panel_ids[p, a + 1, b], panel_ids[p, a + 1, b + 1], panel_ids[p, a, b + 1]]
                    q = [x + ns_ * k for x in q]
                    if prism:
                        bn += [(q[0], q[1], q[2]), (q[0], q[2], q[3])]
                        bt += [tag, tag]
                    else:
                        bn.append(tuple(q))
                        bt.append(tag)
    return _mixed_finish(types, off, nodes, xyz, slot, bn, bt, n_slots,
                         name=f"mixedshell{n_panel}x{n_r}", r_in=r_in, r_out=r_out)


def mixed_box_mesh(n: int = 4, length: float = 4.0, prism_frac: float = 0.25, pyramid_frac: float = 0.2,
                   seed: int = DEFAULT_SEED + 7):
    """Box [0, L]^3 of n^3 cubic hex slots (planar faces), each kept as a hex,
    split into two prisms (whole z columns, seeded) or into six pyramids.
    Levels: slots, then 2x2x2 blocks (n even).  Every boundary face is far
    field."""
    assert n % 2 == 0
    h = length / n
    nid = lambda i, j, k: (k * (n + 1) + j) * (n + 1) + i
    I, J, Kz = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    blk = ((I // 2) * (n // 2) + J // 2) * (n // 2) + Kz // 2
    sub = ((I % 2) * 2 + (J % 2)) * 2 + (Kz % 2)
    order = np.argsort((blk * 8 + sub).ravel(), kind="stable")
    If, Jf, Kf = (x.ravel()[order] for x in (I, J, Kz))
    n_slots = len(If)
    cid = np.zeros((n_slots, 8), np.int64)
    cxyz = np.zeros((n_slots, 8, 3))
    for v, (di, dj, dk) in enumerate(_HEX_CORNERS):
        cid[:, v] = nid(If + di, Jf + dj, Kf + dk)
        cxyz[:, v] = np.stack([(If + di) * h, (Jf + dj) * h, (Kf + dk) * h], 1)
    kinds_cols = _slot_kinds(n * n, n, prism_frac, pyramid_frac, seed)
    kind = kinds_cols[If * n + Jf, Kf]
    types, off, nodes, xyz, slot = _mixed_cells(cid, cxyz, kind, (n + 1) ** 3)
    bn, bt = [], []
    for a in range(n):
        for b in range(n):
            prism = kinds_cols[a * n + b, 0] == 1
            for k in (0, n):  # z faces: triangles on prism columns
                q = [nid(a, b, k), nid(a + 1, b, k), nid(a + 1, b + 1, k), nid(a, b + 1, k)]
                if prism:
                    bn += [(q[0], q[1], q[2]), (q[0], q[2], q[3])]
                    bt += [TAG_FARFIELD, TAG_FARFIELD]
                else:
                    bn.append(tuple(q))
                    bt.append(TAG_FARFIELD)
            for s in (0, n):  # x and y faces: quads
                bn.append((nid(s, a, b), nid(s, a + 1, b), nid(s, a + 1, b + 1), nid(s, a, b + 1)))
                bn.append((nid(a, s, b), nid(a + 1, s, b), nid(a + 1, s, b + 1), nid(a, s, b + 1)))
                bt += [TAG_FARFIELD, TAG_FARFIELD]
    return _mixed_finish(types, off, nodes, xyz, slot, bn, bt, n_slots, name=f"mixedbox{n}", length=length)

