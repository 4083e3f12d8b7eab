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
