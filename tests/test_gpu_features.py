"""GPU parity of the learned correction's input features (76 per cell) against a
numpy reconstruction from the state, the residual and the mesh.  Per cell: W,
slopes times |Omega|^(1/2), R dt_imp / |Omega| and the DF factor, scaled by the
free stream (rho, rho c, rho c, rho c^2); then the three face neighbours in
stored face order (face k opposite vertex k), with wall (mirror) and far-field
(free stream on inflow, copy on outflow) ghosts across boundary faces; then
the fine residual summed over the cell's parent and grandparent, times
dt_imp (|Omega_I| / |Omega|)^(1/2) / |Omega_I|, scaled like W.  With
learned_scale = 1 the 24 residual-type inputs are further divided by the cell's
dt_imp times the RMS over the variables of the mesh's residual norms (RMS over
cells of R_v / |Omega|, free-stream units).  The GPU rounds to bfloat16, so the
bound is 2^-8 relative."""
import numpy as np
import pytest

from paper_2509_06347_b300 import synth
from helpers import GAMMA, face_neighbours
import test_gpu_parity as tp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    return cgks


def _ghost(tag, w, n, W, G):
    if tag == synth.TAG_WALL:
        Wg = W.copy()
        Wg[1:3] = W[1:3] - 2.0 * (W[1:3] @ n) * n
        t = G - 2.0 * np.outer(G @ n, n)
        for d in range(2):
            s = n @ t[1:3, d]
            t[1:3, d] -= 2.0 * n * s
        return Wg, t
    if w[1:3] @ n < 0.0:  # inflow
        return w.copy(), np.zeros_like(G)
    return W.copy(), G.copy()


# the residual-type inputs: the residual increments of the cell and of its three
# neighbours, then the parent's and the grandparent's defects
RES_COLS = np.r_[12:16, 29:33, 46:50, 63:67, 68:76]


@pytest.mark.parametrize("learned_scale", [0, 1])
def test_features_match_numpy(cg, learned_scale):
    m = tp.MESHES["cylinder"]
    rng = np.random.default_rng(21)
    W, G, w = tp.state_for("cylinder", m, rng)
    n = len(W)
    ctx = cg.Context(learned_scale=learned_scale)
    try:
        ctx.cgks_mlp_set_params(synth.mlp_init_params())
        ctx.setup(1, m, w, W, G)
        R, al = np.zeros((n, 4)), np.zeros(n)
        ctx.cgks_residual(1, 0, None, R, None, al)
        dte, dti = np.zeros(n), np.zeros(n)
        ctx.cgks_reconstruct(1, None, dte, dti)
        X = ctx.cgks_mlp_features(1).astype(np.float64)
    finally:
        ctx.close()

    p = m["cell_xyz"]
    V = 0.5 * np.abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                     - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    h = np.sqrt(V)
    u = w[1:3] / w[0]
    pinf = (GAMMA - 1) * (w[3] - 0.5 * w[0] * (u @ u))
    c = np.sqrt(GAMMA * pinf / w[0])
    sc = np.array([w[0], w[0] * c, w[0] * c, w[0] * c * c])

    def block(Wc, Gc, hc, Rc, ac):
        out = np.empty(17)
        out[0:4] = Wc / sc
        out[4:12] = (Gc * hc / sc[:, None]).reshape(-1)
        out[12:16] = Rc / sc
        out[16] = ac
        return out

    cn = np.asarray(m["cell_nodes"], np.int64)
    nb, faces = face_neighbours(cn)
    btag = {tuple(sorted(r)): int(t) for r, t in zip(np.asarray(m["bface_nodes"]), m["bface_tag"])}
    E = np.empty((n, 76))
    for i in range(n):
        E[i, :17] = block(W[i], G[i], h[i], R[i] * dti[i] / V[i], al[i])
        for k in range(3):
            j = nb[i, k]
            if j >= 0:
                E[i, 17 * (k + 1):17 * (k + 2)] = block(W[j], G[j], h[j], R[j] * dti[j] / V[j], al[j])
                continue
            a, b = [q for q in range(3) if q != k]
            t = p[i, b] - p[i, a]
            nrm = np.array([t[1], -t[0]]) / np.hypot(t[0], t[1])
            if nrm @ (0.5 * (p[i, a] + p[i, b]) - p[i, k]) < 0:
                nrm = -nrm
            tag = btag[tuple(sorted(faces[i, k]))]
            Wg, Gg = _ghost(tag, w, nrm, W[i], G[i])
            E[i, 17 * (k + 1):17 * (k + 2)] = block(Wg, Gg, h[i], np.zeros(4), al[i])
    # restricted residuals of the parent (level 1) and grandparent (level 2)
    p1 = np.asarray(m["parents"][0], np.int64)
    p2 = np.asarray(m["parents"][1], np.int64)
    n1, n2 = p1.max() + 1, p2.max() + 1
    R1, V1 = np.zeros((n1, 4)), np.zeros(n1)
    np.add.at(R1, p1, R)
    np.add.at(V1, p1, V)
    R2, V2 = np.zeros((n2, 4)), np.zeros(n2)
    np.add.at(R2, p2, R1)
    np.add.at(V2, p2, V1)
    I, J = p1, p2[p1]
    E[:, 68:72] = R1[I] * (dti * np.sqrt(V1[I] / V) / V1[I])[:, None] / sc
    E[:, 72:76] = R2[J] * (dti * np.sqrt(V2[J] / V) / V2[J])[:, None] / sc
    if learned_scale:
        rms = np.sqrt(np.mean((R / V[:, None]) ** 2, axis=0)) / sc
        s = dti * np.sqrt(np.mean(rms ** 2))
        assert np.all(s > 0)
        E[:, RES_COLS] /= s[:, None]
    err = np.abs(X - E)
    bound = 2.0 ** -8 * np.abs(E) + 1e-30
    assert np.all(err <= bound), (np.unravel_index(np.argmax(err - bound), err.shape), np.max(err / (np.abs(E) + 1e-30)))
    # the boundary cells of the mesh were exercised
    assert (nb < 0).any()
