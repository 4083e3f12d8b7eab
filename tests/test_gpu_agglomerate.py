"""Agglomeration coarsening (Sec 5.1) through the C ABI against the oracle:
the parent arrays bit-exact on the synthetic meshes and the hand-built cases
(the decisions are FP64 comparisons on both sides; every tested sin(alpha)
is checked to lie well away from the limit, so rounding order cannot flip
one), argument errors as status codes, and the V-cycle on an agglomerated
hierarchy against the oracle's V-cycle on the same hierarchy."""
import math

import numpy as np
import pytest

import oracle
from oracle import agglomerate as oa
import test_gpu_parity as tp
import test_oracle_agglomerate as hand

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    return cgks


@pytest.fixture(scope="module")
def ctx(cg):
    c = cg.Context()
    yield c
    c.close()


@pytest.mark.parametrize("name", list(tp.MESHES))
@pytest.mark.parametrize("min_skew", [0.0, 0.1, 0.3])
def test_parents_bit_exact(ctx, name, min_skew):
    m = tp.MESHES[name]
    st = {}
    po = oa.agglomerate(m, 3, 3, min_skew, st)
    assert st["margin"] > 1e-9
    pg = ctx.cgks_agglomerate(m, 3, 3, min_skew)
    assert len(pg) == len(po) == 2
    for a, b in zip(pg, po):
        np.testing.assert_array_equal(a, b)


def test_hand_built_cases(ctx):
    s = 14.0 / math.sqrt(340.0)
    m = hand._trapezoid()
    assert list(ctx.cgks_agglomerate(m, 2, 1, s - 1e-9)[0]) == [0, 0]
    assert list(ctx.cgks_agglomerate(m, 2, 1, s + 1e-9)[0]) == [0, 1]
    assert list(ctx.cgks_agglomerate(m, 2, 1, 0.72)[0]) == [0, 0]
    m = hand._bipyramid(1.0, 1.0)
    s = 3.0 / math.sqrt(10.0)
    assert list(ctx.cgks_agglomerate(m, 2, 1, s - 1e-9)[0]) == [0, 0]
    assert list(ctx.cgks_agglomerate(m, 2, 1, s + 1e-9)[0]) == [0, 1]
    xyz = {0: (0.0, 0.0), 1: (1.0, 0.0), 2: (2.0, 0.0), 3: (0.0, 1.0), 4: (1.0, 1.0), 5: (2.0, 1.0)}
    cells = [[0, 1, 3], [1, 2, 4], [1, 4, 3], [2, 5, 4]]
    bf = [[0, 1], [1, 2], [2, 5], [5, 4], [4, 3], [3, 0]]
    strip = hand._mesh(2, cells, xyz, bf, [2] * 6)
    assert list(ctx.cgks_agglomerate(strip, 2, 1, 0.5)[0]) == [0, 1, 0, 2]
    assert ctx.cgks_agglomerate(strip, 1) == []


def test_argument_errors(cg, ctx):
    m = tp.MESHES["cylinder"]
    for kw in (dict(n_levels=0), dict(n_levels=9), dict(passes=0), dict(passes=9), dict(min_skew=1.0),
               dict(min_skew=float("nan"))):
        with pytest.raises(cg.CgksError) as e:
            ctx.cgks_agglomerate(m, **kw)
        assert e.value.code == -1
    m = hand._trapezoid()
    m["bface_nodes"] = m["bface_nodes"][1:]
    m["bface_tag"] = m["bface_tag"][1:]
    with pytest.raises(cg.CgksError) as e:
        ctx.cgks_agglomerate(m, 2, 1)
    assert e.value.code == -2
    # the context stays usable
    assert len(ctx.cgks_agglomerate(tp.MESHES["vortex"], 2, 1)) == 1


@pytest.mark.parametrize("name,ncyc", [("vortex", 4), ("cylinder", 4), ("sphere", 2)])
def test_vcycle_on_agglomerated_hierarchy(ctx, name, ncyc):
    """Level sizes, colourings, and plain-FP64 V-cycles on the agglomerated
    hierarchy against the oracle on the same parents."""
    m = dict(tp.MESHES[name])
    m["parents"] = ctx.cgks_agglomerate(m, 3, 3, 0.1)
    mid = 40 + list(tp.MESHES).index(name)
    W, G, w = tp.state_for(name, m, np.random.default_rng(12))
    ctx.setup(mid, m, w, W, G)
    om = oracle.OracleMesh(m)
    info = ctx.cgks_mesh_info(mid)
    for l, lv in enumerate(info):
        assert lv["cells"] == om.n_cells(l)
        assert lv["faces"] == len(om.faces(l)["S"])
        np.testing.assert_array_equal(ctx.cgks_get_coloring(mid, l, lv["cells"]), om.colors(l))
    dim, nv, n = m["dim"], m["dim"] + 2, len(W)
    norms = np.zeros((ncyc, nv, 2))
    ctx.cgks_vcycle([mid], ncyc, 0, norms)
    Wd = np.zeros_like(W)
    ctx.cgks_get_state(mid, Wd)
    out = om.vcycle(oracle.cfg_vector(dim, winf=w), W, G, np.ones(n), ncyc)
    np.testing.assert_allclose(norms, out["norms"], rtol=1e-8)
    np.testing.assert_allclose(Wd, out["W"], rtol=0, atol=1e-9 * np.max(np.abs(W)))
