"""The exponential and erfc of the half-space moments (special.cuh) on the
GPU, against mpmath at 30 digits and against the CUDA library's functions:
exp(-|x|) by the table-driven reduction within 4 ulp (0 below -700); erfcx(|x|)
from its piecewise polynomials within 4 ulp (the polynomials are within
3.6e-16); erfc(x) = exp(-x^2) erfcx(x) (x >= 0), 2 - exp(-x^2) erfcx(-x)
(x < 0) within 1e-15 relative plus the rounding of x^2 inside exp,
2 |x|^2 * 2^-52; 0 where x^2 >= 700 (erfc(x) < 2^-1000 there)."""
import mpmath as mp
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06347_b300 import build, cgks
    build.build()
    c = cgks.Context()
    yield c
    c.close()


def _inputs():
    rng = np.random.default_rng(77)
    x = np.concatenate([
        rng.uniform(-6.0, 6.0, 3000),
        rng.uniform(-27.0, 27.0, 500),
        np.arange(0, 129) / 16.0,            # interval edges
        -np.arange(0, 129) / 16.0,
        np.nextafter(np.arange(1, 129) / 16.0, 0),
        [0.0, -0.0, 1e-300, 1e-10, 7.999999999, 8.0, 8.000000001, 12.0, 26.5, 30.0, 1e3, 1e10, np.inf],
        -np.array([1e-10, 1.0, 5.0, 30.0, np.inf]),
        rng.uniform(-700.0, 700.0, 500),         # exp(-|x|) over its whole range
        [699.999, 700.0, 745.0, 800.0],
        np.arange(0, 128) * np.log(2.0) / 64.0,  # table points of the exponential
    ])
    return x


def test_erfcx_and_erfc(ctx):
    mp.mp.dps = 30
    x = _inputs()
    out = ctx.cgks_special_selftest(x)
    ours, ex, ox, lib, lx = out[:, 0], out[:, 1], out[:, 2], out[:, 3], out[:, 4]
    worst_x, worst_e, worst_p = 0.0, 0.0, 0.0
    for i, v in enumerate(x):
        a = abs(float(v))
        if a >= 700.0:
            assert ox[i] == 0.0
        else:
            rp = mp.exp(-mp.mpf(a))
            p_err = abs(mp.mpf(ox[i]) - rp) / rp
            worst_p = max(worst_p, float(p_err))
            assert p_err <= 4 * 2.0 ** -53, (v, ox[i], float(rp))
            assert abs(ox[i] - lx[i]) <= 8 * 2.0 ** -53 * lx[i]
        if np.isinf(a):
            assert ex[i] == 0.0
            assert ours[i] == (0.0 if v > 0 else 2.0)
            continue
        rx = mp.exp(mp.mpf(a) ** 2) * mp.erfc(mp.mpf(a))
        ex_err = abs(mp.mpf(ex[i]) - rx) / rx
        worst_x = max(worst_x, float(ex_err))
        assert ex_err <= 4 * 2.0 ** -53, (v, ex[i], float(rx))
        re = mp.erfc(mp.mpf(float(v)))
        if v > 0 and v * v >= 700.0:  # exp(-x^2) below 2^-1009 is returned as 0
            assert ours[i] == 0.0 and re < mp.mpf(2.0) ** -1000
            continue
        bound = 1e-15 + 2 * a * a * 2.0 ** -52
        e_err = abs(mp.mpf(ours[i]) - re) / re
        worst_e = max(worst_e, float(e_err))
        assert e_err <= bound, (v, ours[i], float(re), float(e_err))
        # and beside the library's erfc
        assert abs(ours[i] - lib[i]) <= 2 * bound * abs(lib[i]) + 1e-300
    print(f"\nexp worst {worst_p:.2e}, erfcx worst {worst_x:.2e}, erfc worst {worst_e:.2e}")


def test_empty(ctx):
    assert ctx.cgks_special_selftest(np.zeros(0)).shape == (0, 5)
