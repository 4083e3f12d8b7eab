"""CPU checks of the C-ABI library: it loads without a GPU and exports every
entry point declared in include/cgks.h; the binding names match."""
import os
import re

import pytest

from paper_2509_06347_b300 import build, cgks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "cgks.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cgks_[a-z_]+)\s*\(", txt)))


def test_header_declares_binding_exports():
    assert declared() == sorted(cgks.EXPORTS)


def test_library_loads_and_exports_every_symbol():
    path = build.build()
    lib = cgks.load_library(path)
    for name in declared():
        assert hasattr(lib, name), name


def test_default_config_values():
    cfg = cgks.default_config()
    assert cfg.gamma == 1.4 and cfg.cfl_imp == 10.0 and cfg.cfl_exp == 0.5
    assert cfg.n_sweep_coarse == 6 and cfg.n_pre == 1 and cfg.n_post == 0
    assert cfg.tol == 1e-10
    assert cfg.weno_gamma_high == 0.95 and cfg.slope_relax == 1.0 and cfg.alpha_relax == 1.0
    assert cfg.learned_scale == 0


@pytest.mark.parametrize("kw", [dict(tau_c1=0.0), dict(tau_c1=float("nan")), dict(tau_c2=-1.0), dict(mu=-1.0),
                                dict(gamma=1.0), dict(df_relax=3), dict(df_relax=2, relax_beta=1.5),
                                dict(n_pre=2), dict(n_sweep_coarse=0), dict(flux_precision=2),
                                dict(cfl_imp=0.0), dict(cfl_exp=-0.5), dict(weno_eps=0.0),
                                dict(slope_relax=0.0), dict(alpha_relax=1.5), dict(weno_gamma_high=0.0),
                                dict(learned_scale=2)])
def test_invalid_config_rejected_before_any_device_call(kw):
    """cgks_create checks the configuration before it touches the device, so
    every rejection holds on a host without a GPU."""
    with pytest.raises(cgks.CgksError) as e:
        cgks.Context(**kw)
    assert e.value.code == -1
