"""The C-ABI library loads and exports every symbol include/hmc.h declares;
argument validation runs on the host (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def libhmc():
    from conftest import build_libhmc
    return C.CDLL(build_libhmc())


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hmc_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(libhmc):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(libhmc, n), n


def test_binding_covers_the_abi(libhmc):
    import paper_1009_0457_gb300 as G
    for n in declared_functions():
        assert callable(getattr(G, n, None)), n


def test_invalid_parameters_rejected_on_host(libhmc):
    import paper_1009_0457_gb300 as G
    bad = [dict(nx=5), dict(ny=2), dict(n_orient=0), dict(n_orient=70000), dict(kT=-1.0),
           dict(c11=100.0, c12=150.0), dict(precision=7), dict(bc=3), dict(trial=9), dict(elastic=4),
           dict(mpm_steps_per_mcs=-1), dict(damping=1.5), dict(load_axis=(0.0, 0.0, 0.0)),
           dict(J=float("nan")),
           # one site over the 2^32 - 1 limit needs an odd edge; the smallest even grid over it
           dict(nx=2048, ny=2048, nz=1024),
           dict(elastic=2, nx=4, ny=6, nz=6)]
    for kw in bad:
        p = G.hmc_default_params(**kw)
        with pytest.raises(G.HMCError) as e:
            G.hmc_create(p)
        assert e.value.status == G.HMC_ERR_ARG
        assert G.lib.hmc_last_error(None)


def test_default_params(libhmc):
    import paper_1009_0457_gb300 as G
    p = G.hmc_default_params()
    assert (p.nx, p.ny, p.nz, p.n_orient) == (32, 32, 32, 64)
    assert p.precision == G.HMC_FP32 and p.elastic == G.HMC_ELASTIC_TRACTION
    assert p.elastic_scale < 0 and p.dt < 0 and p.damping < 0


def test_fma_peak_rejects_bad_arguments_on_host(libhmc):
    import paper_1009_0457_gb300 as G
    t = C.c_double(-1.0)
    for prec, iters in [(7, 16), (G.HMC_FP32, 0), (G.HMC_FP64, -3), (G.HMC_FP32, (1 << 16) + 1)]:
        assert G.lib.hmc_fma_peak(prec, iters, C.byref(t)) == G.HMC_ERR_ARG
    assert G.lib.hmc_fma_peak(G.HMC_FP32, 16, None) == G.HMC_ERR_ARG
    assert t.value == -1.0
