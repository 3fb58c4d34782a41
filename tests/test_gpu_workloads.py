"""Parity with the FP64 CPU oracle on the named workloads, as configured.

* ni32  (32^3, Q = 64, 200 Voronoi grains, uniaxial 1e-3 along z, 50 MPM steps per
  MCS, FP64): all 10 Monte Carlo steps through ``hmc_mc_sweeps`` (the captured
  graph) against the oracle's schedule (Sec. "Results": equilibrate, then one MC
  step): spins identical after every step, stress and mean strain to 1e-12.
* ni128 (128^3, Q = 256, 5 000 grains, 2e-3 along [001], 50 steps per MCS): two
  Monte Carlo steps in FP64 (spins identical, stress to 1e-12) and in FP32, where the
  precision contract is a stated error: the FP32 stress against the oracle's (relative
  L2) and the fraction of half-sweep decisions that differ when both sides sweep the
  same spins, each with its own stress, with every differing decision's distance to
  its threshold reported.
"""
import numpy as np
import pytest

import hmc_synth as S
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    return G


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _pair_args(spec):
    kw = dict(J=spec["J"], kT=spec["kT"], c11=spec["c11"], c12=spec["c12"], c44=spec["c44"],
              load_axis=tuple(spec["axis"]), strain=spec["strain"], mpm_steps_per_mcs=spec["mpm_steps"],
              seed=0x5EED0000 + spec["euler_seed"])
    return kw


def _oracle(spec, euler, spins):
    kw = _pair_args(spec)
    o = O.OracleHMC(spec["shape"], spec["Q"], **kw)
    o.set_orientations(euler, spins.copy())   # the oracle sweeps its spin array in place
    return o


def test_ni32_ten_mcs_fp64_match_the_oracle(G):
    spec, euler, spins = S.workload_inputs("ni32")
    assert spec["shape"] == (32, 32, 32) and spec["Q"] == 64 and spec["n_seeds"] == 200
    o = _oracle(spec, euler, spins)
    g = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP64, **_pair_args(spec))
    g.set_orientations(euler, spins)
    total_g = total_o = 0
    for m in range(spec["n_mcs"]):
        total_g += g.mc_sweeps(1)
        total_o += o.mc_sweeps(1)
        assert total_g == total_o, f"MCS {m}: accepted counts differ"
        assert (g.spins() == o.spins).all(), f"MCS {m}: spins differ"
        assert rel(g.stress(), o.sig) < 1e-12, f"MCS {m}: stress"
        assert rel(g.strain(), o.Ebar) < 1e-12, f"MCS {m}: mean strain"
    assert g.info().mcs == spec["n_mcs"]
    assert total_g > 0
    g.close()


@pytest.fixture(scope="module")
def ni128():
    """The oracle's first two Monte Carlo steps of the 128^3 workload, with the spins
    before each half sweep, the stress of each step and every site's decision data."""
    spec, euler, spins = S.workload_inputs("ni128")
    assert spec["shape"] == (128, 128, 128) and spec["Q"] == 256 and spec["n_seeds"] == 5000
    o = _oracle(spec, euler, spins)
    rec = []
    for m in range(2):
        o.mpm_steps(spec["mpm_steps"])
        sig = o.stress().copy()
        halves = []
        for colour in (0, 1):
            pre = o.spins.copy()
            acc, changed, dH, t = o.half_sweep(colour)
            halves.append(dict(pre=pre, post=o.spins.copy(), acc=acc, dH=dH.reshape(spec["shape"]).copy(),
                               t=t.reshape(spec["shape"]).copy()))
        o.end_mcs()
        rec.append(dict(sig=sig, halves=halves, ebar=o.Ebar.copy(), u=o.u.copy()))
    return spec, euler, spins, rec


def test_ni128_two_mcs_fp64_match_the_oracle(G, ni128):
    spec, euler, spins, rec = ni128
    g = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP64, **_pair_args(spec))
    g.set_orientations(euler, spins)
    for m, r in enumerate(rec):
        acc = g.mc_sweeps(1)
        assert acc == r["halves"][0]["acc"] + r["halves"][1]["acc"], f"MCS {m}"
        assert (g.spins() == r["halves"][1]["post"]).all(), f"MCS {m}: spins differ"
        assert rel(g.stress(), r["sig"]) < 1e-12, f"MCS {m}: stress"
        assert rel(g.nodal()[0], r["u"]) < 1e-11, f"MCS {m}: displacement"
        assert rel(g.strain(), r["ebar"]) < 1e-12, f"MCS {m}: mean strain"
    g.close()


def test_ni128_two_mcs_fp32_error_is_stated(G, ni128):
    """FP32 stress and FP32 decisions against the FP64 oracle, lock-step: before each
    half sweep the device takes the oracle's spins, while the stress of each step is the
    FP32 path's own (50 FP32 MPM steps per step from its own state)."""
    spec, euler, spins, rec = ni128
    g = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP32, **_pair_args(spec))
    g.set_orientations(euler, spins)
    nz, ny, nx = spec["shape"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    col = (x + y + z) & 1
    report = []
    for m, r in enumerate(rec):
        g.mpm_steps(spec["mpm_steps"])
        g.compute_stress()
        err = rel(g.stress(), r["sig"])
        # 50 explicit steps per Monte Carlo step: well inside the 1e-4 bar set for 200 steps
        assert err < 1e-4, f"MCS {m}: FP32 stress relative L2 {err:.2e}"
        for colour, hv in enumerate(r["halves"]):
            g.set_spins(hv["pre"])
            g.sweep_half(colour)
            mask = col == colour
            diff = (g.spins() != hv["post"]) & mask
            n_mis = int(diff.sum())
            gap = np.abs(hv["dH"] - hv["t"])[diff] / np.maximum(1.0, np.abs(hv["t"][diff]))
            outside = int((gap > 1e-6).sum())
            report.append((m, colour, err, n_mis / int(mask.sum()), outside, float(gap.max()) if n_mis else 0.0))
            # sites of the other colour are untouched
            assert (g.spins()[~mask] == hv["pre"][~mask]).all()
            # a differing decision is a trial whose own dH is within the FP32 stress error of its
            # threshold: |dH - t| / max(1, |t|) below 1e-3 (the elastic term is ~10 MC units at
            # 128^3; 1e-5 of it is 1e-4), and few of them
            assert n_mis <= 1e-3 * int(mask.sum()), report[-1]
            if n_mis:
                assert gap.max() < 1e-3, report[-1]
        g.end_mcs()
    for m, colour, err, frac, outside, gmax in report:
        print(f"ni128 FP32 MCS {m} colour {colour}: stress rel L2 {err:.2e}, decision mismatch fraction "
              f"{frac:.2e}, outside the 1e-6 margin {outside}, largest |dH - t| {gmax:.2e}")
    g.close()
