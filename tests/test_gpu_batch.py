"""Batched ensemble: every replica of a batch equals the same replica run alone,
bit for bit, and every MPM patch shape the autotuner can pick gives the same bits."""
import os

import numpy as np
import pytest

import hmc_synth as S
import oracle as O

pytestmark = pytest.mark.gpu

C3 = dict(c11=246.5, c12=147.3, c44=124.7)


@pytest.fixture(scope="module")
def G():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    return G


def _replicas():
    shapes = [(8, 18, 34), (12, 12, 12), (6, 34, 20), (20, 16, 30), (10, 10, 64)]
    rng = np.random.default_rng(21)
    reps = []
    for r, sh in enumerate(shapes):
        ax = rng.normal(size=3)
        reps.append(dict(shape=sh, kw=dict(load_axis=tuple(ax / np.linalg.norm(ax)), strain=float(rng.uniform(5e-4, 3e-3)),
                                           seed=1000 + r, replica=r),
                         spins=S.voronoi_spins(sh, 12, 16, 300 + r)))
    return reps


@pytest.mark.parametrize("precision", [1, 0])
def test_batch_replicas_equal_solo_runs(G, precision):
    reps = _replicas()
    eul = S.euler_uniform_so3(16, 5)
    common = dict(precision=precision, mpm_steps_per_mcs=6, **C3)
    b = G.HMCBatch([r["shape"] for r in reps], 16, [r["kw"] for r in reps], **common)
    b.set_orientations(eul, [r["spins"] for r in reps])
    acc_b = b.mc_sweeps(3)
    acc_s = 0
    for i, r in enumerate(reps):
        g = G.HMC(r["shape"], 16, **r["kw"], **common)
        g.set_orientations(eul, r["spins"])
        acc_s += g.mc_sweeps(3)
        assert (b.spins(i) == g.spins()).all(), f"replica {i}"
        assert np.array_equal(b.nodal(i)[0], g.nodal()[0]), f"replica {i}"
        assert np.array_equal(b.strain(i), g.strain()), f"replica {i}"
        g.close()
    assert acc_b == acc_s
    b.close()


@pytest.mark.parametrize("variants", [("0", "1", "2"), ("3", "4", "5"), ("0", "6")])
def test_patch_shapes_are_bitwise_equal(G, variants):
    shape = (10, 40, 50)
    eul = S.euler_uniform_so3(9, 2)
    sp = S.voronoi_spins(shape, 20, 9, 4)
    rng = np.random.default_rng(3)
    u0 = rng.normal(size=(np.prod(shape) // 8, 3)) * 1e-3
    out = []
    old = os.environ.get("HMC_MPM_SHAPE")
    try:
        for shp in variants:
            os.environ["HMC_MPM_SHAPE"] = shp
            g = G.HMC(shape, 9, load_axis=(1, 2, 3.0), strain=2e-3, **C3)
            g.set_orientations(eul, sp)
            g.set_nodal(u0, None)
            g.mpm_steps(15)
            assert g.tuning()[0] == int(shp)
            out.append(g.nodal())
            g.close()
    finally:
        if old is None:
            os.environ.pop("HMC_MPM_SHAPE", None)
        else:
            os.environ["HMC_MPM_SHAPE"] = old
    for u, v in out[1:]:
        assert np.array_equal(u, out[0][0]) and np.array_equal(v, out[0][1])


def test_batch_mpm_matches_oracle_fp64(G):
    """One FP64 batch of three replicas against the oracle, replica by replica."""
    reps = _replicas()[:3]
    eul = S.euler_uniform_so3(16, 5)
    common = dict(precision=0, mpm_steps_per_mcs=0, **C3)
    b = G.HMCBatch([r["shape"] for r in reps], 16, [r["kw"] for r in reps], **common)
    b.set_orientations(eul, [r["spins"] for r in reps])
    b.mpm_steps(12)
    for i, r in enumerate(reps):
        o = O.OracleHMC(r["shape"], 16, load_axis=r["kw"]["load_axis"], strain=r["kw"]["strain"], **C3)
        o.set_orientations(eul, r["spins"])
        o.mpm_steps(12)
        u = b.nodal(i)[0]
        assert np.linalg.norm(u - o.u) < 1e-12 * np.linalg.norm(o.u)
    b.close()


def test_paired_hooke_bitwise_equal_to_scalar(G):
    shape = (10, 40, 50)
    eul = S.euler_uniform_so3(9, 2)
    sp = S.voronoi_spins(shape, 20, 9, 4)
    rng = np.random.default_rng(3)
    u0 = rng.normal(size=(np.prod(shape) // 8, 3)) * 1e-3
    out = []
    old = os.environ.get("HMC_MPM_SHAPE")
    try:
        for shp in ("0", "3"):
            os.environ["HMC_MPM_SHAPE"] = shp
            g = G.HMC(shape, 9, load_axis=(1, 2, 3.0), strain=2e-3, **C3)
            g.set_orientations(eul, sp)
            g.set_nodal(u0, None)
            g.mpm_steps(15)
            out.append(g.nodal()[0])
            g.close()
    finally:
        if old is None:
            os.environ.pop("HMC_MPM_SHAPE", None)
        else:
            os.environ["HMC_MPM_SHAPE"] = old
    assert np.array_equal(out[1], out[0])   # same products and fused adds in the same order


@pytest.mark.parametrize("precision,elastic", [(1, 1), (1, 3), (1, 0), (0, 0)])
def test_large_uneven_batch_equals_solo_runs(G, precision, elastic):
    """Replicas of uneven size, the largest spanning several waves of sweep CTAs:
    each replica of the batch equals its own single-replica run bit for bit
    (spins, accepted count, nodal state), for the stored-stress elastic forms and
    pure Potts."""
    shapes = [(128, 128, 96), (34, 18, 8), (64, 50, 46)]
    eul = S.euler_uniform_so3(64, 3)
    fields = [S.voronoi_spins(sh, 40, 64, 50 + i) for i, sh in enumerate(shapes)]
    per = [dict(seed=11 + r, load_axis=(0.2 * r, 0.3, 1.0), strain=1e-3 * (r + 1), replica=r) for r in range(3)]
    common = dict(precision=precision, mpm_steps_per_mcs=4, elastic=elastic, elastic_scale=3e3, **C3)
    b = G.HMCBatch(shapes, 64, per, **common)
    b.set_orientations(eul, fields)
    acc_b = b.mc_sweeps(3)
    acc_s = 0
    for r, sh in enumerate(shapes):
        kw = dict(common)
        kw.update(per[r])
        g = G.HMC(sh, 64, **kw)
        g.set_orientations(eul, fields[r])
        acc_s += g.mc_sweeps(3)
        assert np.array_equal(b.spins(r), g.spins()), r
        assert np.array_equal(b.nodal(r)[0], g.nodal()[0]), r
        g.close()
    b.close()
    assert acc_b == acc_s and acc_b > 0


def test_configured_ensemble_200_mcs(G):
    """The batched ensemble as configured: 64 replicas with edges from {48, 64, 96, 128, 160},
    independent seeds, axes uniform on the sphere, strains uniform in [5e-4, 3e-3], Q = 256,
    FP32, 200 Monte Carlo steps of 50 MPM steps in one handle.  Every replica accepts trials
    and keeps its spins in range, its mean strain stays finite, and replica 0's spins equal
    its own single-replica run over the first 5 steps."""
    specs, euler, fields = S.ensemble_inputs()
    per = [dict(load_axis=sp["axis"], strain=sp["strain"], seed=sp["mc_seed"], replica=r)
           for r, sp in enumerate(specs)]
    common = dict(S.COMMON)
    b = G.HMCBatch([sp["shape"] for sp in specs], specs[0]["Q"], per, precision=G.HMC_FP32,
                   mpm_steps_per_mcs=50, **common)
    try:
        b.set_orientations(euler, fields)
        b.mc_sweeps(5)
        kw = dict(common)
        kw.update(per[0])
        solo = G.HMC(specs[0]["shape"], specs[0]["Q"], precision=G.HMC_FP32, mpm_steps_per_mcs=50, **kw)
        solo.set_orientations(euler, fields[0])
        solo.mc_sweeps(5)
        assert (solo.spins() == b.spins(0)).all()
        solo.close()
        acc = b.mc_sweeps(195)
        assert acc > 0
        for r, sp in enumerate(specs):
            s = b.spins(r)
            assert s.shape == tuple(sp["shape"]) and int(s.max()) < sp["Q"], r
            assert (s != fields[r]).any(), r
            assert np.all(np.isfinite(b.strain(r))), r
    finally:
        b.close()
