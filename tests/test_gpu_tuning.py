"""Autotuner knobs never change a result: every choice of the sweep's CTA size and,
in auto mode (store_stress = 2), of stored against recomputed stress gives the same
spins, displacement and mean strain as the defaults, for single handles and for a
batch of uneven replicas."""
import numpy as np
import pytest

import hmc_synth as S

pytestmark = pytest.mark.gpu

C3 = dict(c11=246.5, c12=147.3, c44=124.7)


@pytest.fixture(scope="module")
def G():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    return G


def _run(G, shape, precision, elastic=1, store=1, n_mcs=3):
    Q = 12
    eul = S.euler_uniform_so3(Q, 6)
    sp = S.voronoi_spins(shape, 18, Q, 6)
    g = G.HMC(shape, Q, precision=precision, load_axis=(1, 1, 1.0), strain=2e-3, mpm_steps_per_mcs=6,
              elastic=elastic, elastic_scale=2e3, store_stress=store, seed=91, **C3)
    g.set_orientations(eul, sp)
    acc = g.mc_sweeps(n_mcs)
    out = (acc, g.spins().copy(), g.nodal()[0], g.strain())
    g.close()
    return out


def _same(a, b):
    assert a[0] == b[0] and a[0] > 0
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


@pytest.mark.parametrize("precision,elastic", [(1, 1), (0, 1), (1, 0), (1, 3)])
def test_sweep_cta_size_gives_the_same_bits(G, monkeypatch, precision, elastic):
    shape = (12, 22, 70)   # 3 080 blocks: tiles split over two 128-thread CTAs, a ragged last tile
    res = []
    for cta in ("256", "128"):
        monkeypatch.setenv("HMC_SWEEP_CTA", cta)
        res.append(_run(G, shape, precision, elastic))
    _same(res[0], res[1])


@pytest.mark.parametrize("precision", [1, 0])
def test_auto_stored_or_recomputed_stress_gives_the_same_bits(G, monkeypatch, precision):
    shape = (14, 18, 36)
    monkeypatch.setenv("HMC_AUTOTUNE", "1")
    ref = _run(G, shape, precision, store=1)
    _same(ref, _run(G, shape, precision, store=0))
    _same(ref, _run(G, shape, precision, store=2))


def test_batch_with_half_ctas_equals_solo_runs(G, monkeypatch):
    Q = 10
    eul = S.euler_uniform_so3(Q, 8)
    shapes = [(8, 10, 34), (12, 12, 12)]
    fields = [S.voronoi_spins(s, 9, Q, 20 + i) for i, s in enumerate(shapes)]
    per = [dict(load_axis=(0.2, 0.5, 1.0), strain=1.5e-3, seed=5, replica=0),
           dict(load_axis=(1.0, 0.0, 0.3), strain=2.5e-3, seed=6, replica=1)]
    common = dict(precision=G.HMC_FP32, mpm_steps_per_mcs=5, elastic_scale=3e3, **C3)
    monkeypatch.setenv("HMC_SWEEP_CTA", "128")
    b = G.HMCBatch(shapes, Q, per, **common)
    b.set_orientations(eul, fields)
    b.mc_sweeps(2)
    got = [b.spins(r) for r in range(2)]
    b.close()
    monkeypatch.setenv("HMC_SWEEP_CTA", "256")
    for r, (shape, f) in enumerate(zip(shapes, fields)):
        g = G.HMC(shape, Q, **per[r], **common)
        g.set_orientations(eul, f)
        g.mc_sweeps(2)
        assert np.array_equal(g.spins(), got[r]), f"replica {r}"
        g.close()


def _run_tuned(G, shape, precision):
    Q = 12
    eul = S.euler_uniform_so3(Q, 6)
    sp = S.voronoi_spins(shape, 18, Q, 6)
    g = G.HMC(shape, Q, precision=precision, load_axis=(1, 1, 1.0), strain=2e-3, mpm_steps_per_mcs=6,
              elastic=1, elastic_scale=2e3, seed=91, **C3)
    g.set_orientations(eul, sp)
    acc = g.mc_sweeps(3)
    out = (acc, g.spins().copy(), g.nodal()[0], g.strain())
    tuning = g.tuning()
    g.close()
    return out, tuning


@pytest.mark.parametrize("precision", [1, 0])
def test_mpm_grid_size_gives_the_same_bits(G, monkeypatch, precision):
    """A small grid (12 node planes of one tile): the tuner's persistent grid (it may take
    one plane per CTA) and the default one for the same patch shape (at least four planes
    per CTA) give the same spins, displacement and mean strain; the CTAs split the planes
    differently, and every CTA recomputes the cells below its first plane."""
    shape = (24, 16, 16)
    monkeypatch.delenv("HMC_MPM_SHAPE", raising=False)
    monkeypatch.setenv("HMC_AUTOTUNE", "1")
    tuned, (shp, grid_tuned) = _run_tuned(G, shape, precision)
    monkeypatch.setenv("HMC_MPM_SHAPE", str(shp))
    forced, (shp2, grid_default) = _run_tuned(G, shape, precision)
    assert shp2 == shp
    _same(tuned, forced)
    assert grid_default >= 1 and grid_tuned >= 1, (grid_tuned, grid_default)
    print(f"MPM grid tuned {grid_tuned}, default {grid_default} (shape {shp})")
