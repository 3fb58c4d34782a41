"""Oracle pins of the grain count and the Gauss-Seidel step, and the grain-growth
behaviour of Sec. "Microstructural Evolution" (V^(3/2) linear in MC time; the
red/black update grows grains faster than the Gauss-Seidel one)."""
import numpy as np
import pytest

import hmc_synth as S
import oracle as O


def periodic_label_count(sp):
    """Independent count: scipy's face-connected labelling of the unwrapped
    field, then the labels that touch across each periodic face merged."""
    ndimage = pytest.importorskip("scipy.ndimage")
    nz, ny, nx = sp.shape
    parent = {}

    def find(a):
        while parent.get(a, a) != a:
            a = parent[a]
        return a

    lab = np.zeros(sp.shape, dtype=np.int64)
    off = 0
    for q in np.unique(sp):
        l, n = ndimage.label(sp == q)
        lab[l > 0] = l[l > 0] + off
        off += n
    for axis in range(3):
        a = np.take(lab, 0, axis=axis)
        b = np.take(lab, sp.shape[axis] - 1, axis=axis)
        sa = np.take(sp, 0, axis=axis)
        sb = np.take(sp, sp.shape[axis] - 1, axis=axis)
        for u, v in zip(a[sa == sb], b[sa == sb]):
            ru, rv = find(int(u)), find(int(v))
            if ru != rv:
                parent[max(ru, rv)] = min(ru, rv)
    return len({find(int(v)) for v in np.unique(lab)})


def test_grain_count_closed_forms():
    assert O.grain_count(np.zeros((4, 6, 8), dtype=np.uint16)) == 1
    z, y, x = np.meshgrid(np.arange(4), np.arange(6), np.arange(8), indexing="ij")
    assert O.grain_count(((x + y + z) & 1).astype(np.uint16)) == 4 * 6 * 8   # every site isolated
    assert O.grain_count((x & 1).astype(np.uint16)) == 8                      # one grain per x plane
    wrap = ((x == 0) | (x == 7)).astype(np.uint16)                            # joined across the periodic face
    assert O.grain_count(wrap) == 2
    n, lab = O.grain_count(wrap, want_labels=True)
    assert n == 2 and len(np.unique(lab[wrap == 1])) == 1


@pytest.mark.parametrize("shape,Q,seed", [((6, 8, 10), 3, 1), ((10, 6, 4), 5, 2), ((12, 12, 12), 2, 3)])
def test_grain_count_matches_independent_labelling(shape, Q, seed):
    sp = S.random_spins(shape, Q, seed)
    assert O.grain_count(sp) == periodic_label_count(sp)
    v = S.voronoi_spins(shape, 9, Q, seed)
    assert O.grain_count(v) == periodic_label_count(v)


def test_gs_step_energy_bookkeeping():
    sp = S.voronoi_spins((10, 12, 14), 12, 9, 5).copy()
    for m in range(3):
        before = O.unlike_bonds(sp)
        acc, de = O.gs_sweep(sp, 7, m, 0, 1.0, 0.7, O.TRIAL_NEIGHBOR, 9)
        assert acc > 0
        assert O.unlike_bonds(sp) - before == de


def test_gs_step_at_zero_temperature_never_raises_energy():
    sp = S.random_spins((8, 8, 8), 4, 3).copy()
    for m in range(4):
        before = O.unlike_bonds(sp)
        acc, de = O.gs_sweep(sp, 11, m, 0, 1.0, 0.0, O.TRIAL_NEIGHBOR, 4)
        assert de <= 0 and O.unlike_bonds(sp) == before + de


def test_gs_step_uniform_field_and_trial_set():
    sp = np.full((6, 6, 6), 3, dtype=np.uint16)
    assert O.gs_sweep(sp, 1, 0, 0, 1.0, 5.0, O.TRIAL_NEIGHBOR, 8) == (0, 0)
    sp = S.voronoi_spins((8, 8, 8), 5, 20, 4).copy()
    present = set(np.unique(sp))
    O.gs_sweep(sp, 1, 0, 0, 1.0, 5.0, O.TRIAL_NEIGHBOR, 20)
    assert set(np.unique(sp)) <= present   # neighbour-copy trials never introduce an orientation


def _growth(mode, shape, Q, kT, n_mcs, every, seed):
    sp = S.random_spins(shape, Q, seed).copy()
    t, V = [], []
    for m in range(1, n_mcs + 1):
        if mode == "RB":
            O.half_sweep(sp, 0, 7, m, 0, 1.0, kT, O.TRIAL_NEIGHBOR, Q, 0, 0.0, None, None)
            O.half_sweep(sp, 1, 7, m, 0, 1.0, kT, O.TRIAL_NEIGHBOR, Q, 0, 0.0, None, None)
        else:
            O.gs_sweep(sp, 7, m, 0, 1.0, kT, O.TRIAL_NEIGHBOR, Q)
        if m % every == 0:
            t.append(m)
            V.append(sp.size / O.grain_count(sp))
    return np.array(t, dtype=float), np.array(V)


def test_grain_growth_law_and_rb_faster_than_gs():
    """40^3, 99 orientations, kT/J = 1 from a random start: after a transient the
    mean grain volume follows V^(3/2) = c2 t + c0 under both updates, and c2 of
    the red/black update exceeds that of the Gauss-Seidel update."""
    c2 = {}
    for mode in ("RB", "GS"):
        t, V = _growth(mode, (40, 40, 40), 99, 1.0, 200, 20, 1)
        sel = t >= 60
        y = V[sel] ** 1.5
        slope, icpt = np.polyfit(t[sel], y, 1)
        r = np.corrcoef(t[sel], y)[0, 1]
        assert r > 0.98, (mode, r)
        assert np.all(np.diff(V) > 0), mode
        c2[mode] = slope
    assert c2["RB"] > 1.5 * c2["GS"], c2
