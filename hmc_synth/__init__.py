"""Seeded synthetic inputs for the hybrid Monte Carlo hot path.

This module is shared by the CUDA library's tests/bench and by the CPU oracle's
tests: it draws inputs only and holds none of the method's arithmetic.

* Orientations: Euler triples (z-y-z, radians) uniform on SO(3), or the
  paper's single-angle set (rotation about z in 1-degree steps, Sec. "Results").
* Microstructure: periodic Voronoi polycrystal.  Seeds uniform in the periodic
  box (voxel units), each with a uniformly drawn orientation index; a voxel
  centre takes the orientation of the nearest seed under the minimum-image
  distance, ties going to the lowest seed index.  The paper starts from random
  synthetic microstructures as well (Sec. "Microstructural Evolution", 60^3 grid
  with 99 random orientations; Sec. "Results", random initial orientations).
* Workloads: the five named configurations (polycrystal sizes, orientation
  counts, Voronoi seed counts, loads, step counts) used by the tests and bench.
"""
from __future__ import annotations

import numpy as np

NI_CONSTANTS = dict(c11=246.5, c12=147.3, c44=124.7)   # GPa, cubic Ni used by the workloads
PAPER_NI_CONSTANTS = dict(c11=250.8, c12=150.0, c44=123.5)  # Sec. "Elastic Deformation"


def euler_uniform_so3(Q: int, seed: int) -> np.ndarray:
    """(Q,3) Euler triples (phi, theta, psi) with the rotations uniform on SO(3)."""
    rng = np.random.default_rng([0x5EED, 1, int(seed)])
    u = rng.random((Q, 3))
    return np.stack([2 * np.pi * u[:, 0], np.arccos(1.0 - 2.0 * u[:, 1]), 2 * np.pi * u[:, 2]], axis=1)


def euler_z_rotations(n: int = 91, step_deg: float = 1.0) -> np.ndarray:
    """(n,3) rotations about z by 0, step, 2 step, ... degrees; the other two angles zero."""
    phi = np.radians(step_deg * np.arange(n))
    return np.stack([phi, np.zeros(n), np.zeros(n)], axis=1)


def voronoi_seeds(shape, n_seeds: int, Q: int, seed: int):
    """Seed positions (S,3) in voxel units, (x,y,z) order, and their orientations (S,)."""
    nz, ny, nx = shape
    rng = np.random.default_rng([0x5EED, 2, int(seed)])
    pos = rng.random((n_seeds, 3)) * np.array([nx, ny, nz], dtype=np.float64)
    ori = rng.integers(0, Q, size=n_seeds).astype(np.uint16)
    return pos, ori


def _min_image_d2(pts, seeds, box):
    d = np.abs(pts[:, None, :] - seeds[None, :, :])
    d = np.minimum(d, box - d)
    return (d * d).sum(axis=2)


def voronoi_owner_brute(shape, pos) -> np.ndarray:
    """Nearest-seed index of every voxel by testing all seeds (O(N S)); natural order."""
    nz, ny, nx = shape
    box = np.array([nx, ny, nz], dtype=np.float64)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([xx.ravel() + 0.5, yy.ravel() + 0.5, zz.ravel() + 0.5], axis=1)
    out = np.empty(pts.shape[0], dtype=np.int64)
    for a in range(0, pts.shape[0], 4096):
        d2 = _min_image_d2(pts[a:a + 4096], pos, box)
        out[a:a + 4096] = np.argmin(d2, axis=1)  # first minimum = lowest index on ties
    return out


def voronoi_owner(shape, pos) -> np.ndarray:
    """Same result as ``voronoi_owner_brute`` through a periodic k-d tree: the three
    nearest candidates are re-ranked by the exact minimum-image distance."""
    from scipy.spatial import cKDTree
    nz, ny, nx = shape
    box = np.array([nx, ny, nz], dtype=np.float64)
    S = pos.shape[0]
    if S < 4:
        return voronoi_owner_brute(shape, pos)
    tree = cKDTree(np.mod(pos, box), boxsize=box)
    out = np.empty(nx * ny * nz, dtype=np.int64)
    xs = np.arange(nx) + 0.5
    plane = nx * ny
    for z in range(nz):
        yy, xx = np.meshgrid(np.arange(ny) + 0.5, xs, indexing="ij")
        pts = np.stack([xx.ravel(), yy.ravel(), np.full(plane, z + 0.5)], axis=1)
        _, idx = tree.query(pts, k=3, workers=-1)
        d = np.abs(pts[:, None, :] - pos[idx])
        d = np.minimum(d, box - d)
        d2 = (d * d).sum(axis=2)
        # rank by exact distance, then by seed index
        dmin = d2.min(axis=1, keepdims=True)
        cand = np.where(d2 == dmin, idx, np.iinfo(np.int64).max)
        out[z * plane:(z + 1) * plane] = cand.min(axis=1)
    return out


def voronoi_spins(shape, n_seeds: int, Q: int, seed: int) -> np.ndarray:
    """(nz,ny,nx) uint16 orientation field of a periodic Voronoi polycrystal."""
    pos, ori = voronoi_seeds(shape, n_seeds, Q, seed)
    owner = voronoi_owner(shape, pos)
    return ori[owner].reshape(shape)


def random_spins(shape, Q: int, seed: int) -> np.ndarray:
    """(nz,ny,nx) uint16 independent uniform orientations (the paper's random start)."""
    rng = np.random.default_rng([0x5EED, 3, int(seed)])
    return rng.integers(0, Q, size=shape).astype(np.uint16)


def box_grain_spins(shape, edge: int, Q: int, seed: int) -> np.ndarray:
    """(nz,ny,nx) uint16 field of box-shaped grains: the orientation of voxel (x, y, z) is
    (a[x // edge] ^ b[y // edge] ^ c[z // edge]) mod Q with a, b, c seeded uniform 16-bit
    words.  Built one layer of boxes at a time, so it serves grids of billions of sites (a
    grain boundary every edge voxels along each axis)."""
    nz, ny, nx = shape
    rng = np.random.default_rng([0x5EED, 5, int(seed)])
    a = rng.integers(0, 1 << 16, size=nx // edge + 1, dtype=np.uint32)
    b = rng.integers(0, 1 << 16, size=ny // edge + 1, dtype=np.uint32)
    c = rng.integers(0, 1 << 16, size=nz // edge + 1, dtype=np.uint32)
    ax = a[np.arange(nx) // edge]
    by = b[np.arange(ny) // edge]
    out = np.empty(shape, dtype=np.uint16)
    plane = (by[:, None] ^ ax[None, :])
    for z0 in range(0, nz, edge):
        out[z0:z0 + edge] = ((plane ^ c[z0 // edge]) % Q).astype(np.uint16)[None]
    return out


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

COMMON = dict(J=1.0, kT=0.7, **NI_CONSTANTS)

WORKLOADS = {
    # 32^3, 64 orientations, 200 Voronoi grains, uniaxial 1e-3 along z, 10 MCS x 50 steps, FP64
    "ni32": dict(shape=(32, 32, 32), Q=64, euler_seed=1, n_seeds=200, voronoi_seed=1,
                 axis=(0.0, 0.0, 1.0), strain=1e-3, n_mcs=10, mpm_steps=50, precision="fp64"),
    # 128^3, 256 orientations, 5000 grains, 2e-3 along [001], 100 MCS, FP64 vs FP32
    "ni128": dict(shape=(128, 128, 128), Q=256, euler_seed=2, n_seeds=5000, voronoi_seed=2,
                  axis=(0.0, 0.0, 1.0), strain=2e-3, n_mcs=100, mpm_steps=50, precision="fp32"),
    # 256^3, 1024 orientations, 40000 grains, 2e-3 along [111], 500 MCS, FP32, histogram every 10 MCS
    "ni256": dict(shape=(256, 256, 256), Q=1024, euler_seed=3, n_seeds=40000, voronoi_seed=3,
                  axis=(1.0, 1.0, 1.0), strain=2e-3, n_mcs=500, mpm_steps=50, precision="fp32",
                  hist_every=10),
}


def workload_inputs(name: str):
    """(spec, euler (Q,3), spins (nz,ny,nx) uint16) of a named workload.  With
    HMC_SYNTH_CACHE set to a directory, the Voronoi field is kept there as .npy
    (it is a pure function of the workload's seeds)."""
    import os
    w = dict(WORKLOADS[name])
    w.update(COMMON)
    euler = euler_uniform_so3(w["Q"], w["euler_seed"])
    cache = os.environ.get("HMC_SYNTH_CACHE")
    path = None
    if cache:
        os.makedirs(cache, exist_ok=True)
        path = os.path.join(cache, f"{name}_voronoi_{w['n_seeds']}_{w['voronoi_seed']}.npy")
        if os.path.exists(path):
            spins = np.load(path)
            if spins.shape == tuple(w["shape"]) and spins.dtype == np.uint16:
                return w, euler, spins
    spins = voronoi_spins(w["shape"], w["n_seeds"], w["Q"], w["voronoi_seed"])
    if path:
        np.save(path + ".tmp.npy", spins)
        os.replace(path + ".tmp.npy", path)
    return w, euler, spins


ENSEMBLE_EDGES = (48, 64, 96, 128, 160)


def ensemble_specs(n_replicas: int = 64, seed: int = 4, Q: int = 256, grain_volume: float = 419.4):
    """Replica descriptions of the batched ensemble: cubic edge uniform from
    {48,64,96,128,160}, loading axis uniform on the unit sphere, uniaxial strain
    uniform in [5e-4, 3e-3], independent seeds; Voronoi grains of about
    ``grain_volume`` voxels (the mean grain volume of the 128^3 and 256^3 workloads)."""
    rng = np.random.default_rng([0x5EED, 4, int(seed)])
    out = []
    for r in range(n_replicas):
        e = int(rng.choice(ENSEMBLE_EDGES))
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        strain = float(rng.uniform(5e-4, 3e-3))
        out.append(dict(shape=(e, e, e), axis=tuple(ax), strain=strain, Q=Q,
                        n_seeds=max(2, int(round(e ** 3 / grain_volume))),
                        voronoi_seed=int(rng.integers(1 << 31)), mc_seed=int(rng.integers(1 << 62)),
                        euler_seed=4))
    return out


def ensemble_inputs(n_replicas: int = 64, seed: int = 4, Q: int = 256):
    """(specs, euler (Q,3), [spins per replica]) of the batched ensemble; the
    Voronoi fields are cached like ``workload_inputs`` when HMC_SYNTH_CACHE is set."""
    import os
    specs = ensemble_specs(n_replicas, seed, Q)
    euler = euler_uniform_so3(Q, specs[0]["euler_seed"])
    cache = os.environ.get("HMC_SYNTH_CACHE")
    fields = []
    for sp in specs:
        path = None
        if cache:
            os.makedirs(cache, exist_ok=True)
            e = sp["shape"][0]
            path = os.path.join(cache, f"ens_{e}_{sp['n_seeds']}_{sp['voronoi_seed']}.npy")
            if os.path.exists(path):
                f = np.load(path)
                if f.shape == tuple(sp["shape"]):
                    fields.append(f)
                    continue
        f = voronoi_spins(sp["shape"], sp["n_seeds"], Q, sp["voronoi_seed"])
        if path:
            np.save(path + ".tmp.npy", f)
            os.replace(path + ".tmp.npy", path)
        fields.append(f)
    return specs, euler, fields
