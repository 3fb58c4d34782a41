#!/usr/bin/env python
"""Throughput of the hybrid Monte Carlo hot path on GB300.

One step = one Monte Carlo step (MCS) of the whole hot path on the 256^3
workload: 50 fused explicit MPM steps, the stress of every point, the red and
the black half sweep, and the end-of-step reduction / loading update -- one
replay of the captured CUDA graph behind ``hmc_mc_sweeps``.

Prints ONE JSON line (rank 0):
  value   site-updates/s of the whole job (every site is visited once per MCS),
          CUDA events on the library's stream, inputs resident in HBM
  e2e     the same metric through the C ABI with host buffers: every step
          uploads the spin field from pinned host memory and reads it back
  roofline        the dominant kernel (the fused MPM step), ALU-bound (FP32)
  roofline_sweep  the red/black half sweep, HBM-bound
  cpu_baseline    the FP64 CPU oracle on a bounded crop of the same workload

``--impl reference`` times the oracle instead (the CPU arm): each step is one
full oracle MCS on a 64^3 crop of the workload's microstructure.

Multi-GPU (torchrun): every rank runs an independent replica (Philox replica
id = rank) of the workload -- replicas only, weak scaling, no collective on the
data path; the timed region is bracketed by barriers and the max time over
ranks is used.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP32 peak of the ALU roofline: SMs (read from the device) x 128 FP32 lanes x 2 flop per FMA x clock
FP32_LANES = 128
# algorithmic flops of one point in one fused FP32 MPM step, separable trilinear form
# (corner differences, gradient interpolation, strain, Hooke's law in the cubic form
# (66 flop), traction sums, force interpolation, corner assembly, node update), FMA = 2 flop
MPM_FLOP_PER_POINT = 132
# the FP64 step's Hooke product is the 21-entry symmetric row (72 flop instead of 66)
MPM_FLOP_PER_POINT_F64 = 138
MPM_BYTES_PER_POINT = {"f32": 8, "f64": 14}      # spin 2 + (u,v) read + (u,v) write, per point
SWEEP_BYTES_PER_SITE = {"f32": 28, "f64": 52}    # spin read + write + stored stress read
STRESS_BYTES_PER_SITE = {"f32": 27.5, "f64": 53}  # spin 2 + u read (per point) + stress write
# plain FP64 step, per point: stress read (P2G) 48 + cell forces written and read 2 x 24 + node
# u, v read and written 4 x 3 + stress read and written (G2P) 96 + spins 2 (once per kernel pair)
PLAIN_BYTES_PER_POINT = 48 + 2 * 24 + 12 + 96 + 2
CROP = 64
ENSEMBLE_STEPS = 10


def measured_fma_peaks(G):
    """The device's FP32 and FP64 fused multiply-add rates, measured by the library's
    micro-benchmark (eight independent FMA chains per thread, best of three launches):
    what the FP32 and FP64 pipes deliver at the clock they run at under that load."""
    return {"fp32_tflops": G.hmc_fma_peak(G.HMC_FP32, 4096), "fp64_tflops": G.hmc_fma_peak(G.HMC_FP64, 256),
            "how": "hmc_fma_peak: every thread of (resident CTAs per SM x SMs) CTAs of 256 runs 8 independent "
                   "FMA chains, 2 flop per FMA, best of three launches after one warm-up"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ni256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--store-stress", type=int, default=1, choices=[0, 1],
                    help="1: the stress pass stores every point's stress for the sweeps; 0: sweeps recompute it")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class Clocks:
    """nvidia-smi samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            d = os.environ.get("HMC_CLOCKS_DIR") or None   # where to keep the sampled clock log
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv", dir=d)
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_traffic(kernel):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel's
    source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = {"mpm": "k_mpm.cu", "sweep": "k_sweep.cu", "zone": "k_zone.cu"}[kernel]
    try:
        csrc = os.path.join(ROOT, "paper_1009_0457_gb300", "csrc")
        blob = b"".join(open(os.path.join(csrc, f), "rb").read() for f in (src, "hmc_device.cuh", "hmc_internal.h"))
        sha = hashlib.sha256(blob).hexdigest()[:16]
        for line in open(path):
            f = line.split()
            if len(f) >= 4 and not line.startswith("#") and f[0] == kernel and f[1] == sha:
                return float(f[2])
    except Exception:
        pass
    return None


def mpm_variant_name(v):
    if v == 6:
        return "16x16 two cells per thread (paired FP32)"
    return ["16x16", "32x8", "8x32"][v % 3] + (" paired-FMA Hooke" if v >= 3 else "")


def dist_reduce(t_local, units_local, device="cpu"):
    """(max time over ranks, total work units over ranks); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(t_local), float(units_local)
    x = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    y = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    dist.all_reduce(y, op=dist.ReduceOp.SUM)
    return float(x.item()), float(y.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def crops(spins, n):
    """n disjoint CROP^3 crops of the field (as many as it holds, at most n); a field
    smaller than CROP along any axis is taken whole, n times (independent runs of the
    whole workload, one per process)."""
    nz, ny, nx = spins.shape
    if min(nz, ny, nx) < CROP:
        return [np.ascontiguousarray(spins) for _ in range(n)]
    out = []
    for z in range(0, nz - CROP + 1, CROP):
        for y in range(0, ny - CROP + 1, CROP):
            for x in range(0, nx - CROP + 1, CROP):
                if len(out) < n:
                    out.append(np.ascontiguousarray(spins[z:z + CROP, y:y + CROP, x:x + CROP]))
    return out


def crop_desc(spins, nproc, sites):
    """What the oracle processes ran on, for the sample strings."""
    if min(spins.shape) < CROP:
        edge = "x".join(str(d) for d in spins.shape[::-1])
        return f"{nproc} independent runs of the whole {edge} field ({sites} sites in all)"
    return f"{nproc} disjoint {CROP}^3 crops ({sites} sites)"


def _oracle_crop_worker(spec, euler, crop, warmup, n_mcs, barrier, out):
    """One host process: the unchanged FP64 oracle (single-threaded C) on one crop; the
    timed part starts when every process has finished its set-up and warm-up."""
    sys.path.insert(0, ROOT)
    import oracle as O
    try:
        o = O.OracleHMC(crop.shape, spec["Q"], J=spec["J"], kT=spec["kT"], c11=spec["c11"], c12=spec["c12"],
                        c44=spec["c44"], load_axis=spec["axis"], strain=spec["strain"],
                        mpm_steps_per_mcs=spec["mpm_steps"], seed=12345)
        o.set_orientations(euler, crop)
        o.mc_sweeps(warmup)
        barrier.wait(timeout=600)
        t0 = time.time()
        o.mc_sweeps(n_mcs)
        out.put((crop.size * n_mcs, t0, time.time()))
    except Exception as e:  # reported by the parent
        out.put(("error", repr(e), 0.0))


def oracle_rate(spec, euler, spins, n_mcs, procs, warmup=0):
    """site-updates/s of the oracle over n_mcs full MCS in each of `procs` host processes,
    each on its own disjoint CROP^3 crop (one process per core; spawned, never forked,
    since the parent may already hold a CUDA context).  Returns (rate, seconds, sites, procs)."""
    import multiprocessing as mp
    parts = crops(spins, procs)
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(len(parts))
    q = ctx.Queue()
    ps = [ctx.Process(target=_oracle_crop_worker, args=(spec, euler, c, warmup, n_mcs, barrier, q), daemon=True)
          for c in parts]
    for p in ps:
        p.start()
    res = [q.get(timeout=1800) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    bad = [r for r in res if r[0] == "error"]
    if bad:
        raise RuntimeError(f"oracle worker failed: {bad[0][1]}")
    units = sum(r[0] for r in res)
    t = max(r[2] for r in res) - min(r[1] for r in res)
    return units / t, t, sum(c.size for c in parts), len(parts)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import hmc_synth as S
    spec, euler, spins = S.workload_inputs(args.workload)
    cores = host_cores()
    value, t, sites, nproc = oracle_rate(spec, euler, spins, args.steps, cores, warmup=args.warmup)
    sample = (f"{crop_desc(spins, nproc, sites)} of the {args.workload} microstructure, one "
              f"single-threaded oracle process per host core; each step one full oracle MCS in every crop "
              f"({spec['mpm_steps']} MPM steps, stress, red+black sweep), FP64")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(spec, args.workload),
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": "site-updates/s", "cores": nproc,
                             "sample": sample},
            "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


METRIC = "HMC site-updates/s and MPM cell-steps/s at 1 GB300; fraction of HBM roofline"


def workload_config(spec, name):
    nz, ny, nx = spec["shape"]
    return {"workload": f"{name}: {nx}x{ny}x{nz} Ni polycrystal, Q={spec['Q']} orientations uniform on SO(3), "
                        f"periodic Voronoi of {spec['n_seeds']} grains, uniaxial strain {spec['strain']} along "
                        f"{list(spec['axis'])} with traction-free sides, J=1, kT=0.7, {spec['mpm_steps']} explicit "
                        f"MPM steps per MCS, FP32 stress and zone energy, FP64 reductions",
            "sites": nx * ny * nz, "orientations": spec["Q"], "mpm_steps_per_mcs": spec["mpm_steps"],
            "l2": l2_statement(nx * ny * nz)}


L2_BYTES = 129e6   # GB300's L2
# FP32 bytes resident per site: spin 2, stored stress 24, two displacement buffers and the
# velocity at one node per 8 sites (3 x 12 / 8)
RESIDENT_BYTES_PER_SITE = 2 + 24 + 36 / 8


def l2_statement(sites):
    mb = RESIDENT_BYTES_PER_SITE * sites / 1e6
    if mb * 1e6 > L2_BYTES:
        return f"inputs larger than L2 ({mb:.0f} MB of spins, nodal state and stored stress resident in HBM)"
    return (f"inputs smaller than L2 ({mb:.1f} MB resident): the steps run L2-resident, with no flush between "
            f"them; a per-configuration figure, not an HBM measurement")


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import hmc_synth as S
    import paper_1009_0457_gb300 as G

    spec, euler, spins = S.workload_inputs(args.workload)
    nz, ny, nx = spec["shape"]
    N = nx * ny * nz
    stream = torch.cuda.Stream()
    common = dict(J=spec["J"], kT=spec["kT"], c11=spec["c11"], c12=spec["c12"], c44=spec["c44"],
                  load_axis=spec["axis"], strain=spec["strain"], mpm_steps_per_mcs=spec["mpm_steps"],
                  seed=0x5EED0000 + 3, replica=rank, stream=stream.cuda_stream, store_stress=args.store_stress)
    h = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP32, **common)
    h.set_orientations(euler, spins)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def tmax(t):
        return dist_reduce(t, 0, "cuda")[0]

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    # warm-up (captures the graph)
    G.lib.hmc_mc_sweeps(h.h, args.warmup, None)
    h.synchronize()
    # the workload logs the texture (angle to the nearest <100>, 10-degree bins) every hist_every MCS
    hist_every = int(spec.get("hist_every", 0))
    hist = np.zeros(9)
    hist_p = hist.ctypes.data_as(G.C.POINTER(G.C.c_double))

    def run_mcs(n):
        done, nh = 0, 0
        while done < n:
            k = min(n - done, hist_every) if hist_every else n
            st = G.lib.hmc_mc_sweeps(h.h, k, None)
            assert st == 0, G.hmc_last_error(h.h)
            done += k
            if hist_every and k == hist_every:
                st = G.lib.hmc_texture_histogram(h.h, G.HMC_HIST_ANGLE_100, 9, hist_p, None)
                assert st == 0, G.hmc_last_error(h.h)
                nh += 1
        return nh

    # ---- timed region: K MCS --------------------------------------------------
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_hist = run_mcs(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    t_local = e0.elapsed_time(e1) / 1e3
    t, units = dist_reduce(t_local, N * args.steps, "cuda")
    value = units / t
    launches = args.steps * (spec["mpm_steps"] + 4) + 2 * n_hist
    texture = [float(x) for x in hist] if n_hist else None

    # ---- per-kernel timing on the same stream (roofline) ----------------------
    n_mpm = 50
    t_mpm = timed(lambda: G.lib.hmc_mpm_steps(h.h, n_mpm, None)) / n_mpm
    t_stress = timed(lambda: G.lib.hmc_compute_stress(h.h, None, None))
    # the half sweeps as a step runs them: red after a stress pass, black after red (eight rounds;
    # each half sweep's time depends on the state, so the median of sixteen)
    t_sweep = []
    for _ in range(8):
        assert G.lib.hmc_compute_stress(h.h, None, None) == 0
        t_sweep += [timed(lambda c=c: G.lib.hmc_sweep_half(h.h, c, None)) for c in (0, 1)]
    t_red, t_black = statistics.median(t_sweep[0::2]), statistics.median(t_sweep[1::2])
    t_sweep = statistics.median(t_sweep)
    mcs_ms = 1e3 * t / args.steps
    sum_ms = 1e3 * (spec["mpm_steps"] * t_mpm + t_stress + 2 * t_sweep)
    mcs_phases = {"mpm_ms": 1e3 * spec["mpm_steps"] * t_mpm, "stress_and_reduction_ms": 1e3 * t_stress,
                  "half_sweeps_ms": 2e3 * t_sweep, "sum_ms": sum_ms, "mcs_ms": mcs_ms,
                  "graph_minus_phases_fraction": (mcs_ms - sum_ms) / mcs_ms}
    hbm, sm_max, peak_src = peaks()
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = n_sms * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    mpm_tflops = MPM_FLOP_PER_POINT * N / t_mpm / 1e12
    fma = measured_fma_peaks(G)
    sweep_gbs = SWEEP_BYTES_PER_SITE["f32"] * (N / 2) / t_sweep / 1e9
    roofline = {"kernel": "k_mpm_step<float> (fused explicit MPM step)", "bound": "alu",
                "achieved": mpm_tflops, "peak": fp32_peak, "unit": "TFLOP/s", "frac": mpm_tflops / fp32_peak,
                "traffic": kernel_traffic("mpm"),
                "algorithmic": f"{MPM_FLOP_PER_POINT} flop/point x {N} points per launch",
                "peak_source": f"derived: {n_sms} SMs x {FP32_LANES} FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                               f"(max SM clock, {peak_src})",
                "hbm_view": {"achieved_gbs": MPM_BYTES_PER_POINT["f32"] * N / t_mpm / 1e9, "peak": hbm,
                             "frac": MPM_BYTES_PER_POINT["f32"] * N / t_mpm / 1e9 / hbm},
                "measured_fma_peaks": dict(fma, frac_of_measured_fp32=mpm_tflops / fma["fp32_tflops"])}
    roofline_sweep = {"kernel": "k_sweep<float, elastic> (red/black half sweep)", "bound": "hbm",
                      "achieved": sweep_gbs, "peak": hbm, "unit": "GB/s", "frac": sweep_gbs / hbm,
                      "traffic": kernel_traffic("sweep"),
                      "algorithmic": f"{SWEEP_BYTES_PER_SITE['f32']} B/site x {N // 2} sites per launch",
                      "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})"}

    # ---- end to end through the C ABI with host buffers -----------------------
    pin_in = torch.from_numpy(spins.reshape(-1).view(np.int16)).pin_memory()
    pin_out = torch.empty(N, dtype=torch.int16).pin_memory()
    a_in = pin_in.numpy().view(np.uint16)
    a_out = pin_out.numpy().view(np.uint16)
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(1):
        G.hmc_set_spins(h.h, a_in)
        G.lib.hmc_mc_sweeps(h.h, 1, None)
        G.hmc_get_spins(h.h, a_out)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        G.hmc_set_spins(h.h, a_in)
        G.lib.hmc_mc_sweeps(h.h, 1, None)
        G.hmc_get_spins(h.h, a_out)
    torch.cuda.synchronize()
    t_e2e = tmax(time.perf_counter() - t0)
    e2e = {"value": N * e2e_steps * ws / t_e2e, "unit": "site-updates/s", "h2d_bytes_per_step": 2 * N,
           "d2h_bytes_per_step": 2 * N, "steps": e2e_steps,
           "path": "hmc_set_spins(pinned host) + hmc_mc_sweeps(1) + hmc_get_spins(pinned host), wall clock"}

    # ---- plain FP64 form on the same GPU --------------------------------------
    fp64 = None
    if not args.no_fp64:
        h64 = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP64, **common)
        h64.set_orientations(euler, spins)
        G.lib.hmc_mc_sweeps(h64.h, 1, None)
        h64.synchronize()
        k64 = 2
        t64 = timed(lambda: G.lib.hmc_mc_sweeps(h64.h, k64, None))
        t64_mpm = timed(lambda: G.lib.hmc_mpm_steps(h64.h, 5, None)) / 5
        v64 = N * k64 / t64
        # the plain form of the explicit step: unfused, incremental, FP64 (one call of 5 steps
        # includes its total-form stress start, a sixth of a step's work)
        G.lib.hmc_mpm_steps_plain(h64.h, 1)
        h64.synchronize()
        t_plain = timed(lambda: G.lib.hmc_mpm_steps_plain(h64.h, 5)) / 5
        mcs_plain = t64 / k64 - spec["mpm_steps"] * t64_mpm + spec["mpm_steps"] * t_plain
        fp64 = {"form": "the fused kernels instantiated in FP64", "value": v64, "unit": "site-updates/s",
                "steps": k64, "speedup_fp32_over_fp64": value / ws / v64,
                "mpm_cell_steps_per_s": N / t64_mpm, "mpm_ms_per_step": t64_mpm * 1e3,
                "mpm_tflops": MPM_FLOP_PER_POINT_F64 * N / t64_mpm / 1e12,
                "mpm_frac_of_measured_fp64": MPM_FLOP_PER_POINT_F64 * N / t64_mpm / 1e12 / fma["fp64_tflops"],
                "mpm_hbm_frac": MPM_BYTES_PER_POINT["f64"] * N / t64_mpm / 1e9 / hbm,
                "plain_unfused": {
                    "form": "the explicit step in the plain form: unfused G2P/stress-increment, P2G and node kernels "
                            "with every point's FP64 stress and every cell's corner forces in global memory "
                            "(hmc_mpm_steps_plain)",
                    "mpm_ms_per_step": t_plain * 1e3, "mpm_cell_steps_per_s": N / t_plain,
                    "algorithmic_bytes_per_point_step": PLAIN_BYTES_PER_POINT,
                    "mpm_hbm_frac": PLAIN_BYTES_PER_POINT * N / t_plain / 1e9 / hbm,
                    "mcs_ms": mcs_plain * 1e3,
                    "mcs_composition": "the FP64 MCS with its 50 fused steps replaced by 50 plain steps",
                    "site_updates_per_s": N / mcs_plain,
                    "speedup_fp32_over_plain_fp64": value / ws / (N / mcs_plain),
                    "mpm_speedup_fp32_over_plain_fp64": t_plain / t_mpm}}
        h64.close()

    # ---- error of the FP32 path against the FP64 path (outside the timed region) ----
    err32 = None
    if rank == 0 and ws == 1 and not args.no_fp64:
        err32 = fp32_error(G, spec, euler, spins, common)

    # ---- CPU oracle on the host cores (rank 0, one GPU only) ------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v1, t1, n1, _ = oracle_rate(spec, euler, spins, 1, 1)
        cores = host_cores()
        v, tt, n, nproc = oracle_rate(spec, euler, spins, 1, cores)
        cpu = {"kind": "oracle", "value": v, "unit": "site-updates/s", "cores": nproc,
               "sample": f"{crop_desc(spins, nproc, n)} of the workload's microstructure, one "
                         f"single-threaded oracle process per host core, one full MCS each ({spec['mpm_steps']} "
                         f"MPM steps, stress, red+black sweep), FP64, {tt:.1f} s wall",
               "one_core": {"value": v1, "unit": "site-updates/s", "cores": 1,
                            "sample": f"{crop_desc(spins, 1, n1)}, one full MCS, {t1:.1f} s"}}

    # ---- the batched ensemble (64 uneven replicas in one handle), one GPU only ----
    ens = None
    if rank == 0 and ws == 1 and not args.no_ensemble:
        ens = ensemble_measure(torch, G, S, ENSEMBLE_STEPS, 3, local)
        ens["workload"] = ENSEMBLE_WORKLOAD(S, ens)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(spec, args.workload), store_stress=args.store_stress),
            "mpm_cell_steps_per_s": N * ws / t_mpm, "mpm_ms_per_step": t_mpm * 1e3,
            "stress_ms": t_stress * 1e3, "half_sweep_ms": t_sweep * 1e3,
            "red_half_sweep_ms": t_red * 1e3, "black_half_sweep_ms": t_black * 1e3,
            "roofline": roofline, "roofline_sweep": roofline_sweep,
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "fp64_form": fp64, "fp32_error": err32,
            "texture_angle100_10deg": texture, "ensemble": ens, "mcs_phases": mcs_phases, "cpu_baseline": cpu,
            "mpm_variant": mpm_variant_name(h.tuning()[0]), "mpm_grid": h.tuning()[1],
            "sweep_cta": h.sweep_tuning()[0], "sweeps_read_stored_stress": h.sweep_tuning()[1],
        }
        print(json.dumps(line), flush=True)
    h.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


FP32_ERR_STEPS = 200


def fp32_error(G, spec, euler, spins, common):
    """The error of the FP32 path against the FP64 path of the same library (which the
    oracle parity tests pin to the oracle), on the workload itself:
      * stress: relative L2 of the FP32 stress after 200 explicit MPM steps from the same
        state (zero displacement, the initial mean strain);
      * decisions: one red and one black half sweep in FP32 and in FP64 on the same spins
        and the same stress (the FP64 stress, rounded for the FP32 handle); the fraction
        of the colour's sites whose decision differs, and how many of those differing
        decisions lie outside the 1e-6 margin |H - t| <= 1e-6 max(1, |t|) of the FP64 sweep."""
    kw = dict(common)
    kw["store_stress"] = 1
    h64 = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP64, **kw)
    h32 = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP32, **kw)
    try:
        for h in (h64, h32):
            h.set_orientations(euler, spins)
            h.mpm_steps(FP32_ERR_STEPS)
            h.compute_stress()
        s64 = h64.stress()
        s32 = h32.stress()
        rel_l2 = float(np.linalg.norm(s32 - s64) / np.linalg.norm(s64))
        del s32
        h32.set_stress(s64)
        del s64
        nz, ny, nx = spec["shape"]
        par = (np.arange(nz)[:, None, None] + np.arange(ny)[None, :, None] + np.arange(nx)[None, None, :]) & 1
        halves = []
        for colour in (0, 1):
            h32.set_spins(h64.spins())
            _, m64 = h64.sweep_half_margins(colour)
            h32.sweep_half(colour)
            mis = (h64.spins() != h32.spins()) & (par == colour)
            n_mis = int(mis.sum())
            gaps = np.abs(m64[mis])
            halves.append({"colour": colour, "sites": int((par == colour).sum()), "mismatched": n_mis,
                           "mismatch_fraction": n_mis / int((par == colour).sum()),
                           "outside_1e-6_margin": int((gaps > 1e-6).sum()),
                           "largest_margin_of_a_mismatch": float(gaps.max()) if n_mis else 0.0,
                           "evaluated_trials": int((~np.isnan(m64) & (par == colour)).sum())})
        return {"stress_rel_l2": rel_l2, "stress_steps": FP32_ERR_STEPS, "half_sweeps": halves,
                "reference": "the library's FP64 path from the same state (pinned to the FP64 oracle by the "
                             "parity tests)"}
    finally:
        h64.close()
        h32.close()


def ensemble_measure(torch, G, S, steps, warmup, clocks_index=0, rank=0, ws=1):
    """The batched ensemble (64 replicas of uneven size in one handle, every phase one
    launch over all replicas, one CUDA graph per MCS): site-updates/s over all replicas,
    the time of each phase launched on its own (50 MPM steps, stress pass with the
    end-of-step reduction, red and black half sweep) and what the graph saves or loses
    against their sum (launch gaps).  With ws ranks, this rank takes its share of the
    replicas (balanced by sites, replica ids kept) and the rates are this rank's."""
    from paper_1009_0457_gb300.shard import balance_replicas
    specs, euler, fields = S.ensemble_inputs()
    if ws > 1:
        mine = balance_replicas([int(np.prod(sp["shape"])) for sp in specs], ws)[rank]
        specs = [dict(sp, replica=r) for r, sp in enumerate(specs)]
        specs, fields = [specs[r] for r in mine], [fields[r] for r in mine]
    else:
        specs = [dict(sp, replica=r) for r, sp in enumerate(specs)]
    stream = torch.cuda.Stream()
    per = [dict(load_axis=sp["axis"], strain=sp["strain"], seed=sp["mc_seed"], replica=sp["replica"])
           for sp in specs]
    b = G.HMCBatch([sp["shape"] for sp in specs], specs[0]["Q"], per, precision=G.HMC_FP32,
                   mpm_steps_per_mcs=50, stream=stream.cuda_stream, **S.COMMON)
    try:
        b.set_orientations(euler, fields)
        G.lib.hmc_mc_sweeps(b.h, warmup, None)
        b.synchronize()
        N = sum(int(np.prod(sp["shape"])) for sp in specs)

        def timed(fn):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a0.record(stream)
            st = fn()
            a1.record(stream)
            torch.cuda.synchronize()
            assert st == 0, G.hmc_last_error(b.h)
            return a0.elapsed_time(a1)

        clocks = Clocks(clocks_index)
        torch.cuda.synchronize()
        clocks.start()
        ms = timed(lambda: G.lib.hmc_mc_sweeps(b.h, steps, None))
        clk = clocks.stop()
        phases = {"mpm_50_steps_ms": timed(lambda: G.lib.hmc_mpm_steps(b.h, 50, None)),
                  "stress_and_reduction_ms": timed(lambda: G.lib.hmc_compute_stress(b.h, None, None)),
                  "red_half_sweep_ms": timed(lambda: G.lib.hmc_sweep_half(b.h, 0, None)),
                  "black_half_sweep_ms": timed(lambda: G.lib.hmc_sweep_half(b.h, 1, None))}
        mcs_ms = ms / steps
        tot = sum(phases.values())
        shape, grid = b.tuning()
        return {"value": N * steps / (ms / 1e3), "unit": "site-updates/s", "steps": steps, "warmup": warmup,
                "ms_per_mcs": mcs_ms, "sites": N, "replicas": len(specs),
                "edges": [sp["shape"][0] for sp in specs],
                "phases_ms": phases, "phase_fractions": {k: v / tot for k, v in phases.items()},
                "sum_of_phases_ms": tot, "graph_minus_phases_fraction": (mcs_ms - tot) / mcs_ms,
                "mpm_variant": mpm_variant_name(shape), "mpm_grid": grid,
                "gpu_launches": steps * (50 + 4), "clocks": clk}
    finally:
        b.close()


def run_ensemble(args):
    """The batched ensemble on its own: one JSON line (site-updates/s over all replicas).
    Under torchrun the replicas are shared out over the ranks (replicas only, no
    collective on the data path): the job's rate is all ranks' site-updates over the
    slowest rank's time, and the ensemble is the same 64 replicas at every N (strong
    scaling)."""
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import hmc_synth as S
    import paper_1009_0457_gb300 as G
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    e = ensemble_measure(torch, G, S, args.steps, args.warmup, local, rank, ws)
    t, units = dist_reduce(e["ms_per_mcs"] * args.steps / 1e3, e["sites"] * args.steps, "cuda")
    if rank == 0:
        line = {"metric": METRIC, "value": units / t, "unit": "site-updates/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": ENSEMBLE_WORKLOAD(S, e), "sites": int(units / args.steps), "replicas": 64,
                           "replicas_on_rank0": e["replicas"], "parallelism": f"replicas over {ws} ranks"},
                "phases_ms": e["phases_ms"], "graph_minus_phases_fraction": e["graph_minus_phases_fraction"],
                "mpm_variant": e["mpm_variant"], "mpm_grid": e["mpm_grid"], "gpu_launches": e["gpu_launches"],
                "clocks": e["clocks"]}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def ENSEMBLE_WORKLOAD(S, e):
    return (f"ensemble: 64 replicas, cubic edges from {S.ENSEMBLE_EDGES}, Q=256, axis uniform on S2, "
            f"strain U[5e-4, 3e-3], 50 MPM steps per MCS, FP32, one launch per phase over all replicas")


# a fixed unit for the zone's rate: the flops of the first sparse block elimination of a trial
# (assembly 8.1k adds, block Cholesky 56k, forward solve and G 4.6k, 6x6 solve 1k); the current
# kernel's bordered form does less work for the same trial
ZONE_FLOP_PER_TRIAL = 70_000


def zone_fp32_error(G, spec, euler, spins, kw):
    """The 27-point zone's FP32 decisions against the library's FP64 zone path (pinned to the
    oracle's zone re-solve by the parity tests), on the workload itself: both handles start
    from the same state, the FP64 one takes the workload's MPM steps and its nodal state is
    given to the FP32 one (rounded), and both then sweep one red and one black half on the same
    spins; the fraction of the colour's sites whose decision differs."""
    hs = {}
    try:
        for prec in (G.HMC_FP64, G.HMC_FP32):
            hs[prec] = G.HMC(spec["shape"], spec["Q"], precision=prec, bc=G.HMC_BC_UNIAXIAL,
                             load_axis=spec["axis"], strain=spec["strain"], elastic=G.HMC_ELASTIC_ZONE1,
                             mpm_steps_per_mcs=spec["mpm_steps"], **kw)
            hs[prec].set_orientations(euler, spins)
        h64, h32 = hs[G.HMC_FP64], hs[G.HMC_FP32]
        h64.mpm_steps(spec["mpm_steps"])
        u, v = h64.nodal()
        h32.set_nodal(u, v)
        nz, ny, nx = spec["shape"]
        par = (np.arange(nz)[:, None, None] + np.arange(ny)[None, :, None] + np.arange(nx)[None, None, :]) & 1
        halves = []
        for colour in (0, 1):
            h32.set_spins(h64.spins())
            before = h64.spins()
            h64.sweep_half(colour)
            trials = h64.info().zone_trials   # the listed trials of this half sweep
            h32.sweep_half(colour)
            mis = (h64.spins() != h32.spins()) & (par == colour)
            halves.append({"colour": colour, "sites": int((par == colour).sum()), "mismatched": int(mis.sum()),
                           "mismatch_fraction": int(mis.sum()) / int((par == colour).sum()),
                           "zone_trials": int(trials), "accepted_fp64": int((h64.spins() != before).sum())})
        return {"half_sweeps": halves, "mpm_steps": spec["mpm_steps"],
                "reference": "the library's FP64 zone path from the same state (pinned to the FP64 oracle's "
                             "zone re-solve by the parity tests)"}
    finally:
        for h in hs.values():
            h.close()


def run_zone(args):
    """The 27-point constant-traction zone (HMC_ELASTIC_ZONE1) on the 128^3
    microstructure: whole MCS timed with CUDA events, plus the zone half sweep
    alone (trial list, spin copy, zone kernel) against the ALU roofline."""
    import torch
    torch.cuda.set_device(0)
    import hmc_synth as S
    import paper_1009_0457_gb300 as G
    spec, euler, spins = S.workload_inputs("ni128")
    stream = torch.cuda.Stream()
    nz, ny, nx = spec["shape"]
    kw = dict(S.COMMON)
    g = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP32, bc=G.HMC_BC_UNIAXIAL, load_axis=spec["axis"],
              strain=spec["strain"], elastic=G.HMC_ELASTIC_ZONE1, mpm_steps_per_mcs=spec["mpm_steps"],
              stream=stream.cuda_stream, **kw)
    g.set_orientations(euler, spins)
    G.lib.hmc_mc_sweeps(g.h, args.warmup, None)
    g.synchronize()
    N = nx * ny * nz
    clocks = Clocks(0)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = G.lib.hmc_mc_sweeps(g.h, args.steps, None)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    assert st == 0, G.hmc_last_error(g.h)
    t = e0.elapsed_time(e1) / 1e3
    # the zone half sweep alone, both colours, on the current state
    half_ms, trials = [], []
    for c in (0, 1, 0, 1):
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        assert G.lib.hmc_sweep_half(g.h, c, None) == 0
        a1.record(stream)
        torch.cuda.synchronize()
        half_ms.append(a0.elapsed_time(a1))
        trials.append(g.info().zone_trials)
    ms = float(np.mean(half_ms))
    ntr = float(np.mean(trials))
    achieved = ZONE_FLOP_PER_TRIAL * ntr / (ms * 1e-3) / 1e12
    _, sm_max, _ = peaks()
    n_sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = n_sms * FP32_LANES * 2 * sm_max / 1e6
    fma = measured_fma_peaks(G)
    line = {"metric": METRIC, "value": N * args.steps / t, "unit": "site-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "zone128: the 128^3 Ni polycrystal (Q=256, 5000 Voronoi grains, uniaxial 2e-3 "
                                   "along [001]) with the 27-point constant-traction zone, 50 MPM steps per MCS",
                       "sites": N},
            "zone_half_sweep_ms": ms, "zone_trials_per_half_sweep": ntr, "zone_ns_per_trial": ms * 1e6 / ntr,
            "roofline": {"kernel": "k_zone<float> (27-point zone, one warp per trial)", "bound": "alu",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": kernel_traffic("zone"),
                         "algorithmic": f"{ZONE_FLOP_PER_TRIAL} flop/trial x {ntr:.0f} trials per half sweep",
                         "peak_source": f"derived: {n_sms} SMs x {FP32_LANES} FP32 lanes x 2 flop x {sm_max:.0f} MHz",
                         "measured_fma_peaks": dict(fma, frac_of_measured_fp32=achieved / fma["fp32_tflops"])},
            "gpu_launches": args.steps * (spec["mpm_steps"] + 2 + 2 * 2), "clocks": clk}
    g.close()
    if not args.no_fp64:
        line["fp32_error"] = zone_fp32_error(G, spec, euler, spins, kw)
    print(json.dumps(line), flush=True)
    return 0


ADJ_STEPS, ADJ_EVERY = 200, 20


def run_adjoint(args):
    """The adjoint of the explicit MPM solve (the differentiation form) on the 128^3
    microstructure: spins frozen, Ebar = the library's initial mixed-control strain for
    2e-3 along [001], 200 FP32 steps with a checkpoint every 20.  One step = the forward
    map (W and the w field) plus the reverse sweep giving d(gW W + g.w)/d(C11, C12, C44,
    Ebar_1..6); CUDA events around each, on the library's stream."""
    import torch
    torch.cuda.set_device(0)
    import hmc_synth as S
    import paper_1009_0457_gb300 as G
    spec, euler, spins = S.workload_inputs("ni128")
    nz, ny, nx = spec["shape"]
    N = nx * ny * nz
    stream = torch.cuda.Stream()
    kw = dict(c11=spec["c11"], c12=spec["c12"], c44=spec["c44"], stream=stream.cuda_stream)
    u = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP32, load_axis=(0.0, 0.0, 1.0), strain=2e-3,
              mpm_steps_per_mcs=0, **kw)
    u.set_orientations(euler, spins)
    E = u.strain()
    u.close()
    g = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP32, bc=G.HMC_BC_STRAIN6, strain6=tuple(E),
              mpm_steps_per_mcs=0, **kw)
    g.set_orientations(euler, spins)
    g_field = np.random.default_rng(5).random(N)
    nodal0 = g.nodal()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, r

    fw, bw = [], []
    for it in range(args.warmup + args.steps):
        g.set_nodal(*nodal0)
        tf, _ = timed(lambda: g.adjoint_forward(ADJ_STEPS, ADJ_EVERY))
        tb, grad = timed(lambda: g.adjoint_backward(0.5, g_field))
        if it >= args.warmup:
            fw.append(tf)
            bw.append(tb)
    t_mpm, _ = timed(lambda: G.lib.hmc_mpm_steps(g.h, ADJ_STEPS, None))
    tf, tb = float(np.median(fw)), float(np.median(bw))
    line = {"metric": METRIC, "value": N * ADJ_STEPS / (tf + tb), "unit": "cell-steps/s (forward + reverse)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * (tf + tb),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "adjoint128: the 128^3 Ni polycrystal (Q=256, 5000 Voronoi grains) with frozen spins, "
                                   "mean strain = the initial mixed-control strain for 2e-3 along [001], 200 explicit "
                                   "FP32 MPM steps, checkpoint every 20, gradient of 0.5 W + g.w w.r.t. C11, C12, C44 "
                                   "and the 6 mean-strain components", "sites": N},
            "forward_ms": 1e3 * tf, "reverse_ms": 1e3 * tb, "plain_mpm_ms": 1e3 * t_mpm,
            "adjoint_cost_in_forward_steps": (tf + tb) / (t_mpm / ADJ_STEPS) / ADJ_STEPS,
            "gradient": [float(x) for x in grad]}
    g.close()
    if not args.no_fp64:
        # the FP32 gradient against the library's FP64 adjoint (pinned to the oracle's
        # tangent-linear gradient by the parity tests), same map, same cotangent
        h = G.HMC(spec["shape"], spec["Q"], precision=G.HMC_FP64, bc=G.HMC_BC_STRAIN6, strain6=tuple(E),
                  mpm_steps_per_mcs=0, **kw)
        h.set_orientations(euler, spins)
        h.adjoint_forward(ADJ_STEPS, ADJ_EVERY)
        g64 = np.asarray(h.adjoint_backward(0.5, g_field), dtype=np.float64)
        h.close()
        g32 = np.asarray(line["gradient"], dtype=np.float64)
        rel = np.abs(g32 - g64) / np.maximum(np.abs(g64), 1e-300)
        line["fp32_error"] = {"gradient_rel_err_per_component": [float(x) for x in rel],
                              "gradient_rel_err_max": float(rel.max()),
                              "gradient_rel_l2": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64)),
                              "reference": "the library's FP64 adjoint of the same map (pinned to the FP64 "
                                           "oracle's tangent-linear gradient by the parity tests)"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "zone128":
        return run_zone(args)
    if args.workload == "adjoint128":
        return run_adjoint(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
