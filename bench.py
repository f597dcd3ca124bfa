"""Throughput of the FFT-based Yamamoto multipole estimator on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one catalogue through the whole path: mesh assignment (galaxies minus
alpha randoms, TSC, interlaced), the 1 + 6 + 15 line-of-sight fields and their 3D
FFTs, the k-space combination, shell sums and Eqs. (6)-(8).  Workload: the
survey-shaped synthetic catalogue -- 1e7 galaxies and 5e7 randoms uniform in a
600-2000 Mpc/h shell clipped to a 3500 Mpc/h box centred on the observer, 512^3 mesh,
TSC + interlacing, l <= 4, shells of 0.01 h/Mpc up to k = 0.4 h/Mpc (seeded;
inputs are resident in HBM and far larger than L2, so no L2 flush is needed).

Under torchrun (N > 1) every rank runs its own catalogue (independent replicas,
weak scaling, no collective on the data path); value = all catalogues / max time.

--impl reference times the FP64 CPU oracle (oracle/) on this machine's host cores:
each step is a bounded sample of the same workload (a particle subsample and a
subset of the field transforms), extrapolated to seconds per catalogue.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "P0/P2/P4 catalogues/s at 512^3, 1e7 gal, % HBM roofline; batched/learned vs plain"
UNIT = "catalogues/s"
WORKLOAD = "shell512_tsc_il"
N_MESH = 512
K_MAX = 0.4
DK = 0.01
# Other workloads, for profiling captures that must stay small on the device.
WORKLOADS = {
    "shell512_tsc_il": dict(n_mesh=512, k_max=0.4),
    "cone256_tsc_il": dict(n_mesh=256, k_max=None),   # up to Nyquist
}


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        hbm = d.get("hbm_gbs") or d.get("hbm_GBps") or d.get("hbm")
        if hbm:
            return float(hbm), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def rank_seeds(rank, name=WORKLOAD):
    """(galaxy / field seed, random seed) of a replica: every rank draws its own
    catalogue of the same workload."""
    base = {"shell512_tsc_il": (4, 5), "cone256_tsc_il": (2, 3)}[name]
    return base[0] + 100 * rank, base[1] + 100 * rank


def seeds_record(rank, name=WORKLOAD):
    """The seeds of this rank's catalogue, as recorded in the result line."""
    sg, sr = rank_seeds(rank, name)
    return {"galaxies": sg, "randoms": sr, "rank": rank, "other_ranks": "both seeds + 100 per rank"}


def make_workload(rank, name=WORKLOAD, scale=1.0):
    import synth
    sg, sr = rank_seeds(rank, name)
    if name == "shell512_tsc_il":
        return synth.poisson_shell(int(10_000_000 * scale), int(50_000_000 * scale), seed_gal=sg, seed_ran=sr)
    if name == "cone256_tsc_il":
        return synth.zeldovich_cone(int(1_000_000 * scale), int(5_000_000 * scale), seed_field=sg, seed_ran=sr)
    raise KeyError(name)


def max_over_ranks(value, device):
    """The slowest rank's time: the job's time for N replicas (all_reduce MAX)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, steps, seconds):
    """Whole-job catalogues per second: every rank processes `steps` catalogues."""
    return world * steps / seconds


def alg_bytes(n_gal, n_ran, n, m, groups, n_pencils):
    """Algorithmic HBM bytes per catalogue (pruned pencils): particles read once
    (x, y, z, w), each mesh written and read once, each grouped half-spectrum pencil
    written once and read once."""
    return 16 * (n_gal + n_ran) + m * 8 * n ** 3 + m * groups * 16 * n * n_pencils


# FP32 issue peak of the GB300 (derived, not measured): 152 SMs x 128 FP32 lanes x
# 2 flops per FMA x 2.07 GHz maximum SM clock.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def fft_flops(cls, n, m, n_pencils, nzc, pairs=8, fields=16, groups=9):
    """Nominal FFT flops per launch (5 L log2 L per complex line of length L) of the
    two transform kernels: the y,z stage transforms m N^2 lines along z per field
    pair and m N nzc lines along y per basis field; the x stage m G lines per kept
    pencil."""
    line = 5.0 * n * math.log2(n)
    if cls == "yz_stage":
        return line * (m * n * n * pairs + m * n * nzc * fields)
    if cls == "x_combine":
        return line * m * groups * n_pencils
    return 0.0


# DRAM bytes (read + write) per launch that ncu measured for the current build of
# each kernel on the 512^3 survey workload in its tuned launch configuration (one-pass
# dram__bytes_{read,write}.sum capture; profiles/dram_traffic_shell512_tsc_il.md).
# Remove an entry when its kernel changes.  particle_count and particle_bin: the mean
# of the galaxy and random launches.
TRAFFIC = {"yz_stage": 8.86e9, "x_combine": 5.77e9, "tile_deposit": 2.50e9, "particle_bin": 1.26e9,
           "particle_count": 0.58e9}


def kernel_bytes(cls, n_gal, n_ran, n, m, groups, n_pencils, launches_per_step, batch_planes):
    """Algorithmic bytes per launch of one kernel class."""
    if cls == "particle_count":
        return (16 * (n_gal + n_ran) + 4 * n_ran) / 2
    if cls == "particle_bin":
        return 16 * (n_gal + n_ran) / 2
    if cls == "tile_deposit":
        return m * 4 * n ** 3
    if cls == "yz_stage":
        return (m * 4 * n ** 3 + m * groups * 8 * n * n_pencils) / launches_per_step
    if cls == "x_combine":
        return m * groups * 8 * n * n_pencils
    return 0.0


def cpu_sample(gal, ran, geo, frac=0.05, n_fields=7, field_mesh=None):
    """Time the FP64 oracle on a bounded sample of the workload and extrapolate to
    seconds per catalogue: mesh assignment of a particle subsample at the workload's
    mesh (scaled by 1/frac and by the 2 meshes), the l <= 2 field transforms of one
    mesh (A_0 + 6 B_ij; scaled to 22 fields x 2 meshes), and one pass of shell
    binning.  With ``field_mesh`` below the workload's mesh the field transforms and
    the binning run on that smaller mesh and are scaled by the cell-count ratio
    (N / n)^3: their cost is dominated by N^3 elementwise passes (measured 512^3 /
    256^3 time ratio 8.0 for the 7 transforms)."""
    import oracle
    import synth
    from oracle.binning import BinSpec, bin_sums, mode_bins
    from oracle.estimator import mesh_transforms, node_offsets

    workers = _cores()
    fm = field_mesh or N_MESH
    vol = (N_MESH / fm) ** 3
    ng = max(1, int(gal.n * frac))
    nr = max(1, int(ran.n * frac))
    sub = lambda c, k: synth.Catalog(c.x[:k], c.y[:k], c.z[:k], c.w[:k], c.nbar[:k])
    t0 = time.perf_counter()
    F = oracle.assign_mesh(sub(gal, ng), sub(ran, nr), 0.2, geo.box_min, geo.box_len, N_MESH, "tsc", False)
    t_assign = time.perf_counter() - t0
    if fm != N_MESH:
        F = oracle.assign_mesh(sub(gal, ng), sub(ran, nr), 0.2, geo.box_min, geo.box_len, fm, "tsc", False)
    rx, ry, rz = node_offsets(geo.box_min, geo.box_len, fm, geo.observer, False)
    ell = 2 if n_fields >= 7 else 0
    t0 = time.perf_counter()
    T = mesh_transforms(F, rx, ry, rz, ell, workers)
    t_fields = time.perf_counter() - t0
    nf = 7 if ell == 2 else 1
    t0 = time.perf_counter()
    bins = BinSpec.up_to(K_MAX, DK)
    bidx, w, kmag = mode_bins(fm, geo.box_len, bins)
    A0 = T["A0"]
    for key in T:
        bin_sums((A0 * np.conj(T[key])).real, bidx, w, bins.n_bins)
    t_tail = time.perf_counter() - t0
    per_cat = t_assign / frac * 2 + (t_fields / nf * 22 * 2 + t_tail * 3 / len(T)) * vol
    where = f"at {N_MESH}^3" if fm == N_MESH else f"at {fm}^3 scaled by (N/n)^3 = {vol:g}"
    sample = (f"oracle on {frac:.0%} of the particles (1 TSC mesh at {N_MESH}^3), {nf} of the 44 field FFTs "
              f"{where}, one shell-binning pass; scaled to 2 meshes x 22 fields; "
              f"{t_assign + t_fields + t_tail:.1f} s measured")
    return per_cat, sample, workers


def galaxy_sum_rate(seconds=2.0):
    """Terms per second of the oracle's direct galaxy sum (Sec. 4's sum-gal: one
    particle x one k mode x l = 0, 2, 4), timed on a 500 + 2500 point cube with the
    modes of a 16^3 grid.  The context figure beside the CPU baseline: the cost of
    the sum the FFT method replaces."""
    import oracle
    import synth
    from oracle.binning import BinSpec
    gal, ran, geo = synth.poisson_cube(500, 2500, seed=1)
    bins = BinSpec.up_to(math.pi * 16 / geo.box_len, 0.01)
    t0 = time.perf_counter()
    runs = 0
    res = None
    while time.perf_counter() - t0 < seconds or runs == 0:
        res = oracle.sum_gal(gal, ran, geo, 16, bins)
        runs += 1
    dt = (time.perf_counter() - t0) / runs
    modes = float(np.sum(res.n_modes)) / 2.0  # half-grid modes summed (Hermitian weights 2)
    return (gal.n + ran.n) * modes / dt


def half_modes_below(k_max, box_len, n):
    """Half-grid modes with 0 < |k| < min(k_max, k_Nyquist), by counting integer
    vectors (k_z >= 0, half of the k_z = 0 plane)."""
    kf = 2 * math.pi / box_len
    m2max = (min(k_max, kf * n / 2) / kf) ** 2
    r = int(math.sqrt(m2max)) + 1
    g = np.arange(-r, r + 1)
    kx, ky = np.meshgrid(g, g, indexing="ij")
    count = 0.0
    for kz in range(0, r + 1):
        m2 = kx * kx + ky * ky + kz * kz
        c = np.count_nonzero((m2 > 0) & (m2 < m2max))
        count += c if kz > 0 else c / 2.0
    return count


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth  # noqa: F401
    gal, ran, geo = make_workload(0)
    times = []
    sample = ""
    cores = _cores()
    for i in range(args.warmup + args.steps):
        per_cat, sample, cores = cpu_sample(gal, ran, geo, frac=0.01, n_fields=7, field_mesh=N_MESH // 2)
        if i >= args.warmup:
            times.append(per_cat)
    value = 1.0 / statistics.mean(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_mesh": N_MESH, "assign": "tsc", "interlace": True, "ell_max": 4,
                   "n_gal": gal.n, "n_ran": ran.n, "k_max": K_MAX, "dk": DK, "seeds": seeds_record(0)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1505_05341_gb300 as ys

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    global N_MESH, K_MAX
    wl = WORKLOADS[args.workload]
    gal, ran, geo = make_workload(rank, args.workload)
    N_MESH = wl["n_mesh"]
    K_MAX = wl["k_max"] if wl["k_max"] is not None else math.pi * N_MESH / geo.box_len
    dev = lambda c: tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (c.x, c.y, c.z, c.w, c.nbar))
    dgal, dran = dev(gal), dev(ran)
    stream = torch.cuda.current_stream()
    n_bins = int(math.ceil(K_MAX / DK - 1e-9))
    plan = ys.Plan(N_MESH, geo.box_min, geo.box_len, geo.observer, assign="tsc", interlace=True, ell_max=4,
                   dk=DK, n_bins=n_bins, max_particles=gal.n + ran.n, stream=stream.cuda_stream)
    out = torch.empty(5 * n_bins + 5, dtype=torch.float64, device="cuda")

    def step():
        plan.assign(dgal, dran)
        plan.measure_async(out)

    # launch shapes for this configuration (scatter tile, y,z grid and ring lead),
    # chosen once before any timing (--no-tune keeps the defaults, so that a
    # profiler sees a fixed launch sequence)
    if args.no_tune:
        tuning = None
    else:
        tuning = plan.autotune(dgal, dran, reps=2)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.stats(reset=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        # keep the GPU busy while nvidia-smi starts, so that its samples fall under load
        t_spin = time.perf_counter() + 0.6
        while time.perf_counter() < t_spin:
            step()
            torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = plan.stats(reset=True)
    gpu_launches = sum(v[0] for v in st.values())
    if world > 1:
        ms = max_over_ranks(ms, "cuda")
        dist.barrier()
    value = job_rate(world, args.steps, ms / 1e3)

    # Per-kernel device times: a short profiled pass (events around each launch).
    plan.set_profiling(True)
    for _ in range(2):
        step()
    prof = plan.stats(reset=True)
    plan.set_profiling(False)
    plan.measure_async(out)  # re-arm the captured graph path
    torch.cuda.synchronize()

    # End to end through the host entry point: H2D copies of the catalogue inside.
    pin = lambda c: [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in
                     (c.x, c.y, c.z, c.w, c.nbar)]
    hg, hr = pin(gal), pin(ran)
    # each call is synchronous (copies in, result out): time them one by one and take
    # the median, which host-side outliers (page faults, scheduler) do not move
    e2e_steps = max(1, min(args.steps, 10))
    plan.estimate_host(hg, hr)
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        plan.estimate_host(hg, hr)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_times)
    if world > 1:
        e2e_s = max_over_ranks(e2e_s, "cuda")
    res = plan.measure()

    n_pencils, nzc = plan_pencils(plan, with_nzc=True)
    m, groups = 2, 9
    steps_prof = 2
    per_cls = {k: (v[0] / steps_prof, v[1] / max(1, v[0])) for k, v in prof.items() if v[0] > 0}
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    launches_dom = per_cls[dom][0]
    bytes_dom = kernel_bytes(dom, gal.n, ran.n, N_MESH, m, groups, n_pencils, launches_dom, None)
    avg_ms = per_cls[dom][1]
    peak, peak_src = _peaks()
    achieved = bytes_dom / (avg_ms / 1e3) / 1e9
    flops_dom = fft_flops(dom, N_MESH, m, n_pencils, nzc)
    # the ncu DRAM table holds the headline workload in its tuned configuration only
    traffic = TRAFFIC if (args.workload == WORKLOAD and not args.no_tune) else {}
    b_alg = alg_bytes(gal.n, ran.n, N_MESH, m, groups, n_pencils)
    if flops_dom > 0:
        # the transform kernels are bound by FP32 issue, not by HBM
        tflops = flops_dom / (avg_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "kernel": dom, "achieved": tflops, "peak": FP32_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": tflops / FP32_PEAK_TFLOPS, "traffic": traffic.get(dom),
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                    "flops_per_launch": flops_dom, "avg_launch_ms": avg_ms,
                    "hbm_view": {"alg_bytes_per_launch": bytes_dom, "achieved_GBps": achieved, "peak_GBps": peak,
                                 "frac": achieved / peak, "peak_source": peak_src}}
    else:
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic.get(dom), "peak_source": peak_src,
                    "alg_bytes_per_launch": bytes_dom, "avg_launch_ms": avg_ms}
    ms_step = ms / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n_mesh": N_MESH, "assign": "tsc", "interlace": True, "ell_max": 4,
                   "n_gal": gal.n, "n_ran": ran.n, "k_max": K_MAX, "dk": DK, "fields": "1+6+15",
                   "l2": "inputs larger than L2 (0.96 GB catalogue, 1 GB meshes, 11 GB spectra)",
                   "parallelism": f"replicas{world}", "seeds": seeds_record(rank, args.workload),
                   "tuned": ({"tile": list(tuning.tile), "yz_grid": tuning.yz_grid, "ring_lead": tuning.ring_lead,
                              "x_pencils": tuning.x_pencils}
                             if tuning is not None else "defaults (--no-tune)")},
        "roofline": roofline,
        "step_roofline": {"bound": "hbm", "alg_bytes": b_alg, "achieved_GBps": b_alg / (ms_step / 1e3) / 1e9,
                          "peak_GBps": peak, "frac": b_alg / (ms_step / 1e3) / 1e9 / peak, "peak_source": peak_src},
        "kernels": {k: {"launches_per_step": v[0], "avg_ms": v[1], "dram_bytes_ncu": traffic.get(k),
                        "dram_GBps": (traffic[k] / (v[1] / 1e3) / 1e9) if k in traffic and v[1] > 0 else None}
                    for k, v in per_cls.items()},
        "clocks": clk.summary(),
        "e2e": {"value": job_rate(world, 1, e2e_s), "unit": UNIT, "h2d_bytes_per_step": 16 * gal.n + 20 * ran.n,
                "d2h_bytes_per_step": 8 * (5 * n_bins + 5), "calls": e2e_steps, "statistic": "median",
                "ms_min_max": [1e3 * min(e2e_times), 1e3 * max(e2e_times)]},
        "gpu_launches": gpu_launches,
        "p0_first_bins": [float(v) for v in res.p0[:3]],
    }
    if world == 1 and args.workload == WORKLOAD:
        try:
            cmp_ = cufft_comparison()
            cmp_["ours_yz_plus_x_ms"] = sum(per_cls[c][0] * per_cls[c][1] for c in ("yz_stage", "x_combine")
                                            if c in per_cls)
            line["cufft_comparison"] = cmp_
        except Exception as exc:  # a comparison only: never fail the benchmark for it
            line["cufft_comparison"] = {"error": str(exc)[:200]}
    if world == 1 and not args.no_extras and args.workload == WORKLOAD:
        try:
            line["extras"] = run_extras(gal, ran, geo, dgal, dran, n_bins, max(3, min(args.steps, 5)))
        except Exception as exc:  # sub-entries only: never fail the benchmark for them
            line["extras"] = {"error": str(exc)[:300]}
    if world == 1 and not args.no_batched and args.workload == WORKLOAD:
        del dgal, dran
        plan.close()
        torch.cuda.empty_cache()
        line["batched"] = run_batched(max(1, min(args.steps, 3)), 1)
    if world == 1 and not args.no_learned and args.workload == WORKLOAD:
        line["learned"] = run_learned(max(1, min(args.steps, 3)))
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per_cat, sample, cores = cpu_sample(gal, ran, geo)
        line["cpu_baseline"] = {"value": 1.0 / per_cat, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample}
        try:  # context only: the direct galaxy sum the FFT method replaces (Sec. 4)
            rate = galaxy_sum_rate()
            terms = (gal.n + ran.n) * half_modes_below(K_MAX, geo.box_len, N_MESH)
            line["cpu_baseline"]["galaxy_sum"] = {
                "terms_per_s": rate, "terms_per_catalogue": terms, "s_per_catalogue": terms / rate,
                "what": "oracle sum-gal (particles x half-grid modes below k_max, l <= 4) timed on a "
                        "3000-point cube and extrapolated to this workload"}
        except Exception as exc:
            line["cpu_baseline"]["galaxy_sum"] = {"error": str(exc)[:200]}
    plan.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def _event_time_s(fn, steps, stream):
    """Seconds per call of fn (queued on stream), by CUDA events after one warm-up."""
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / steps


def run_extras(gal, ran, geo, dgal, dran, n_bins, steps):
    """Sub-entries for the rows beyond l <= 4 on the survey catalogue: l_max = 6, shared
    randoms, the direct galaxy sum and the wedges' definition (Sec. 4, 5), and the
    paper-shaped mock on the meshes of Table 1.  Each is timed with CUDA events on
    device-resident inputs; none is the headline metric."""
    import torch

    import paper_1505_05341_gb300 as ys
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    out = {}

    # l <= 6 on the same 512^3 TSC interlaced survey catalogue (28 more fields)
    with ys.Plan(N_MESH, geo.box_min, geo.box_len, geo.observer, assign="tsc", interlace=True, ell_max=6,
                 dk=DK, n_bins=n_bins, max_particles=gal.n + ran.n, stream=sp) as p6:
        row = torch.empty(p6.row_len, dtype=torch.float64, device="cuda")
        t = _event_time_s(lambda: (p6.assign(dgal, dran), p6.measure_async(row)), steps, stream)
        out["l6"] = {"value": 1.0 / t, "unit": UNIT, "ms_per_catalogue": 1e3 * t, "fields": "1+6+15+28",
                     "what": "ys_assign + ys_measure_multipoles_async with ell_max = 6, 512^3 TSC interlaced, "
                             "1e7 + 5e7, shells to 0.4"}
    torch.cuda.empty_cache()

    # shared randoms: the 5e7 randoms deposited once, each catalogue's 1e7 galaxies after
    with ys.Plan(N_MESH, geo.box_min, geo.box_len, geo.observer, assign="tsc", interlace=True, ell_max=4,
                 dk=DK, n_bins=n_bins, max_particles=gal.n + ran.n, stream=sp) as pc:
        row = torch.empty(pc.row_len, dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        pc.cache_randoms(dran)
        torch.cuda.synchronize()
        t_cache = time.perf_counter() - t0
        t = _event_time_s(lambda: (pc.assign_cached(dgal), pc.measure_async(row)), steps, stream)
        out["shared_randoms"] = {"value": 1.0 / t, "unit": UNIT, "ms_per_catalogue": 1e3 * t,
                                 "cache_ms_once": 1e3 * t_cache,
                                 "what": "ys_assign_cached (1e7 galaxies against 5e7 kept randoms) + "
                                         "ys_measure_multipoles_async, 512^3 TSC interlaced"}
    torch.cuda.empty_cache()

    # the direct galaxy sum on the GPU: its rate, and the paper's comparison (Sec. 4: the
    # FFT method is > 1000x faster than the sums) on this catalogue
    import synth
    from oracle.binning import BinSpec
    cg, cr, cgeo, _ = synth.workload("cube32_cic")
    cbins = BinSpec.up_to(math.pi * 32 / cgeo.box_len, 0.01)
    dev = lambda c: tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (c.x, c.y, c.z, c.w, c.nbar))
    dcg, dcr = dev(cg), dev(cr)
    sg = lambda: ys.sum_gal(32, cgeo.box_min, cgeo.box_len, dcg, dcr, observer=cgeo.observer, dk=cbins.dk,
                            n_bins=cbins.n_bins, stream=sp)
    sg()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        sg()
    t_sg = (time.perf_counter() - t0) / 3
    terms = (cg.n + cr.n) * half_modes_below(math.pi * 32 / cgeo.box_len, cgeo.box_len, 32)
    rate = terms / t_sg
    survey_terms = (gal.n + ran.n) * half_modes_below(K_MAX, geo.box_len, N_MESH)
    out["sum_gal"] = {"terms_per_s": rate, "s_per_c1_catalogue": t_sg,
                      "survey_terms": survey_terms, "survey_s_extrapolated": survey_terms / rate,
                      "what": "ys_sum_gal (l <= 4) on the 2000 + 10000-point cube, 32^3 lattice, synchronous "
                              "call; extrapolated by terms to the 512^3 survey catalogue for the FFT-vs-sum ratio"}

    # Fig. 2's comparison: wedges by their definition against Eqs. 16-17, four mocks
    gaps_perp, gaps_para = [], []
    for seed in (301, 302, 303, 304):
        wg, wr, wgeo = synth.zeldovich_cube(20_000, 100_000, n_lattice=64, seed=seed)
        n = 32
        wb = BinSpec.up_to(math.pi * n / wgeo.box_len, 0.02)
        dwg, dwr = dev(wg), dev(wr)
        res, (pp, pq) = ys.sum_gal(n, wgeo.box_min, wgeo.box_len, dwg, dwr, observer=wgeo.observer, dk=wb.dk,
                                   n_bins=wb.n_bins, wedges=True, stream=sp)
        with ys.Plan(n, wgeo.box_min, wgeo.box_len, wgeo.observer, assign="tsc", interlace=True, ell_max=4,
                     dk=wb.dk, n_bins=wb.n_bins, stream=sp) as pw:
            pw.assign(dwg, dwr)
            rowd = torch.empty((1, pw.row_len), dtype=torch.float64, device="cuda")
            pw.measure_async(rowd[0])
            wout = torch.empty((1, 2, wb.n_bins), dtype=torch.float64, device="cuda")
            ys.wedges(rowd, wb.n_bins, wout, stream=sp)
            torch.cuda.synchronize()
            approx = wout.cpu().numpy()[0]
        k = res.k
        sel = (res.n_modes > 0) & (k > 0.05) & (k < 0.2)
        raw = res.p0[sel] + res.shot_noise   # the monopole before shot noise: P_perp can cross zero
        gaps_perp.append(np.abs(approx[0][sel] - pp[sel]) / raw)
        gaps_para.append(np.abs(approx[1][sel] - pq[sel]) / raw)
    out["wedges_definition_vs_eqs16_17"] = {
        "mean_gap_perp_over_raw_p0": float(np.mean(np.concatenate(gaps_perp))),
        "mean_gap_para_over_raw_p0": float(np.mean(np.concatenate(gaps_para))),
        "what": "Sec. 5 / Fig. 2 on synthetic mocks: P_perp, P_para by their definition (GPU galaxy sum, "
                "top hats at |mu| = 1/2) against Eqs. 16-17 from the GPU FFT multipoles (32^3 TSC interlaced); "
                "mean |gap| / (P_0 + S/I) over shells 0.05 < k < 0.2 h/Mpc of four 20 000-galaxy Zel'dovich cubes"}
    torch.cuda.empty_cache()

    # the paper-shaped mock (525 000 galaxies, 10x randoms, CIC) on Table 1's meshes
    pg, pr, pgeo, _ = synth.workload("paper512_cic")
    dpg, dpr = dev(pg), dev(pr)
    shaped = {}
    for n in (512, 1024):
        nb = int(math.ceil(math.pi * n / pgeo.box_len / DK - 1e-9))
        with ys.Plan(n, pgeo.box_min, pgeo.box_len, pgeo.observer, assign="cic", interlace=False, ell_max=4,
                     dk=DK, n_bins=nb, max_particles=pg.n + pr.n, stream=sp) as pp_:
            row = torch.empty(pp_.row_len, dtype=torch.float64, device="cuda")
            t = _event_time_s(lambda: (pp_.assign(dpg, dpr), pp_.measure_async(row)), max(2, steps - 2), stream)
            shaped[str(n)] = {"value": 1.0 / t, "unit": UNIT, "s_per_catalogue": t,
                              "paper_s_per_catalogue": {512: 72.0, 1024: 450.0}[n]}
        torch.cuda.empty_cache()
    out["paper_shaped"] = {"meshes": shaped, "what": "paper512_cic / paper1024_cic: 525 000 Zel'dovich galaxies, "
                           "5.25e6 randoms, 3500 Mpc/h box, CIC, shells of 0.01 to Nyquist; the paper's times "
                           "(Table 1, 16 CPU cores, its own PTHalos mock) are context only"}
    return out


def batched_catalogues(n_cat=256, first_seed=1000):
    """The batched-mock workload on the GPU: per catalogue (seed, n_gal, mesh) from
    synth.batched_cube_specs; config-1-style clustered mocks (Zel'dovich + RSD in the
    500 Mpc/h cube centred on (600, 600, 600), observer at the origin, randoms 5 n_gal,
    unit weights) drawn on the device from generators seeded with the catalogue seed."""
    import synth
    import synth.gpu as sg
    specs = synth.batched_cube_specs(n_cat, first_seed)
    gals, rans = [], []
    for seed, ng, nr, mesh in specs:
        g, r, _ = sg.zeldovich_cube(ng, nr, seed)
        gals.append(g)
        rans.append(r)
    return specs, gals, rans


def run_batched(steps, warmup):
    """Batched-mock throughput: one graph launch over all catalogues, against the same
    catalogues run one at a time through the plain path (one plan per mesh size)."""
    import torch
    import paper_1505_05341_gb300 as ys
    specs, gals, rans = batched_catalogues()
    cfgs = [ys.make_config(mesh, (350.0,) * 3, 500.0, (0.0, 0.0, 0.0), assign="cic", interlace=False, dk=0.01,
                           max_particles=ng + nr) for seed, ng, nr, mesh in specs]
    batch = ys.Batch(cfgs, lanes=8)
    out = torch.zeros((batch.n, batch.stride), dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    batch.autotune(gals, rans, reps=2)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    for _ in range(max(1, warmup)):
        batch.run(gals, rans, out, stream.cuda_stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        batch.run(gals, rans, out, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1) / steps
    rows = batch.results(out)
    bad = sum(1 for r in rows if r.status != 0)
    batch.close()
    # plain path: one plan per mesh size, catalogues one after another
    plans = {}
    for (seed, ng, nr, mesh) in specs:
        if mesh not in plans:
            cap = max(g + r for s_, g, r, m in specs if m == mesh)
            plans[mesh] = ys.Plan(mesh, (350.0,) * 3, 500.0, (0.0, 0.0, 0.0), assign="cic", dk=0.01,
                                  max_particles=cap, stream=stream.cuda_stream)
    def plain_pass():
        for i, (seed, ng, nr, mesh) in enumerate(specs):
            plans[mesh].assign(gals[i], rans[i])
            plans[mesh].measure_async(out[i])
    plain_pass()
    torch.cuda.synchronize()
    e0.record(stream)
    plain_pass()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    for pl in plans.values():
        pl.close()
    meshes = {m: sum(1 for s_ in specs if s_[3] == m) for m in (128, 192, 256)}
    return {"value": len(specs) / (ms_batch / 1e3), "unit": UNIT, "n_catalogs": len(specs),
            "ms_per_batch": ms_batch, "plain_value": len(specs) / (ms_plain / 1e3),
            "speedup_vs_plain": ms_plain / ms_batch, "meshes": meshes, "assign": "cic", "lanes": 8,
            "autotune_s": tune_s, "rows_with_errors": bad, "seeds": [specs[0][0], specs[-1][0]],
            "particles": int(sum(g + r for s_, g, r, m in specs))}


def run_learned(steps, n_heldout=200):
    """Learned correction on the held-out mocks (seeds 20000-20199): the coarse 128^3
    CIC measurement of every mock in one batched graph launch plus one correction
    launch, against the plain 512^3 TSC+interlaced path on the same mocks, with the
    residual of both coarse and corrected multipoles against the 512^3 result."""
    import torch
    import paper_1505_05341_gb300 as ys
    import synth.gpu as sg
    from paper_1505_05341_gb300 import learned
    if not os.path.exists(learned.WEIGHTS):
        return {"unavailable": "no trained weights at " + os.path.relpath(learned.WEIGHTS, ROOT)}
    mlp, meta = learned.load()
    seeds = list(range(learned.HELDOUT_SEEDS, learned.HELDOUT_SEEDS + n_heldout))
    gals, rans, caps = [], [], []
    for sd in seeds:
        ng, nr = sg.mock_sizes(sd)
        g, r, _ = sg.zeldovich_cube(ng, nr, sd)
        gals.append(g)
        rans.append(r)
        caps.append(ng + nr)
    n = len(seeds)
    cfgs = [ys.make_config(learned.COARSE["n_mesh"], learned.BOX_MIN, learned.BOX_LEN, learned.OBSERVER,
                           assign=learned.COARSE["assign"], interlace=learned.COARSE["interlace"], dk=learned.DK,
                           n_bins=learned.N_BINS, max_particles=c) for c in caps]
    batch = ys.Batch(cfgs, lanes=8)
    rows = torch.zeros((n, batch.stride), dtype=torch.float64, device="cuda")
    corr = torch.empty_like(rows)
    batch.autotune(gals, rans, reps=2)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def learned_pass():
        batch.run(gals, rans, rows, sp)
        mlp.correct(rows, learned.N_BINS, learned.K_NYQ, corr, sp)

    for _ in range(2):
        learned_pass()
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    for _ in range(steps):
        learned_pass()
    e1.record(stream)
    for _ in range(steps):
        mlp.correct(rows, learned.N_BINS, learned.K_NYQ, corr, sp)
    e2.record(stream)
    torch.cuda.synchronize()
    ms_learned = e0.elapsed_time(e1) / steps
    ms_mlp = e1.elapsed_time(e2) / steps
    batch.close()
    # plain 512^3 path on the same mocks: the target of the correction and the comparison
    fine = ys.Plan(learned.FINE["n_mesh"], learned.BOX_MIN, learned.BOX_LEN, learned.OBSERVER,
                   assign=learned.FINE["assign"], interlace=learned.FINE["interlace"], dk=learned.DK,
                   n_bins=learned.N_BINS, max_particles=max(caps), stream=sp)
    rows_f = torch.zeros_like(rows)
    fine.assign(gals[0], rans[0])
    fine.measure_async(rows_f[0])
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(n):
        fine.assign(gals[i], rans[i])
        fine.measure_async(rows_f[i])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fine = e0.elapsed_time(e1)
    fine.close()
    before = learned.residual_stats(rows, rows_f)
    after = learned.residual_stats(corr, rows_f)
    mlp.close()
    return {"value": n / (ms_learned / 1e3), "unit": UNIT, "n_catalogs": n, "ms_per_pass": ms_learned,
            "mlp_ms_per_pass": ms_mlp, "plain_512_value": n / (ms_fine / 1e3),
            "speedup_vs_plain_512": ms_fine / ms_learned,
            "residual_vs_512": {"uncorrected_128": before, "corrected_128": after,
                                "definition": "|P_l - P_l(512^3)| / (P_0 + S/I) over shells with modes, "
                                              "k < 0.80 h/Mpc; rms and max"},
            "coarse": "128^3 CIC, no interlacing, batched (waves of 8)",
            "fine": "512^3 TSC, interlaced, plain path",
            "heldout_seeds": [seeds[0], seeds[-1]],
            "trained": {k: meta[k] for k in ("train_seeds", "rows", "steps", "lr", "lr_final")}}


def cufft_comparison(n=512, fields=16, meshes=2, reps=3):
    """cuFFT (through torch.fft) on the same transforms, as a comparison only: one
    full real-to-complex 3D FFT of each of the 16 basis fields of each mesh, with no
    pruning and none of the field construction, folding, combination or shell sums
    that the library's y,z and x stages fuse around their own transforms."""
    import torch
    x = torch.randn((n, n, n), device="cuda", dtype=torch.float32)
    out = torch.empty((n, n, n // 2 + 1), device="cuda", dtype=torch.complex64)
    for _ in range(2):
        torch.fft.rfftn(x, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        for _ in range(fields * meshes):
            torch.fft.rfftn(x, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del x, out
    torch.cuda.empty_cache()
    return {"library": "cuFFT via torch.fft.rfftn", "transforms": fields * meshes, "n": n,
            "ms_per_catalogue": ms,
            "what": "full 3D R2C FFTs of the 16 basis fields x 2 meshes only; no pruning, field "
                    "construction, folding, combination or shell sums"}


def plan_pencils(plan, with_nzc=False):
    """Number of (k_y, k_z) pencils the plan keeps: k_y^2 + k_z^2 < n2_hi, derived
    from the shell edges exactly as the library does (integer |m|^2 test)."""
    L = plan.cfg.box_len
    kf = 2 * math.pi / L
    n = plan.cfg.n_mesh
    n2_hi = 0
    for n2 in range(1, (n // 2) ** 2):
        k = kf * math.sqrt(n2)
        if k < kf * n / 2 and 0 <= math.floor((k - plan.cfg.k_min) / plan.cfg.dk) < plan.cfg.n_bins:
            n2_hi = n2 + 1
    cnt = 0
    kz = 0
    while kz * kz < n2_hi:
        kymax = 0
        while (kymax + 1) ** 2 + kz * kz < n2_hi:
            kymax += 1
        cnt += 2 * kymax + 1
        kz += 1
    return (cnt, kz) if with_nzc else cnt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (fixed launch sequence for profiling)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=WORKLOAD)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
